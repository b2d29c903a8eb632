"""Float32 passes whose input tiles are staged by TMA copies issued by one
thread (a column tile as 2-D boxes of S columns x up to 256 rows, the tile
of a single pass or a row pass as one contiguous bulk copy; completion
counted on a shared-memory barrier) against the same plans staged with
16-byte cp.async copies: bitwise-equal outputs, parity with the oracle,
ragged last units, fault injection and correction in TMA-staged passes,
misaligned inputs refused before any launch, host-buffer execs in chunks."""
import numpy as np
import pytest

import oracle
import synth_signals as ss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_05824_gb300 as tfl  # noqa: E402


def make(n, batch, direction, ft, structure, tma):
    tfl.set_tma_staging("always" if tma else "never")
    try:
        return tfl.Plan(n, batch, "complex64", direction, ft, structure=structure)
    finally:
        tfl.set_tma_staging("auto")


def bits(y):
    return torch.view_as_real(y).contiguous().view(torch.int32)


def expected(x, direction):
    if direction == "forward":
        return oracle.fft(x)
    return oracle.fft(x, inverse=True, scaled=(direction == "inverse"))


@pytest.mark.parametrize("n,batch,structure", [(1 << 14, 7, "default"), (1 << 15, 3, "default"),
                                               (1 << 16, 5, "default"), (1 << 18, 2, "default"),
                                               (1 << 20, 3, "default"), (1 << 21, 1, "default"),
                                               (1 << 22, 2, "split"), (1 << 24, 1, "split")])
@pytest.mark.parametrize("direction", ["forward", "inverse"])
@pytest.mark.parametrize("ft", ["off", "correct"])
def test_tma_staging_is_bitwise_cp_async(n, batch, structure, direction, ft):
    a = make(n, batch, direction, ft, structure, True)
    b = make(n, batch, direction, ft, structure, False)
    ia, ib = a.info(), b.info()
    assert ia["num_passes"] == 2 and ia["tma_passes"] & 1 and ib["tma_passes"] == 0
    # row passes of 256 points and more keep their tile unswizzled: one bulk copy
    assert bool(ia["tma_passes"] & 2) == (ia["sub_n"][1] >= 256), ia
    x = ss.uniform_complex(81, batch, n, np.float32)
    xd = torch.from_numpy(x).cuda()
    ya, yb = a.exec(xd), b.exec(xd)
    assert torch.equal(bits(ya), bits(yb))
    if n <= 1 << 21:
        err = oracle.rel_l2(ya.cpu().numpy(), expected(x, direction))
        assert float(np.max(err)) <= oracle.tolerance(np.float32, n), float(np.max(err))
    ra = a.report()
    assert ra["status"] == tfl.SUCCESS, ra
    if ft != "off":
        assert ra["detected"] == 0 and ra["groups_checked"] == b.report()["groups_checked"] > 0, ra
    a.close()
    b.close()


def test_default_staging_choice():
    # TMA where it measured faster (bit p: pass p): row passes; column tiles
    # with 64-byte rows at N1 >= 512 or with checksums on; single passes of
    # 4096, of 1024 / 2048 with checksums, of 256 / 8192 without
    cases = [((1 << 20, 2, "complex64"), 3), ((1 << 18, 2, "complex64"), 3),
             ((1 << 16, 2, "complex64", "forward", "correct"), 3), ((1 << 16, 2, "complex64"), 2),
             ((1 << 14, 2, "complex64"), 0), ((1 << 14, 2, "complex64", "forward", "correct"), 1),
             ((1 << 22, 1, "complex64", "forward", "off", "split"), 2),
             ((1 << 12, 2, "complex64"), 1), ((1 << 12, 2, "complex64", "forward", "correct"), 1),
             ((1 << 10, 2, "complex64"), 0), ((1 << 10, 2, "complex64", "forward", "correct"), 1),
             ((1 << 13, 2, "complex64"), 1), ((1 << 13, 2, "complex64", "forward", "correct"), 0),
             ((1 << 6, 2, "complex64"), 0), ((1 << 16, 2, "complex128"), 0), ((1 << 22, 1, "complex64"), 0)]
    for args, want in cases:
        kw = {"structure": args[5]} if len(args) > 5 else {}
        q = tfl.Plan(*args[:5], **kw)  # float64, tiny and three-pass plans: cp.async staging
        assert q.info()["tma_passes"] == want, args
        q.close()


@pytest.mark.parametrize("n,batch", [(1 << 8, 1001), (1 << 9, 37), (1 << 10, 300), (1 << 11, 77),
                                     (1 << 12, 50), (1 << 13, 9)])
@pytest.mark.parametrize("direction", ["forward", "inverse"])
@pytest.mark.parametrize("ft", ["off", "correct"])
def test_single_pass_bulk_copies_are_bitwise_cp_async(n, batch, direction, ft):
    """One contiguous bulk copy per tile of S whole transforms; batches
    that leave a ragged last unit copy only its valid transforms."""
    a = make(n, batch, direction, ft, "default", True)
    b = make(n, batch, direction, ft, "default", False)
    assert a.info()["num_passes"] == 1 and a.info()["tma_passes"] == 1 and b.info()["tma_passes"] == 0
    x = ss.uniform_complex(85, batch, n, np.float32)
    xd = torch.from_numpy(x).cuda()
    ya, yb = a.exec(xd), b.exec(xd)
    assert torch.equal(bits(ya), bits(yb))
    err = oracle.rel_l2(ya.cpu().numpy(), expected(x, direction))
    assert float(np.max(err)) <= oracle.tolerance(np.float32, n), float(np.max(err))
    ra = a.report()
    assert ra["status"] == tfl.SUCCESS and (ft == "off" or ra["detected"] == 0), ra
    a.close()
    b.close()


@pytest.mark.parametrize("n,batch", [(1 << 16, 6), (1 << 20, 3)])
def test_tma_staged_pass_detects_and_corrects(n, batch):
    x = ss.uniform_complex(82, batch, n, np.float32)
    xd = torch.from_numpy(x).cuda()
    ref = oracle.fft(x)
    tol = oracle.tolerance(np.float32, n)
    p = make(n, batch, "forward", "correct", "default", True)
    info = p.info()
    assert info["tma_passes"] == 3
    rng = np.random.default_rng(9)
    for pass_ in range(2):
        for stage in sorted({0, 1, info["stages"][pass_]}):
            tr = int(rng.integers(0, batch))
            el = int(rng.integers(0, n))
            p.inject(tr, pass_, stage, el, int(rng.integers(0, 2)), 30)
            y = p.exec(xd).cpu().numpy()
            rep = p.report()
            assert rep["detected"] >= 1 and rep["corrected"] >= 1 and rep["first_pass"] == pass_, (stage, rep)
            assert rep["first_transform"] == tr and rep["uncorrectable"] == 0 and rep["status"] == tfl.SUCCESS
            assert float(np.max(oracle.rel_l2(y, ref))) <= tol, (pass_, stage)
    p.exec(xd)
    assert p.report()["detected"] == 0
    p.close()


def test_misaligned_input_is_rejected_before_any_launch():
    n, batch = 1 << 16, 3
    # a view starting 8 bytes into its buffer: neither TMA nor 16-byte
    # cp.async copies can read it, and the exec refuses it up front
    buf = torch.zeros(batch * n + 1, dtype=torch.complex64, device="cuda")
    xd = buf[1:].view(batch, n)
    assert xd.data_ptr() % 16 == 8
    p = make(n, batch, "forward", "correct", "default", True)
    assert p.info()["tma_passes"] == 3
    with pytest.raises(tfl.TurboFFTError):
        p.exec(xd)
    y = p.exec(torch.zeros(batch, n, dtype=torch.complex64, device="cuda"))
    assert int(torch.count_nonzero(y)) == 0 and p.report()["status"] == tfl.SUCCESS
    p.close()


def test_tma_through_host_chunks():
    n, batch = 1 << 20, 40  # 320 MiB: several 128 MiB host-staging chunks
    x = ss.uniform_complex(84, batch, n, np.float32)
    xh = torch.from_numpy(x).pin_memory()
    a = make(n, batch, "forward", "correct", "default", True)
    b = make(n, batch, "forward", "correct", "default", False)
    ya = a.exec_host(xh, torch.empty_like(xh).pin_memory())
    yb = b.exec_host(xh, torch.empty_like(xh).pin_memory())
    assert torch.equal(bits(ya), bits(yb))
    sample = [0, 17, batch - 1]
    err = oracle.rel_l2(ya.numpy()[sample], oracle.fft(x[sample]))
    assert float(np.max(err)) <= oracle.tolerance(np.float32, n)
    assert a.report()["status"] == tfl.SUCCESS and a.report()["detected"] == 0
    a.close()
    b.close()
