"""Three-pass plans (N = N1 * N2 * N3: a column pass over N1, then each
length-M = N2 * N3 row transformed by a column and a row pass whose store
lands in the final order): parity with the oracle, agreement with the
two-pass plan, fault injection in each of the three passes, host-buffer
exec in chunks and the no-allocation entry point."""
import numpy as np
import pytest

import oracle
import synth_signals as ss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_05824_gb300 as tfl  # noqa: E402

CDT = {np.float32: "complex64", np.float64: "complex128"}


def three(n, batch, rdt, direction="forward", ft="off"):
    return tfl.Plan(n, batch, CDT[rdt], direction, ft, structure="three_pass")


def expected(x, direction):
    if direction == "forward":
        return oracle.fft(x)
    return oracle.fft(x, inverse=True, scaled=(direction == "inverse"))


@pytest.mark.parametrize("rdt,n", [(np.float32, 1 << 21), (np.float32, 1 << 22), (np.float32, 1 << 24),
                                   (np.float64, 1 << 18), (np.float64, 1 << 20)])
def test_three_pass_info(rdt, n):
    p = three(n, 2, rdt)
    i = p.info()
    assert i["num_passes"] == 3 and i["sub_n"][0] * i["sub_n"][1] * i["sub_n"][2] == n
    assert i["sub_n"][0] <= i["sub_n"][1] <= i["sub_n"][2]
    assert i["scratch_bytes"] == 2 * n * (8 if rdt == np.float32 else 16)
    p.close()


def test_default_structure_for_large_float32():
    p = tfl.Plan(1 << 22, 1, "complex64")
    assert p.info()["num_passes"] == 3
    p.close()
    q = tfl.Plan(1 << 22, 1, "complex64", structure="split")
    assert q.info()["num_passes"] == 2
    q.close()
    with pytest.raises(tfl.TurboFFTError):
        three(256, 4, np.float32)  # too small to split three ways


@pytest.mark.parametrize("rdt,n,batch", [(np.float32, 1 << 21, 3), (np.float32, 1 << 22, 2),
                                         (np.float32, 1 << 24, 1), (np.float64, 1 << 18, 5),
                                         (np.float64, 1 << 21, 1)])
@pytest.mark.parametrize("direction", ["forward", "inverse", "inverse_unscaled"])
@pytest.mark.parametrize("ft", ["off", "correct"])
def test_three_pass_matches_oracle(rdt, n, batch, direction, ft):
    x = ss.uniform_complex(71, batch, n, rdt)
    p = three(n, batch, rdt, direction, ft)
    y = p.exec(torch.from_numpy(x).cuda()).cpu().numpy()
    err = oracle.rel_l2(y, expected(x, direction))
    assert float(np.max(err)) <= oracle.tolerance(rdt, n), float(np.max(err))
    if ft != "off":
        rep = p.report()
        assert rep["detected"] == 0 and rep["status"] == tfl.SUCCESS and rep["groups_checked"] > 0, rep
    p.close()


@pytest.mark.parametrize("rdt,n", [(np.float32, 1 << 22), (np.float64, 1 << 19)])
def test_three_pass_agrees_with_two_pass(rdt, n):
    x = ss.uniform_complex(72, 2, n, rdt)
    xd = torch.from_numpy(x).cuda()
    a = three(n, 2, rdt, "forward", "correct")
    b = tfl.Plan(n, 2, CDT[rdt], "forward", "correct", structure="split")
    ya, yb = a.exec(xd).cpu().numpy(), b.exec(xd).cpu().numpy()
    assert float(np.max(oracle.rel_l2(ya, yb))) <= 2 * oracle.tolerance(rdt, n)
    a.close()
    b.close()


@pytest.mark.parametrize("rdt,n,batch", [(np.float32, 1 << 21, 3), (np.float64, 1 << 18, 3)])
def test_three_pass_injection_every_pass(rdt, n, batch):
    x = ss.uniform_complex(73, batch, n, rdt)
    xd = torch.from_numpy(x).cuda()
    ref = oracle.fft(x)
    tol = oracle.tolerance(rdt, n)
    p = three(n, batch, rdt, "forward", "correct")
    info = p.info()
    bit = 30 if rdt == np.float32 else 62
    rng = np.random.default_rng(5)
    for pass_ in range(3):
        for stage in sorted({0, 1, info["stages"][pass_]}):
            tr = int(rng.integers(0, batch))
            el = int(rng.integers(0, n))
            p.inject(tr, pass_, stage, el, int(rng.integers(0, 2)), bit)
            y = p.exec(xd).cpu().numpy()
            rep = p.report()
            assert rep["detected"] >= 1 and rep["corrected"] >= 1, (pass_, stage, rep)
            assert rep["first_transform"] == tr and rep["first_pass"] == pass_, (pass_, stage, rep)
            assert rep["uncorrectable"] == 0 and rep["status"] == tfl.SUCCESS
            assert float(np.max(oracle.rel_l2(y, ref))) <= tol, (pass_, stage)
    p.exec(xd)
    assert p.report()["detected"] == 0
    p.close()


def test_three_pass_exec_host_chunks_and_injection():
    n, batch = 1 << 22, 5  # 32 MiB per transform: several exec_host chunks
    x = ss.uniform_complex(74, batch, n, np.float32)
    ref = oracle.fft(x)
    p = three(n, batch, np.float32, "forward", "correct")
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    p.inject(3, 2, 1, 12345, 0, 30)
    p.exec_host(xh, yh)
    rep = p.report()
    assert rep["detected"] >= 1 and rep["first_transform"] == 3 and rep["status"] == tfl.SUCCESS, rep
    assert float(np.max(oracle.rel_l2(yh.numpy(), ref))) <= oracle.tolerance(np.float32, n)
    p.close()


def test_three_pass_static_scratch():
    n = 1 << 21  # 16 MiB intermediate: fits the static area
    x = ss.uniform_complex(75, 1, n, np.float32)
    p = three(n, 1, np.float32, "forward", "correct")
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    st = tfl.lib().turbofft_exec_static_scratch(p.handle, xd.data_ptr(), yd.data_ptr(),
                                                torch.cuda.current_stream().cuda_stream)
    assert st == tfl.SUCCESS
    torch.cuda.synchronize()
    assert float(np.max(oracle.rel_l2(yd.cpu().numpy(), oracle.fft(x)))) <= oracle.tolerance(np.float32, n)
    p.close()
