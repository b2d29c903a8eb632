"""Single-pass cluster plans (both four-step phases in one kernel whose
thread-block clusters share each transform): parity with the oracle, equal
results to the two-pass plan of the same size, and the two-sided ABFT with
injected faults in either phase."""
import numpy as np
import pytest

import oracle
import synth_signals as ss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_05824_gb300 as tfl  # noqa: E402

CL_SIZES = [1 << 13, 1 << 14, 1 << 15, 1 << 16]


def cluster_plan(n, batch, direction="forward", ft="off"):
    return tfl.Plan(n, batch, "complex64", direction, ft, structure="cluster")


def expected(x, direction):
    if direction in ("forward", "forward_scaled"):
        y = oracle.fft(x)
        return y / x.shape[1] if direction == "forward_scaled" else y
    return oracle.fft(x, inverse=True, scaled=(direction == "inverse"))


@pytest.mark.parametrize("n", CL_SIZES)
def test_cluster_plan_info(n):
    p = cluster_plan(n, 7, ft="correct")
    i = p.info()
    assert i["cluster"] >= 2 and i["num_passes"] == 2 and i["scratch_bytes"] == 0
    assert i["sub_n"][0] * i["sub_n"][1] == n
    assert i["grid"][0] % i["cluster"] == 0
    p.close()


@pytest.mark.parametrize("n", CL_SIZES)
@pytest.mark.parametrize("direction", ["forward", "inverse", "inverse_unscaled", "forward_scaled"])
@pytest.mark.parametrize("ft", ["off", "correct"])
def test_cluster_matches_oracle(n, direction, ft):
    batch = max(3, (1 << 19) // n) + 1
    x = ss.uniform_complex(41, batch, n, np.float32)
    p = cluster_plan(n, batch, direction, ft)
    y = p.exec(torch.from_numpy(x).cuda()).cpu().numpy()
    err = oracle.rel_l2(y, expected(x, direction))
    assert float(np.max(err)) <= oracle.tolerance(np.float32, n), float(np.max(err))
    if ft != "off":
        rep = p.report()
        assert rep["detected"] == 0 and rep["status"] == tfl.SUCCESS and rep["groups_checked"] > 0, rep
        assert 0 < rep["max_clean_ratio"] < 0.8
    p.close()


@pytest.mark.parametrize("n", CL_SIZES)
@pytest.mark.parametrize("batch", [1, 2, 5])
def test_cluster_small_batches_and_bounds(n, batch):
    """Fewer transforms than clusters; nothing outside [0, batch*n) is written."""
    x = ss.uniform_complex(43, batch, n, np.float32)
    guard = 4096
    out = torch.full((batch * n + 2 * guard,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
    p = cluster_plan(n, batch, "forward", "correct")
    xd = torch.from_numpy(x).cuda().view(-1)
    st = p.exec_ptr(xd.data_ptr(), out[guard:].data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == tfl.SUCCESS
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.all(o[:guard] == np.complex64(7 - 7j)) and np.all(o[guard + batch * n:] == np.complex64(7 - 7j))
    y = o[guard:guard + batch * n].reshape(batch, n)
    assert float(np.max(oracle.rel_l2(y, oracle.fft(x)))) <= oracle.tolerance(np.float32, n)
    p.close()


@pytest.mark.parametrize("n", CL_SIZES)
def test_cluster_and_split_agree(n):
    batch = 9
    x = ss.uniform_complex(45, batch, n, np.float32)
    xd = torch.from_numpy(x).cuda()
    a = cluster_plan(n, batch, "forward", "correct")
    b = tfl.Plan(n, batch, "complex64", "forward", "correct", structure="split")
    assert a.info()["cluster"] > 0 and b.info()["cluster"] == 0
    ya = a.exec(xd).cpu().numpy()
    yb = b.exec(xd).cpu().numpy()
    tol = oracle.tolerance(np.float32, n)
    assert float(np.max(oracle.rel_l2(ya, yb))) <= 2 * tol
    a.close()
    b.close()


def test_structured_create_rejects():
    with pytest.raises(tfl.TurboFFTError):
        tfl.Plan(1024, 4, "complex64", "forward", "off", structure="cluster")  # no cluster configuration
    L = tfl.lib()
    import ctypes
    h = ctypes.c_void_p()
    assert L.turbofft_plan_create_structured(1 << 14, 4, 0, -1, 0, 7, ctypes.byref(h)) == tfl.INVALID_VALUE
    assert not h.value


@pytest.mark.parametrize("n", CL_SIZES)
def test_cluster_clean_runs_no_alarm(n):
    batch = max(8, (1 << 20) // n)
    p = cluster_plan(n, batch, "forward", "correct")
    worst = 0.0
    for seed in range(12):
        x = ss.uniform_complex(100 + seed, batch, n, np.float32)
        p.exec(torch.from_numpy(x).cuda())
        rep = p.report()
        assert rep["detected"] == 0 and rep["status"] == tfl.SUCCESS
        worst = max(worst, rep["max_clean_ratio"])
    assert 0 < worst < 0.8, worst
    p.close()


@pytest.mark.parametrize("n", CL_SIZES)
def test_cluster_injection_every_stage_both_phases(n):
    batch = 11
    x = ss.uniform_complex(47, batch, n, np.float32)
    xd = torch.from_numpy(x).cuda()
    ref = oracle.fft(x)
    tol = oracle.tolerance(np.float32, n)
    p = cluster_plan(n, batch, "forward", "correct")
    off = cluster_plan(n, batch, "forward", "off")
    det = cluster_plan(n, batch, "forward", "detect")
    info = p.info()
    rng = np.random.default_rng(n)
    for pass_ in range(2):
        for stage in range(info["stages"][pass_] + 1):
            tr = int(rng.integers(0, batch))
            el = int(rng.integers(0, n))
            comp = int(rng.integers(0, 2))
            for bit in (30, 22):
                off.inject(tr, pass_, stage, el, comp, bit)
                with np.errstate(all="ignore"):
                    err_off = oracle.rel_l2(off.exec(xd).cpu().numpy(), ref)
                p.inject(tr, pass_, stage, el, comp, bit)
                y = p.exec(xd).cpu().numpy()
                rep = p.report()
                err = oracle.rel_l2(y, ref)
                breaking = not (float(np.max(err_off)) <= tol)
                if breaking:
                    assert rep["detected"] >= 1 and rep["corrected"] >= 1, (pass_, stage, bit, rep)
                    assert rep["first_transform"] == tr and rep["status"] == tfl.SUCCESS, rep
                if rep["detected"]:
                    assert rep["uncorrectable"] == 0 and rep["recomputed"] >= 1, rep
                assert float(np.max(err)) <= tol, (pass_, stage, bit, float(np.max(err)))
                # the same fault in DETECT mode is reported, not corrected
                if breaking:
                    det.inject(tr, pass_, stage, el, comp, bit)
                    det.exec(xd)
                    rd = det.report()
                    assert rd["detected"] >= 1 and rd["status"] == tfl.FT_UNCORRECTABLE and rd["corrected"] == 0
    # after the faults, a clean exec reports nothing
    p.exec(xd)
    assert p.report()["detected"] == 0
    for q in (p, off, det):
        q.close()


def test_cluster_inverse_injection():
    n, batch = 1 << 15, 6
    x = ss.uniform_complex(49, batch, n, np.float32)
    ref = oracle.fft(x, inverse=True, scaled=True)
    p = cluster_plan(n, batch, "inverse", "correct")
    p.inject(4, 1, 1, 1000, 1, 30)
    y = p.exec(torch.from_numpy(x).cuda()).cpu().numpy()
    rep = p.report()
    assert rep["detected"] >= 1 and rep["first_transform"] == 4 and rep["status"] == tfl.SUCCESS
    assert float(np.max(oracle.rel_l2(y, ref))) <= oracle.tolerance(np.float32, n)
    p.close()


def test_cluster_full_size_sampled():
    """N = 2^16 at the sweep's 2^28 elements (4096 transforms), ABFT on;
    sampled transforms against the oracle."""
    n, batch = 1 << 16, 1 << 12
    xd = ss.uniform_complex_torch(2, batch, n, "float32")
    p = cluster_plan(n, batch, "forward", "correct")
    assert p.info()["cluster"] > 0
    y = p.exec(xd)
    torch.cuda.synchronize()
    rep = p.report()
    assert rep["detected"] == 0 and rep["groups_checked"] > 0
    for b in (0, 1, 1777, batch - 1):
        xr = ss.uniform_complex(2, 1, n, np.float32, first_element=b * n)
        got = y[b].cpu().numpy()[None]
        assert float(oracle.rel_l2(got, oracle.fft(xr))[0]) <= oracle.tolerance(np.float32, n)
    p.close()
