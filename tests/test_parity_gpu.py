"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Element-by-element comparison on the same seeded inputs: the accuracy bar is
relative L2 error per transform <= 2e-6 log2 N (complex64) and
<= 5e-15 log2 N (complex128), taken as the maximum over transforms.
"""
import math

import numpy as np
import pytest

import oracle
import synth_signals as ss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_05824_gb300 as tfl  # noqa: E402

DT = {"c64": np.float32, "c128": np.float64}


def run_gpu(x: np.ndarray, direction="forward", ft="off"):
    batch, n = x.shape
    plan = tfl.Plan(n, batch, "complex64" if x.dtype == np.complex64 else "complex128", direction, ft)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    y = plan.exec(xd)
    torch.cuda.synchronize()
    rep = plan.report() if ft != "off" else None
    out = y.cpu().numpy()
    plan.close()
    return out, rep


def expected(x, direction):
    if direction == "forward":
        return oracle.fft(x)
    return oracle.fft(x, inverse=True, scaled=(direction == "inverse"))


def check(x, direction="forward", ft="off"):
    n = x.shape[1]
    y, rep = run_gpu(x, direction, ft)
    ref = expected(x, direction)
    err = oracle.rel_l2(y, ref)
    tol = oracle.tolerance(np.float32 if x.dtype == np.complex64 else np.float64, n)
    assert np.all(np.isfinite(y))
    assert float(np.max(err)) <= tol, (n, direction, float(np.max(err)), tol)
    if rep is not None:
        assert rep["detected"] == 0 and rep["uncorrectable"] == 0, rep
        assert rep["groups_checked"] > 0
    return float(np.max(err))


def batch_for(n, target=1 << 19):
    # several tiles and a ragged tail: not a multiple of the signals per block
    b = max(1, target // n)
    return b + 3 if b > 4 else b


SIZES = [1 << k for k in range(3, 25)]


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", SIZES)
def test_forward_uniform(dt, n):
    x = ss.uniform_complex(2, batch_for(n), n, DT[dt])
    check(x, "forward")


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("direction", ["inverse", "inverse_unscaled"])
@pytest.mark.parametrize("n", [8, 64, 512, 4096, 1 << 13, 1 << 14, 1 << 17, 1 << 20, 1 << 24])
def test_inverse_uniform(dt, direction, n):
    x = ss.uniform_complex(3, batch_for(n, 1 << 18), n, DT[dt])
    check(x, direction)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", [8, 64, 4096, 1 << 14, 1 << 22])
def test_scaled_inverse_is_exact_power_of_two_scaling(dt, n):
    """The scaled inverse is the unscaled inverse times 2^-log2(N), bit for
    bit, whichever way the kernel applies the scale: rows of ordinary
    values, exact zeros, values whose scaled result is subnormal, subnormal
    inputs, infinities and NaNs (the last ones must not change a transform's
    neighbours either)."""
    rdt = DT[dt]
    batch = max(4, min(64, (1 << 18) // n))
    x = ss.uniform_complex(11, batch, n, rdt)
    tiny = np.finfo(rdt).tiny
    x[1] = 0
    x[2] *= tiny * 4          # outputs near the bottom of the normal range
    x[3] *= tiny / 1024       # subnormal inputs
    if batch > 5:
        x[5, n // 3] = np.inf
        x[5, n // 2] = complex(np.nan, 1.0)
    ys, _ = run_gpu(x, "inverse")
    yu, _ = run_gpu(x, "inverse_unscaled")
    scale = rdt(1.0) / rdt(n)
    with np.errstate(all="ignore"):
        want = (yu.view(rdt) * scale).view(yu.dtype)
    np.testing.assert_array_equal(ys.view(rdt), want.view(rdt))
    ok = [r for r in range(batch) if r != 5]
    assert np.all(np.isfinite(ys[ok]))


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("kind", ["impulse", "constant", "tone"])
@pytest.mark.parametrize("n", [8, 32, 256, 2048, 1 << 14, 1 << 16, 1 << 21])
def test_structured_inputs(dt, kind, n):
    x = ss.structured(kind, batch_for(n, 1 << 17), n, DT[dt])
    check(x, "forward")


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", SIZES)
def test_ft_correct_clean_parity(dt, n):
    """ABFT on, no fault: same accuracy, no detection."""
    x = ss.uniform_complex(4, batch_for(n, 1 << 18), n, DT[dt])
    check(x, "forward", "correct")


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", [16, 1024, 1 << 15])
def test_ft_inverse_clean(dt, n):
    x = ss.uniform_complex(5, batch_for(n, 1 << 17), n, DT[dt])
    check(x, "inverse", "correct")


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("batch", [1, 2, 3, 5, 17])
@pytest.mark.parametrize("n", [8, 256, 2048, 1 << 14])
def test_small_and_ragged_batches(dt, batch, n):
    x = ss.uniform_complex(6, batch, n, DT[dt])
    check(x, "forward", "correct")


def test_output_only_written_in_range():
    """Guard bands around the output stay untouched."""
    n, batch = 1024, 37
    x = ss.uniform_complex(7, batch, n, np.float32)
    plan = tfl.Plan(n, batch, "complex64", "forward", "correct")
    xd = torch.from_numpy(x).cuda()
    guard = 4096
    buf = torch.full((batch * n + 2 * guard,), 123.0 + 7j, dtype=torch.complex64, device="cuda")
    out = buf[guard:guard + batch * n].view(batch, n)
    plan.exec(xd, out)
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    assert np.all(b[:guard] == 123.0 + 7j) and np.all(b[-guard:] == 123.0 + 7j)
    assert float(np.max(oracle.rel_l2(out.cpu().numpy(), oracle.fft(x)))) <= oracle.tolerance(np.float32, n)
    # the input is never written
    np.testing.assert_array_equal(xd.cpu().numpy(), x)


def test_in_place_rejected():
    plan = tfl.Plan(64, 4, "complex64")
    x = torch.zeros(4, 64, dtype=torch.complex64, device="cuda")
    st = plan.exec_ptr(x.data_ptr(), x.data_ptr(), 0)
    assert st == tfl.UNSUPPORTED
    st = plan.exec_ptr(x.data_ptr() + 8, x.data_ptr() + 512, 0)
    assert st == tfl.INVALID_VALUE  # misaligned


@pytest.mark.parametrize("dt,n", [("c64", 8), ("c64", 1024), ("c64", 1 << 16), ("c64", 1 << 24),
                                  ("c128", 1024), ("c128", 1 << 20)])
def test_full_size_sampled(dt, n):
    """The benchmark's workload size (2^28 elements per call for complex64,
    2^27 here for complex128 to bound host memory), checked on sampled
    transforms that the oracle computes one by one."""
    total = (1 << 28) if dt == "c64" else (1 << 27)
    batch = total // n
    name = "float32" if dt == "c64" else "float64"
    x = ss.uniform_complex_torch(8, batch, n, name, device="cuda")
    plan = tfl.Plan(n, batch, x.dtype, "forward", "correct")
    y = plan.exec(x)
    torch.cuda.synchronize()
    rep = plan.report()
    assert rep["detected"] == 0 and rep["uncorrectable"] == 0
    rng = np.random.default_rng(n)
    rows = sorted(set([0, batch - 1] + list(rng.integers(0, batch, size=6))))
    for r in rows:
        xr = ss.uniform_complex(8, 1, n, DT[dt], first_element=r * n)
        np.testing.assert_array_equal(x[r].cpu().numpy(), xr[0])
        err = float(oracle.rel_l2(y[r].cpu().numpy()[None], oracle.fft(xr))[0])
        assert err <= oracle.tolerance(DT[dt], n), (r, err)
    plan.close()
    del x, y
    torch.cuda.empty_cache()


def test_plan_info():
    p = tfl.Plan(1 << 20, 2, "complex64", "forward", "correct")
    i = p.info()
    assert i["num_passes"] == 2 and i["sub_n"][0] * i["sub_n"][1] == 1 << 20
    assert i["stages"][0] >= 1 and i["block"][0] > 0 and i["grid"][0] > 0
    p1 = tfl.Plan(1024, 8, "complex128")
    assert p1.info()["num_passes"] == 1 and p1.info()["sub_n"][0] == 1024


def test_float64_column_tables_are_plan_owned():
    """float64 two-pass plans own an n-point twiddle table for the column
    pass (and an n-point checksum-weight table with fault tolerance on),
    counted in workspace_bytes and freed with the plan."""
    n = 1 << 16
    free0, _ = torch.cuda.mem_get_info()
    off = tfl.Plan(n, 3, "complex128", "forward", "off")
    ft = tfl.Plan(n, 3, "complex128", "forward", "correct")
    io, ic = off.info(), ft.info()
    assert io["num_passes"] == 2
    assert io["workspace_bytes"] >= io["scratch_bytes"] + n * 16
    assert ic["workspace_bytes"] >= ic["scratch_bytes"] + 2 * n * 16
    x = ss.uniform_complex(12, 3, n, np.float64)
    xd = torch.from_numpy(x).cuda()
    ref = oracle.fft(x)
    for y in (off.exec(xd).cpu().numpy(), ft.exec(xd).cpu().numpy()):
        assert float(np.max(oracle.rel_l2(y, ref))) <= oracle.tolerance(np.float64, n)
    assert ft.report()["detected"] == 0
    off.close()
    ft.close()
    del xd
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (1 << 20)


def test_exec_host_matches_device_path():
    n, batch = 4096, 300
    x = ss.uniform_complex(9, batch, n, np.float32)
    plan = tfl.Plan(n, batch, "complex64", "forward", "correct")
    xh = torch.from_numpy(x).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    plan.exec_host(xh, yh)
    yd = plan.exec(xh.cuda())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(yh.numpy(), yd.cpu().numpy())
    assert float(np.max(oracle.rel_l2(yh.numpy(), oracle.fft(x)))) <= oracle.tolerance(np.float32, n)
