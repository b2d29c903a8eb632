"""turbofft_exec_static_scratch: the transform for callers that may not
allocate device memory when they transform (their device memory belongs to
another allocator, or a budget fixed at start-up).  A two-pass plan's
intermediate then lives in the library's fixed 32 MiB device array instead of
a cudaMalloc'd buffer.  Checked through the C ABI against turbofft_exec on two
calls in a row.  Kept in its own file, collected last."""
import ctypes

import numpy as np
import pytest

import oracle
import synth_signals as ss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_05824_gb300 as tfl  # noqa: E402

DT = {"complex64": np.float32, "complex128": np.float64}


def _call(plan, x, y):
    st = tfl.lib().turbofft_exec_static_scratch(plan.handle, x.data_ptr(), y.data_ptr(),
                                                 torch.cuda.current_stream().cuda_stream)
    return st


@pytest.mark.parametrize("dtype,n,batch,ft", [
    ("complex64", 1 << 16, 24, "off"),      # two passes, 12 MiB intermediate
    ("complex64", 1 << 20, 4, "correct"),   # two passes with checksums
    ("complex128", 1 << 14, 64, "off"),     # two passes, 16 MiB intermediate
    ("complex64", 1024, 100, "off"),        # one pass: no intermediate needed
])
def test_matches_exec_on_two_calls(dtype, n, batch, ft):
    plan = tfl.Plan(n, batch, dtype, "forward", ft)
    info = plan.info()
    assert info["scratch_bytes"] <= tfl.STATIC_SCRATCH_BYTES
    tol = oracle.tolerance(DT[dtype], n)
    for call in range(2):
        x = ss.uniform_complex(40 + call, batch, n, DT[dtype])
        xd = torch.from_numpy(x).cuda()
        y_ref = plan.exec(xd)
        y_new = torch.full_like(xd, float("nan"))
        assert _call(plan, xd, y_new) == tfl.SUCCESS
        torch.cuda.synchronize()
        if ft != "off":
            rep = plan.report()
            assert rep["detected"] == 0 and rep["groups_checked"] > 0
        a, b = y_new.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert float(np.max(oracle.rel_l2(a, b))) <= tol
        assert float(np.max(oracle.rel_l2(a, oracle.fft(x)))) <= tol
    plan.close()


def test_allocates_nothing_after_setup():
    n, batch = 1 << 15, 32
    plan = tfl.Plan(n, batch, "complex64", "forward", "off")
    xd = torch.from_numpy(ss.uniform_complex(50, batch, n, np.float32)).cuda()
    yd = torch.empty_like(xd)
    assert _call(plan, xd, yd) == tfl.SUCCESS   # first call: address lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _call(plan, xd, yd) == tfl.SUCCESS
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # the plan never allocated its own intermediate either (only its tables)
    info = plan.info()
    assert info["workspace_bytes"] - info["scratch_bytes"] < 1 << 20
    plan.close()


def test_rejects_plans_beyond_the_static_size():
    n, batch = 1 << 16, 80        # 40 MiB intermediate > 32 MiB
    plan = tfl.Plan(n, batch, "complex64", "forward", "off")
    assert plan.info()["scratch_bytes"] > tfl.STATIC_SCRATCH_BYTES
    xd = torch.zeros(batch, n, dtype=torch.complex64, device="cuda")
    yd = torch.full_like(xd, 7.0)
    assert _call(plan, xd, yd) == tfl.INVALID_VALUE
    torch.cuda.synchronize()
    assert tfl.lib().turbofft_last_error(plan.handle).decode().startswith("turbofft_exec_static_scratch")
    assert bool(torch.all(yd == 7.0))
    plan.close()


def test_null_plan_rejected():
    assert tfl.lib().turbofft_exec_static_scratch(None, None, None, None) == tfl.INVALID_VALUE
