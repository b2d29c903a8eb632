"""C-ABI library checks that need no GPU: the shared library loads, exports
every function include/turbofft.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

import paper_2412_05824_gb300 as tfl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "turbofft.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(turbofft_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(tfl.LIB_PATH):
        from paper_2412_05824_gb300 import build as b
        b.build()
    return tfl.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["turbofft_plan_create", "turbofft_exec", "turbofft_inject", "turbofft_destroy",
                     "turbofft_get_report", "turbofft_exec_host"]:
        assert required in names


def test_every_declared_symbol_is_exported(L):
    for name in _declared_functions():
        assert hasattr(L, name), name
    assert sorted(tfl.EXPORTS) == sorted(_declared_functions())


def test_status_strings(L):
    for code in range(7):
        assert L.turbofft_status_string(code).decode().startswith("TURBOFFT_")
    assert L.turbofft_status_string(99) == b"TURBOFFT_UNKNOWN_STATUS"


@pytest.mark.parametrize("n,batch,dtype,direction,ft", [
    (12, 4, 0, -1, 0),          # not a power of two
    (4, 4, 0, -1, 0),           # below the minimum length 8
    (1 << 25, 1, 0, -1, 0),     # above the maximum length 2^24
    (64, 0, 0, -1, 0),          # empty batch
    (64, 1 << 30, 0, -1, 0),    # too many elements
    (64, 4, 7, -1, 0),          # bad dtype
    (64, 4, 0, 0, 0),           # bad direction
    (64, 4, 0, -1, 9),          # bad ft mode
])
def test_plan_create_rejects_bad_arguments(L, n, batch, dtype, direction, ft):
    h = ctypes.c_void_p(123)
    st = L.turbofft_plan_create(n, batch, dtype, direction, ft, ctypes.byref(h))
    assert st == tfl.INVALID_VALUE
    assert not h.value


def test_null_handles_are_rejected(L):
    assert L.turbofft_exec(None, None, None, None) == tfl.INVALID_VALUE
    assert L.turbofft_exec_host(None, None, None, None) == tfl.INVALID_VALUE
    assert L.turbofft_inject(None, tfl.Site(0, 0, 0, 0, 0), 3) == tfl.INVALID_VALUE
    r = tfl.Report()
    assert L.turbofft_get_report(None, ctypes.byref(r)) == tfl.INVALID_VALUE
    assert L.turbofft_plan_get_info(None, None) == tfl.INVALID_VALUE
    assert L.turbofft_set_threshold_scale(None, 1.0) == tfl.INVALID_VALUE
    assert L.turbofft_destroy(None) == tfl.SUCCESS
    assert L.turbofft_plan_create(64, 4, 0, -1, 0, None) == tfl.INVALID_VALUE


def test_null_handles_are_rejected_by_the_other_calls(L):
    assert L.turbofft_set_group_transactions(None, 4) == tfl.INVALID_VALUE
    assert L.turbofft_set_workspace(None, None, 0) == tfl.INVALID_VALUE
    assert L.turbofft_set_profiling(None, 1) == tfl.INVALID_VALUE
    assert L.turbofft_get_kernel_times(None, None, 0, None) == tfl.INVALID_VALUE
    assert L.turbofft_exec_static_scratch(None, None, None, None) == tfl.INVALID_VALUE
    assert L.turbofft_last_error(None) == b""


@pytest.mark.parametrize("structure", [-1, 0, 5, 99])
def test_structured_create_rejects_unknown_structures(L, structure):
    h = ctypes.c_void_p(123)
    st = L.turbofft_plan_create_structured(1 << 14, 4, 0, -1, 0, structure, ctypes.byref(h))
    assert st == tfl.INVALID_VALUE
    assert not h.value


@pytest.mark.parametrize("dtype,ft", [(0, 0), (1, 1), (1, 2), (1, 3), (1, 4)])
def test_float_pairs_only_for_plain_float64(L, dtype, ft):
    # float-pair arithmetic: complex128 without checksums only (decided
    # before any device call)
    h = ctypes.c_void_p(123)
    st = L.turbofft_plan_create_structured(1024, 4, dtype, -1, ft, 4, ctypes.byref(h))
    assert st == tfl.UNSUPPORTED
    assert not h.value


def test_no_gpu_reports_cuda_error_not_crash(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = L.turbofft_plan_create(64, 4, 0, -1, 0, ctypes.byref(h))
    assert st == tfl.CUDA_ERROR and not h.value


def _ragged(L, sizes, offsets, dtype=0, direction=-1, ft=0, count=None):
    arr = ctypes.c_int64 * max(1, len(sizes))
    h = ctypes.c_void_p(123)
    st = L.turbofft_plan_create_ragged(arr(*sizes), arr(*offsets), len(sizes) if count is None else count,
                                       dtype, direction, ft, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("sizes,offsets,dtype,direction,ft,count", [
    ([64, 128], [0, 64], 0, -1, 0, 0),          # empty batch
    ([64, 96], [0, 64], 0, -1, 0, None),        # not a power of two
    ([64, 4], [0, 64], 0, -1, 0, None),         # below the minimum length 8
    ([64, 1 << 25], [0, 64], 0, -1, 0, None),   # above the maximum length
    ([64, 128], [0, -2], 0, -1, 0, None),       # negative offset
    ([64, 128], [0, 65], 0, -1, 0, None),       # odd complex64 offset: not 16-byte aligned
    ([64, 128], [0, 32], 0, -1, 0, None),       # overlapping transforms
    ([128, 64], [40, 0], 0, -1, 0, None),       # overlap found after sorting by offset
    ([64, 128], [0, 64], 3, -1, 0, None),       # bad dtype
    ([64, 128], [0, 64], 0, 5, 0, None),        # bad direction
    ([64, 128], [0, 64], 0, -1, 8, None),       # bad ft mode
])
def test_ragged_create_rejects_bad_arguments(L, sizes, offsets, dtype, direction, ft, count):
    st, h = _ragged(L, sizes, offsets, dtype, direction, ft, count)
    assert st == tfl.INVALID_VALUE
    assert not h.value


def test_ragged_null_arrays_are_rejected(L):
    h = ctypes.c_void_p(123)
    assert L.turbofft_plan_create_ragged(None, None, 3, 0, -1, 0, ctypes.byref(h)) == tfl.INVALID_VALUE
    assert L.turbofft_plan_get_member_info(None, 0, None) == tfl.INVALID_VALUE
    assert L.turbofft_set_autotune(0) == tfl.SUCCESS


def test_ragged_odd_offset_is_fine_for_complex128(L):
    # every complex128 element is 16 bytes: any offset is aligned; without a
    # GPU the call gets as far as the device query
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = _ragged(L, [64, 128], [1, 65], dtype=1)
    assert st == tfl.CUDA_ERROR and not h.value


def test_static_scratch_size_is_exported(L):
    """The static scratch size comes from the library itself, and matches
    the header's TURBOFFT_STATIC_SCRATCH_BYTES."""
    src = open(HEADER).read()
    m = re.search(r"#define TURBOFFT_STATIC_SCRATCH_BYTES \((\d+)u << (\d+)\)", src)
    assert m, "header macro not found"
    assert "extern const uint64_t turbofft_static_scratch_bytes;" in src
    assert tfl.static_scratch_bytes() == int(m.group(1)) << int(m.group(2))
    assert tfl.STATIC_SCRATCH_BYTES == tfl.static_scratch_bytes()


def test_fma_peak_rejects_bad_arguments(L):
    out = ctypes.c_double()
    assert L.turbofft_fma_peak(0, 0.5, None, None) == tfl.INVALID_VALUE
    assert L.turbofft_fma_peak(0, 0.0, None, ctypes.byref(out)) == tfl.INVALID_VALUE
    assert L.turbofft_fma_peak(0, 100.0, None, ctypes.byref(out)) == tfl.INVALID_VALUE
    assert L.turbofft_fma_peak(5, 0.5, None, ctypes.byref(out)) == tfl.INVALID_VALUE


def test_thread_level_mode_rejected_where_it_cannot_apply(L):
    h = ctypes.c_void_p()
    sizes = (ctypes.c_int64 * 2)(8, 16)
    offs = (ctypes.c_int64 * 2)(0, 8)
    # ragged plans and cluster / three-pass structures have no one-thread shape
    assert L.turbofft_plan_create_ragged(sizes, offs, 2, 0, -1, 4, ctypes.byref(h)) == tfl.UNSUPPORTED
    assert L.turbofft_plan_create_structured(1 << 14, 4, 0, -1, 4, 2, ctypes.byref(h)) == tfl.UNSUPPORTED
    assert L.turbofft_plan_create_structured(1 << 22, 1, 0, -1, 4, 3, ctypes.byref(h)) == tfl.UNSUPPORTED
    assert L.turbofft_plan_create(64, 4, 0, -1, 5, ctypes.byref(h)) == tfl.INVALID_VALUE


def test_process_wide_switches_need_no_device(L):
    """The staging / launch-form switches only record a choice for plans
    created afterwards."""
    for f in (L.turbofft_set_tma_staging, L.turbofft_set_ragged_single_launch):
        assert f(0) == tfl.SUCCESS
        assert f(1) == tfl.SUCCESS
    assert L.turbofft_set_tma_staging(2) == tfl.SUCCESS
    assert L.turbofft_set_tma_staging(3) == tfl.INVALID_VALUE
    assert L.turbofft_set_tma_staging(-1) == tfl.INVALID_VALUE
    assert L.turbofft_set_tma_staging(1) == tfl.SUCCESS


def test_plan_info_layout_matches_header():
    """The binding's PlanInfo mirrors the header's field list."""
    src = open(HEADER).read()
    body = src[src.index("/* Static facts about a plan. */"):src.index("} turbofft_plan_info;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b(?:int32_t|int64_t)\s+([^;]+);", body)
    fields = []
    for decl in names:
        for part in decl.split(","):
            fields.append(re.sub(r"\[.*\]", "", part).strip())
    assert fields == [name for name, _ in tfl.PlanInfo._fields_]
