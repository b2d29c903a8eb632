"""Python binding of libturbofft (include/turbofft.h): argument marshalling
only.  Every step of the transform and of the fault tolerance runs in the
library's CUDA kernels; PyTorch provides device memory and streams.

    import paper_2412_05824_gb300 as tf
    plan = tf.Plan(n=1024, batch=4096, dtype="complex64", direction="forward", ft="correct")
    y = plan.exec(x)                      # x: CUDA complex tensor [batch, n]
    rep = plan.report()                   # fault-tolerance outcome of that exec

There is no fallback: if the compiled library is missing the import of
`lib()` raises, and so does every call that needs it.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libturbofft.so")

# status codes
SUCCESS = 0
INVALID_VALUE = 1
UNSUPPORTED = 2
ALLOC_FAILED = 3
CUDA_ERROR = 4
FT_UNCORRECTABLE = 5
TIMEOUT = 6

C2C_F32 = 0
C2C_F64 = 1
FORWARD = -1
INVERSE = 1
INVERSE_UNSCALED = 2
FORWARD_SCALED = -2
FT_OFF = 0
FT_DETECT = 1
FT_CORRECT = 2
FT_CORRECT_REGISTERS = 3
FT_CORRECT_THREAD = 4

_DIRS = {"forward": FORWARD, "inverse": INVERSE, "inverse_unscaled": INVERSE_UNSCALED,
         "forward_scaled": FORWARD_SCALED, FORWARD: FORWARD, INVERSE: INVERSE,
         INVERSE_UNSCALED: INVERSE_UNSCALED, FORWARD_SCALED: FORWARD_SCALED}
STRUCTURE_SPLIT = 1
STRUCTURE_CLUSTER = 2
STRUCTURE_THREE_PASS = 3
STRUCTURE_FLOAT_PAIRS = 4
_STRUCT = {"split": STRUCTURE_SPLIT, "cluster": STRUCTURE_CLUSTER, "three_pass": STRUCTURE_THREE_PASS,
           "float_pairs": STRUCTURE_FLOAT_PAIRS}
_FT = {"off": FT_OFF, "detect": FT_DETECT, "correct": FT_CORRECT, "correct_registers": FT_CORRECT_REGISTERS,
       "correct_thread": FT_CORRECT_THREAD,
       None: FT_OFF, False: FT_OFF, FT_OFF: FT_OFF, FT_DETECT: FT_DETECT, FT_CORRECT: FT_CORRECT,
       FT_CORRECT_REGISTERS: FT_CORRECT_REGISTERS, FT_CORRECT_THREAD: FT_CORRECT_THREAD}


class Site(ctypes.Structure):
    _fields_ = [("transform", ctypes.c_int64), ("pass_", ctypes.c_int32), ("stage", ctypes.c_int32),
                ("element", ctypes.c_int64), ("component", ctypes.c_int32)]


class Report(ctypes.Structure):
    _fields_ = [("groups_checked", ctypes.c_int64), ("detected", ctypes.c_int64),
                ("located", ctypes.c_int64), ("corrected", ctypes.c_int64),
                ("recomputed", ctypes.c_int64), ("uncorrectable", ctypes.c_int64),
                ("first_transform", ctypes.c_int64), ("first_pass", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("first_residual", ctypes.c_double),
                ("first_threshold", ctypes.c_double), ("max_clean_ratio", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("batch", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("direction", ctypes.c_int32), ("ft_mode", ctypes.c_int32),
                ("num_passes", ctypes.c_int32), ("sub_n", ctypes.c_int64 * 3),
                ("stages", ctypes.c_int32 * 3), ("radix", ctypes.c_int32 * 3),
                ("group_transactions", ctypes.c_int32), ("grid", ctypes.c_int32 * 3),
                ("block", ctypes.c_int32 * 3), ("workspace_bytes", ctypes.c_int64),
                ("scratch_bytes", ctypes.c_int64), ("per_block", ctypes.c_int32 * 3),
                ("num_members", ctypes.c_int32), ("autotuned", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("single_launch", ctypes.c_int32),
                ("transform_checks", ctypes.c_int32), ("tma_passes", ctypes.c_int32)]


class KernelTime(ctypes.Structure):
    _fields_ = [("pass_", ctypes.c_int32), ("is_correction", ctypes.c_int32), ("ms", ctypes.c_double)]


EXPORTS = [
    "turbofft_plan_create", "turbofft_exec", "turbofft_exec_host", "turbofft_inject",
    "turbofft_get_report", "turbofft_plan_get_info", "turbofft_set_threshold_scale",
    "turbofft_destroy", "turbofft_status_string", "turbofft_last_error",
    "turbofft_set_workspace", "turbofft_set_profiling", "turbofft_get_kernel_times",
    "turbofft_exec_static_scratch", "turbofft_plan_create_ragged", "turbofft_plan_get_member_info",
    "turbofft_set_autotune", "turbofft_plan_create_structured", "turbofft_set_group_transactions",
    "turbofft_fma_peak", "turbofft_set_ragged_single_launch", "turbofft_set_tma_staging",
]

_lib = None


def lib() -> ctypes.CDLL:
    """Load libturbofft.so (built by build.py / __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libturbofft.so is not built (%s); run paper_2412_05824_gb300/build.py" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.turbofft_plan_create.argtypes = [i64, i64, i32, i32, i32, ctypes.POINTER(vp)]
    L.turbofft_exec.argtypes = [vp, vp, vp, vp]
    L.turbofft_exec_host.argtypes = [vp, vp, vp, vp]
    L.turbofft_exec_static_scratch.argtypes = [vp, vp, vp, vp]
    L.turbofft_plan_create_ragged.argtypes = [ctypes.POINTER(i64), ctypes.POINTER(i64), i64, i32, i32, i32,
                                              ctypes.POINTER(vp)]
    L.turbofft_plan_get_member_info.argtypes = [vp, i32, ctypes.POINTER(PlanInfo)]
    L.turbofft_set_autotune.argtypes = [i32]
    L.turbofft_set_ragged_single_launch.argtypes = [i32]
    L.turbofft_set_tma_staging.argtypes = [i32]
    L.turbofft_set_group_transactions.argtypes = [vp, i32]
    L.turbofft_plan_create_structured.argtypes = [i64, i64, i32, i32, i32, i32, ctypes.POINTER(vp)]
    L.turbofft_inject.argtypes = [vp, Site, i32]
    L.turbofft_get_report.argtypes = [vp, ctypes.POINTER(Report)]
    L.turbofft_plan_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    L.turbofft_set_threshold_scale.argtypes = [vp, ctypes.c_double]
    L.turbofft_destroy.argtypes = [vp]
    L.turbofft_set_workspace.argtypes = [vp, vp, ctypes.c_size_t]
    L.turbofft_set_profiling.argtypes = [vp, i32]
    L.turbofft_get_kernel_times.argtypes = [vp, ctypes.POINTER(KernelTime), i32, ctypes.POINTER(i32)]
    L.turbofft_fma_peak.argtypes = [i32, ctypes.c_double, vp, ctypes.POINTER(ctypes.c_double)]
    L.turbofft_status_string.argtypes = [i32]
    L.turbofft_status_string.restype = ctypes.c_char_p
    L.turbofft_last_error.argtypes = [vp]
    L.turbofft_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("turbofft_status_string", "turbofft_last_error"):
            getattr(L, name).restype = i32
    _lib = L
    return L


def fma_peak(dtype="complex128", seconds: float = 0.5, stream=None) -> float:
    """Measured FMA throughput (TFLOP/s) of the current device in the real
    type of `dtype` (turbofft_fma_peak)."""
    out = ctypes.c_double()
    s = 0 if stream is None else stream.cuda_stream
    _check(lib().turbofft_fma_peak(_dtype_code(dtype), float(seconds), s, ctypes.byref(out)), "turbofft_fma_peak")
    return out.value


def static_scratch_bytes() -> int:
    """Size of the library's static scratch array (turbofft_static_scratch_bytes)."""
    return int(ctypes.c_uint64.in_dll(lib(), "turbofft_static_scratch_bytes").value)


def __getattr__(name):
    # STATIC_SCRATCH_BYTES is read from the loaded library, not restated here
    if name == "STATIC_SCRATCH_BYTES":
        return static_scratch_bytes()
    raise AttributeError(name)


class TurboFFTError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        name = lib().turbofft_status_string(status).decode()
        super().__init__("%s: %s%s" % (what, name, (" (" + detail + ")") if detail else ""))
        self.status = status


def _check(status: int, what: str, plan=None):
    if status != SUCCESS:
        detail = lib().turbofft_last_error(plan).decode() if plan else ""
        raise TurboFFTError(status, what, detail)


def _dtype_code(dtype) -> int:
    import torch
    if dtype in ("complex64", "c64", "f32", torch.complex64, C2C_F32):
        return C2C_F32
    if dtype in ("complex128", "c128", "f64", torch.complex128, C2C_F64):
        return C2C_F64
    raise ValueError("dtype must be complex64 or complex128, got %r" % (dtype,))


class Plan:
    """A turbofft plan: batch transforms of length n (owns its device tables)."""

    def __init__(self, n: int, batch: int, dtype="complex64", direction="forward", ft="off",
                 structure="default"):
        """structure: "default" (chosen by the library), "split" (one pass or
        two four-step passes), "cluster" (one pass over thread-block
        clusters), "three_pass", or "float_pairs" (complex128, ft "off":
        the split passes in float-pair arithmetic instead of on the FP64
        pipe)."""
        self.n, self.batch = int(n), int(batch)
        self.dtype_code = _dtype_code(dtype)
        self.direction = _DIRS[direction]
        self.ft_mode = _FT[ft]
        h = ctypes.c_void_p()
        if structure == "default":
            _check(lib().turbofft_plan_create(self.n, self.batch, self.dtype_code, self.direction,
                                              self.ft_mode, ctypes.byref(h)), "turbofft_plan_create")
        else:
            _check(lib().turbofft_plan_create_structured(self.n, self.batch, self.dtype_code, self.direction,
                                                         self.ft_mode, _STRUCT[structure], ctypes.byref(h)),
                   "turbofft_plan_create_structured")
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def torch_dtype(self):
        import torch
        return torch.complex64 if self.dtype_code == C2C_F32 else torch.complex128

    def exec(self, x, out=None, stream=None):
        """y = transform(x) for a contiguous CUDA tensor x of shape [batch, n]."""
        import torch
        if not (x.is_cuda and x.dtype == self.torch_dtype and x.is_contiguous() and x.numel() == self.n * self.batch):
            raise ValueError("x must be a contiguous CUDA %s tensor with %d elements" % (self.torch_dtype, self.n * self.batch))
        if out is None:
            out = torch.empty_like(x)
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        _check(lib().turbofft_exec(self._h, x.data_ptr(), out.data_ptr(), stream.cuda_stream), "turbofft_exec", self._h)
        return out

    def exec_ptr(self, in_ptr: int, out_ptr: int, stream_ptr: int = 0) -> int:
        """Raw call through the C ABI; returns the status code."""
        return lib().turbofft_exec(self._h, in_ptr, out_ptr, stream_ptr)

    def exec_host(self, x_host, out_host=None, stream=None):
        """Transform CPU (ideally pinned) tensors: copies in, transforms, copies out."""
        import torch
        span = self.extent if isinstance(self, RaggedPlan) else self.n * self.batch
        if x_host.is_cuda or x_host.dtype != self.torch_dtype or not x_host.is_contiguous() or x_host.numel() < span:
            raise ValueError("x_host must be a contiguous CPU %s tensor of >= %d elements" % (self.torch_dtype, span))
        if out_host is None:
            out_host = torch.empty_like(x_host)
        if out_host.is_cuda or out_host.dtype != self.torch_dtype or not out_host.is_contiguous() or out_host.numel() < span:
            raise ValueError("out_host must be a contiguous CPU %s tensor of >= %d elements" % (self.torch_dtype, span))
        s = 0 if stream is None else stream.cuda_stream
        _check(lib().turbofft_exec_host(self._h, x_host.data_ptr(), out_host.data_ptr(), s), "turbofft_exec_host", self._h)
        return out_host

    def inject(self, transform: int, pass_: int, stage: int, element: int, component: int, bit: int):
        site = Site(int(transform), int(pass_), int(stage), int(element), int(component))
        _check(lib().turbofft_inject(self._h, site, int(bit)), "turbofft_inject")

    def report(self) -> dict:
        r = Report()
        st = lib().turbofft_get_report(self._h, ctypes.byref(r))
        if st not in (SUCCESS, FT_UNCORRECTABLE):
            _check(st, "turbofft_get_report", self._h)
        d = {name: getattr(r, name) for name, _ in Report._fields_ if name != "reserved"}
        d["status"] = st
        return d

    def info(self) -> dict:
        i = PlanInfo()
        _check(lib().turbofft_plan_get_info(self._h, ctypes.byref(i)), "turbofft_plan_get_info")
        return _info_dict(i)

    def set_workspace(self, buf):
        """Use the CUDA tensor `buf` (kept alive by the plan object) as the
        intermediate buffer of a two-pass plan."""
        self._workspace = buf
        _check(lib().turbofft_set_workspace(self._h, buf.data_ptr(), buf.numel() * buf.element_size()),
               "turbofft_set_workspace")

    def set_profiling(self, enable: bool = True):
        _check(lib().turbofft_set_profiling(self._h, 1 if enable else 0), "turbofft_set_profiling")

    def kernel_times(self) -> list:
        """[(pass, is_correction, ms)] of the last exec (profiling on)."""
        buf = (KernelTime * 8)()
        cnt = ctypes.c_int()
        _check(lib().turbofft_get_kernel_times(self._h, buf, 8, ctypes.byref(cnt)), "turbofft_get_kernel_times", self._h)
        return [(buf[i].pass_, buf[i].is_correction, buf[i].ms) for i in range(cnt.value)]

    def set_threshold_scale(self, factor: float):
        _check(lib().turbofft_set_threshold_scale(self._h, float(factor)), "turbofft_set_threshold_scale")

    def set_group_transactions(self, transactions: int):
        """Transactions per checksum group (default 4, range 1..16)."""
        _check(lib().turbofft_set_group_transactions(self._h, int(transactions)), "turbofft_set_group_transactions")

    def close(self):
        if getattr(self, "_h", None):
            lib().turbofft_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _info_dict(i: PlanInfo) -> dict:
    d = {}
    for name, _ in PlanInfo._fields_:
        v = getattr(i, name)
        d[name] = list(v) if hasattr(v, "__len__") else v
    return d


def set_autotune(enable: bool = True):
    """Process-wide: plans created afterwards time their candidate launch
    shapes and keep the fastest (turbofft_set_autotune)."""
    _check(lib().turbofft_set_autotune(1 if enable else 0), "turbofft_set_autotune")


def set_ragged_single_launch(enable: bool = True):
    """Process-wide: ragged plans created afterwards run as one launch of the
    persistent ragged kernel where they can (default), or as a graph of
    per-size kernels (turbofft_set_ragged_single_launch)."""
    _check(lib().turbofft_set_ragged_single_launch(1 if enable else 0), "turbofft_set_ragged_single_launch")


def set_tma_staging(mode="auto"):
    """Process-wide: how float32 one- and two-pass plans created afterwards
    stage their input tiles (turbofft_set_tma_staging): "auto" (TMA copies
    where they measured faster, else cp.async), "always" (TMA wherever the
    kernel's tile allows it) or "never" (16-byte cp.async copies)."""
    modes = {"never": 0, "auto": 1, "always": 2}
    _check(lib().turbofft_set_tma_staging(modes[mode]), "turbofft_set_tma_staging")


def packed_offsets(sizes, dtype="complex64"):
    """Offsets of transforms of the given sizes packed back to back in order
    (every size is a power of two >= 8, so each start stays 16-byte aligned);
    returns (offsets, total elements)."""
    offs, o = [], 0
    for n in sizes:
        offs.append(o)
        o += int(n)
    return offs, o


class RaggedPlan(Plan):
    """Transforms of mixed power-of-two sizes at given element offsets of one
    packed buffer, run as one CUDA graph (turbofft_plan_create_ragged)."""

    def __init__(self, sizes, offsets, dtype="complex64", direction="forward", ft="off"):
        sizes = [int(v) for v in sizes]
        offsets = [int(v) for v in offsets]
        if len(sizes) != len(offsets):
            raise ValueError("sizes and offsets differ in length")
        self.sizes, self.offsets = sizes, offsets
        self.n, self.batch = 0, len(sizes)
        self.extent = max((o + n for o, n in zip(offsets, sizes)), default=0)
        self.dtype_code = _dtype_code(dtype)
        self.direction = _DIRS[direction]
        self.ft_mode = _FT[ft]
        arr = ctypes.c_int64 * max(1, len(sizes))
        h = ctypes.c_void_p()
        _check(lib().turbofft_plan_create_ragged(arr(*sizes), arr(*offsets), len(sizes), self.dtype_code,
                                                 self.direction, self.ft_mode, ctypes.byref(h)),
               "turbofft_plan_create_ragged")
        self._h = h

    def exec(self, x, out=None, stream=None):
        """Transform the packed CUDA tensor x (1-D, at least `extent` elements)."""
        import torch
        if not (x.is_cuda and x.dtype == self.torch_dtype and x.is_contiguous() and x.numel() >= self.extent):
            raise ValueError("x must be a contiguous CUDA %s tensor with >= %d elements" % (self.torch_dtype, self.extent))
        if out is None:
            out = torch.empty_like(x)
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        _check(lib().turbofft_exec(self._h, x.data_ptr(), out.data_ptr(), stream.cuda_stream), "turbofft_exec", self._h)
        return out

    def member_info(self, index: int) -> dict:
        i = PlanInfo()
        _check(lib().turbofft_plan_get_member_info(self._h, int(index), ctypes.byref(i)),
               "turbofft_plan_get_member_info")
        return _info_dict(i)

    def members(self) -> list:
        return [self.member_info(k) for k in range(self.info()["num_members"])]


_plan_cache: dict = {}


def fft(x, inverse: bool = False, scaled: bool = True, ft="off"):
    """Batched 1-D FFT over the last dimension of a CUDA complex tensor."""
    n = x.shape[-1]
    batch = x.numel() // n
    direction = (INVERSE if scaled else INVERSE_UNSCALED) if inverse else FORWARD
    key = (n, batch, _dtype_code(x.dtype), direction, _FT[ft], x.device.index)
    plan = _plan_cache.get(key)
    if plan is None:
        plan = _plan_cache[key] = Plan(n, batch, x.dtype, direction, ft)
    xc = x.contiguous()
    return plan.exec(xc.view(batch, n)).view(x.shape)
