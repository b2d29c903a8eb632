// Kernel launches of an exec: per-pass arguments, the pass sequence with its
// correction kernels, the exec helpers shared by every entry point, and the
// host-buffer exec with its pipelined staging.
#include <cuda.h>
#include <cudaTypedefs.h>  // PFN_cuTensorMapEncodeTiled
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <complex>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "tf_cluster.cuh"
#include "tf_device.cuh"
#include "tf_internal.h"
#include "tf_plan.h"
#include "tf_ragged_kernel.h"

namespace tfh {

// kernel variant of an ft_mode: 0 none, 1 checksums, 2 checksums + register sums
int ft_variant(int ft_mode) {
  if (ft_mode == TURBOFFT_FT_OFF) return 0;
  if (ft_mode == TURBOFFT_FT_CORRECT_REGISTERS) return 2;
  if (ft_mode == TURBOFFT_FT_CORRECT_THREAD) return 3;
  return 1;
}

int kernel_dtype(const turbofft_plan* p) { return p->dtype == TURBOFFT_C2C_F32 ? 0 : (p->pairs ? 2 : 1); }
int plan_variant(const turbofft_plan* p) { return p->tchk ? 4 : ft_variant(p->ft_mode); }

// cluster kernels have no register-sums variant: that mode runs as CORRECT
int cl_variant(int ft_mode) { return ft_mode == TURBOFFT_FT_OFF ? 0 : 1; }

int occupancy_blocks(const KernelEntry* ke, int variant) {
  int nb = 0;
  const void* fn = ke->fn_main[variant];
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, ke->nt, ke->smem_main[variant]) != cudaSuccess) {
    cudaGetLastError();
    nb = 1;
  }
  return std::max(1, nb);
}

bool set_smem_attrs(const KernelEntry* ke) {
  // the attribute is per function; setting it again is harmless
  for (int v = 0; v < 5; ++v)
    if (ke->fn_main[v] && cudaFuncSetAttribute(ke->fn_main[v], cudaFuncAttributeMaxDynamicSharedMemorySize, ke->smem_main[v]) !=
        cudaSuccess)
      return false;
  if (ke->fn_fix &&
      cudaFuncSetAttribute(ke->fn_fix, cudaFuncAttributeMaxDynamicSharedMemorySize, ke->smem_fix) != cudaSuccess)
    return false;
  if (ke->fn_tcfix && cudaFuncSetAttribute(ke->fn_tcfix, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           ke->smem_main[0]) != cudaSuccess)
    return false;
  for (int v = 0; v < 2; ++v)
    if (ke->fn_main_tma[v] && cudaFuncSetAttribute(ke->fn_main_tma[v], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   ke->smem_tma[v]) != cudaSuccess)
      return false;
  return true;
}

std::atomic<int> g_tma_staging{1};

// TMA staging where it measured faster than cp.async on one GB300 (float32,
// 2^28 elements per call, forward, with and without checksums):
//  - row passes (one bulk copy of S adjacent rows): 1-4% faster at every
//    measured N1 x N2 (2^16 .. 2^21);
//  - column passes: tile rows of 64 bytes or more, at N1 >= 512 or with
//    checksums on (N1 = 128, 256 without checksums ran 2-5% slower; tile
//    rows of 16-32 bytes 1-24% slower);
//  - single passes: where it won by more than the run-to-run spread, N =
//    4096 (+9% / +5% without / with checksums), 1024 and 2048 with checksums
//    (+6%, +3%), 256 and 8192 without (+3%, +5%); the other cases ran 1-5%
//    slower and stay on cp.async.
bool tma_faster(const KernelEntry* ke, int ft_mode) {
  const bool ft = ft_mode != TURBOFFT_FT_OFF;
  if (ke->kind == tf::KIND_ROW) return true;
  if (ke->kind == tf::KIND_COL) return ke->s * 8 >= 64 && (ke->ns >= 512 || ft);
  return ke->ns == 4096 || (ft ? (ke->ns == 1024 || ke->ns == 2048) : (ke->ns == 256 || ke->ns == 8192));
}

namespace {
// the driver's tensor-map encoder, looked up once through the runtime
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}
}  // namespace

// Tensor map of a float32 two-pass plan's column-pass input `in` (batch
// transforms): the input viewed as rows of n2 complex values (8-byte
// elements), boxes of S columns x min(N1, 256) rows.  False where TMA cannot
// describe it (input not 16-byte aligned, 2^31 rows or more, no encoder):
// the exec then stages with cp.async.
bool encode_column_map(const turbofft_plan* p, const void* in, int64_t batch, CUtensorMap* m) {
  const PassPlan& pp = p->pass[0];
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || ((uintptr_t)in & 15u) != 0 || pp.kind != tf::KIND_COL) return false;
  const uint64_t n2 = (uint64_t)pp.g_n2;
  const uint64_t rows = (uint64_t)batch * (uint64_t)pp.bm * ((uint64_t)pp.g_n / n2);
  if (rows == 0 || rows >= (1ull << 31) || (n2 * 8) % 16 != 0) return false;
  const cuuint64_t dims[2] = {n2, rows};
  const cuuint64_t strides[1] = {n2 * 8};
  const cuuint32_t box[2] = {(cuuint32_t)pp.ke->s, (cuuint32_t)std::min(pp.ke->ns, 256)};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(in), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

long long units_for(const turbofft_plan* p, int pi, int64_t batch) {
  const PassPlan& pp = p->pass[pi];
  if (pp.kind == tf::KIND_SP) return (batch + pp.ke->s - 1) / pp.ke->s;
  if (pp.kind == tf::KIND_COL) return batch * pp.bm * (pp.g_n2 / pp.ke->s);
  return batch * pp.bm * (pp.g_n1 / pp.ke->s);
}

// sub-transforms ("signals") of pass pi per transform of the plan
int64_t signals_per_transform(const turbofft_plan* p, int pi) {
  const PassPlan& pp = p->pass[pi];
  if (pp.kind == tf::KIND_SP) return 1;
  return pp.bm * (pp.kind == tf::KIND_COL ? pp.g_n2 : pp.g_n1);
}

namespace {

// Transform-level check of float64 two-pass plans: one thread per transform
// compares e.y (row pass) with v.x (column pass) against
// tau = gamma u sqrt(log2 N) sqrt(N energy); a mismatch appends a record
// (unit_stride 0, signal = the transform) for the recompute kernels.
__global__ void tc_check_kernel(const double* tacc, long long batch, double tau_coef, double n, tf::FtState* fts,
                                int correct, long long tbase) {
  float mr = 0.f;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < batch;
       b += (long long)gridDim.x * blockDim.x) {
    const double* a = tacc + b * 6;
    const double rr = a[2] - a[0], ri = a[3] - a[1];
    const double tau = tau_coef * sqrt(n * a[4]);
    const double mag = sqrt(rr * rr + ri * ri);
    if (isfinite(mag) && isfinite(tau) && mag <= tau) {
      if (tau > 0) mr = fmaxf(mr, (float)(mag / tau));
      continue;
    }
    atomicAdd(&fts->detected, 1ull);
    if (!correct) atomicAdd(&fts->located, 1ull);
    const unsigned long long r = atomicAdd(&fts->num_records, 1ull);
    if (r < (unsigned long long)tf::MAX_RECORDS) {
      tf::FtRecord& R0 = fts->rec[r];
      R0.pass_id = 1;
      R0.slot = 0;
      R0.count = 1;
      R0.located = 0;
      R0.unit0 = b;
      R0.unit_stride = 0;
      R0.transform_base = tbase;
      R0.s1r = rr; R0.s1i = ri; R0.s2r = rr; R0.s2i = ri;
      R0.tau = tau;
      R0.energy = a[4];
      R0.result = correct ? tf::FT_RES_PENDING : tf::FT_RES_LOCATED;
      R0.has_sums = 0;
      R0.signal = b;
    } else {
      atomicAdd(&fts->dropped, 1ull);
    }
  }
  const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(mr));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(reinterpret_cast<int*>(&fts->max_clean_ratio), (int)m);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&fts->groups, (unsigned long long)batch);
}

template <typename R>
void fill_args(const turbofft_plan* p, int pi, const void* in, void* out, int64_t batch, int64_t tbase,
               const tf::InjectSite& inj, tf::PassArgs<R>& A) {
  typedef typename tf::CT<R>::c c;
  const PassPlan& pp = p->pass[pi];
  memset(&A, 0, sizeof(A));
  A.in = static_cast<const c*>(in);
  A.out = static_cast<c*>(out);
  A.tw = static_cast<const c*>(pp.d_tw);
  A.ev = static_cast<const c*>(pp.d_ev);
  A.vv = static_cast<const c*>(pp.d_vv);
  A.ev4 = static_cast<const float4*>(pp.d_ev4);
  A.vv4 = static_cast<const float4*>(pp.d_vv4);
  A.tlo = static_cast<const c*>(pp.d_tlo ? pp.d_tlo : p->d_tlo);
  A.thi = static_cast<const c*>(pp.d_thi ? pp.d_thi : p->d_thi);
  A.colw = static_cast<const c*>(pp.d_colw);
  A.colwe = static_cast<const c*>(pp.d_colwe);
  A.geo.n = pp.g_n;
  A.geo.n1 = pp.g_n1;
  A.geo.n2 = pp.g_n2;
  A.geo.batch = batch * pp.bm;
  A.geo.in_tab = (pi == 0) ? p->d_tab : nullptr;
  A.geo.out_tab = (pi == p->num_passes - 1) ? p->d_tab : nullptr;
  A.geo.outer = pp.outer;
  A.geo.n_outer = p->n;
  A.geo.l2n1 = ilog2_exact(pp.g_n1);
  A.geo.l2n2 = ilog2_exact(pp.g_n2);
  A.geo.l2outer = pp.outer > 1 ? ilog2_exact(pp.outer) : 0;
  A.num_units = p->cl ? batch : units_for(p, pi, batch);  // cluster plans: one unit per transform
  const bool inverse = p->direction > 0;
  const bool scaled = p->direction == TURBOFFT_INVERSE || p->direction == TURBOFFT_FORWARD_SCALED;
  const bool last = (pi == p->num_passes - 1);
  A.conj_in = (inverse && pi == 0) ? 1 : 0;
  A.conj_out = (inverse && last) ? 1 : 0;
  A.out_scale = (last && scaled) ? (R)(1.0 / (double)p->n) : (R)1;
  A.tau_coef = pp.tau_coef * p->threshold_scale;
  A.ft = (p->ft_mode == TURBOFFT_FT_CORRECT_REGISTERS || p->ft_mode == TURBOFFT_FT_CORRECT_THREAD)
             ? TURBOFFT_FT_CORRECT
             : p->ft_mode;
  A.T = p->T;
  A.pass_id = pi;
  A.transform_base = tbase;
  A.fts = p->d_fts;
  A.tacc = p->d_tacc;
  A.vcol = static_cast<const c*>(p->d_vcol);
  A.erow = static_cast<const c*>(p->d_erow);
  A.geo.col_tfast = p->tchk ? 0 : 1;
  A.rec_sums = p->d_rec_sums;
  A.rec_stride = p->rec_stride;
  A.inj = inj;
  A.err = p->d_err;
}

}  // namespace

void fill_pass_args_f32(const turbofft_plan* p, int pi, const void* in, void* out, const tf::InjectSite& inj,
                        tf::PassArgs<float>* A) {
  fill_args<float>(p, pi, in, out, p->batch, 0, inj, *A);
}

namespace {

template <typename R>
void fill_cl_args(const turbofft_plan* p, const void* in, void* out, int64_t batch, int64_t tbase,
                  const tf::InjectSite& inj, tf::ClArgs<R>& A) {
  typedef typename tf::CT<R>::c c;
  fill_args<R>(p, 0, in, out, batch, tbase, inj, A.p);
  const bool inverse = p->direction > 0;
  const bool scaled = p->direction == TURBOFFT_INVERSE || p->direction == TURBOFFT_FORWARD_SCALED;
  A.p.geo.out_tab = p->d_tab;
  A.p.conj_out = inverse ? 1 : 0;
  A.p.out_scale = scaled ? (R)(1.0 / (double)p->n) : (R)1;
  A.p.num_units = batch;
  A.twB = static_cast<const c*>(p->pass[1].d_tw);
  A.evB = static_cast<const c*>(p->pass[1].d_ev);
  A.vvB = static_cast<const c*>(p->pass[1].d_vv);
}

// Device staging of turbofft_exec_host, shared by all plans of a device:
// two input and two output chunk buffers (about 128 MiB each: enough
// transforms per chunk to fill the GPU even at large N) plus a chunk-sized
// intermediate,
// three streams (copy in, transform, copy out) and their events.  Grown on
// demand, kept until the process exits; one exec_host runs at a time per
// device (the call is synchronous).
struct HostStage {
  std::mutex mu;
  size_t chunk_bytes = 0;
  void* in[2] = {nullptr, nullptr};
  void* out[2] = {nullptr, nullptr};
  void* scratch = nullptr;
  cudaStream_t st[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev[8] = {};
  bool ready = false;
};
HostStage g_stage[16];
const size_t kStageChunkBytes = (size_t)128 << 20;

cudaError_t stage_reserve(HostStage& hs, size_t need) {
  cudaError_t e;
  if (!hs.ready) {
    for (auto& s : hs.st)
      if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    for (auto& v : hs.ev)
      if ((e = cudaEventCreateWithFlags(&v, cudaEventDisableTiming)) != cudaSuccess) return e;
    hs.ready = true;
  }
  if (need <= hs.chunk_bytes) return cudaSuccess;
  for (void** b : {&hs.in[0], &hs.in[1], &hs.out[0], &hs.out[1], &hs.scratch}) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  hs.chunk_bytes = 0;
  for (void** b : {&hs.in[0], &hs.in[1], &hs.out[0], &hs.out[1], &hs.scratch})
    if ((e = cudaMalloc(b, need)) != cudaSuccess) return e;
  hs.chunk_bytes = need;
  return cudaSuccess;
}

}  // namespace


turbofft_status run(turbofft_plan* p, const void* in, void* out, void* scratch, int64_t batch, int64_t tbase,
                    cudaStream_t stream, const tf::InjectSite& inj) {
  const bool ft = p->ft_mode != TURBOFFT_FT_OFF;
  // CUDA events around each kernel when profiling (kind = 2 * pass + is_correction)
  auto timed = [&](int kind, auto&& launch) {
    const bool prof = p->profiling && p->nprof < 8;
    if (prof) cudaEventRecord(p->prof_ev[p->nprof][0], stream);
    launch();
    if (prof) {
      cudaEventRecord(p->prof_ev[p->nprof][1], stream);
      p->prof_kind[p->nprof++] = kind;
    }
  };
  if (p->cl) {
    const ClEntry* ce = p->cl;
    const int grid = (int)std::min<long long>((long long)p->cl_grid, (long long)batch * ce->cluster);
    if (p->dtype == TURBOFFT_C2C_F32) {
      tf::ClArgs<float> A;
      fill_cl_args<float>(p, in, out, batch, tbase, inj, A);
      timed(0, [&] { ce->main[cl_variant(p->ft_mode)](&A, grid, stream); });
      if (ft) timed(1, [&] { ce->fix(&A, ce->cluster, stream); });
    } else {
      tf::ClArgs<double> A;
      fill_cl_args<double>(p, in, out, batch, tbase, inj, A);
      timed(0, [&] { ce->main[cl_variant(p->ft_mode)](&A, grid, stream); });
      if (ft) timed(1, [&] { ce->fix(&A, ce->cluster, stream); });
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(p, e, "kernel launch");
    return TURBOFFT_SUCCESS;
  }
  for (int pi = 0; pi < p->num_passes; ++pi) {
    const PassPlan& pp = p->pass[pi];
    // two passes: in -> scratch -> out; three: in -> out -> scratch -> out
    const void* pin = (pi == 0) ? in : (p->num_passes == 3 && pi == 1 ? out : scratch);
    void* pout = (pi == p->num_passes - 1 || (p->num_passes == 3 && pi == 0)) ? out : scratch;
    long long units = units_for(p, pi, batch);
    int grid = (int)std::min<long long>(units, pp.grid);
    if (grid < 1) grid = 1;
    if (p->dtype == TURBOFFT_C2C_F32) {
      tf::PassArgs<float> A;
      fill_args<float>(p, pi, pin, pout, batch, tbase, inj, A);
      const int v = ft_variant(p->ft_mode);
      // tiles staged by TMA where the plan chose it and the exec's input
      // allows it (a column pass: a tensor map of the input; others copy
      // contiguous tiles and ignore the map)
      CUtensorMap tm;
      memset(&tm, 0, sizeof(tm));
      const bool tma = ((p->tma_mask >> pi) & 1) && p->num_passes <= 2 && p->d_tab == nullptr && v <= 1 &&
                       pp.ke->main_tma[v] && (pp.kind != tf::KIND_COL || encode_column_map(p, pin, batch, &tm));
      timed(2 * pi, [&] {
        if (tma)
          pp.ke->main_tma[v](&A, &tm, grid, stream);
        else
          pp.ke->main[v](&A, grid, stream);
      });
      if (ft) timed(2 * pi + 1, [&] { pp.ke->fix(&A, 8, stream); });
    } else if (p->pairs) {
      tf::PassArgs<tf::dd> A;  // no checksums: no correction kernel
      fill_args<tf::dd>(p, pi, pin, pout, batch, tbase, inj, A);
      timed(2 * pi, [&] { pp.ke->main[0](&A, grid, stream); });
    } else {
      tf::PassArgs<double> A;
      fill_args<double>(p, pi, pin, pout, batch, tbase, inj, A);
      timed(2 * pi, [&] { pp.ke->main[plan_variant(p)](&A, grid, stream); });
      if (ft && !p->tchk) timed(2 * pi + 1, [&] { pp.ke->fix(&A, 8, stream); });
      if (p->tchk && pi == p->num_passes - 1) {
        // compare the whole transforms' sums, then recompute the recorded
        // transforms: column pass, then row pass
        const double tau = kGamma[1] * kUnitRoundoff[1] * sqrt((double)ilog2_exact(p->n)) * p->threshold_scale;
        const int cgrid = (int)std::min<long long>((batch + 255) / 256, 1024);
        timed(2 * pi + 1, [&] {
          tc_check_kernel<<<cgrid, 256, 0, stream>>>(p->d_tacc, batch, tau, (double)p->n, p->d_fts,
                                                      p->ft_mode == TURBOFFT_FT_DETECT ? 0 : 1, tbase);
          tf::PassArgs<double> A0;
          fill_args<double>(p, 0, in, scratch, batch, tbase, inj, A0);
          p->pass[0].ke->tcfix(&A0, p->pass[0].grid, stream);
          pp.ke->tcfix(&A, pp.grid, stream);
        });
      }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(p, e, "kernel launch");
  }
  return TURBOFFT_SUCCESS;
}

bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

// queue one complete exec of a (member) plan on `s`: report reset, kernels,
// report copy to the pinned host mirror
turbofft_status queue_plan(turbofft_plan* p, const void* in, void* out, void* scratch, cudaStream_t s,
                           const tf::InjectSite& inj) {
  const bool ft = p->ft_mode != TURBOFFT_FT_OFF;
  if (ft) {
    cudaError_t e = cudaMemsetAsync(p->d_fts, 0, tf::FT_HEADER_BYTES, s);
    if (e == cudaSuccess && p->tchk) e = cudaMemsetAsync(p->d_tacc, 0, (size_t)p->batch * 6 * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(p, e, "report reset");
  }
  turbofft_status st = run(p, in, out, scratch, p->batch, 0, s, inj);
  if (st != TURBOFFT_SUCCESS) return st;
  if (ft) {
    cudaError_t e = cudaMemcpyAsync(p->h_fts, p->d_fts, sizeof(FtState), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(p, e, "report copy");
  }
  return TURBOFFT_SUCCESS;
}

// the buffers a (non-ragged) exec may use: 16-byte aligned, not overlapping
turbofft_status check_io(const turbofft_plan* p, const void* in, void* out) {
  if (!in || !out) return TURBOFFT_INVALID_VALUE;
  if (!aligned16(in) || !aligned16(out)) return TURBOFFT_INVALID_VALUE;
  const size_t bytes = (size_t)(p->ragged ? p->extent : p->batch * p->n) * elem_bytes(p->dtype);
  const char* a = static_cast<const char*>(in);
  const char* b = static_cast<const char*>(out);
  if (a < b + bytes && b < a + bytes) return TURBOFFT_UNSUPPORTED;
  return TURBOFFT_SUCCESS;
}

// one exec of a plan on `s` with the armed site (then disarmed); the plan's
// `done` event marks its end for turbofft_get_report
turbofft_status exec_on_stream(turbofft_plan* p, const void* in, void* out, void* scratch, cudaStream_t s) {
  const tf::InjectSite inj = p->armed;
  p->armed.active = 0;
  p->nprof = 0;
  turbofft_status st = queue_plan(p, in, out, scratch, s, inj);
  if (st != TURBOFFT_SUCCESS) return st;
  cudaError_t e = cudaEventRecord(p->done, s);
  if (e != cudaSuccess) return cuda_fail(p, e, "event record");
  p->have_exec = true;
  return TURBOFFT_SUCCESS;
}

}  // namespace tfh

using namespace tfh;

extern "C" {

turbofft_status turbofft_exec(turbofft_plan* p, const void* in, void* out, turbofft_stream stream) {
  if (!p) return TURBOFFT_INVALID_VALUE;
  turbofft_status st = check_io(p, in, out);
  if (st != TURBOFFT_SUCCESS) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (p->ragged) return exec_ragged(p, in, out, s);
  if (p->scratch_bytes > 0 && !p->d_scratch) {
    if (!dev_alloc(p, &p->d_scratch, p->scratch_bytes)) return TURBOFFT_ALLOC_FAILED;
    p->scratch_owned = true;
  }
  return exec_on_stream(p, in, out, p->d_scratch, s);
}

turbofft_status turbofft_exec_host(turbofft_plan* p, const void* host_in, void* host_out, turbofft_stream stream) {
  if (!p || !host_in || !host_out) return TURBOFFT_INVALID_VALUE;
  if (p->device < 0 || p->device >= 16) return TURBOFFT_UNSUPPORTED;
  const size_t eb = elem_bytes(p->dtype);
  if (p->ragged) {
    // one copy in, the graph, one copy out, ordered on `stream`
    HostStage& hs = g_stage[p->device];
    std::lock_guard<std::mutex> lock(hs.mu);
    const size_t bytes = (size_t)p->extent * eb;
    cudaError_t e = stage_reserve(hs, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(p, e, "exec_host staging");
    }
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    if ((e = cudaMemcpyAsync(hs.in[0], host_in, bytes, cudaMemcpyHostToDevice, user)) != cudaSuccess)
      return cuda_fail(p, e, "h2d");
    turbofft_status st = exec_ragged(p, hs.in[0], hs.out[0], user);
    if (st != TURBOFFT_SUCCESS) return st;
    if ((e = cudaMemcpyAsync(host_out, hs.out[0], bytes, cudaMemcpyDeviceToHost, user)) != cudaSuccess)
      return cuda_fail(p, e, "d2h");
    if ((e = cudaEventRecord(p->done, user)) != cudaSuccess) return cuda_fail(p, e, "event record");
    if ((e = cudaEventSynchronize(p->done)) != cudaSuccess) return cuda_fail(p, e, "exec_host");
    return TURBOFFT_SUCCESS;
  }
  const size_t per = (size_t)p->n * eb;
  // chunk: whole transforms, about 64 MiB (at least one transform)
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(p->batch, (int64_t)(kStageChunkBytes / per)));
  HostStage& hs = g_stage[p->device];
  std::lock_guard<std::mutex> lock(hs.mu);
  cudaError_t e = stage_reserve(hs, (size_t)chunk * per);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(p, e, "exec_host staging");
  }
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  cudaStream_t sh = hs.st[0], sc = hs.st[1], sd = hs.st[2];
  cudaEvent_t* ev = hs.ev;  // 0..1 h2d done, 2..3 transform done, 4..5 d2h done, 6 start, 7 report
  if ((e = cudaEventRecord(ev[6], user)) != cudaSuccess) return cuda_fail(p, e, "event record");
  cudaStreamWaitEvent(sh, ev[6], 0);
  cudaStreamWaitEvent(sc, ev[6], 0);
  cudaStreamWaitEvent(sd, ev[6], 0);
  const bool ft = p->ft_mode != TURBOFFT_FT_OFF;
  if (ft && (e = cudaMemsetAsync(p->d_fts, 0, tf::FT_HEADER_BYTES, sc)) != cudaSuccess)
    return cuda_fail(p, e, "report reset");
  tf::InjectSite inj = p->armed;
  p->armed.active = 0;
  p->nprof = 0;
  const char* hin = static_cast<const char*>(host_in);
  char* hout = static_cast<char*>(host_out);
  int ci = 0;
  for (int64_t b0 = 0; b0 < p->batch; b0 += chunk, ++ci) {
    const int sl = ci & 1;
    const int64_t nb = std::min<int64_t>(chunk, p->batch - b0);
    const size_t off = (size_t)b0 * per, bytes = (size_t)nb * per;
    if (ci >= 2) cudaStreamWaitEvent(sh, ev[2 + sl], 0);  // stage-in slot consumed
    if ((e = cudaMemcpyAsync(hs.in[sl], hin + off, bytes, cudaMemcpyHostToDevice, sh)) != cudaSuccess)
      return cuda_fail(p, e, "h2d");
    cudaEventRecord(ev[sl], sh);
    cudaStreamWaitEvent(sc, ev[sl], 0);
    if (ci >= 2) cudaStreamWaitEvent(sc, ev[4 + sl], 0);  // stage-out slot drained
    tf::InjectSite cinj = inj;
    if (inj.active) {
      // the armed transform belongs to exactly one chunk
      const int64_t per_tr = signals_per_transform(p, inj.pass);
      const int64_t tr = inj.signal / per_tr;
      if (tr >= b0 && tr < b0 + nb) cinj.signal = inj.signal - b0 * per_tr;
      else cinj.active = 0;
    }
    // whole-transform sums start at zero for every chunk (its transforms
    // are indexed from 0)
    if (p->tchk && (e = cudaMemsetAsync(p->d_tacc, 0, (size_t)nb * 6 * sizeof(double), sc)) != cudaSuccess)
      return cuda_fail(p, e, "report reset");
    turbofft_status st = run(p, hs.in[sl], hs.out[sl], hs.scratch, nb, b0, sc, cinj);
    if (st != TURBOFFT_SUCCESS) return st;
    cudaEventRecord(ev[2 + sl], sc);
    cudaStreamWaitEvent(sd, ev[2 + sl], 0);
    if ((e = cudaMemcpyAsync(hout + off, hs.out[sl], bytes, cudaMemcpyDeviceToHost, sd)) != cudaSuccess)
      return cuda_fail(p, e, "d2h");
    cudaEventRecord(ev[4 + sl], sd);
  }
  if (ft) {
    cudaStreamWaitEvent(sc, ev[4 + ((ci - 1) & 1)], 0);
    if ((e = cudaMemcpyAsync(p->h_fts, p->d_fts, sizeof(FtState), cudaMemcpyDeviceToHost, sc)) != cudaSuccess)
      return cuda_fail(p, e, "report copy");
    cudaEventRecord(ev[7], sc);
    cudaStreamWaitEvent(sd, ev[7], 0);
  }
  cudaEventRecord(p->done, sd);
  cudaStreamWaitEvent(user, p->done, 0);
  p->have_exec = true;
  if ((e = cudaEventSynchronize(p->done)) != cudaSuccess) return cuda_fail(p, e, "exec_host");
  return TURBOFFT_SUCCESS;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// library-internal helpers (tf_internal.h)
// ---------------------------------------------------------------------------
namespace tf {

size_t plan_scratch_bytes(const turbofft_plan* p) { return p->ragged ? 0 : p->scratch_bytes; }

int plan_device(const turbofft_plan* p) { return p->device; }

void plan_set_error(turbofft_plan* p, const char* msg) { p->last_error = msg; }

turbofft_status exec_given_scratch(turbofft_plan* p, const void* in, void* out, void* scratch, cudaStream_t s) {
  if (!p) return TURBOFFT_INVALID_VALUE;
  if (p->ragged) return TURBOFFT_UNSUPPORTED;
  if (p->scratch_bytes > 0 && (!scratch || !aligned16(scratch))) return TURBOFFT_INVALID_VALUE;
  turbofft_status st = check_io(p, in, out);
  if (st != TURBOFFT_SUCCESS) return st;
  return exec_on_stream(p, in, out, scratch, s);
}

}  // namespace tf
