// Host side of the C ABI declared in include/turbofft.h: plan creation (tables,
// pass split, launch shapes), exec, injection, report.
//
// Tables (TurboFFT Sec. 5.1.2: twiddles precomputed instead of evaluating
// trigonometric functions on the device; Sec. 4.2.2: the left encoding
// vector e^T W precomputed outside the transform) are evaluated on the host
// in long double and rounded once to the plan's precision.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <complex>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/turbofft.h"
#include "tf_cluster.cuh"
#include "tf_device.cuh"
#include "tf_internal.h"
#include "tf_registry.h"

using tf::FtRecord;
using tf::FtState;
using tf::ClEntry;
using tf::KernelEntry;

namespace {

// ---------------------------------------------------------------------------
// kernel registry
// ---------------------------------------------------------------------------
struct Registry {
  std::vector<const KernelEntry*> all;
  std::vector<const ClEntry*> cl;
  Registry() {
    tf::ClTableFn cfns[] = {tf::entries_f32_cl};
    for (auto fn : cfns) {
      int n = 0;
      const ClEntry* t = fn(&n);
      for (int i = 0; i < n; ++i) cl.push_back(&t[i]);
    }
    tf::EntryTableFn fns[] = {tf::entries_f32_sp, tf::entries_f32_col, tf::entries_f32_row,
                              tf::entries_f64_sp, tf::entries_f64_col, tf::entries_f64_row,
                              tf::entries_f32_alt_sp, tf::entries_f32_alt_cr, tf::entries_f64_alt};
    for (auto fn : fns) {
      int n = 0;
      const KernelEntry* t = fn(&n);
      for (int i = 0; i < n; ++i) all.push_back(&t[i]);
    }
  }
  // the first registered entry is the default shape; later ones are
  // alternatives the autotuner may pick
  const KernelEntry* find(int dtype, int kind, int ns) const {
    for (auto e : all)
      if (e->dtype == dtype && e->kind == kind && e->ns == ns) return e;
    return nullptr;
  }
  std::vector<const KernelEntry*> find_all(int dtype, int kind, int ns) const {
    std::vector<const KernelEntry*> v;
    for (auto e : all)
      if (e->dtype == dtype && e->kind == kind && e->ns == ns) v.push_back(e);
    return v;
  }
  const ClEntry* find_cl(int dtype, int64_t n) const {
    for (auto e : cl)
      if (e->dtype == dtype && e->n == n) return e;
    return nullptr;
  }
  int max_sp(int dtype) const {
    int m = 0;
    for (auto e : all)
      if (e->dtype == dtype && e->kind == tf::KIND_SP) m = std::max(m, e->ns);
    return m;
  }
};
const Registry& registry() {
  static Registry r;
  return r;
}

// ---------------------------------------------------------------------------
// host tables (long double)
// ---------------------------------------------------------------------------
typedef long double ld;
typedef std::complex<ld> cld;
const ld kTwoPi = 6.283185307179586476925286766559005768394338798750L;

// w_n^q = exp(-2 pi i q / n), phase reduced exactly in integers
cld root(int64_t n, int64_t q) {
  q %= n;
  if (q < 0) q += n;
  ld ang = -kTwoPi * (ld)q / (ld)n;
  return cld(cosl(ang), sinl(ang));
}

// forward DFT of a (length power of two), recursive radix-2, long double
void host_fft(std::vector<cld>& a) {
  const size_t n = a.size();
  if (n <= 1) return;
  std::vector<cld> ev(n / 2), od(n / 2);
  for (size_t k = 0; k < n / 2; ++k) { ev[k] = a[2 * k]; od[k] = a[2 * k + 1]; }
  host_fft(ev);
  host_fft(od);
  for (size_t k = 0; k < n / 2; ++k) {
    cld t = root((int64_t)n, (int64_t)k) * od[k];
    a[k] = ev[k] + t;
    a[k + n / 2] = ev[k] - t;
  }
}

// SplitMix64 (Steele, Lea, Flood 2014): phase of the checksum vector
uint64_t splitmix_mix(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// output-side encoding vector e: unit-modulus, seeded random phases
std::vector<cld> encoding_vector(int ns) {
  std::vector<cld> e(ns);
  const uint64_t seed = 0x5EEDull;
  for (int j = 0; j < ns; ++j) {
    uint64_t w = splitmix_mix(seed + (uint64_t)(j + 1) * 0x9E3779B97F4A7C15ull);
    ld theta = (ld)(w >> 11) * 0x1p-53L;
    e[j] = cld(cosl(kTwoPi * theta), sinl(kTwoPi * theta));
  }
  return e;
}

template <typename R> struct DevC;
template <> struct DevC<float> { typedef float2 t; };
template <> struct DevC<double> { typedef double2 t; };

template <typename R> std::vector<typename DevC<R>::t> round_table(const std::vector<cld>& v) {
  std::vector<typename DevC<R>::t> out(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    out[i].x = (R)v[i].real();
    out[i].y = (R)v[i].imag();
  }
  return out;
}

int ilog2_exact(int64_t n) {
  int l = 0;
  while (((int64_t)1 << l) < n) ++l;
  return (((int64_t)1 << l) == n) ? l : -1;
}

// default threshold factor gamma per working precision: chosen from clean-run
// residuals so that the largest clean |S1| stays far below tau
const double kGamma[2] = {8.0, 16.0};

// float32 sizes from 2^this use three passes by default
const int kThreePassLog2F32 = 22;
const double kUnitRoundoff[2] = {0x1p-24, 0x1p-53};

int g_num_sms = 0;

}  // namespace

// ---------------------------------------------------------------------------
// the plan
// ---------------------------------------------------------------------------
struct PassPlan {
  const KernelEntry* ke = nullptr;
  int kind = 0;
  int ns = 0;
  int grid = 0;
  // geometry the pass works on: sub-transforms of length g_n = g_n1 * g_n2,
  // bm of them per transform of the plan (three-pass plans: N1 for the
  // second and third passes); outer = N1 for the third pass's output mapping
  long long g_n = 0;
  int g_n1 = 0, g_n2 = 1;
  long long bm = 1;
  int outer = 0;
  void* d_tlo = nullptr;  // inter-pass twiddles of a column pass over length g_n
  void* d_thi = nullptr;
  void* d_tw = nullptr;
  void* d_ev = nullptr;
  void* d_vv = nullptr;
  void* d_ev4 = nullptr;  // float32: (re, re, im, im) arrangement for paired FMAs
  void* d_vv4 = nullptr;
  double tau_coef = 0;
};

struct turbofft_plan {
  int64_t n = 0, batch = 0;
  int dtype = 0, direction = -1, ft_mode = 0;
  int device = 0;
  int num_passes = 1;
  int n1 = 0, n2 = 1;
  PassPlan pass[3];
  void* d_tlo = nullptr;
  void* d_thi = nullptr;
  void* d_scratch = nullptr;      // intermediate of two-pass plans (owned or caller's)
  size_t scratch_bytes = 0;       // bytes a two-pass exec needs
  bool scratch_owned = false;
  FtState* d_fts = nullptr;
  FtState* h_fts = nullptr;
  void* d_rec_sums = nullptr;
  int rec_stride = 0;
  tf::InjectSite armed{};
  double threshold_scale = 1.0;
  int T = 4;
  cudaEvent_t done = nullptr;
  bool have_exec = false;
  std::string last_error;
  int64_t workspace_bytes = 0;
  std::vector<void*> allocs;
  // per-kernel timing (turbofft_set_profiling)
  bool profiling = false;
  int nprof = 0;
  cudaEvent_t prof_ev[8][2] = {};
  int prof_kind[8] = {};
  // member of a ragged plan: element offsets of its transforms in the
  // caller's packed buffers (device), null for the contiguous layout
  long long* d_tab = nullptr;
  // ragged plan: one member plan per distinct size, run as the parallel
  // branches of one CUDA graph
  bool ragged = false;
  std::vector<turbofft_plan*> members;
  std::vector<std::vector<int64_t>> member_ids;  // global transform index of each member transform
  int64_t extent = 0;                             // elements spanned by the packed buffers
  std::vector<cudaStream_t> branch_streams;
  std::vector<cudaEvent_t> branch_events;
  cudaGraphExec_t graph_exec = nullptr;
  const void* graph_in = nullptr;
  void* graph_out = nullptr;
  bool armed_any = false;
  std::vector<int32_t> member_of;  // ragged: member plan of each global transform
  std::vector<int64_t> local_of;   // ragged: index of each global transform within its member
  bool autotuned = false;          // launch shapes chosen by timing (turbofft_set_autotune)
  // single-pass cluster plan: both four-step phases in one kernel
  const ClEntry* cl = nullptr;
  int cl_grid = 0;
};

namespace {

size_t elem_bytes(int dtype) { return dtype == TURBOFFT_C2C_F32 ? 8 : 16; }

turbofft_status cuda_fail(turbofft_plan* p, cudaError_t e, const char* what) {
  if (p) {
    p->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  }
  return TURBOFFT_CUDA_ERROR;
}

bool dev_alloc(turbofft_plan* p, void** ptr, size_t bytes) {
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return false;
  }
  p->allocs.push_back(*ptr);
  p->workspace_bytes += (int64_t)bytes;
  return true;
}

template <typename R>
bool upload(turbofft_plan* p, void** dst, const std::vector<cld>& v) {
  auto t = round_table<R>(v);
  size_t bytes = t.size() * sizeof(t[0]);
  if (!dev_alloc(p, dst, bytes)) return false;
  return cudaMemcpy(*dst, t.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
}

bool upload_tables(turbofft_plan* p, PassPlan& pp) {
  const int ns = pp.ns;
  std::vector<cld> tw(ns);
  for (int q = 0; q < ns; ++q) tw[q] = root(ns, q);
  std::vector<cld> e = encoding_vector(ns);
  std::vector<cld> v = e;
  host_fft(v);  // v = W e = (e^T W)^T, W symmetric (Eq. 1)
  if (p->dtype == TURBOFFT_C2C_F32) {
    bool ok = upload<float>(p, &pp.d_tw, tw) && upload<float>(p, &pp.d_ev, e) && upload<float>(p, &pp.d_vv, v);
#ifdef TF_PAIRED_CHECKSUMS
    // weights arranged as (re, re, im, im) for the paired-FMA checksum build
    auto arranged = [&](void** dst, const std::vector<cld>& src) {
      std::vector<float4> t4(src.size());
      for (size_t i = 0; i < src.size(); ++i) {
        const float re = (float)src[i].real(), im = (float)src[i].imag();
        t4[i] = make_float4(re, re, im, im);
      }
      const size_t bytes = t4.size() * sizeof(float4);
      return dev_alloc(p, dst, bytes) && cudaMemcpy(*dst, t4.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    ok = ok && arranged(&pp.d_ev4, e) && arranged(&pp.d_vv4, v);
#endif
    return ok;
  }
  return upload<double>(p, &pp.d_tw, tw) && upload<double>(p, &pp.d_ev, e) && upload<double>(p, &pp.d_vv, v);
}

// kernel variant of an ft_mode: 0 none, 1 checksums, 2 checksums + register sums
int ft_variant(int ft_mode) { return ft_mode == TURBOFFT_FT_OFF ? 0 : (ft_mode == TURBOFFT_FT_CORRECT_REGISTERS ? 2 : 1); }

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
  for (int v = 0; v < 3; ++v)
    if (cudaFuncSetAttribute(ke->fn_main[v], cudaFuncAttributeMaxDynamicSharedMemorySize, ke->smem_main[v]) !=
        cudaSuccess)
      return false;
  if (cudaFuncSetAttribute(ke->fn_fix, cudaFuncAttributeMaxDynamicSharedMemorySize, ke->smem_fix) != cudaSuccess)
    return false;
  return true;
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
  A.geo.n = pp.g_n;
  A.geo.n1 = pp.g_n1;
  A.geo.n2 = pp.g_n2;
  A.geo.batch = batch * pp.bm;
  A.geo.in_tab = (pi == 0) ? p->d_tab : nullptr;
  A.geo.out_tab = (pi == p->num_passes - 1) ? p->d_tab : nullptr;
  A.geo.outer = pp.outer;
  A.geo.n_outer = p->n;
  A.num_units = p->cl ? batch : units_for(p, pi, batch);  // cluster plans: one unit per transform
  const bool inverse = p->direction > 0;
  const bool scaled = p->direction == TURBOFFT_INVERSE || p->direction == TURBOFFT_FORWARD_SCALED;
  const bool last = (pi == p->num_passes - 1);
  A.conj_in = (inverse && pi == 0) ? 1 : 0;
  A.conj_out = (inverse && last) ? 1 : 0;
  A.out_scale = (last && scaled) ? (R)(1.0 / (double)p->n) : (R)1;
  A.tau_coef = pp.tau_coef * p->threshold_scale;
  A.ft = p->ft_mode == TURBOFFT_FT_CORRECT_REGISTERS ? TURBOFFT_FT_CORRECT : p->ft_mode;
  A.T = p->T;
  A.pass_id = pi;
  A.transform_base = tbase;
  A.fts = p->d_fts;
  A.rec_sums = p->d_rec_sums;
  A.rec_stride = p->rec_stride;
  A.inj = inj;
}

// queue one transform of `batch` transforms (device pointers) on `stream`
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

// cluster kernels have no register-sums variant: that mode runs as CORRECT
int cl_variant(int ft_mode) { return ft_mode == TURBOFFT_FT_OFF ? 0 : 1; }

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
      timed(2 * pi, [&] { pp.ke->main[ft_variant(p->ft_mode)](&A, grid, stream); });
      if (ft) timed(2 * pi + 1, [&] { pp.ke->fix(&A, 8, stream); });
    } else {
      tf::PassArgs<double> A;
      fill_args<double>(p, pi, pin, pout, batch, tbase, inj, A);
      timed(2 * pi, [&] { pp.ke->main[ft_variant(p->ft_mode)](&A, grid, stream); });
      if (ft) timed(2 * pi + 1, [&] { pp.ke->fix(&A, 8, stream); });
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(p, e, "kernel launch");
  }
  return TURBOFFT_SUCCESS;
}

bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

// Device staging of turbofft_exec_host, shared by all plans of a device:
// two input and two output chunk buffers plus a chunk-sized intermediate,
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
const size_t kStageChunkBytes = (size_t)64 << 20;

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

// queue one complete exec of a (member) plan on `s`: report reset, kernels,
// report copy to the pinned host mirror
turbofft_status queue_plan(turbofft_plan* p, const void* in, void* out, void* scratch, cudaStream_t s,
                           const tf::InjectSite& inj) {
  const bool ft = p->ft_mode != TURBOFFT_FT_OFF;
  if (ft) {
    cudaError_t e = cudaMemsetAsync(p->d_fts, 0, tf::FT_HEADER_BYTES, s);
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

// ---------------------------------------------------------------------------
// autotuner: every registered shape of a pass (radix = values per thread,
// threads per transform, transforms per block) is timed on the plan's own
// geometry and the fastest kept.  Results are cached per process.
// ---------------------------------------------------------------------------
std::atomic<int> g_autotune{0};
// set while the members of a ragged plan are created: they are tuned after
// their offset tables exist, and keep to one or two passes
thread_local bool t_ragged_member = false;
std::mutex g_tune_mu;
typedef std::tuple<int, int, int64_t, int64_t, int, int> TuneKey;  // dtype, pass, n, batch, variant, indexed
std::map<TuneKey, const KernelEntry*> g_tune_cache;

bool use_entry(turbofft_plan* p, int pi, const KernelEntry* ke) {
  if (!set_smem_attrs(ke)) {
    cudaGetLastError();
    return false;
  }
  p->pass[pi].ke = ke;
  p->pass[pi].grid = occupancy_blocks(ke, ft_variant(p->ft_mode)) * g_num_sms;
  return true;
}

// time each candidate of each pass on (in, out, scratch), which span the
// plan's buffers; keeps the default shape of a pass whose candidates all fail
void autotune(turbofft_plan* p, const void* in, void* out, void* scratch) {
  if (p->cl) {  // one shape per cluster configuration
    p->autotuned = true;
    return;
  }
  const Registry& reg = registry();
  const int dt = p->dtype == TURBOFFT_C2C_F32 ? 0 : 1;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    return;
  }
  const tf::InjectSite none{};
  for (int pi = 0; pi < p->num_passes; ++pi) {
    const PassPlan& pp = p->pass[pi];
    std::vector<const KernelEntry*> cands = reg.find_all(dt, pp.kind, pp.ns);
    if (cands.size() < 2) continue;
    const TuneKey key(dt, pi, p->n, p->batch, ft_variant(p->ft_mode), p->d_tab ? 1 : 0);
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) {
        use_entry(p, pi, it->second);
        continue;
      }
    }
    const KernelEntry* dflt = pp.ke;
    const KernelEntry* best = nullptr;
    float best_ms = 0.f;
    for (const KernelEntry* ke : cands) {
      if (!use_entry(p, pi, ke)) continue;
      bool ok = queue_plan(p, in, out, scratch, s, none) == TURBOFFT_SUCCESS;  // warm-up
      float ms_min = 0.f;
      for (int rep = 0; ok && rep < 3; ++rep) {
        ok = cudaEventRecord(e0, s) == cudaSuccess && queue_plan(p, in, out, scratch, s, none) == TURBOFFT_SUCCESS &&
             cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.f;
        if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (ok && (rep == 0 || ms < ms_min)) ms_min = ms;
      }
      if (!ok) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        continue;
      }
      if (!best || ms_min < best_ms) {
        best = ke;
        best_ms = ms_min;
      }
    }
    if (!best) best = dflt;
    use_entry(p, pi, best);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
  }
  cudaStreamSynchronize(s);
  if (p->d_fts) cudaMemset(p->d_fts, 0, sizeof(FtState));
  if (p->h_fts) memset(p->h_fts, 0, sizeof(FtState));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  cudaGetLastError();
  p->autotuned = true;
}

std::map<TuneKey, int> g_structure_cache;  // 1 split, 2 cluster

// run f(in, out, scratch) on temporary buffers of a contiguous plan's size,
// the input filled with a finite, non-zero pattern (0x3c bytes) so that
// timing sees ordinary arithmetic; nothing runs if they cannot be allocated
template <class F> void with_temp(turbofft_plan* p, F&& f) {
  const size_t bytes = (size_t)(p->batch * p->n) * elem_bytes(p->dtype);
  void *a = nullptr, *b = nullptr, *c = nullptr;
  bool ok = cudaMalloc(&a, bytes) == cudaSuccess && cudaMalloc(&b, bytes) == cudaSuccess &&
            (p->scratch_bytes == 0 || cudaMalloc(&c, p->scratch_bytes) == cudaSuccess);
  if (ok) ok = cudaMemset(a, 0x3c, bytes) == cudaSuccess;
  if (ok) f(a, b, c);
  cudaGetLastError();
  for (void* q : {a, b, c})
    if (q) cudaFree(q);
}

void autotune_with_temp(turbofft_plan* p) {
  with_temp(p, [&](void* a, void* b, void* c) { autotune(p, a, b, c); });
}

// best of three execs in ms (0 if timing failed)
double time_with_temp(turbofft_plan* p) {
  double best = 0;
  with_temp(p, [&](void* a, void* b, void* c) {
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
      const tf::InjectSite none{};
      bool ok = queue_plan(p, a, b, c, s, none) == TURBOFFT_SUCCESS;
      for (int rep = 0; ok && rep < 3; ++rep) {
        ok = cudaEventRecord(e0, s) == cudaSuccess && queue_plan(p, a, b, c, s, none) == TURBOFFT_SUCCESS &&
             cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.f;
        if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (ok && (rep == 0 || ms < best)) best = ms;
      }
      if (!ok) best = 0;
      cudaStreamSynchronize(s);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaGetLastError();
    if (p->d_fts) cudaMemset(p->d_fts, 0, sizeof(FtState));
    if (p->h_fts) memset(p->h_fts, 0, sizeof(FtState));
  });
  return best;
}

// ---------------------------------------------------------------------------
// ragged plans
// ---------------------------------------------------------------------------
void drop_graph(turbofft_plan* p) {
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  p->graph_exec = nullptr;
  p->graph_in = nullptr;
  p->graph_out = nullptr;
}

// capture the members as parallel branches of one graph reading `in` and
// writing `out`
turbofft_status capture_ragged(turbofft_plan* p, const void* in, void* out) {
  drop_graph(p);
  cudaStream_t cs = p->branch_streams[0];
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(p, e, "graph capture");
  turbofft_status st = TURBOFFT_SUCCESS;
  const tf::InjectSite none{};
  e = cudaEventRecord(p->branch_events[0], cs);
  for (size_t k = 0; e == cudaSuccess && st == TURBOFFT_SUCCESS && k < p->members.size(); ++k) {
    turbofft_plan* m = p->members[k];
    cudaStream_t bs = p->branch_streams[k + 1];
    e = cudaStreamWaitEvent(bs, p->branch_events[0], 0);
    if (e != cudaSuccess) break;
    st = queue_plan(m, in, out, m->d_scratch, bs, none);
    if (st != TURBOFFT_SUCCESS) break;
    e = cudaEventRecord(p->branch_events[k + 1], bs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, p->branch_events[k + 1], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess && st == TURBOFFT_SUCCESS) e = cudaGraphInstantiate(&p->graph_exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (st != TURBOFFT_SUCCESS || e != cudaSuccess) {
    p->graph_exec = nullptr;
    cudaGetLastError();
    if (st != TURBOFFT_SUCCESS) {
      for (auto m : p->members)
        if (!m->last_error.empty()) p->last_error = m->last_error;
      return st;
    }
    return cuda_fail(p, e, "graph capture");
  }
  p->graph_in = in;
  p->graph_out = out;
  return TURBOFFT_SUCCESS;
}

turbofft_status exec_ragged(turbofft_plan* p, const void* in, void* out, cudaStream_t s) {
  for (auto m : p->members)
    if (m->scratch_bytes > 0 && !m->d_scratch) {
      if (!dev_alloc(m, &m->d_scratch, m->scratch_bytes)) return TURBOFFT_ALLOC_FAILED;
      m->scratch_owned = true;
    }
  if (p->armed_any) {
    // an armed site: queue the members directly (the graph holds no site)
    p->armed_any = false;
    for (auto m : p->members) {
      tf::InjectSite inj = m->armed;
      m->armed.active = 0;
      turbofft_status st = queue_plan(m, in, out, m->d_scratch, s, inj);
      if (st != TURBOFFT_SUCCESS) {
        p->last_error = m->last_error;
        return st;
      }
    }
  } else {
    if (!p->graph_exec || p->graph_in != in || p->graph_out != out) {
      turbofft_status st = capture_ragged(p, in, out);
      if (st != TURBOFFT_SUCCESS) return st;
    }
    cudaError_t e = cudaGraphLaunch(p->graph_exec, s);
    if (e != cudaSuccess) return cuda_fail(p, e, "graph launch");
  }
  cudaError_t e = cudaEventRecord(p->done, s);
  if (e != cudaSuccess) return cuda_fail(p, e, "event record");
  p->have_exec = true;
  return TURBOFFT_SUCCESS;
}

// add a (member) plan's last report into *r; `ids` maps its transforms to
// global indices (ragged members)
void add_report(const turbofft_plan* m, const std::vector<int64_t>* ids, turbofft_report* r) {
  const FtState& h = *m->h_fts;
  r->groups_checked += (int64_t)h.groups;
  r->detected += (int64_t)h.detected;
  r->located += (int64_t)h.located;
  r->corrected += (int64_t)h.corrected;
  r->recomputed += (int64_t)h.recomputed;
  r->uncorrectable += (int64_t)(h.uncorrectable + h.dropped);
  r->max_clean_ratio = std::max(r->max_clean_ratio, (double)h.max_clean_ratio);
  const int nrec = (int)std::min<unsigned long long>(h.num_records, tf::MAX_RECORDS);
  for (int i = 0; i < nrec; ++i) {
    const FtRecord& rc = h.rec[i];
    if (r->first_pass < 0) {
      r->first_pass = rc.pass_id;
      r->first_residual = sqrt(rc.s1r * rc.s1r + rc.s1i * rc.s1i);
      r->first_threshold = rc.tau;
    }
    if (rc.signal >= 0 && r->first_transform < 0) {
      // cluster plans record the transform itself
      int64_t tr = m->cl ? rc.signal : rc.signal / signals_per_transform(m, rc.pass_id);
      tr += rc.transform_base;
      r->first_transform = (ids && tr >= 0 && tr < (int64_t)ids->size()) ? (*ids)[tr] : tr;
    }
  }
}

void fill_info(const turbofft_plan* p, turbofft_plan_info* info) {
  memset(info, 0, sizeof(*info));
  info->n = p->n;
  info->batch = p->batch;
  info->dtype = p->dtype;
  info->direction = p->direction;
  info->ft_mode = p->ft_mode;
  info->autotuned = p->autotuned ? 1 : 0;
  info->group_transactions = p->T;
  if (p->ragged) {
    info->num_members = (int32_t)p->members.size();
    for (auto m : p->members) {
      info->workspace_bytes += m->workspace_bytes + (m->scratch_owned ? 0 : (int64_t)m->scratch_bytes);
      info->autotuned |= m->autotuned ? 1 : 0;
    }
    return;
  }
  info->num_passes = p->num_passes;
  if (p->cl) {
    const ClEntry* ce = p->cl;
    info->cluster = ce->cluster;
    for (int pi = 0; pi < 2; ++pi) {
      info->sub_n[pi] = p->pass[pi].ns;
      info->stages[pi] = pi == 0 ? ce->stages_a : ce->stages_b;
      info->radix[pi] = ce->e;
      info->grid[pi] = p->cl_grid;
      info->block[pi] = ce->nt;
      info->per_block[pi] = pi == 0 ? ce->sa : ce->sb;
    }
    info->sub_n[2] = 1;
    info->workspace_bytes = p->workspace_bytes;
    info->scratch_bytes = 0;
    return;
  }
  for (int pi = 0; pi < p->num_passes; ++pi) {
    info->sub_n[pi] = p->pass[pi].ns;
    info->stages[pi] = p->pass[pi].ke->stages;
    info->radix[pi] = p->pass[pi].ke->e;
    info->grid[pi] = p->pass[pi].grid;
    info->block[pi] = p->pass[pi].ke->nt;
    info->per_block[pi] = p->pass[pi].ke->s;
  }
  for (int pi = p->num_passes; pi < 3; ++pi) info->sub_n[pi] = 1;
  info->workspace_bytes = p->workspace_bytes + (p->scratch_owned ? 0 : (int64_t)p->scratch_bytes);
  info->scratch_bytes = (int64_t)p->scratch_bytes;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* turbofft_status_string(turbofft_status s) {
  switch (s) {
    case TURBOFFT_SUCCESS: return "TURBOFFT_SUCCESS";
    case TURBOFFT_INVALID_VALUE: return "TURBOFFT_INVALID_VALUE";
    case TURBOFFT_UNSUPPORTED: return "TURBOFFT_UNSUPPORTED";
    case TURBOFFT_ALLOC_FAILED: return "TURBOFFT_ALLOC_FAILED";
    case TURBOFFT_CUDA_ERROR: return "TURBOFFT_CUDA_ERROR";
    case TURBOFFT_FT_UNCORRECTABLE: return "TURBOFFT_FT_UNCORRECTABLE";
    case TURBOFFT_TIMEOUT: return "TURBOFFT_TIMEOUT";
  }
  return "TURBOFFT_UNKNOWN_STATUS";
}

const char* turbofft_last_error(const turbofft_plan* p) { return p ? p->last_error.c_str() : ""; }

turbofft_status turbofft_destroy(turbofft_plan* p) {
  if (!p) return TURBOFFT_SUCCESS;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  for (auto m : p->members) turbofft_destroy(m);
  drop_graph(p);
  for (auto st : p->branch_streams)
    if (st) cudaStreamDestroy(st);
  for (auto ev : p->branch_events)
    if (ev) cudaEventDestroy(ev);
  for (void* a : p->allocs) cudaFree(a);
  if (p->h_fts) cudaFreeHost(p->h_fts);
  if (p->done) cudaEventDestroy(p->done);
  for (auto& pr : p->prof_ev)
    for (auto& e : pr)
      if (e) cudaEventDestroy(e);
  cudaGetLastError();
  cudaSetDevice(cur);
  delete p;
  return TURBOFFT_SUCCESS;
}

// structure: 0 = default, 1 = single pass or two passes, 2 = cluster single pass
static turbofft_status create_plan(int64_t n, int64_t batch, turbofft_dtype dtype, int direction,
                                   turbofft_ft_mode ft_mode, int structure, turbofft_plan** out) {
  if (!out) return TURBOFFT_INVALID_VALUE;
  *out = nullptr;
  const int logn = ilog2_exact(n);
  if (logn < 3 || logn > 24) return TURBOFFT_INVALID_VALUE;
  if (batch < 1 || batch * n > ((int64_t)1 << 31)) return TURBOFFT_INVALID_VALUE;
  if (dtype != TURBOFFT_C2C_F32 && dtype != TURBOFFT_C2C_F64) return TURBOFFT_INVALID_VALUE;
  if (direction != TURBOFFT_FORWARD && direction != TURBOFFT_INVERSE && direction != TURBOFFT_INVERSE_UNSCALED &&
      direction != TURBOFFT_FORWARD_SCALED)
    return TURBOFFT_INVALID_VALUE;
  if (ft_mode != TURBOFFT_FT_OFF && ft_mode != TURBOFFT_FT_DETECT && ft_mode != TURBOFFT_FT_CORRECT &&
      ft_mode != TURBOFFT_FT_CORRECT_REGISTERS)
    return TURBOFFT_INVALID_VALUE;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TURBOFFT_CUDA_ERROR;
  }
  if (g_num_sms == 0) {
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  const Registry& reg = registry();
  turbofft_plan* p = new turbofft_plan();
  p->n = n;
  p->batch = batch;
  p->dtype = dtype;
  p->direction = direction;
  p->ft_mode = ft_mode;
  p->device = dev;
  const int dt = dtype == TURBOFFT_C2C_F32 ? 0 : 1;

  // pass split: one pass up to the largest single-pass size, else N1 x N2
  // passes, or N1 x N2 x N3 for large float32 sizes (three passes whose
  // column tiles stay 64-128 bytes wide); the cluster single pass when
  // asked for (or chosen by timing)
  const ClEntry* ce = reg.find_cl(dt, n);
  const bool three = structure == 3 || (structure == 0 && dt == 0 && logn >= kThreePassLog2F32 && !t_ragged_member);
  if (structure == 3 && (logn < 9 || t_ragged_member)) {
    delete p;
    return TURBOFFT_UNSUPPORTED;
  }
  if (ce && structure == 2) {
    p->cl = ce;
    p->num_passes = 2;
    p->n1 = ce->n1;
    p->n2 = ce->n2;
    p->pass[0].kind = tf::KIND_COL;
    p->pass[0].ns = ce->n1;
    p->pass[1].kind = tf::KIND_ROW;
    p->pass[1].ns = ce->n2;
  } else if (three) {
    const int a = logn / 3, b = (logn - a) / 2, c = logn - a - b;
    p->num_passes = 3;
    p->n1 = 1 << a;
    p->n2 = 1 << (b + c);
    p->pass[0].kind = tf::KIND_COL;
    p->pass[0].ns = 1 << a;
    p->pass[1].kind = tf::KIND_COL;
    p->pass[1].ns = 1 << b;
    p->pass[2].kind = tf::KIND_ROW;
    p->pass[2].ns = 1 << c;
  } else if (n <= reg.max_sp(dt)) {
    p->num_passes = 1;
    p->n1 = (int)n;
    p->n2 = 1;
    p->pass[0].kind = tf::KIND_SP;
    p->pass[0].ns = (int)n;
  } else {
    p->num_passes = 2;
    p->n1 = 1 << (logn / 2);
    p->n2 = 1 << (logn - logn / 2);
    p->pass[0].kind = tf::KIND_COL;
    p->pass[0].ns = p->n1;
    p->pass[1].kind = tf::KIND_ROW;
    p->pass[1].ns = p->n2;
  }
  // geometry of each pass
  for (int pi = 0; pi < p->num_passes; ++pi) {
    PassPlan& pp = p->pass[pi];
    pp.g_n = n;
    pp.g_n1 = p->n1;
    pp.g_n2 = p->n2;
    pp.bm = 1;
    if (p->num_passes == 3 && pi > 0) {
      pp.g_n = p->n2;  // M = N2 * N3, one length-M transform per first-pass output row
      pp.g_n1 = p->pass[1].ns;
      pp.g_n2 = p->pass[2].ns;
      pp.bm = p->n1;
      pp.outer = (pi == 2) ? p->n1 : 0;
    }
  }
  for (int pi = 0; pi < p->num_passes && p->cl; ++pi) {
    if (!upload_tables(p, p->pass[pi])) {
      turbofft_destroy(p);
      return TURBOFFT_ALLOC_FAILED;
    }
  }
  if (p->cl) {
    // the column and row checksums are summed per block: the per-phase
    // factors N log2 N ride on the energy, tau = gamma u sqrt(weighted energy)
    p->pass[0].tau_coef = kGamma[dt] * kUnitRoundoff[dt];
    const int v = cl_variant(ft_mode);
    bool ok = true;
    for (const void* fn : {ce->fn_main[0], ce->fn_main[1], ce->fn_fix})
      ok = ok && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ce->smem[1]) == cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ce->cluster * 64));
    cfg.blockDim = dim3((unsigned)ce->nt);
    cfg.dynamicSmemBytes = (size_t)ce->smem[v];
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)ce->cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    ok = ok && cudaOccupancyMaxActiveClusters(&ncl, ce->fn_main[v], &cfg) == cudaSuccess;
    if (!ok || ncl < 1) {
      cudaGetLastError();
      turbofft_destroy(p);
      return TURBOFFT_CUDA_ERROR;
    }
    p->cl_grid = ncl * ce->cluster;
  }
  for (int pi = 0; pi < p->num_passes && !p->cl; ++pi) {
    PassPlan& pp = p->pass[pi];
    pp.ke = reg.find(dt, pp.kind, pp.ns);
    if (!pp.ke) {
      turbofft_destroy(p);
      return TURBOFFT_UNSUPPORTED;
    }
    if (!set_smem_attrs(pp.ke)) {
      cudaGetLastError();
      turbofft_destroy(p);
      return TURBOFFT_CUDA_ERROR;
    }
    const int occ = occupancy_blocks(pp.ke, ft_variant(ft_mode));
    pp.grid = occ * g_num_sms;
    pp.tau_coef = kGamma[dt] * kUnitRoundoff[dt] * sqrt((double)ilog2_exact(pp.ns));
    if (!upload_tables(p, pp)) {
      turbofft_destroy(p);
      return TURBOFFT_ALLOC_FAILED;
    }
  }
  if (p->num_passes >= 2) {
    // inter-pass twiddles w_L^q = thi[q >> 12] * tlo[q & 4095] of each
    // column pass, over the length L it splits (N, and M for the second
    // pass of a three-pass plan)
    bool ok = true;
    for (int pi = 0; pi + 1 < p->num_passes && ok; ++pi) {
      const int64_t L = p->pass[pi].g_n;
      void** lo_dst = (pi == 0) ? &p->d_tlo : &p->pass[pi].d_tlo;
      void** hi_dst = (pi == 0) ? &p->d_thi : &p->pass[pi].d_thi;
      std::vector<cld> lo(4096), hi((size_t)std::max<int64_t>(1, L / 4096));
      for (int j = 0; j < 4096; ++j) lo[j] = root(L, j);
      for (size_t j = 0; j < hi.size(); ++j) hi[j] = root(L, (int64_t)j * 4096);
      ok = (dt == 0) ? (upload<float>(p, lo_dst, lo) && upload<float>(p, hi_dst, hi))
                     : (upload<double>(p, lo_dst, lo) && upload<double>(p, hi_dst, hi));
    }
    p->scratch_bytes = p->cl ? 0 : (size_t)(batch * n) * elem_bytes(dtype);
    if (!ok) {
      turbofft_destroy(p);
      return TURBOFFT_ALLOC_FAILED;
    }
  }
  if (ft_mode != TURBOFFT_FT_OFF) {
    void* fts = nullptr;
    if (!dev_alloc(p, &fts, sizeof(FtState))) {
      turbofft_destroy(p);
      return TURBOFFT_ALLOC_FAILED;
    }
    p->d_fts = static_cast<FtState*>(fts);
    if (cudaMemset(p->d_fts, 0, sizeof(FtState)) != cudaSuccess ||
        cudaHostAlloc((void**)&p->h_fts, sizeof(FtState), cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      turbofft_destroy(p);
      return TURBOFFT_ALLOC_FAILED;
    }
    memset(p->h_fts, 0, sizeof(FtState));
    p->rec_stride = 0;
    for (int pi = 0; pi < p->num_passes; ++pi) p->rec_stride = std::max(p->rec_stride, p->pass[pi].ns);
    if (!dev_alloc(p, &p->d_rec_sums, (size_t)tf::MAX_RECORDS * 2 * p->rec_stride * elem_bytes(dtype))) {
      turbofft_destroy(p);
      return TURBOFFT_ALLOC_FAILED;
    }
  }
  if (cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    turbofft_destroy(p);
    return TURBOFFT_CUDA_ERROR;
  }
  *out = p;
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_plan_create_structured(int64_t n, int64_t batch, turbofft_dtype dtype, int direction,
                                                turbofft_ft_mode ft_mode, int structure, turbofft_plan** out) {
  if (out) *out = nullptr;
  if (structure != TURBOFFT_STRUCTURE_SPLIT && structure != TURBOFFT_STRUCTURE_CLUSTER &&
      structure != TURBOFFT_STRUCTURE_THREE_PASS)
    return TURBOFFT_INVALID_VALUE;
  turbofft_status st = create_plan(n, batch, dtype, direction, ft_mode, structure, out);
  if (st == TURBOFFT_SUCCESS && structure == TURBOFFT_STRUCTURE_CLUSTER && !(*out)->cl) {
    turbofft_destroy(*out);
    *out = nullptr;
    return TURBOFFT_UNSUPPORTED;
  }
  if (st == TURBOFFT_SUCCESS && g_autotune.load()) autotune_with_temp(*out);
  return st;
}

turbofft_status turbofft_plan_create(int64_t n, int64_t batch, turbofft_dtype dtype, int direction,
                                     turbofft_ft_mode ft_mode, turbofft_plan** out) {
  turbofft_status st = create_plan(n, batch, dtype, direction, ft_mode, 0, out);
  if (st != TURBOFFT_SUCCESS || !g_autotune.load() || t_ragged_member) return st;
  turbofft_plan* p = *out;
  autotune_with_temp(p);
  // where both a cluster plan and a split plan exist for this size, the
  // faster of the two (after shape tuning) is kept
  const int dt = dtype == TURBOFFT_C2C_F32 ? 0 : 1;
  if (registry().find_cl(dt, n)) {
    const TuneKey key(dt, -1, n, batch, ft_variant(ft_mode), 0);
    int choice = -1;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_structure_cache.find(key);
      if (it != g_structure_cache.end()) choice = it->second;
    }
    const int mine = p->cl ? 2 : 1;
    if (choice != mine) {
      turbofft_plan* q = nullptr;
      if (create_plan(n, batch, dtype, direction, ft_mode, mine == 2 ? 1 : 2, &q) == TURBOFFT_SUCCESS) {
        autotune_with_temp(q);
        bool take_q = choice == (mine == 2 ? 1 : 2);
        if (choice < 0) {
          const double tp = time_with_temp(p), tq = time_with_temp(q);
          take_q = tq > 0 && (tp <= 0 || tq < tp);
          std::lock_guard<std::mutex> lock(g_tune_mu);
          g_structure_cache[key] = take_q ? (mine == 2 ? 1 : 2) : mine;
        }
        if (take_q) std::swap(p, q);
        turbofft_destroy(q);
      }
    }
    p->autotuned = true;
    *out = p;
  }
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_plan_create_ragged(const int64_t* sizes, const int64_t* offsets, int64_t count,
                                            turbofft_dtype dtype, int direction, turbofft_ft_mode ft_mode,
                                            turbofft_plan** out) {
  if (!out) return TURBOFFT_INVALID_VALUE;
  *out = nullptr;
  if (!sizes || !offsets || count < 1 || count > ((int64_t)1 << 31)) return TURBOFFT_INVALID_VALUE;
  if (dtype != TURBOFFT_C2C_F32 && dtype != TURBOFFT_C2C_F64) return TURBOFFT_INVALID_VALUE;
  if (direction != TURBOFFT_FORWARD && direction != TURBOFFT_INVERSE && direction != TURBOFFT_INVERSE_UNSCALED &&
      direction != TURBOFFT_FORWARD_SCALED)
    return TURBOFFT_INVALID_VALUE;
  if (ft_mode != TURBOFFT_FT_OFF && ft_mode != TURBOFFT_FT_DETECT && ft_mode != TURBOFFT_FT_CORRECT &&
      ft_mode != TURBOFFT_FT_CORRECT_REGISTERS)
    return TURBOFFT_INVALID_VALUE;
  int64_t extent = 0;
  for (int64_t i = 0; i < count; ++i) {
    const int lg = ilog2_exact(sizes[i]);
    if (lg < 3 || lg > 24 || offsets[i] < 0 || offsets[i] > ((int64_t)1 << 40)) return TURBOFFT_INVALID_VALUE;
    // every transform starts on a 16-byte boundary of the packed buffers
    if (dtype == TURBOFFT_C2C_F32 && (offsets[i] & 1)) return TURBOFFT_INVALID_VALUE;
    extent = std::max(extent, offsets[i] + sizes[i]);
  }
  std::vector<int64_t> order((size_t)count);
  std::iota(order.begin(), order.end(), (int64_t)0);
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return offsets[a] < offsets[b]; });
  for (size_t k = 1; k < order.size(); ++k)
    if (offsets[order[k - 1]] + sizes[order[k - 1]] > offsets[order[k]]) return TURBOFFT_INVALID_VALUE;

  std::map<int64_t, std::vector<int64_t>> groups;  // size -> global indices, ascending
  for (int64_t i = 0; i < count; ++i) groups[sizes[i]].push_back(i);
  for (auto& g : groups)
    if ((int64_t)g.second.size() * g.first > ((int64_t)1 << 31)) return TURBOFFT_INVALID_VALUE;

  turbofft_plan* p = new turbofft_plan();
  p->ragged = true;
  p->n = 0;
  p->batch = count;
  p->dtype = dtype;
  p->direction = direction;
  p->ft_mode = ft_mode;
  p->extent = extent;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return TURBOFFT_CUDA_ERROR;
  }
  p->member_of.assign((size_t)count, 0);
  p->local_of.assign((size_t)count, 0);
  t_ragged_member = true;
  turbofft_status st = TURBOFFT_SUCCESS;
  for (auto& g : groups) {
    turbofft_plan* m = nullptr;
    st = turbofft_plan_create(g.first, (int64_t)g.second.size(), dtype, direction, ft_mode, &m);
    if (st != TURBOFFT_SUCCESS) break;
    p->members.push_back(m);
    p->member_ids.push_back(g.second);
    std::vector<long long> tab(g.second.size());
    for (size_t j = 0; j < tab.size(); ++j) {
      tab[j] = offsets[g.second[j]];
      p->member_of[(size_t)g.second[j]] = (int32_t)(p->members.size() - 1);
      p->local_of[(size_t)g.second[j]] = (int64_t)j;
    }
    void* d = nullptr;
    if (!dev_alloc(m, &d, tab.size() * sizeof(long long)) ||
        cudaMemcpy(d, tab.data(), tab.size() * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      st = TURBOFFT_ALLOC_FAILED;
      break;
    }
    m->d_tab = static_cast<long long*>(d);
  }
  t_ragged_member = false;
  if (st != TURBOFFT_SUCCESS) {
    turbofft_destroy(p);
    return st;
  }
  const size_t nstreams = p->members.size() + 1;
  p->branch_streams.assign(nstreams, nullptr);
  p->branch_events.assign(nstreams, nullptr);
  for (size_t k = 0; k < nstreams; ++k)
    if (cudaStreamCreateWithFlags(&p->branch_streams[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->branch_events[k], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      turbofft_destroy(p);
      return TURBOFFT_CUDA_ERROR;
    }
  if (cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    turbofft_destroy(p);
    return TURBOFFT_CUDA_ERROR;
  }
  if (g_autotune.load()) {
    // tune every member on its real (indexed) geometry in shared temporaries
    const size_t bytes = (size_t)extent * elem_bytes(dtype);
    size_t sbytes = 0;
    for (auto m : p->members) sbytes = std::max(sbytes, m->scratch_bytes);
    void *a = nullptr, *b = nullptr, *c = nullptr;
    bool ok = cudaMalloc(&a, bytes) == cudaSuccess && cudaMalloc(&b, bytes) == cudaSuccess &&
              (sbytes == 0 || cudaMalloc(&c, sbytes) == cudaSuccess);
    if (ok) ok = cudaMemset(a, 0x3c, bytes) == cudaSuccess;
    if (ok)
      for (auto m : p->members) autotune(m, a, b, c);
    cudaGetLastError();
    for (void* q : {a, b, c})
      if (q) cudaFree(q);
  }
  *out = p;
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_plan_get_member_info(const turbofft_plan* p, int32_t index, turbofft_plan_info* info) {
  if (!p || !info || !p->ragged || index < 0 || index >= (int32_t)p->members.size()) return TURBOFFT_INVALID_VALUE;
  fill_info(p->members[(size_t)index], info);
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_set_autotune(int enable) {
  g_autotune.store(enable ? 1 : 0);
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_plan_get_info(const turbofft_plan* p, turbofft_plan_info* info) {
  if (!p || !info) return TURBOFFT_INVALID_VALUE;
  fill_info(p, info);
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_set_threshold_scale(turbofft_plan* p, double factor) {
  if (!p || !(factor > 0) || !isfinite(factor)) return TURBOFFT_INVALID_VALUE;
  p->threshold_scale = factor;
  for (auto m : p->members) m->threshold_scale = factor;
  if (p->ragged) drop_graph(p);  // the captured launches hold the old threshold
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_set_group_transactions(turbofft_plan* p, int transactions) {
  if (!p || transactions < 1 || transactions > 16) return TURBOFFT_INVALID_VALUE;
  p->T = transactions;
  for (auto m : p->members) m->T = transactions;
  if (p->ragged) drop_graph(p);  // the captured launches hold the old group size
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_inject(turbofft_plan* p, turbofft_site site, int bit) {
  if (!p) return TURBOFFT_INVALID_VALUE;
  if (p->ragged) {
    if (site.transform < 0 || site.transform >= p->batch) return TURBOFFT_INVALID_VALUE;
    turbofft_plan* m = p->members[(size_t)p->member_of[(size_t)site.transform]];
    turbofft_site ls = site;
    ls.transform = p->local_of[(size_t)site.transform];
    turbofft_status st = turbofft_inject(m, ls, bit);
    if (st == TURBOFFT_SUCCESS) p->armed_any = true;
    return st;
  }
  const int nbits = p->dtype == TURBOFFT_C2C_F32 ? 32 : 64;
  if (bit < 0 || bit >= nbits) return TURBOFFT_INVALID_VALUE;
  if (site.transform < 0 || site.transform >= p->batch) return TURBOFFT_INVALID_VALUE;
  if (site.pass < 0 || site.pass >= p->num_passes) return TURBOFFT_INVALID_VALUE;
  const int nst = p->cl ? (site.pass == 0 ? p->cl->stages_a : p->cl->stages_b) : p->pass[site.pass].ke->stages;
  if (site.stage < 0 || site.stage > nst) return TURBOFFT_INVALID_VALUE;
  if (site.element < 0 || site.element >= p->n) return TURBOFFT_INVALID_VALUE;
  if (site.component != 0 && site.component != 1) return TURBOFFT_INVALID_VALUE;
  tf::InjectSite s{};
  s.active = 1;
  s.pass = site.pass;
  s.stage = site.stage;
  s.comp = site.component;
  s.bit = bit;
  const PassPlan& ip = p->pass[site.pass];
  if (ip.kind == tf::KIND_SP) {
    s.signal = site.transform;
    s.pos = (int)site.element;
  } else {
    // element = sub * g_n + el: sub-transform `sub` of the pass's bm per transform
    const int64_t sub = site.element / ip.g_n, el = site.element % ip.g_n;
    const int64_t r = site.transform * ip.bm + sub;
    if (ip.kind == tf::KIND_COL) {
      s.signal = r * ip.g_n2 + el % ip.g_n2;
      s.pos = (int)(el / ip.g_n2);
    } else {
      s.signal = r * ip.g_n1 + el / ip.g_n2;
      s.pos = (int)(el % ip.g_n2);
    }
  }
  p->armed = s;
  return TURBOFFT_SUCCESS;
}

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

turbofft_status turbofft_set_workspace(turbofft_plan* p, void* workspace, size_t bytes) {
  if (!p) return TURBOFFT_INVALID_VALUE;
  if (p->ragged) return TURBOFFT_UNSUPPORTED;
  if (p->scratch_bytes == 0) return TURBOFFT_SUCCESS;  // nothing to place
  if (!workspace || bytes < p->scratch_bytes || !aligned16(workspace)) return TURBOFFT_INVALID_VALUE;
  if (p->scratch_owned) {
    cudaStreamSynchronize(nullptr);
    cudaDeviceSynchronize();
    for (auto it = p->allocs.begin(); it != p->allocs.end(); ++it)
      if (*it == p->d_scratch) {
        cudaFree(*it);
        p->allocs.erase(it);
        p->workspace_bytes -= (int64_t)p->scratch_bytes;
        break;
      }
    p->scratch_owned = false;
  }
  p->d_scratch = workspace;
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_set_profiling(turbofft_plan* p, int enable) {
  if (!p) return TURBOFFT_INVALID_VALUE;
  if (p->ragged) return TURBOFFT_UNSUPPORTED;
  if (enable && !p->prof_ev[0][0]) {
    for (auto& pr : p->prof_ev)
      for (auto& e : pr) {
        cudaError_t ce = cudaEventCreate(&e);
        if (ce != cudaSuccess) return cuda_fail(p, ce, "event create");
      }
  }
  p->profiling = enable != 0;
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_get_kernel_times(turbofft_plan* p, turbofft_kernel_time* out, int capacity, int* count) {
  if (!p || !count || (capacity > 0 && !out)) return TURBOFFT_INVALID_VALUE;
  *count = 0;
  if (!p->profiling) return TURBOFFT_SUCCESS;
  for (int i = 0; i < p->nprof && i < capacity; ++i) {
    cudaError_t ce = cudaEventSynchronize(p->prof_ev[i][1]);
    if (ce != cudaSuccess) return cuda_fail(p, ce, "profiling wait");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p->prof_ev[i][0], p->prof_ev[i][1]);
    out[i].pass = p->prof_kind[i] / 2;
    out[i].is_correction = p->prof_kind[i] % 2;
    out[i].ms = ms;
    ++*count;
  }
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_get_report(turbofft_plan* p, turbofft_report* r) {
  if (!p || !r) return TURBOFFT_INVALID_VALUE;
  memset(r, 0, sizeof(*r));
  r->first_transform = -1;
  r->first_pass = -1;
  if (p->ft_mode == TURBOFFT_FT_OFF || !p->have_exec) return TURBOFFT_SUCCESS;
  cudaError_t e = cudaEventSynchronize(p->done);
  if (e != cudaSuccess) return cuda_fail(p, e, "report wait");
  if (p->ragged) {
    for (size_t k = 0; k < p->members.size(); ++k) add_report(p->members[k], &p->member_ids[k], r);
  } else {
    add_report(p, nullptr, r);
  }
  if (r->uncorrectable > 0) return TURBOFFT_FT_UNCORRECTABLE;
  if (p->ft_mode == TURBOFFT_FT_DETECT && r->detected > 0) return TURBOFFT_FT_UNCORRECTABLE;
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
