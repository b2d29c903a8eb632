// Host-side internals shared by the library's translation units: the plan
// object, the kernel registry, host tables and the launch, autotuning and
// ragged-batch helpers.  Not part of the C ABI (include/turbofft.h).
#pragma once

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

#include "../../include/turbofft.h"
#include "tf_registry.h"
#include "tf_types.h"

namespace tfh {

using tf::ClEntry;
using tf::FtRecord;
using tf::FtState;
using tf::KernelEntry;

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
                              tf::entries_f32_alt_sp, tf::entries_f32_alt_cr, tf::entries_f64_alt,
                              tf::entries_pairs};
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
  // first entry that has a kernel of checksum variant `variant`
  const KernelEntry* find_variant(int dtype, int kind, int ns, int variant) const {
    for (auto e : all)
      if (e->dtype == dtype && e->kind == kind && e->ns == ns && e->main[variant]) return e;
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
const Registry& registry();

// ---------------------------------------------------------------------------
// host tables (long double; tf_tables.cu)
// ---------------------------------------------------------------------------
typedef long double ld;
typedef std::complex<ld> cld;

cld root(int64_t n, int64_t q);                // w_n^q = exp(-2 pi i q / n)
void host_fft(std::vector<cld>& a);            // forward DFT, recursive radix-2
std::vector<cld> encoding_vector(int ns);      // output-side checksum vector e
int ilog2_exact(int64_t n);                    // log2 n, -1 if not a power of two

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

// default threshold factor gamma per working precision: chosen from clean-run
// residuals so that the largest clean |S1| stays far below tau
// (index: 0 float32, 1 float64, 2 float64 data in float-pair arithmetic,
// which has no checksums)
constexpr double kGamma[3] = {8.0, 16.0, 16.0};
constexpr double kUnitRoundoff[3] = {0x1p-24, 0x1p-53, 0x1p-47};
// thread-level checks test one transform at a time: the rounding residual of
// a single transform has a heavier tail relative to its energy than that of
// a group's sum, so their threshold takes twice the group's gamma
constexpr double kThreadLevelGammaFactor = 2.0;
// float32 sizes from 2^this use three passes by default
constexpr int kThreePassLog2F32 = 22;

extern int g_num_sms;

}  // namespace tfh

// ---------------------------------------------------------------------------
// the plan
// ---------------------------------------------------------------------------
struct PassPlan {
  const tf::KernelEntry* ke = nullptr;
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
  void* d_colw = nullptr;   // float64 column pass: twiddles in access order (g_n entries)
  void* d_colwe = nullptr;  // and e_k1 conj(w) (checksummed plans)
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
  bool pairs = false;  // float64 data transformed in float-pair arithmetic
  // float64 two-pass plan with checksums over whole transforms (column pass
  // v.x, row pass e.y, check and recompute kernels after the row pass)
  bool tchk = false;
  // float32 one- and two-pass plans: bit pi set if pass pi stages its tiles
  // with TMA copies (a column pass where encode_column_map can describe the
  // exec's input); d_err receives the kernels' timeout flag (the FtState's
  // error field with checksums on)
  int tma_mask = 0;
  int* d_err = nullptr;
  void* d_vcol = nullptr;
  void* d_erow = nullptr;
  double* d_tacc = nullptr;
  int device = 0;
  int num_passes = 1;
  int n1 = 0, n2 = 1;
  PassPlan pass[3];
  void* d_tlo = nullptr;
  void* d_thi = nullptr;
  void* d_scratch = nullptr;      // intermediate of two-pass plans (owned or caller's)
  size_t scratch_bytes = 0;       // bytes a two-pass exec needs
  bool scratch_owned = false;
  tf::FtState* d_fts = nullptr;
  tf::FtState* h_fts = nullptr;
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
  void* rg = nullptr;               // ragged: state of the one-launch persistent kernel, if used
  std::vector<int32_t> member_of;  // ragged: member plan of each global transform
  std::vector<int64_t> local_of;   // ragged: index of each global transform within its member
  bool autotuned = false;          // launch shapes chosen by timing (turbofft_set_autotune)
  // single-pass cluster plan: both four-step phases in one kernel
  const tf::ClEntry* cl = nullptr;
  int cl_grid = 0;
};

namespace tfh {

// ---------------------------------------------------------------------------
// allocation and tables (tf_tables.cu)
// ---------------------------------------------------------------------------
size_t elem_bytes(int dtype);
turbofft_status cuda_fail(turbofft_plan* p, cudaError_t e, const char* what);
bool dev_alloc(turbofft_plan* p, void** ptr, size_t bytes);
template <typename R>
bool upload(turbofft_plan* p, void** dst, const std::vector<cld>& v) {
  auto t = round_table<R>(v);
  size_t bytes = t.size() * sizeof(t[0]);
  if (!dev_alloc(p, dst, bytes)) return false;
  return cudaMemcpy(*dst, t.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
}
// a table as float pairs (hi, lo) per component, for float-pair plans
bool upload_pairs(turbofft_plan* p, void** dst, const std::vector<cld>& v);
bool upload_tables(turbofft_plan* p, PassPlan& pp);
bool col_tables(turbofft_plan* p, PassPlan& pp, bool weights);  // float64 column-pass tables, host-built
bool tc_tables(turbofft_plan* p);  // N-point weights of transform-level checksums, host-built

// ---------------------------------------------------------------------------
// launches (tf_launch.cu)
// ---------------------------------------------------------------------------
int ft_variant(int ft_mode);   // 0 none, 1 checksums, 2 checksums + register sums, 3 thread-level
int kernel_dtype(const turbofft_plan* p);  // registry dtype: 0 float32, 1 float64, 2 float pairs
int plan_variant(const turbofft_plan* p);  // kernel variant of the plan's passes (4: transform-level)
int cl_variant(int ft_mode);   // cluster kernels: 0 none, 1 checksums
int occupancy_blocks(const KernelEntry* ke, int variant);
bool set_smem_attrs(const KernelEntry* ke);
long long units_for(const turbofft_plan* p, int pi, int64_t batch);
int64_t signals_per_transform(const turbofft_plan* p, int pi);
bool aligned16(const void* ptr);
turbofft_status run(turbofft_plan* p, const void* in, void* out, void* scratch, int64_t batch, int64_t tbase,
                    cudaStream_t stream, const tf::InjectSite& inj);
turbofft_status queue_plan(turbofft_plan* p, const void* in, void* out, void* scratch, cudaStream_t s,
                           const tf::InjectSite& inj);
turbofft_status check_io(const turbofft_plan* p, const void* in, void* out);
turbofft_status exec_on_stream(turbofft_plan* p, const void* in, void* out, void* scratch, cudaStream_t s);

// ---------------------------------------------------------------------------
// autotuning (tf_autotune.cu)
// ---------------------------------------------------------------------------
extern std::atomic<int> g_autotune;
// set while the members of a ragged plan are created: they are tuned after
// their offset tables exist, and keep to one or two passes
extern thread_local bool t_ragged_member;
typedef std::tuple<int, int, int64_t, int64_t, int, int> TuneKey;  // dtype, pass, n, batch, variant, indexed
extern std::mutex g_tune_mu;
extern std::map<TuneKey, int> g_structure_cache;  // 1 split, 2 cluster
void autotune(turbofft_plan* p, const void* in, void* out, void* scratch);
void autotune_with_temp(turbofft_plan* p);
double time_with_temp(turbofft_plan* p);

// ---------------------------------------------------------------------------
// ragged plans (tf_ragged.cu)
// ---------------------------------------------------------------------------
void drop_graph(turbofft_plan* p);
turbofft_status exec_ragged(turbofft_plan* p, const void* in, void* out, cudaStream_t s);
extern std::atomic<int> g_ragged_single;  // new ragged plans use the persistent kernel where they can
extern std::atomic<int> g_tma_staging;    // TMA staging of new float32 plans: 0 never, 1 where faster, 2 always
bool tma_faster(const KernelEntry* ke, int ft_mode);  // mode 1's rule (tf_launch.cu)
void rg_free(turbofft_plan* p);
bool rg_timed_out(const turbofft_plan* p);  // the last exec's grid barrier gave up waiting

// ---------------------------------------------------------------------------
// plans, reports (tf_capi.cu)
// ---------------------------------------------------------------------------
// structure: 0 = default, 1 = single pass or two passes, 2 = cluster single
// pass, 3 = three passes, 4 = float pairs, 5 = as 1 with one pass only up to
// 4096 (members of a ragged plan run by the persistent kernel)
turbofft_status create_plan(int64_t n, int64_t batch, turbofft_dtype dtype, int direction, turbofft_ft_mode ft_mode,
                            int structure, turbofft_plan** out);
void add_report(const turbofft_plan* m, const std::vector<int64_t>* ids, turbofft_report* r);
void fill_info(const turbofft_plan* p, turbofft_plan_info* info);

}  // namespace tfh
