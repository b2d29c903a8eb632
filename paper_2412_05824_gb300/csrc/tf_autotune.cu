// Autotuning of launch shapes: every registered shape of a pass (radix =
// values per thread, threads per transform, transforms per block) is timed
// on the plan's own geometry and the fastest kept; where a cluster and a
// split structure exist for a size, both are timed.  Results are cached per
// process.
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

#include "tf_plan.h"

namespace tfh {

std::atomic<int> g_autotune{0};
thread_local bool t_ragged_member = false;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_structure_cache;

namespace {
std::map<TuneKey, const KernelEntry*> g_tune_cache;

bool use_entry(turbofft_plan* p, int pi, const KernelEntry* ke) {
  if (!set_smem_attrs(ke)) {
    cudaGetLastError();
    return false;
  }
  p->pass[pi].ke = ke;
  p->pass[pi].grid = occupancy_blocks(ke, plan_variant(p)) * g_num_sms;
  return true;
}

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
}  // namespace

// time each candidate of each pass on (in, out, scratch), which span the
// plan's buffers; keeps the default shape of a pass whose candidates all fail
void autotune(turbofft_plan* p, const void* in, void* out, void* scratch) {
  if (p->cl) {  // one shape per cluster configuration
    p->autotuned = true;
    return;
  }
  const Registry& reg = registry();
  const int dt = kernel_dtype(p);
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
    const TuneKey key(dt, pi, p->n, p->batch, plan_variant(p), p->d_tab ? 1 : 0);
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
      if (!ke->main[plan_variant(p)]) continue;  // no kernel of this checksum variant
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

}  // namespace tfh

extern "C" turbofft_status turbofft_set_autotune(int enable) {
  tfh::g_autotune.store(enable ? 1 : 0);
  return TURBOFFT_SUCCESS;
}
