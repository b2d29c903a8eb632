// Ragged batches: one member plan per distinct size addressing its
// transforms through a device offset table, run as the parallel branches of
// one CUDA graph captured per (in, out) pair.
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

void drop_graph(turbofft_plan* p) {
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  p->graph_exec = nullptr;
  p->graph_in = nullptr;
  p->graph_out = nullptr;
}

namespace {

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

}  // namespace

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

}  // namespace tfh

using namespace tfh;

extern "C" {

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
  if (ft_mode == TURBOFFT_FT_CORRECT_THREAD) return TURBOFFT_UNSUPPORTED;  // one thread per transform only
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

}  // extern "C"
