// Ragged batches: one member plan per distinct size addressing its
// transforms through a device offset table.  A float32 batch of lengths
// 8 .. 2^16 runs as ONE launch of the persistent ragged kernel
// (tf_ragged_kernel.cu) over a size-sorted work queue; other batches (and
// plans created with the single launch switched off) run the members as the
// parallel branches of one CUDA graph.  Either form is captured per
// (in, out) pair.
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
#include "tf_ragged_kernel.h"

namespace tfh {

std::atomic<int> g_ragged_single{1};

// state of a ragged plan run by the persistent kernel
struct RgState {
  std::vector<int> ca_member, ca_pass, ca_cls, ca_phase;  // pass entries
  std::vector<long long> ca_units;
  tf::RgItem* d_items[2] = {nullptr, nullptr};
  long long num_items[2] = {0, 0};
  int num_phases = 1;
  int ftm = 0;
  int grid = 0;
  size_t smem = 0;
  tf::RgCtl* d_ctl = nullptr;
  tf::RgCtl* h_ctl = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraphExec_t graph = nullptr;
  const void* g_in = nullptr;
  void* g_out = nullptr;
};

void rg_free(turbofft_plan* p) {
  RgState* r = static_cast<RgState*>(p->rg);
  if (!r) return;
  if (r->graph) cudaGraphExecDestroy(r->graph);
  for (auto d : r->d_items)
    if (d) cudaFree(d);
  if (r->d_ctl) cudaFree(r->d_ctl);
  if (r->h_ctl) cudaFreeHost(r->h_ctl);
  if (r->cs) cudaStreamDestroy(r->cs);
  delete r;
  p->rg = nullptr;
}

void drop_graph(turbofft_plan* p) {
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  p->graph_exec = nullptr;
  p->graph_in = nullptr;
  p->graph_out = nullptr;
  if (RgState* r = static_cast<RgState*>(p->rg)) {
    if (r->graph) cudaGraphExecDestroy(r->graph);
    r->graph = nullptr;
    r->g_in = nullptr;
    r->g_out = nullptr;
  }
}

bool rg_timed_out(const turbofft_plan* p) {
  const RgState* r = static_cast<const RgState*>(p->rg);
  return r && r->h_ctl && r->h_ctl->error != 0;
}

namespace {

// size class of pass pi of a member of length n (-1: none)
int rg_class_of(int64_t n, int pi, int num_passes, int n1, int n2) {
  const tf::RgClassInfo* ci = tf::ragged_classes();
  const int kind = num_passes == 1 ? tf::KIND_SP : (pi == 0 ? tf::KIND_COL : tf::KIND_ROW);
  const int ns = num_passes == 1 ? (int)n : (pi == 0 ? n1 : n2);
  for (int c = 0; c < tf::kRgClasses; ++c)
    if (ci[c].kind == kind && ci[c].ns == ns) return c;
  return -1;
}

// work units of pass entry (member m, pass pi) in class c
long long rg_units(const turbofft_plan* m, int pi, const tf::RgClassInfo& c) {
  if (c.kind == tf::KIND_SP) return (m->batch + c.s - 1) / c.s;
  if (c.kind == tf::KIND_COL) return m->batch * (m->n2 / c.s);
  return m->batch * (m->n1 / c.s);
}

// Build the work queue of a ragged plan whose members the persistent kernel
// can run; false (and no state) otherwise.
bool rg_setup(turbofft_plan* p) {
  if (p->dtype != TURBOFFT_C2C_F32) return false;
  if (p->ft_mode != TURBOFFT_FT_OFF && p->ft_mode != TURBOFFT_FT_DETECT && p->ft_mode != TURBOFFT_FT_CORRECT)
    return false;
  const tf::RgClassInfo* ci = tf::ragged_classes();
  RgState* r = new RgState();
  r->ftm = p->ft_mode == TURBOFFT_FT_OFF ? 0 : 1;
  struct Piece {
    int ca;
    long long u0, u1;
    long long bytes;
  };
  std::vector<Piece> pieces[2];
  size_t smem = 0;
  bool ok = true;
  for (size_t k = 0; k < p->members.size() && ok; ++k) {
    const turbofft_plan* m = p->members[k];
    if (m->cl || m->num_passes > 2 || m->T < 1) ok = false;
    for (int pi = 0; ok && pi < m->num_passes; ++pi) {
      const int c = rg_class_of(m->n, pi, m->num_passes, m->n1, m->n2);
      if (c < 0 || (int)r->ca_cls.size() >= tf::kRgMaxPasses) {
        ok = false;
        break;
      }
      const int phase = (m->num_passes == 2 && pi == 1) ? 1 : 0;
      const int ca = (int)r->ca_cls.size();
      const long long units = rg_units(m, pi, ci[c]);
      r->ca_member.push_back((int)k);
      r->ca_pass.push_back(pi);
      r->ca_cls.push_back(c);
      r->ca_phase.push_back(phase);
      r->ca_units.push_back(units);
      smem = std::max(smem, (size_t)(r->ftm ? std::max(ci[c].smem_ft, ci[c].smem_fix) : ci[c].smem_plain));
      // items of about 512 KB of input (each item restarts the block's
      // copy pipeline), whole checksum groups of T units
      const long long ubytes = (long long)ci[c].s * ci[c].ns * 8;
      long long per = std::max<long long>(1, (512 << 10) / ubytes);
      per = (per + m->T - 1) / m->T * m->T;
      for (long long u = 0; u < units; u += per)
        pieces[phase].push_back({ca, u, std::min(units, u + per), ubytes * (std::min(units, u + per) - u)});
      if (phase == 1) r->num_phases = 2;
    }
  }
  if (ok) {
    r->smem = smem;
    const void* fn = tf::ragged_kernel_fn(r->ftm);
    int per_sm = 0;
    ok = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
         cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, tf::kRgThreads, smem) == cudaSuccess &&
         per_sm >= 1;
    r->grid = per_sm * g_num_sms;
  }
  for (int ph = 0; ok && ph < r->num_phases; ++ph) {
    // largest items first: the queue's tail holds the small ones
    std::stable_sort(pieces[ph].begin(), pieces[ph].end(), [&](const Piece& a, const Piece& b) {
      return ci[r->ca_cls[a.ca]].ns * ci[r->ca_cls[a.ca]].s > ci[r->ca_cls[b.ca]].ns * ci[r->ca_cls[b.ca]].s;
    });
    std::vector<tf::RgItem> items(pieces[ph].size());
    for (size_t i = 0; i < items.size(); ++i) items[i] = tf::RgItem{pieces[ph][i].ca, 0, pieces[ph][i].u0, pieces[ph][i].u1};
    r->num_items[ph] = (long long)items.size();
    const size_t bytes = std::max<size_t>(1, items.size()) * sizeof(tf::RgItem);
    ok = cudaMalloc((void**)&r->d_items[ph], bytes) == cudaSuccess &&
         cudaMemcpy(r->d_items[ph], items.data(), items.size() * sizeof(tf::RgItem), cudaMemcpyHostToDevice) ==
             cudaSuccess;
  }
  if (ok)
    ok = cudaMalloc((void**)&r->d_ctl, sizeof(tf::RgCtl)) == cudaSuccess &&
         cudaHostAlloc((void**)&r->h_ctl, sizeof(tf::RgCtl), cudaHostAllocDefault) == cudaSuccess &&
         cudaStreamCreateWithFlags(&r->cs, cudaStreamNonBlocking) == cudaSuccess;
  if (ok) memset(r->h_ctl, 0, sizeof(tf::RgCtl));
  p->rg = r;
  if (!ok) {
    cudaGetLastError();
    rg_free(p);
  }
  return ok;
}

// one exec on `s`: control block and reports cleared, the kernel, reports
// and control block copied to their host mirrors
turbofft_status rg_queue(turbofft_plan* p, const void* in, void* out, cudaStream_t s, bool with_sites) {
  RgState* r = static_cast<RgState*>(p->rg);
  tf::RgParams P;
  memset(&P, 0, sizeof(P));
  const tf::InjectSite none{};
  for (size_t i = 0; i < r->ca_cls.size(); ++i) {
    turbofft_plan* m = p->members[(size_t)r->ca_member[i]];
    const int pi = r->ca_pass[i];
    const void* pin = pi == 0 ? in : m->d_scratch;
    void* pout = (m->num_passes == 2 && pi == 0) ? m->d_scratch : out;
    fill_pass_args_f32(m, pi, pin, pout, with_sites ? m->armed : none, &P.ca[i].A);
    P.ca[i].A.num_units = r->ca_units[i];
    P.ca[i].cls = r->ca_cls[i];
    P.ca[i].phase = r->ca_phase[i];
  }
  P.num_ca = (int)r->ca_cls.size();
  P.num_phases = r->num_phases;
  for (int ph = 0; ph < 2; ++ph) {
    P.num_items[ph] = r->num_items[ph];
    P.items[ph] = r->d_items[ph];
  }
  P.ctl = r->d_ctl;
  cudaError_t e = cudaMemsetAsync(r->d_ctl, 0, sizeof(tf::RgCtl), s);
  const bool ft = p->ft_mode != TURBOFFT_FT_OFF;
  for (size_t k = 0; ft && e == cudaSuccess && k < p->members.size(); ++k)
    e = cudaMemsetAsync(p->members[k]->d_fts, 0, tf::FT_HEADER_BYTES, s);
  if (e == cudaSuccess) e = tf::launch_ragged_kernel(r->ftm, P, r->grid, r->smem, s);
  for (size_t k = 0; ft && e == cudaSuccess && k < p->members.size(); ++k)
    e = cudaMemcpyAsync(p->members[k]->h_fts, p->members[k]->d_fts, sizeof(FtState), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->h_ctl, r->d_ctl, sizeof(tf::RgCtl), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(p, e, "ragged persistent launch");
  return TURBOFFT_SUCCESS;
}

turbofft_status rg_exec(turbofft_plan* p, const void* in, void* out, cudaStream_t s) {
  RgState* r = static_cast<RgState*>(p->rg);
  if (p->armed_any) {
    // an armed site: the launch carries it (not the captured graph)
    p->armed_any = false;
    turbofft_status st = rg_queue(p, in, out, s, true);
    for (auto m : p->members) m->armed.active = 0;
    return st;
  }
  if (!r->graph || r->g_in != in || r->g_out != out) {
    if (r->graph) cudaGraphExecDestroy(r->graph);
    r->graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(r->cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(p, e, "graph capture");
    turbofft_status st = rg_queue(p, in, out, r->cs, false);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(r->cs, &g);
    if (st == TURBOFFT_SUCCESS && e == cudaSuccess) e = cudaGraphInstantiate(&r->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st != TURBOFFT_SUCCESS) return st;
    if (e != cudaSuccess) {
      r->graph = nullptr;
      return cuda_fail(p, e, "graph capture");
    }
    r->g_in = in;
    r->g_out = out;
  }
  cudaError_t e = cudaGraphLaunch(r->graph, s);
  if (e != cudaSuccess) return cuda_fail(p, e, "graph launch");
  return TURBOFFT_SUCCESS;
}

}  // namespace


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
  if (p->rg) {
    turbofft_status st = rg_exec(p, in, out, s);
    if (st != TURBOFFT_SUCCESS) return st;
  } else if (p->armed_any) {
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
  // one persistent launch for float32 lengths up to 2^16 (members with one
  // pass up to 4096, two passes above, as the kernel's size classes)
  bool single = g_ragged_single.load() != 0 && dtype == TURBOFFT_C2C_F32 &&
                (ft_mode == TURBOFFT_FT_OFF || ft_mode == TURBOFFT_FT_DETECT || ft_mode == TURBOFFT_FT_CORRECT);
  for (auto& g : groups) single = single && g.first <= (int64_t)1 << 16;
  t_ragged_member = true;
  turbofft_status st = TURBOFFT_SUCCESS;
  for (auto& g : groups) {
    turbofft_plan* m = nullptr;
    st = single ? create_plan(g.first, (int64_t)g.second.size(), dtype, direction, ft_mode, 5, &m)
                : turbofft_plan_create(g.first, (int64_t)g.second.size(), dtype, direction, ft_mode, &m);
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
  if (single) rg_setup(p);  // else (or if it cannot be set up) the graph of members
  *out = p;
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_set_ragged_single_launch(int enable) {
  g_ragged_single.store(enable ? 1 : 0);
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_plan_get_member_info(const turbofft_plan* p, int32_t index, turbofft_plan_info* info) {
  if (!p || !info || !p->ragged || index < 0 || index >= (int32_t)p->members.size()) return TURBOFFT_INVALID_VALUE;
  fill_info(p->members[(size_t)index], info);
  return TURBOFFT_SUCCESS;
}

}  // extern "C"
