// Host side of the C ABI declared in include/turbofft.h: plan creation
// (pass split, launch shapes, tables), destruction, injection, reports,
// settings.  Launches live in tf_launch.cu, ragged plans in tf_ragged.cu,
// the autotuner in tf_autotune.cu, host tables in tf_tables.cu.
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
      int64_t tr = (m->cl || m->tchk) ? rc.signal : rc.signal / signals_per_transform(m, rc.pass_id);
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
    info->single_launch = p->rg ? 1 : 0;
    for (auto m : p->members) {
      info->workspace_bytes += m->workspace_bytes + (m->scratch_owned ? 0 : (int64_t)m->scratch_bytes);
      info->autotuned |= m->autotuned ? 1 : 0;
    }
    return;
  }
  info->num_passes = p->num_passes;
  info->transform_checks = p->tchk ? 1 : 0;
  info->tma_passes = p->tma_mask;
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

turbofft_status create_plan(int64_t n, int64_t batch, turbofft_dtype dtype, int direction,
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
      ft_mode != TURBOFFT_FT_CORRECT_REGISTERS && ft_mode != TURBOFFT_FT_CORRECT_THREAD)
    return TURBOFFT_INVALID_VALUE;
  // thread-level checksums need one thread per whole transform: single-pass
  // sizes only, and not inside a ragged plan
  if (ft_mode == TURBOFFT_FT_CORRECT_THREAD && (structure == 2 || structure == 3 || t_ragged_member))
    return TURBOFFT_UNSUPPORTED;
  // float-pair arithmetic: float64 data, no checksums (its rounding is above
  // the float64 detection threshold), not inside a ragged plan
  const bool pairs = structure == TURBOFFT_STRUCTURE_FLOAT_PAIRS;
  if (pairs && (dtype != TURBOFFT_C2C_F64 || ft_mode != TURBOFFT_FT_OFF || t_ragged_member))
    return TURBOFFT_UNSUPPORTED;

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
  p->pairs = pairs;
  const int dt = kernel_dtype(p);

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
  } else if (n <= reg.max_sp(dt) && !(structure == 5 && n > 4096)) {
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
  // float64 two-pass plans with checksums check whole transforms
  p->tchk = dt == 1 && p->num_passes == 2 && !p->cl && !t_ragged_member &&
            (ft_mode == TURBOFFT_FT_DETECT || ft_mode == TURBOFFT_FT_CORRECT);
  for (int pi = 0; pi < p->num_passes && !p->cl; ++pi) {
    PassPlan& pp = p->pass[pi];
    pp.ke = reg.find_variant(dt, pp.kind, pp.ns, plan_variant(p));
    if (!pp.ke) {
      turbofft_destroy(p);
      return TURBOFFT_UNSUPPORTED;
    }
    if (!set_smem_attrs(pp.ke)) {
      cudaGetLastError();
      turbofft_destroy(p);
      return TURBOFFT_CUDA_ERROR;
    }
    const int occ = occupancy_blocks(pp.ke, plan_variant(p));
    pp.grid = occ * g_num_sms;
    pp.tau_coef = kGamma[dt] * kUnitRoundoff[dt] * sqrt((double)ilog2_exact(pp.ns));
    if (ft_mode == TURBOFFT_FT_CORRECT_THREAD) pp.tau_coef *= kThreadLevelGammaFactor;
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
      ok = (dt == 0)   ? (upload<float>(p, lo_dst, lo) && upload<float>(p, hi_dst, hi))
           : (dt == 2) ? (upload_pairs(p, lo_dst, lo) && upload_pairs(p, hi_dst, hi))
                       : (upload<double>(p, lo_dst, lo) && upload<double>(p, hi_dst, hi));
      if (ok && dt == 1 && !p->cl) ok = col_tables(p, p->pass[pi], ft_mode != TURBOFFT_FT_OFF && !p->tchk);
    }
    p->scratch_bytes = p->cl ? 0 : (size_t)(batch * n) * elem_bytes(dtype);
    if (ok && p->tchk) {
      void* acc = nullptr;
      ok = tc_tables(p) && dev_alloc(p, &acc, (size_t)batch * 6 * sizeof(double));
      p->d_tacc = static_cast<double*>(acc);
    }
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
  // float32 one- and two-pass plans may stage their tiles with TMA copies:
  // always (mode 2) or where that measured faster than cp.async on GB300
  // (mode 1, tma_faster); the kernels' timeout flag
  p->tma_mask = 0;
  if (dt == 0 && p->num_passes <= 2 && !p->cl && !t_ragged_member) {
    const int mode = g_tma_staging.load();
    for (int pi = 0; pi < p->num_passes; ++pi) {
      const KernelEntry* ke = p->pass[pi].ke;
      if (ke && ke->main_tma[0] && (mode == 2 || (mode == 1 && tma_faster(ke, ft_mode))))
        p->tma_mask |= 1 << pi;
    }
  }
  if (p->tma_mask) {
    if (p->d_fts) {
      p->d_err = &p->d_fts->error;
    } else {
      void* e = nullptr;
      if (!dev_alloc(p, &e, 16) || cudaMemset(e, 0, 16) != cudaSuccess) {
        cudaGetLastError();
        turbofft_destroy(p);
        return TURBOFFT_ALLOC_FAILED;
      }
      p->d_err = static_cast<int*>(e);
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

}  // namespace tfh

using namespace tfh;

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
  rg_free(p);
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

turbofft_status turbofft_plan_create_structured(int64_t n, int64_t batch, turbofft_dtype dtype, int direction,
                                                turbofft_ft_mode ft_mode, int structure, turbofft_plan** out) {
  if (out) *out = nullptr;
  if (structure != TURBOFFT_STRUCTURE_SPLIT && structure != TURBOFFT_STRUCTURE_CLUSTER &&
      structure != TURBOFFT_STRUCTURE_THREE_PASS && structure != TURBOFFT_STRUCTURE_FLOAT_PAIRS)
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

turbofft_status turbofft_plan_get_info(const turbofft_plan* p, turbofft_plan_info* info) {
  if (!p || !info) return TURBOFFT_INVALID_VALUE;
  fill_info(p, info);
  return TURBOFFT_SUCCESS;
}

turbofft_status turbofft_set_tma_staging(int mode) {
  if (mode < 0 || mode > 2) return TURBOFFT_INVALID_VALUE;
  g_tma_staging.store(mode);
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
  if (p->rg && p->have_exec) {
    // one-launch ragged exec: a grid barrier that gave up waiting
    cudaError_t e = cudaEventSynchronize(p->done);
    if (e != cudaSuccess) return cuda_fail(p, e, "report wait");
    if (rg_timed_out(p)) {
      p->last_error = "ragged persistent kernel: grid barrier timed out";
      return TURBOFFT_TIMEOUT;
    }
  }
  if (p->tma_mask && p->have_exec) {
    // TMA-staged pass: a tile copy that never completed
    cudaError_t e = cudaEventSynchronize(p->done);
    if (e != cudaSuccess) return cuda_fail(p, e, "report wait");
    int err = 0;
    if (p->ft_mode != TURBOFFT_FT_OFF) {
      err = p->h_fts->error;
    } else if ((e = cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) {
      return cuda_fail(p, e, "report read");
    }
    if (err) {
      p->last_error = "a TMA tile copy did not complete in time";
      return TURBOFFT_TIMEOUT;
    }
  }
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
