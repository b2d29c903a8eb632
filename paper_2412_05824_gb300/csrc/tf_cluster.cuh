// Single-pass transforms of length N = N1 * N2 spread over a thread-block
// cluster (one HBM round trip where one block's shared memory cannot hold
// a whole transform).
//
// The four-step split of the kernel-level tiling (Sec. 3.1) runs inside one
// kernel: C blocks of a cluster share each transform.
//   phase A: block r of the cluster loads columns n2 in [r*SA, (r+1)*SA) of
//            the N1 x N2 row-major input (SA contiguous values per row),
//            transforms them (length N1, slot-fast like the column pass)
//            and multiplies by w_N^{k1 n2};
//   exchange: each value A[k1][n2] is stored into the shared memory of the
//            block that owns row k1 in phase B (distributed shared memory,
//            between two cluster barriers);
//   phase B: block r holds rows k1 in [r*SB, (r+1)*SB), transforms them
//            (length N2) and stores y[k2 * N1 + k1] through shared memory so
//            that the SB adjacent rows leave as contiguous runs.
// Each block keeps a two-sided checksum of its own columns (phase A, with the
// output weights e_k conj(w) after the twiddle, as in the two-pass plan) and
// rows (phase B), summed over the block, per transform, with the location
// encoding over the transforms of its group (Sec. 4.1, 4.3).  A detected
// group is repaired on the rare path by recomputing its transforms from the
// untouched input (tf_cl_fix_kernel).
#pragma once

#include <cooperative_groups.h>

#include "tf_device.cuh"

namespace tf {

namespace cg = cooperative_groups;

// KA: column configuration (KIND_COL, S = SA columns per block);
// KB: row configuration (KIND_ROW, S = SB rows per block).
template <class KA_, class KB_> struct ClCfg {
  using KA = KA_;
  using KB = KB_;
  using real = typename KA::real;
  using c = typename KA::c;
  static constexpr int N1 = KA::NS, N2 = KB::NS;
  static constexpr int SA = KA::S, SB = KB::S;
  static constexpr int C = N2 / SA;            // blocks per cluster
  static constexpr int NT = KA::NT;
  static constexpr int SLICE = N1 * SA;        // values per block
  static constexpr long long N = (long long)N1 * N2;
  static constexpr int STAGE_BYTES = (SLICE * (int)sizeof(c) + 127) / 128 * 128;
  static constexpr int TAB_BYTES = 2 * (N1 + N2) * (int)sizeof(c);  // e and v of both phases
  // inter-phase twiddles w_N^{k1 n2} of every thread's E values: the block's
  // columns never change, so they are formed once per block
  static constexpr int TW_BYTES = STAGE_BYTES;
  // energy weights: tau^2 = (gamma u)^2 (N1 log2 N1 E_A + N2 log2 N2 E_B)
  static constexpr double WA = (double)N1 * KA::LOG_NS, WB = (double)N2 * KB::LOG_NS;
  static_assert(KA::KIND == KIND_COL && KB::KIND == KIND_ROW, "column then row configuration");
  static_assert(sizeof(typename KB::c) == sizeof(c), "one precision");
  static_assert(KA::NT == KB::NT, "both phases use every thread");
  static_assert(N2 % SA == 0 && N1 % SB == 0 && N1 / SB == C, "the cluster splits columns and rows alike");
  static_assert(C >= 2 && C <= 8, "portable cluster size");
  static_assert(SA * (int)sizeof(c) % 16 == 0, "16-byte runs per row");
  // resident blocks per SM the register allocation must allow (128 registers
  // per thread at 512 threads per SM)
  static constexpr int MINB = NT >= 512 ? 1 : 512 / NT;
};

// 32-bit shared::cluster address of `p` (this block's shared memory) in
// block `rank` of the cluster, and a store through it
__device__ __forceinline__ unsigned dsmem_map(const void* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void dsmem_store(unsigned addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};\n" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void dsmem_store(unsigned addr, double2 v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};\n" ::"r"(addr), "d"(v.x), "d"(v.y) : "memory");
}
// cluster barrier halves: a relaxed arrive orders nothing (enough when the
// barrier only says "my reads of my buffer are done": those values are
// already in registers); a release arrive makes this thread's prior stores
// (the distributed shared-memory exchange) visible to the cluster, and the
// acquire wait makes the others' visible here
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

template <typename R> struct ClArgs {
  using c = typename CT<R>::c;
  PassArgs<R> p;  // phase A tables (tw, ev, vv), inter-pass twiddles, geometry, flags, fault tolerance
  const c* twB;   // phase B tables
  const c* evB;
  const c* vvB;
};

template <class CL> constexpr int cl_smem_bytes(int ftm) {
  return 2 * CL::STAGE_BYTES + CL::TW_BYTES + (ftm ? CL::TAB_BYTES : 0);
}

// copies of transform `unit`'s phase-A tile (N1 rows x SA columns) of block
// `rank` into `stage`, position-major [n1][column]
template <class CL>
__device__ __forceinline__ void cl_issue(const ClArgs<typename CL::real>& A, long long unit, int rank, char* stage,
                                         int tid) {
  using c = typename CL::c;
  constexpr int cpr = CL::SA * (int)sizeof(c) / 16;  // 16-byte chunks per row
  constexpr int chunks = CL::N1 * cpr;
  const c* base = A.p.in + tr_base(A.p.geo.in_tab, unit, CL::N) + rank * CL::SA;
  for (int q = tid; q < chunks; q += CL::NT) {
    const int row = q / cpr, j = q - row * cpr;
    cp_async16(stage + (size_t)row * CL::SA * sizeof(c) + 16 * j,
               reinterpret_cast<const char*>(base + (long long)row * CL::N2) + 16 * j);
  }
}

// per-thread outcome of one transform's slice
template <typename R> struct ClRes {
  R rr, ri;  // (e.y - v.x) summed over both phases' signals of this thread
  R en;      // weighted energy (WA |x_A|^2 + WB |x_B|^2)
  bool finite;
};

// Transform `unit`'s slice, staged in `sm`, through both phases and the
// exchange; stores the output.  Every block of the cluster must call it for
// the same unit (two cluster barriers inside).
template <class CL, bool FT, class TWA, class TWB>
__device__ __forceinline__ void cl_body(const ClArgs<typename CL::real>& A, long long unit, int rank,
                                        typename CL::c* sm, const TWA& twa, const TWB& twb,
                                        const typename CL::c* twc, const typename CL::c* evA, const typename CL::c* vvA,
                                        const typename CL::c* evB, const typename CL::c* vvB,
                                        const InjectSite& inj, cg::cluster_group& cluster,
                                        ClRes<typename CL::real>& res) {
  using KA = typename CL::KA;
  using KB = typename CL::KB;
  using R = typename CL::real;
  using c = typename CL::c;
  constexpr int E = KA::E, PA = KA::P, SA = CL::SA, PB = KB::P, SB = CL::SB, N1 = CL::N1, N2 = CL::N2;
  const int tid = threadIdx.x;
  const int slotA = tid % SA, tA = tid / SA;  // phase A: column slotA, positions tA + i*PA
  const int slotB = tid / PB, tB = tid % PB;  // phase B: row slotB, positions tB + i*PB
  const int n2 = rank * SA + slotA;
  const int k1b = rank * SB + slotB;
  const unsigned long long mask_in = sign_mask<c>(A.p.conj_in), mask_out = sign_mask<c>(A.p.conj_out);
  res.rr = res.ri = res.en = 0;
  res.finite = true;

  // ---- phase A: columns
  c a[E];
#pragma unroll
  for (int i = 0; i < E; ++i) a[i] = conj_mask(sm[(tA + i * PA) * SA + slotA], mask_in);
  __syncthreads();  // the tile is consumed; the stage becomes the exchange buffer
  c pin = mk<c>(0, 0), pout = mk<c>(0, 0);
  R en = 0;
  if constexpr (FT) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      cmac(pin, vvA[tA + i * PA], a[i]);
      en = fma(a[i].x, a[i].x, en);
      en = fma(a[i].y, a[i].y, en);
    }
  }
  {
    InjCtx ic{false, 0, 0, 0, 0};
    if (inj.active && inj.pass == 0 && inj.signal == unit * N2 + n2) {
      ic.on = true;
      ic.stage = inj.stage;
      ic.pos = inj.pos;
      ic.comp = inj.comp;
      ic.bit = inj.bit;
    }
    Passes<KA, 0>::run(a, sm, twa, slotA, tA, ic);
  }
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int k1 = tA + i * PA;
    const c w = twc[i * CL::NT + tid];
    a[i] = cmul(a[i], w);
    if constexpr (FT) cmac(pout, cmulconj(evA[k1], w), a[i]);
  }
  if constexpr (FT) {
    res.rr = pout.x - pin.x;
    res.ri = pout.y - pin.y;
    res.en = (R)CL::WA * en;
  }

  // ---- exchange: A[k1][n2] -> row k1 % SB of block k1 / SB.  Rows are
  // stored with the columns XOR-swizzled by (row % RPW) * PB so that the
  // RPW rows one warp reads in phase B fall on different banks
  constexpr int RPW = (PB * (int)sizeof(c) < 128) ? 32 / PB : 1;
  cluster_arrive_relaxed();  // every block has finished phase A with its stage
  cluster_wait_acquire();
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int k1 = tA + i * PA;
    const int r = k1 % SB;
    dsmem_store(dsmem_map(sm + r * N2 + (n2 ^ ((r % RPW) * PB)), (unsigned)(k1 / SB)), a[i]);
  }
  cluster_arrive_release();  // every value of this block's rows has arrived
  cluster_wait_acquire();

  // ---- phase B: rows
#pragma unroll
  for (int i = 0; i < E; ++i) a[i] = sm[slotB * N2 + ((tB + i * PB) ^ ((slotB % RPW) * PB))];
  __syncthreads();
  pin = mk<c>(0, 0);
  pout = mk<c>(0, 0);
  en = 0;
  if constexpr (FT) {
#pragma unroll
    for (int i = 0; i < E; ++i) {
      cmac(pin, vvB[tB + i * PB], a[i]);
      en = fma(a[i].x, a[i].x, en);
      en = fma(a[i].y, a[i].y, en);
    }
  }
  {
    InjCtx ic{false, 0, 0, 0, 0};
    if (inj.active && inj.pass == 1 && inj.signal == unit * N1 + k1b) {
      ic.on = true;
      ic.stage = inj.stage;
      ic.pos = inj.pos;
      ic.comp = inj.comp;
      ic.bit = inj.bit;
    }
    Passes<KB, 0>::run(a, sm, twb, slotB, tB, ic);
  }
  if constexpr (FT) {
#pragma unroll
    for (int i = 0; i < E; ++i) cmac(pout, evB[tB + i * PB], a[i]);
    res.rr += pout.x - pin.x;
    res.ri += pout.y - pin.y;
    res.en += (R)CL::WB * en;
    res.finite = isfinite(res.rr) && isfinite(res.ri);
  }
  if (A.p.out_scale != (R)1) {
#pragma unroll
    for (int i = 0; i < E; ++i) a[i] = cscale(a[i], A.p.out_scale);
  }
  // ---- transposed store: for each k2 the block's SB rows are contiguous
#pragma unroll
  for (int i = 0; i < E; ++i) sm[slotB * N2 + ((tB + i * PB) ^ tsw<KB>(slotB))] = a[i];
  __syncthreads();
  {
    const int s2 = tid % SB, t2 = tid / SB;
    c* const ob = A.p.out + tr_base(A.p.geo.out_tab, unit, CL::N) + rank * SB + s2;
#pragma unroll
    for (int i = 0; i < E; ++i) {
      const int k2 = t2 + i * PB;
      const c v = conj_mask(sm[s2 * N2 + (k2 ^ tsw<KB>(s2))], mask_out);
      __stcs(ob + (long long)k2 * N1, v);
    }
  }
  __syncthreads();
}

// this thread's inter-phase twiddles w_N^{k1 n2}, k1 = tA + i PA, into
// tw[i * NT + tid] (each thread reads back only its own entries)
template <class CL>
__device__ __forceinline__ const typename CL::c* cl_twiddles(const ClArgs<typename CL::real>& A, int rank,
                                                             typename CL::c* tw) {
  const int tid = threadIdx.x;
  const int n2 = rank * CL::SA + tid % CL::SA, tA = tid / CL::SA;
#pragma unroll
  for (int i = 0; i < CL::KA::E; ++i) {
    const unsigned q = (unsigned)(tA + i * CL::KA::P) * (unsigned)n2;
    tw[i * CL::NT + tid] = cmul(ldg(A.p.thi + (q >> 12)), ldg(A.p.tlo + (q & 4095u)));
  }
  return tw;
}

// block-wide sums in double (thread 0 gets the totals)
__device__ __forceinline__ void cl_block_sum(double* red, int nt, double (&v)[5], int& lo, int& hi) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  __syncthreads();
  if ((tid & 31) == 0) {
    double* d = red + (tid >> 5) * 8;
#pragma unroll
    for (int k = 0; k < 5; ++k) d[k] = v[k];
    d[5] = (double)lo;
    d[6] = (double)hi;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = 0;
    lo = 0x7fffffff;
    hi = -1;
    for (int w = 0; w < nt / 32; ++w) {
      const double* d = red + w * 8;
#pragma unroll
      for (int k = 0; k < 5; ++k) v[k] += d[k];
      lo = min(lo, (int)d[5]);
      hi = max(hi, (int)d[6]);
    }
  }
  __syncthreads();
}

// checksum tables of both phases into shared memory
template <class CL>
__device__ __forceinline__ void cl_tables(const ClArgs<typename CL::real>& A, typename CL::c* tab) {
  for (int q = threadIdx.x; q < CL::N1; q += CL::NT) {
    tab[q] = A.p.ev[q];
    tab[CL::N1 + q] = A.p.vv[q];
  }
  for (int q = threadIdx.x; q < CL::N2; q += CL::NT) {
    tab[2 * CL::N1 + q] = A.evB[q];
    tab[2 * CL::N1 + CL::N2 + q] = A.vvB[q];
  }
  __syncthreads();
}

template <class CL> constexpr int cl_tw_budget() { return 32; }

// ---------------------------------------------------------------------------
// the cluster transform kernel: persistent clusters, transform `unit` =
// cluster id + k * clusters; its input tile is copied one transform ahead
// FTM: 0 = no checksums, 1 = checksums
// ---------------------------------------------------------------------------
template <class CL, int FTM>
__global__ void __launch_bounds__(CL::NT, CL::MINB) tf_cl_kernel(const ClArgs<typename CL::real> A) {
  using KA = typename CL::KA;
  using KB = typename CL::KB;
  using R = typename CL::real;
  using c = typename CL::c;
  constexpr bool FT = FTM != 0;
  extern __shared__ __align__(128) unsigned char smem_raw_[];
  char* smem = reinterpret_cast<char*>(smem_raw_);
  __shared__ double red[32 * 8];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const long long ncl = gridDim.x / CL::C;
  const long long cid = blockIdx.x / CL::C;
  const int tid = threadIdx.x;

  TwReg<KA, cl_tw_budget<CL>()> twa;
  twa.load(A.p.tw, tid / CL::SA);
  TwReg<KB, cl_tw_budget<CL>()> twb;
  twb.load(A.twB, tid % KB::P);
  c* tab = reinterpret_cast<c*>(smem + 2 * CL::STAGE_BYTES + CL::TW_BYTES);
  const c* twc = cl_twiddles<CL>(A, rank, reinterpret_cast<c*>(smem + 2 * CL::STAGE_BYTES));
  if constexpr (FT) cl_tables<CL>(A, tab);
  const c* evA = tab;
  const c* vvA = tab + CL::N1;
  const c* evB = tab + 2 * CL::N1;
  const c* vvB = tab + 2 * CL::N1 + CL::N2;

  R s1r = 0, s1i = 0, s2r = 0, s2i = 0, en = 0;
  int bad_lo = 0x7fffffff, bad_hi = -1;
  int gi = 0;
  long long g_unit0 = cid;
  long long groups = 0;
  float max_ratio = 0.f;

  if (cid < A.p.num_units) cl_issue<CL>(A, cid, rank, smem, tid);
  cp_async_commit();
  int it = 0;
  for (long long unit = cid; unit < A.p.num_units; unit += ncl, ++it) {
    {
      const long long un = unit + ncl;
      if (un < A.p.num_units) cl_issue<CL>(A, un, rank, smem + ((it + 1) & 1) * CL::STAGE_BYTES, tid);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
    }
    c* sm = reinterpret_cast<c*>(smem + (it & 1) * CL::STAGE_BYTES);
    ClRes<R> rs;
    cl_body<CL, FT>(A, unit, rank, sm, twa, twb, twc, evA, vvA, evB, vvB, A.p.inj, cluster, rs);
    if constexpr (FT) {
      if (!rs.finite) {
        bad_lo = min(bad_lo, gi);
        bad_hi = max(bad_hi, gi);
      }
      s1r += rs.rr;
      s1i += rs.ri;
      s2r += (R)(gi + 1) * rs.rr;
      s2i += (R)(gi + 1) * rs.ri;
      en += rs.en;
    }
    ++gi;
    const bool group_end = (gi == A.p.T) || (unit + ncl >= A.p.num_units);
    if constexpr (FT) {
      if (group_end) {
        double v[5] = {(double)s1r, (double)s1i, (double)s2r, (double)s2i, (double)en};
        int lo = bad_lo, hi = bad_hi;
        cl_block_sum(red, CL::NT, v, lo, hi);
        if (tid == 0) {
          const double S1r = v[0], S1i = v[1], S2r = v[2], S2i = v[3], EN = v[4];
          const double tau = A.p.tau_coef * sqrt(EN);
          const double mag = sqrt(S1r * S1r + S1i * S1i);
          const bool finite = isfinite(S1r) && isfinite(S1i) && isfinite(EN);
          if (finite && mag <= tau) {
            if (tau > 0) max_ratio = fmaxf(max_ratio, (float)(mag / tau));
          } else {
            int located = -1;
            if (hi >= 0) {
              located = (lo == hi) ? lo : -2;
            } else if (isfinite(S1r) && isfinite(S1i)) {
              // (an overflowed energy does not stop the location: a fault
              // upstream in the cluster can push the phase-B inputs of every
              // block beyond the float32 range of |x|^2)
              const double den = S1r * S1r + S1i * S1i;
              const double qr = (S2r * S1r + S2i * S1i) / den, qi = (S2i * S1r - S2r * S1i) / den;
              const double kk = floor(qr + 0.5);
              if (isfinite(qr) && isfinite(qi) && kk >= 1 && kk <= gi &&
                  sqrt((qr - kk) * (qr - kk) + qi * qi) < 0.25)
                located = (int)kk - 1;
            }
            atomicAdd(&A.p.fts->detected, 1ull);
            const unsigned long long r = atomicAdd(&A.p.fts->num_records, 1ull);
            if (r < (unsigned long long)MAX_RECORDS) {
              FtRecord& R0 = A.p.fts->rec[r];
              R0.pass_id = 0;
              R0.slot = rank;
              R0.count = gi;
              R0.located = located;
              R0.unit0 = g_unit0;
              R0.unit_stride = ncl;
              R0.transform_base = A.p.transform_base;
              R0.s1r = S1r; R0.s1i = S1i; R0.s2r = S2r; R0.s2i = S2i;
              R0.tau = tau;
              R0.energy = EN;
              R0.result = FT_RES_PENDING;
              R0.has_sums = 0;
              R0.signal = -1;
            } else {
              atomicAdd(&A.p.fts->dropped, 1ull);
            }
          }
        }
        ++groups;
        s1r = s1i = s2r = s2i = en = 0;
        bad_lo = 0x7fffffff;
        bad_hi = -1;
      }
    }
    if (group_end) {
      gi = 0;
      g_unit0 = unit + ncl;
    }
  }
  if constexpr (FT) {
    if (tid == 0 && groups > 0) {
      atomicAdd(&A.p.fts->groups, (unsigned long long)groups);
      if (max_ratio > 0.f) atomic_max_nonneg(&A.p.fts->max_clean_ratio, max_ratio);
    }
  }
}

// ---------------------------------------------------------------------------
// rare path: one cluster walks the records of the exec.  A located or
// ambiguous group is repaired by recomputing each of its transforms from the
// untouched input (the right-side correction Delta = y_bar - W x_bar would
// itself need a full-length transform of x_bar); every recomputed slice is
// checked again and a failing one makes the group uncorrectable.  DETECT
// mode only reports.
// ---------------------------------------------------------------------------
template <class CL>
__global__ void __launch_bounds__(CL::NT, CL::MINB) tf_cl_fix_kernel(const ClArgs<typename CL::real> A) {
  using KA = typename CL::KA;
  using KB = typename CL::KB;
  using R = typename CL::real;
  using c = typename CL::c;
  extern __shared__ __align__(128) unsigned char smem_raw_[];
  char* smem = reinterpret_cast<char*>(smem_raw_);
  __shared__ double red[32 * 8];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x;
  FtState* fs = A.p.fts;
  const int nrec = (int)min((unsigned long long)MAX_RECORDS, fs->num_records);
  if (nrec == 0) return;  // uniform over the cluster: no barrier is skipped by some blocks only
  TwReg<KA, cl_tw_budget<CL>()> twa;
  twa.load(A.p.tw, tid / CL::SA);
  TwReg<KB, cl_tw_budget<CL>()> twb;
  twb.load(A.twB, tid % KB::P);
  c* tab = reinterpret_cast<c*>(smem + 2 * CL::STAGE_BYTES + CL::TW_BYTES);
  const c* twc = cl_twiddles<CL>(A, rank, reinterpret_cast<c*>(smem + 2 * CL::STAGE_BYTES));
  cl_tables<CL>(A, tab);
  const InjectSite none{};
  c* sm = reinterpret_cast<c*>(smem);
  // every record of this exec is pending (the transform kernel wrote them);
  // each block walks all of them, so the cluster barriers stay paired
  for (int r = 0; r < nrec; ++r) {
    FtRecord& rc = fs->rec[r];
    // several blocks of one cluster may flag the same group (a fault in one
    // block's phase A reaches every block's phase B): the first record of a
    // group repairs it, the others are settled with it
    int first = r;
    for (int q = 0; q < r; ++q)
      if (fs->rec[q].unit0 == rc.unit0) {
        first = q;
        break;
      }
    if (first != r) {
      if (rank == 0 && tid == 0) {
        rc.signal = fs->rec[first].signal;
        rc.result = FT_RES_CLEAR;
      }
      continue;
    }
    if (A.p.ft == FT_CORRECT) {
      for (int j = 0; j < rc.count; ++j) {
        const long long unit = rc.unit0 + (long long)j * rc.unit_stride;
        cl_issue<CL>(A, unit, rank, smem, tid);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        ClRes<R> rs;
        cl_body<CL, true>(A, unit, rank, sm, twa, twb, twc, tab, tab + CL::N1, tab + 2 * CL::N1,
                          tab + 2 * CL::N1 + CL::N2, none, cluster, rs);
        double v[5] = {(double)rs.rr, (double)rs.ri, 0.0, 0.0, (double)rs.en};
        int lo = rs.finite ? 0x7fffffff : 0, hi = rs.finite ? -1 : 0;
        cl_block_sum(red, CL::NT, v, lo, hi);
        if (tid == 0) {
          const double tau = A.p.tau_coef * sqrt(v[4]);
          const double mag = sqrt(v[0] * v[0] + v[1] * v[1]);
          if (hi >= 0 || !(mag <= tau)) atomicMax(&rc.result, (int)FT_RES_UNCORRECTABLE);
        }
      }
    }
    __threadfence();
    cluster.sync();
    if (rank == 0 && tid == 0) {
      int loc = rc.located;  // or the location another block of the cluster found
      for (int q = r + 1; q < nrec && loc < 0; ++q)
        if (fs->rec[q].unit0 == rc.unit0 && fs->rec[q].located >= 0) loc = fs->rec[q].located;
      if (loc >= 0) atomicAdd(&fs->located, 1ull);
      rc.signal = loc >= 0 ? rc.unit0 + (long long)loc * rc.unit_stride : -1;
      if (A.p.ft != FT_CORRECT) {
        rc.result = loc >= 0 ? FT_RES_LOCATED : FT_RES_UNCORRECTABLE;
      } else if (rc.result == FT_RES_UNCORRECTABLE) {
        atomicAdd(&fs->uncorrectable, 1ull);
      } else {
        rc.result = FT_RES_RECOMPUTE;
        atomicAdd(&fs->corrected, 1ull);
        atomicAdd(&fs->recomputed, 1ull);
      }
    }
    cluster.sync();  // the record's outcome is settled before any block reads the next
  }
}

}  // namespace tf
