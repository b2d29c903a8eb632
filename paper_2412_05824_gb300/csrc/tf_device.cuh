// Device code of the batched complex FFT with fused two-sided ABFT.
//
// Transform (TurboFFT Sec. 2.2.1 definition; Sec. 3.1 tiling; Sec. 3.2
// Stockham autosort with a padding-free, swizzled shared-memory exchange):
//   A length-NS sub-transform is held by P = NS/E threads, E complex values
//   per thread in registers.  Thread t always holds the "home" positions
//   t + i*P, i < E.  The transform runs as Stockham radix passes; pass p has
//   radix R (E, or a smaller radix for the last pass) and sub-transform
//   length L = E^p before it.  In pass p thread t computes E/R butterflies
//   j = t + u*P: inputs X[j + m*NS/R] (exactly its home registers),
//   twiddle w_{L*R}^{(j mod L)*m}, a radix-R DFT in registers, outputs to
//   Y[(j div L)*L*R + (j mod L) + m*L].  Every pass but the last writes Y to
//   shared memory and reads its home positions back; the last pass's
//   outputs land in the thread's own home registers.
//
// Kernel kinds:
//   KIND_SP   one pass over HBM, S whole transforms per transaction
//   KIND_COL  first pass of the four-step plan N = N1*N2: S adjacent
//             columns (stride N2) per transaction, length-N1 FFTs, then the
//             inter-pass twiddle w_N^{k1*n2}
//   KIND_ROW  second pass: S adjacent rows (contiguous) per transaction,
//             length-N2 FFTs, transposed store y[k1 + N1*k2] through shared
//             memory so that global stores stay coalesced
//
// Fault tolerance (TurboFFT Sec. 4.1-4.3), per thread block, per slot:
//   a checksum group is the T consecutive transactions a block processes;
//   per transaction each thread accumulates its share of
//       r = e . y_hat - v . x       (left checksum, v = W^T e, Eq. 1-2)
//   into S1 += r and S2 += (g+1) r  (location encoding, Sec. 4.1 / 4.3)
//   and the right-side sums x_bar += x, y_bar += y_hat (Eq. 4-5).  At the
//   end of a group the block reduces S1, S2 and the input energy (warp
//   shuffles in the working precision, cross-warp in float64), compares
//   |S1| with tau = gamma u sqrt(log2 NS) sqrt(NS * energy) in float64 and,
//   on a mismatch, appends a record (location and right-side sums) that the
//   correction kernel consumes right after this pass (delayed, batched
//   correction, Sec. 4.1.2).
#pragma once

#include <cuda.h>  // CUtensorMap (the tensor-map type of TMA copies)
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "tf_dd.cuh"
#include "tf_dft_constants.h"
#include "tf_types.h"

namespace tf {

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename R> struct CT;
template <> struct CT<float> { using c = float2; };
template <> struct CT<double> { using c = double2; };
template <> struct CT<dd> { using c = cdd; };  // float64 data in float-pair arithmetic

template <typename C> __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// float32 complex add / subtract as one paired FP32 instruction each
// (sm_100+ FADD2: two independent round-to-nearest additions, the same
// results as the scalar code)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulconj(C a, C b) {
  return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// conjugation as an integer sign flip of the imaginary part under a mask
// (0 or the sign bit), so that no floating-point pipe is used for it
__device__ __forceinline__ float2 conj_mask(float2 v, unsigned long long m) {
  return make_float2(v.x, __uint_as_float(__float_as_uint(v.y) ^ (unsigned)m));
}
__device__ __forceinline__ double2 conj_mask(double2 v, unsigned long long m) {
  return make_double2(v.x, __longlong_as_double(__double_as_longlong(v.y) ^ (long long)m));
}
__device__ __forceinline__ cdd conj_mask(cdd v, unsigned long long m) {
  const unsigned f = m ? 0x80000000u : 0u;
  return cdd{v.x, dd(__uint_as_float(__float_as_uint(v.y.hi) ^ f), __uint_as_float(__float_as_uint(v.y.lo) ^ f))};
}
// |v| 2^-down of a double as a float built with integer operations from its
// exponent and top 20 mantissa bits (relative error < 2^-20): for the energy
// that only scales the checksum threshold.  Exponents below the float range
// give 0 or a subnormal, above it the float exponent 254 (the callers keep a
// second sum with down = 64 for sums that overflow).
__device__ __forceinline__ float abs_as_float(double v, int down = 0) {
  const int hi = __double2hiint(v);
  int fe = ((hi >> 20) & 0x7FF) - 1023 + 127 - down;
  fe = fe < 0 ? 0 : (fe > 254 ? 254 : fe);
  return __uint_as_float(((unsigned)fe << 23) | (((unsigned)hi & 0xFFFFFu) << 3));
}

// Power-of-two scaling of a double by integer operations.  For s = 2^-k,
// v * s only lowers the exponent field by k when the result stays normal,
// and a zero stays the same; pow2_scalable says whether v is such a value
// (then pow2_scale gives bit for bit the floating-point product), else
// (subnormal result, infinity, NaN) the caller multiplies.
__device__ __forceinline__ int scaled_exponent_shift(double s) {
  return 1023 - ((__double2hiint(s) >> 20) & 0x7FF);
}
__device__ __forceinline__ bool pow2_scalable(double v, int k) {
  const int hi = __double2hiint(v);
  const int ex = (hi >> 20) & 0x7FF;
  return (ex > k && ex < 0x7FF) || ((hi & 0x7FFFFFFF) | __double2loint(v)) == 0;
}
__device__ __forceinline__ double pow2_scale(double v, int k) {
  const int hi = __double2hiint(v);
  return ((hi >> 20) & 0x7FF) == 0 ? v : __hiloint2double(hi - (k << 20), __double2loint(v));
}

template <typename C> __device__ __forceinline__ unsigned long long sign_mask(int on) {
  return on ? (sizeof(decltype(C::x)) == 4 ? 0x80000000ull : 0x8000000000000000ull) : 0ull;
}
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// acc += a*b as four chained fused multiply-adds
template <typename C> __device__ __forceinline__ void cmac(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

template <typename C> __device__ __forceinline__ C ldg(const C* p) { return __ldg(p); }
__device__ __forceinline__ cdd ldg(const cdd* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return cdd{dd(v.x, v.y), dd(v.z, v.w)};
}

// Values of a staged input tile and of the global output.  Float-pair plans
// keep float64 data in memory and float pairs in registers and in the
// shared-memory exchanges: the tile is read as float64 and split, the
// output joined back to float64.
template <typename C> __device__ __forceinline__ C tile_val(const C* p) { return *p; }
__device__ __forceinline__ cdd tile_val(const cdd* p) { return cdd_from(*reinterpret_cast<const double2*>(p)); }
template <typename C> __device__ __forceinline__ void store_out(C* p, C v) { __stcs(p, v); }
__device__ __forceinline__ void store_out(cdd* p, cdd v) { __stcs(reinterpret_cast<double2*>(p), cdd_to(v)); }

template <int N> struct ILog2 { static constexpr int v = 1 + ILog2<N / 2>::v; };
template <> struct ILog2<1> { static constexpr int v = 0; };

template <int I> using IC = std::integral_constant<int, I>;
template <int B, int E, class F> __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(IC<B>{});
    static_for<B + 1, E>(f);
  }
}

// ---------------------------------------------------------------------------
// register-level radix-R DFT (R <= 32), forward sign, natural order in/out.
// Radix-2 decimation in time, applied recursively; constant twiddles
// w_R^k = cos(2 pi k/R) - i sin(2 pi k/R) are compile-time immediates, and the
// trivial ones (1, -i, (1-i)/sqrt2, (-1-i)/sqrt2) are special-cased.
// ---------------------------------------------------------------------------
template <typename C, int R, int K> __device__ __forceinline__ C twc(C v) {
  using T = decltype(C::x);
  constexpr int q = K * (32 / R);  // index into the 32-point circle
  if constexpr (q == 0) {
    return v;
  } else if constexpr (q == 8) {  // -i
    return mk<C>(v.y, -v.x);
  } else if constexpr (q == 4) {  // (1 - i)/sqrt2
    constexpr T s = (T)0.707106781186547524401;
    return mk<C>((v.x + v.y) * s, (v.y - v.x) * s);
  } else if constexpr (q == 12) {  // (-1 - i)/sqrt2
    constexpr T s = (T)0.707106781186547524401;
    return mk<C>((v.y - v.x) * s, -(v.x + v.y) * s);
  } else {
    constexpr T c = (T)cos32(q), s = (T)sin32(q);
    // (a + ib)(c - is) = (ac + bs) + i(bc - as)
    return mk<C>(v.x * c + v.y * s, v.y * c - v.x * s);
  }
}

template <typename C, int R> struct Dft {
  static __device__ __forceinline__ void run(C* x) {
    C ev[R / 2], od[R / 2];
#pragma unroll
    for (int k = 0; k < R / 2; ++k) { ev[k] = x[2 * k]; od[k] = x[2 * k + 1]; }
    Dft<C, R / 2>::run(ev);
    Dft<C, R / 2>::run(od);
    static_for<0, R / 2>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      C t = twc<C, R, k>(od[k]);
      x[k] = cadd(ev[k], t);
      x[k + R / 2] = csub(ev[k], t);
    });
  }
};
template <typename C> struct Dft<C, 1> { static __device__ __forceinline__ void run(C*) {} };
template <typename C> struct Dft<C, 2> {
  static __device__ __forceinline__ void run(C* x) {
    C a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

// ---------------------------------------------------------------------------
// float64 twiddled radix-R DFT (R = 2, 4, 8) as radix-2 decimation-in-time
// layers whose twiddles are folded into the butterflies (Linzer and Feig,
// "Modified FFTs for fused multiply-add architectures", Math. Comp. 1993):
// a +- w b with w = c (1 + i t), |t| <= 1, costs 6 FMAs instead of 8 (a
// complex product and two complex additions).  Where |Im w| > |Re w| the
// factorisation is w = Im(w) (1 - i Re(w)/Im(w)) applied to i b; the
// choice is carried in the lowest mantissa bit of the stored t (a change
// of at most one ulp of t).  On GB300, whose float64 kernels are bound by
// the FP64 pipe, this is 9 FP64 operations per value and radix-8 pass
// instead of 10.5 (twiddle products, then the DFT).
//
// The pass twiddles of a thread, w = w_{LR}^{k m}, enter as the layer
// twiddles (omega = w_{LR}^k, W_n = w_n):
//   R = 8: omega^4, omega^2, W_4 omega^2, omega, W_4 omega, W_8 omega, W_8^3 omega
//   R = 4: omega^2, omega, W_4 omega
//   R = 2: omega
// ---------------------------------------------------------------------------
__device__ __forceinline__ void lf_bfly(double2& a, double2& b, double2 w) {
  const bool sw = (__double2loint(w.y) & 1) != 0;
  const double t = w.y, cc = w.x;
  // b' = b, or i b = (-b.im, b.re).  The sign is flipped by an integer xor
  // of the high word in inline PTX: written as a plain C++ bit operation
  // the compiler recognises a negation and may emit it as a float64
  // instruction, which on GB300 costs a slot of the FP64 pipe
  int nbi_hi = __double2hiint(b.y);
  asm("xor.b32 %0, %0, 0x80000000;" : "+r"(nbi_hi));
  const double nbi = __hiloint2double(nbi_hi, __double2loint(b.y));
  const double pr = sw ? nbi : b.x;
  const double pi = sw ? b.x : b.y;
  const double u = fma(-t, pi, pr);
  const double v = fma(t, pr, pi);
  const double ar = a.x, ai = a.y;
  a = make_double2(fma(cc, u, ar), fma(cc, v, ai));
  b = make_double2(fma(-cc, u, ar), fma(-cc, v, ai));
}
template <int R> struct LfDft;
template <> struct LfDft<2> {
  static __device__ __forceinline__ void run(double2* x, const double2* w) { lf_bfly(x[0], x[1], w[0]); }
};
template <> struct LfDft<4> {
  static __device__ __forceinline__ void run(double2* x, const double2* w) {
    lf_bfly(x[0], x[2], w[0]);
    lf_bfly(x[1], x[3], w[0]);
    lf_bfly(x[0], x[1], w[1]);  // X0, X2
    lf_bfly(x[2], x[3], w[2]);  // X1, X3
    const double2 x1 = x[1];
    x[1] = x[2];
    x[2] = x1;
  }
};
template <> struct LfDft<8> {
  static __device__ __forceinline__ void run(double2* x, const double2* w) {
#pragma unroll
    for (int m = 0; m < 4; ++m) lf_bfly(x[m], x[m + 4], w[0]);  // p_m, q_m
    lf_bfly(x[0], x[2], w[1]);                                  // P0+, P0-
    lf_bfly(x[1], x[3], w[1]);                                  // P1+, P1-
    lf_bfly(x[4], x[6], w[2]);                                  // Q0+, Q0-
    lf_bfly(x[5], x[7], w[2]);                                  // Q1+, Q1-
    lf_bfly(x[0], x[1], w[3]);                                  // X0, X4
    lf_bfly(x[2], x[3], w[4]);                                  // X2, X6
    lf_bfly(x[4], x[5], w[5]);                                  // X1, X5
    lf_bfly(x[6], x[7], w[6]);                                  // X3, X7
    const double2 y0 = x[0], y4 = x[1], y2 = x[2], y6 = x[3], y1 = x[4], y5 = x[5], y3 = x[6], y7 = x[7];
    x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3; x[4] = y4; x[5] = y5; x[6] = y6; x[7] = y7;
  }
};

// ---------------------------------------------------------------------------
// compile-time configuration of one kernel
// ---------------------------------------------------------------------------
template <typename R_, int NS_, int E_, int S_, int KIND_>
struct Cfg {
  using real = R_;
  using c = typename CT<R_>::c;
  static constexpr int NS = NS_;
  static constexpr int E = E_;
  static constexpr int S = S_;
  static constexpr int KIND = KIND_;
  static constexpr int P = NS / E;
  static constexpr int NT = P * S;
  static constexpr bool SLOT_FAST = (KIND == KIND_COL);
  static constexpr int LOG_NS = ILog2<NS>::v;
  static constexpr int LOG_E = ILog2<E>::v;
  static constexpr int NP = (LOG_NS + LOG_E - 1) / LOG_E;   // radix passes
  static constexpr int LOG_RL = LOG_NS - (NP - 1) * LOG_E;  // log radix of the last pass
  static constexpr int B = (sizeof(c) == 8) ? 4 : 3;         // 128-byte bank row, in elements
  static constexpr int SMEM_BYTES = S * NS * (int)sizeof(c);

  static_assert(E <= NS && NS % E == 0, "E must divide NS");
  static_assert(NT >= 32 && NT <= 1024 && NT % 32 == 0, "block size");
  static_assert(!SLOT_FAST || (32 % S == 0), "slot-fast mapping needs S | 32");
};

template <class K, int p> struct PassInfo {
  static constexpr int LOG_R = (p == K::NP - 1) ? K::LOG_RL : K::LOG_E;
  static constexpr int R = 1 << LOG_R;
  static constexpr int NB = K::E / R;           // butterflies per thread
  static constexpr int LOG_L = p * K::LOG_E;
  static constexpr int L = 1 << LOG_L;
  static constexpr bool LAST = (p == K::NP - 1);
  static constexpr int TWS = K::NS / (L * R);   // twiddle table stride
};

// Shared-memory index of (slot, pos) in the exchange written by pass p.
// Slot-major layouts XOR bits [l, B) of the position with bits
// [l + r, l + r + B - l) when the pass writes with a stride (l < B), and,
// when a slot's threads cover less than a 128-byte bank row, add a per-slot
// offset: a padding-free swizzle that keeps both the pass's scattered
// writes and the next pass's contiguous reads free of bank conflicts
// (Sec. 3.2).
template <class K, int p> __device__ __forceinline__ int sidx(int slot, int pos) {
  if constexpr (K::SLOT_FAST) {
    // Position-major rows of S values.  When a 128-byte bank row holds
    // G = W/S > 1 positions, the first pass (twiddle stride 1) writes
    // positions j*R + m for the 32/S adjacent j of a warp, R/G bank rows
    // apart, all at the same offset: XOR the position's offset inside its
    // bank row with bits of j (the row index over max(R/G, 1)), which keeps
    // the later contiguous reads conflict-free (a permutation inside each
    // bank row).
    constexpr int W = 1 << K::B;
    if constexpr (p == 0 && K::S < W) {
      constexpr int G = W / K::S;
      constexpr int LOG_G = ILog2<G>::v;
      constexpr int R = PassInfo<K, 0>::R;
      constexpr int SH = (R > G) ? ILog2<R / G>::v : 0;
      const int key = ((pos >> LOG_G) >> SH) & (G - 1);
      return (pos ^ key) * K::S + slot;
    } else {
      return pos * K::S + slot;
    }
  } else {
    constexpr int l = PassInfo<K, p>::LOG_L, r = PassInfo<K, p>::LOG_R;
    int q = pos;
    if constexpr (l < K::B) q ^= ((pos >> (l + r)) & ((1 << (K::B - l)) - 1)) << l;
    // when a slot's P threads span less than a bank row, the 32/P slots of a
    // warp take different parts of it
    constexpr int RUN = K::P * (int)sizeof(typename K::c);
    if constexpr (K::P < 32 && RUN < 128 && K::NS >= (1 << K::B)) q ^= (slot % (128 / RUN)) * K::P;
    return slot * K::NS + q;
  }
}

// Injection context of one thread for the current transaction.
struct InjCtx {
  bool on;
  int stage, pos, comp, bit;
};

__device__ __forceinline__ float flip1(float f, int bit) { return __uint_as_float(__float_as_uint(f) ^ (1u << bit)); }
__device__ __forceinline__ double flip1(double f, int bit) {
  return __longlong_as_double(__double_as_longlong(f) ^ (1ll << bit));
}
// a float pair stands for a float64 value: flip the bit of that value
__device__ __forceinline__ dd flip1(dd f, int bit) { return dd_from_double(flip1(dd_to_double(f), bit)); }
template <typename C> __device__ __forceinline__ void flip_bit(C& v, int comp, int bit) {
  if (comp) v.y = flip1(v.y, bit);
  else v.x = flip1(v.x, bit);
}

template <class K> __device__ __forceinline__ void inject_stage(typename K::c (&a)[K::E], int stage,
                                                                const InjCtx& ic, int t) {
  if (ic.on && ic.stage == stage) {
#pragma unroll
    for (int i = 0; i < K::E; ++i)
      if (t + i * K::P == ic.pos) flip_bit(a[i], ic.comp, ic.bit);
  }
}

// Pass twiddles of one thread.  Thread t's butterflies j = t + u*P need
// w_NS^{TWS*(j mod L)*m}, the same values in every transaction, so when
// they fit in a register budget they are loaded once per block and kept in
// registers; otherwise they are read from the table in each pass.
template <class K, int p> struct TwCount {
  static constexpr int v = (PassInfo<K, p>::L > 1) ? PassInfo<K, p>::NB * (PassInfo<K, p>::R - 1) : 0;
};
template <class K, int p> struct TwOff { static constexpr int v = TwOff<K, p - 1>::v + TwCount<K, p - 1>::v; };
template <class K> struct TwOff<K, 0> { static constexpr int v = 0; };
template <class K> struct TwTotal { static constexpr int v = TwOff<K, K::NP>::v; };
#ifndef TF_FT_TW_BUDGET
#define TF_FT_TW_BUDGET 64
#endif
template <class K, int BUDGET = 64> struct TwMode {
  // passes whose twiddles fit, in order, in BUDGET 32-bit registers keep
  // them in registers; later passes read the table
  template <int p> static constexpr bool reg() {
    return TwOff<K, p + 1>::v * (int)sizeof(typename K::c) / 4 <= BUDGET;
  }
  static constexpr int count_reg() {
    int n = 0;
    for (int p = 0; p < K::NP; ++p) {
      int off = 0, cnt = 0;
      // recompute offsets without templates
      for (int q = 0; q <= p; ++q) {
        const int lr = (q == K::NP - 1) ? K::LOG_RL : K::LOG_E;
        const int L = 1 << (q * K::LOG_E), R = 1 << lr, NB = K::E / R;
        cnt = (L > 1) ? NB * (R - 1) : 0;
        off += cnt;
      }
      if (off * (int)sizeof(typename K::c) / 4 <= BUDGET) n = off;
    }
    return n;
  }
  static constexpr int N = count_reg() > 0 ? count_reg() : 1;
  static constexpr bool ANY = count_reg() > 0;
  // resident blocks per SM that the register allocation must allow
  static constexpr int MINB_RAW = (ANY ? 512 : 768) / K::NT;
  static constexpr int MINB = MINB_RAW < 1 ? 1 : (MINB_RAW > 8 ? 8 : MINB_RAW);
#ifndef TF_FT_MINB_DELTA
#define TF_FT_MINB_DELTA 0
#endif
  // checksum variants: optionally fewer resident blocks for more registers
  static constexpr int MINB_FT = (MINB - TF_FT_MINB_DELTA) < 1 ? 1 : (MINB - TF_FT_MINB_DELTA);
};

// float64 kernels read the folded layer twiddles (c, t) of each pass from
// one table: pass p (L > 1) holds L groups of R - 1 entries, k-major
template <class K> constexpr bool lf_twiddles() { return std::is_same<typename K::real, double>::value; }
template <class K, int p> struct LfOff {
  static constexpr int v = LfOff<K, p - 1>::v + ((PassInfo<K, p - 1>::L > 1) ? PassInfo<K, p - 1>::L * (PassInfo<K, p - 1>::R - 1) : 0);
};
template <class K> struct LfOff<K, 0> { static constexpr int v = 0; };
template <class K, int p> __device__ __forceinline__ int tw_index(int k, int m) {
  using PI = PassInfo<K, p>;
  if constexpr (lf_twiddles<K>()) return LfOff<K, p>::v + k * (PI::R - 1) + (m - 1);
  else return PI::TWS * k * m;
}

template <class K, int BUDGET = 64> struct TwReg {
  using c = typename K::c;
  using M = TwMode<K, BUDGET>;
  static_assert(!lf_twiddles<K>() || K::NP == 1 || K::E == 8,
                "the float64 folded twiddle tables are laid out for radix-8 passes");
  c v[M::N];
  const c* __restrict__ tab;
  __device__ __forceinline__ void load(const c* __restrict__ tw, int t) {
    tab = tw;
    static_for<0, K::NP>([&](auto pc) {
      constexpr int p = decltype(pc)::value;
      using PI = PassInfo<K, p>;
      if constexpr (PI::L > 1 && M::template reg<p>()) {
#pragma unroll
        for (int u = 0; u < PI::NB; ++u) {
          const int k = (t + u * K::P) & (PI::L - 1);
#pragma unroll
          for (int m = 1; m < PI::R; ++m) v[TwOff<K, p>::v + u * (PI::R - 1) + m - 1] = ldg(tw + tw_index<K, p>(k, m));
        }
      }
    });
  }
  template <int p> __device__ __forceinline__ c get(int u, int m, int k) const {
    using PI = PassInfo<K, p>;
    if constexpr (M::template reg<p>()) return v[TwOff<K, p>::v + u * (PI::R - 1) + m - 1];
    else return ldg(tab + tw_index<K, p>(k, m));
  }
};

template <class K, int p, class TW>
__device__ __forceinline__ void run_pass(typename K::c (&a)[K::E], typename K::c* sm, const TW& tw, int slot,
                                         int t) {
  using c = typename K::c;
  using PI = PassInfo<K, p>;
  constexpr int R = PI::R, NB = PI::NB, L = PI::L;
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int j = t + u * K::P;
    const int k = j & (L - 1);
    c b[R];
#pragma unroll
    for (int m = 0; m < R; ++m) b[m] = a[u + m * NB];
    if constexpr (L > 1 && lf_twiddles<K>()) {
      c w[R - 1];
#pragma unroll
      for (int m = 1; m < R; ++m) w[m - 1] = tw.template get<p>(u, m, k);
      LfDft<R>::run(b, w);
    } else {
      if constexpr (L > 1) {
#pragma unroll
        for (int m = 1; m < R; ++m) b[m] = cmul(b[m], tw.template get<p>(u, m, k));
      }
      Dft<c, R>::run(b);
    }
    if constexpr (PI::LAST) {
#pragma unroll
      for (int m = 0; m < R; ++m) a[u + m * NB] = b[m];
    } else {
      const int base = (j - k) * R + k;
#pragma unroll
      for (int m = 0; m < R; ++m) sm[sidx<K, p>(slot, base + m * L)] = b[m];
    }
  }
  if constexpr (!PI::LAST) {
    __syncthreads();
#pragma unroll
    for (int i = 0; i < K::E; ++i) a[i] = sm[sidx<K, p>(slot, t + i * K::P)];
    __syncthreads();
  }
}

template <class K, int p, bool END = (p == K::NP)> struct Passes {
  template <class TW>
  static __device__ __forceinline__ void run(typename K::c (&a)[K::E], typename K::c* sm, const TW& tw, int slot,
                                             int t, const InjCtx& ic) {
    inject_stage<K>(a, p, ic, t);
    run_pass<K, p, TW>(a, sm, tw, slot, t);
    Passes<K, p + 1>::run(a, sm, tw, slot, t, ic);
  }
};
template <class K, int p> struct Passes<K, p, true> {
  template <class TW>
  static __device__ __forceinline__ void run(typename K::c (&a)[K::E], typename K::c*, const TW&, int, int t,
                                             const InjCtx& ic) {
    inject_stage<K>(a, p, ic, t);
  }
};

// full sub-transform in registers + shared memory (all threads of the block
// take part; no injection)
template <class K, class TW>
__device__ __forceinline__ void fft_block(typename K::c (&a)[K::E], typename K::c* sm, const TW& tw, int slot,
                                          int t) {
  InjCtx off{false, 0, 0, 0, 0};
  Passes<K, 0>::run(a, sm, tw, slot, t, off);
}

// ---------------------------------------------------------------------------
// addressing of one sub-transform ("signal") of a pass
// ---------------------------------------------------------------------------
struct Geo {
  long long n;   // full transform length N
  int n1, n2;    // N = n1 * n2 (single pass: n1 = N, n2 = 1)
  long long batch;
  // element offset of transform b in this pass's input / output, or null for
  // the contiguous layout b * N (ragged batches index their transforms)
  const long long* in_tab;
  const long long* out_tab;
  // last pass of a three-pass plan (outer > 1): this pass's transforms are
  // the rows b = t * outer + k1 of transform t of length n_outer, and element
  // k' of row b goes to k1 + outer * k' of transform t (0 or 1: no mapping)
  int outer;
  long long n_outer;
  // float64 column passes: 1 = units walk the transforms fastest (shared
  // column tables), 0 = the columns of one transform first (transform-level
  // checksums accumulate per transform)
  int col_tfast;
  // log2 of n1, n2 and outer (all powers of two): the column and row passes
  // split unit and signal indices with shifts and masks.  A 64-bit integer
  // division is a library sequence whose rarely taken branches still issue
  // float64 instructions (predicated off) on the FP64 pipe, the pipe that
  // bounds the float64 kernels.
  int l2n1, l2n2, l2outer;
};

__device__ __forceinline__ long long tr_base(const long long* tab, long long b, long long n) {
  return tab ? __ldg(tab + b) : b * n;
}

// three-pass last pass: first sub-transform of unit `unit` (units walk
// transform t, then row k2, then blocks of S adjacent sub-transforms)
template <class K> __device__ __forceinline__ long long row_unit_first(const Geo& g, long long unit) {
  // per transform n1 * (outer / S) units; kb = unit mod (outer / S)
  constexpr int LS = ILog2<K::S>::v;
  const long long t = unit >> (g.l2n1 + g.l2outer - LS);
  const int kb = (int)(unit & ((1ll << (g.l2outer - LS)) - 1));
  return t * g.outer + (long long)kb * K::S;
}

// Column-pass unit -> (transform b, first column c0).  float64 column passes
// walk the transforms fastest, so that the blocks running at once share their
// column block and the per-column tables in access order (twiddles, checksum
// weights) are read from HBM about once per column block, not per transform;
// float32 column passes (no such tables) walk the columns of a transform.
template <class K>
__device__ __forceinline__ void col_unit(const Geo& g, long long unit, long long& b, int& c0) {
  if (std::is_same<typename K::real, double>::value && g.col_tfast) {
    // (unit indices stay below 2^32: a 32-bit division)
    const unsigned u = (unsigned)unit, bt = (unsigned)g.batch;
    const unsigned cb = u / bt;
    b = (long long)(u - cb * bt);
    c0 = (int)cb * K::S;
  } else {
    constexpr int LS = ILog2<K::S>::v;
    b = unit >> (g.l2n2 - LS);
    c0 = (int)(unit & ((1ll << (g.l2n2 - LS)) - 1)) * K::S;
  }
}

// signal id of slot `slot` of work unit `unit`; -1 if past the end (ragged tail)
template <class K> __device__ __forceinline__ long long signal_of(const Geo& g, long long unit, int slot) {
  if constexpr (K::KIND == KIND_SP) {
    long long s = unit * K::S + slot;
    return s < g.batch ? s : -1;
  } else if constexpr (K::KIND == KIND_COL) {
    long long b;
    int c0;
    col_unit<K>(g, unit, b, c0);
    return b * g.n2 + c0 + slot;
  } else {
    if (g.outer > 1) {
      // last pass of a three-pass plan: the S rows of a unit are row k2 of
      // S adjacent sub-transforms (adjacent first-pass outputs k1), whose
      // results are adjacent in the final output
      constexpr int LS = ILog2<K::S>::v;
      const long long b0 = row_unit_first<K>(g, unit);
      const int k2 = (int)((unit >> (g.l2outer - LS)) & (g.n1 - 1));
      return (b0 + slot) * g.n1 + k2;
    }
    constexpr int LS = ILog2<K::S>::v;
    const long long b = unit >> (g.l2n1 - LS);
    const int k1 = (int)(unit & ((1ll << (g.l2n1 - LS)) - 1)) * K::S + slot;
    return b * g.n1 + k1;
  }
}

// Addressing of signal `sig`: element (pos) of its input sits at
// in_base(sig) + pos * in_step, of its output at out_base(sig) + pos * out_step.
//   SP:  transform sig, contiguous
//   COL: column n2 of transform b = sig / N2 (stride N2)
//   ROW: row k1 of transform b = sig / N1: input contiguous, output stride N1
template <class K> __device__ __forceinline__ long long in_base(const Geo& g, long long sig) {
  if constexpr (K::KIND == KIND_SP) {
    return tr_base(g.in_tab, sig, g.n);
  } else if constexpr (K::KIND == KIND_COL) {
    return tr_base(g.in_tab, sig >> g.l2n2, g.n) + (sig & (g.n2 - 1));
  } else {
    return tr_base(g.in_tab, sig >> g.l2n1, g.n) + (sig & (g.n1 - 1)) * g.n2;
  }
}
template <class K> __device__ __forceinline__ long long in_step(const Geo& g) {
  return K::KIND == KIND_COL ? (long long)g.n2 : 1;
}
template <class K> __device__ __forceinline__ long long out_base(const Geo& g, long long sig) {
  if constexpr (K::KIND == KIND_SP) {
    return tr_base(g.out_tab, sig, g.n);
  } else if constexpr (K::KIND == KIND_COL) {
    return tr_base(g.out_tab, sig >> g.l2n2, g.n) + (sig & (g.n2 - 1));
  } else {
    const long long b = sig >> g.l2n1;
    if (g.outer > 1) {
      return tr_base(g.out_tab, b >> g.l2outer, g.n_outer) + (b & (g.outer - 1)) + (sig & (g.n1 - 1)) * g.outer;
    }
    return tr_base(g.out_tab, b, g.n) + (sig & (g.n1 - 1));
  }
}
template <class K> __device__ __forceinline__ long long out_step(const Geo& g) {
  if constexpr (K::KIND == KIND_ROW) return (long long)g.n1 * (g.outer > 1 ? g.outer : 1);
  return K::KIND == KIND_SP ? 1 : (long long)g.n2;
}
template <class K> __device__ __forceinline__ long long in_off(const Geo& g, long long sig, int pos) {
  return in_base<K>(g, sig) + (long long)pos * in_step<K>(g);
}
template <class K> __device__ __forceinline__ long long out_off(const Geo& g, long long sig, int pos) {
  return out_base<K>(g, sig) + (long long)pos * out_step<K>(g);
}

// inter-pass twiddle w_N^{k1 * n2} for column n2 of signal `sig` (KIND_COL):
// w_N^q = thi[q >> 12] * tlo[q & 4095] (two small tables that stay in L1;
// one table of all N values, read from L2 with no locality, measured slower)
template <class K> __device__ __forceinline__ typename K::c colTwiddle(const Geo& g, const typename K::c* tlo,
                                                                       const typename K::c* thi, long long sig,
                                                                       int k1) {
  const int n2 = (int)(sig & (g.n2 - 1));
  unsigned q = (unsigned)k1 * (unsigned)n2;
  return cmul(ldg(thi + (q >> 12)), ldg(tlo + (q & 4095u)));
}

// ---------------------------------------------------------------------------
// kernel arguments
// ---------------------------------------------------------------------------
template <typename R> struct PassArgs {
  using c = typename CT<R>::c;
  const c* in;
  c* out;
  const c* tw;    // w_NS^q, q < NS (forward sign)
  const c* ev;    // output-side encoding vector e, NS entries
  const c* vv;    // input-side vector v = W^T e, NS entries
  const float4* ev4;  // float32 plans: e arranged as (re, re, im, im) for paired FMAs
  const float4* vv4;  // float32 plans: v arranged the same way
  const c* tlo;   // inter-pass twiddles (KIND_COL)
  const c* thi;
  // float64 column passes: the inter-pass twiddles, and the output-side
  // checksum weights e_k1 conj(w), in the pass's access order
  // (colw[n2 * NS + k1] = w^{k1 n2}); null otherwise
  const c* colw;
  const c* colwe;
  Geo geo;
  long long num_units;
  int conj_in;    // inverse: conjugate on load (first pass)
  int conj_out;   // inverse: conjugate on store (last pass)
  R out_scale;    // 1 or 1/N on store (last pass)
  double tau_coef;  // gamma * u * sqrt(log2 NS) * threshold scale
  int ft;         // FT_OFF / FT_DETECT / FT_CORRECT
  int T;          // transactions per checksum group
  int pass_id;
  long long transform_base;  // first transform of this launch in the caller's batch
  FtState* fts;
  // transform-level checksums (float64 two-pass plans): per transform
  // [v.x re, v.x im, e.y re, e.y im, energy, -], and the N-point weights in
  // the passes' access orders: vcol[n2 * N1 + p] = v[p * N2 + n2],
  // erow[k1 * N2 + k2] = e[k1 + N1 * k2]
  double* tacc;
  const c* vcol;
  const c* erow;
  void* rec_sums; // MAX_RECORDS x 2 x NS_MAX complex (x_bar, y_bar)
  int rec_stride; // complex elements per record half (NS_MAX)
  InjectSite inj;
  int* err;       // TMA-staged passes: set to 1 when a bounded wait expires
};

// column n2 of a column-pass signal (within its transform)
template <class K> __device__ __forceinline__ long long col_of(const Geo& g, long long sig) {
  return sig & (g.n2 - 1);
}
// inter-pass twiddle of a column pass: from the float64 table in access
// order, else the product of the two small tables
template <class K>
__device__ __forceinline__ typename K::c col_w(const PassArgs<typename K::real>& A, long long sig, int k1) {
  if constexpr (std::is_same<typename K::real, double>::value) {
    return ldg(A.colw + col_of<K>(A.geo, sig) * K::NS + k1);
  } else {
    return colTwiddle<K>(A.geo, A.tlo, A.thi, sig, k1);
  }
}

// ---------------------------------------------------------------------------
// block reduction helpers for the checksum group
// ---------------------------------------------------------------------------
template <class K> struct Seg {
  // lanes of one slot inside a warp: pos-fast -> contiguous runs of min(P,32);
  // slot-fast -> lanes congruent mod S.
  static constexpr int RUN = (K::P < 32) ? K::P : 32;
  static constexpr int PER_WARP = K::SLOT_FAST ? K::S : (32 / RUN);
  static constexpr int COUNT = (K::NT / 32) * PER_WARP;
};

template <class K, typename V> __device__ __forceinline__ V seg_reduce_sum(V v) {
  if constexpr (K::SLOT_FAST) {
#pragma unroll
    for (int o = K::S; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  } else {
#pragma unroll
    for (int o = 1; o < Seg<K>::RUN; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}
template <class K> __device__ __forceinline__ int seg_reduce_min(int v) {
  if constexpr (K::SLOT_FAST) {
#pragma unroll
    for (int o = K::S; o < 32; o <<= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  } else {
#pragma unroll
    for (int o = 1; o < Seg<K>::RUN; o <<= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}
template <class K> __device__ __forceinline__ int seg_reduce_max(int v) {
  if constexpr (K::SLOT_FAST) {
#pragma unroll
    for (int o = K::S; o < 32; o <<= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  } else {
#pragma unroll
    for (int o = 1; o < Seg<K>::RUN; o <<= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}
// is this lane the leader of its segment, and the segment id
template <class K> __device__ __forceinline__ bool seg_leader(int tid, int& seg) {
  const int lane = tid & 31, warp = tid >> 5;
  if constexpr (K::SLOT_FAST) {
    seg = warp * K::S + lane;
    return lane < K::S;
  } else {
    seg = warp * Seg<K>::PER_WARP + lane / Seg<K>::RUN;
    return (lane % Seg<K>::RUN) == 0;
  }
}
// segments that hold slot s: calls f(seg) for each
template <class K, class F> __device__ __forceinline__ void for_slot_segments(int s, F&& f) {
  if constexpr (K::SLOT_FAST) {
    for (int w = 0; w < K::NT / 32; ++w) f(w * K::S + s);
  } else if constexpr (K::P >= 32) {
    for (int w = 0; w < K::P / 32; ++w) f(s * (K::P / 32) + w);
  } else {
    f(s);
  }
}

// dynamic shared memory of the transform kernel: the exchange buffer, which
// the checksum-group reduction reuses
// One stage of the shared-memory ring holds a transaction's input tile
// (S x NS values), copied asynchronously one transaction ahead; the stage of
// the current transaction then serves as its exchange buffer and as the
// scratch of the checksum-group reduction.
#ifndef TF_NSTAGE
#define TF_NSTAGE 2
#endif
constexpr int NSTAGE = TF_NSTAGE;
template <class K> constexpr int stage_bytes() {
  constexpr int red = Seg<K>::COUNT * 64 + (K::S + 1) * 4;  // partial sums, slot flags, "any" flag
  constexpr int b = (K::SMEM_BYTES > red) ? K::SMEM_BYTES : red;
  return (b + 127) / 128 * 128;
}
// checksum vectors e and v staged in shared memory once per block when
// they are small (read once per element per transaction)
// Optionally (TF_PAIRED_CHECKSUMS) float32 checksums use paired FP32 FMAs
// (FFMA2) with the weights arranged as (re, re, im, im); the column pass
// weights e by the inter-pass twiddle per element and keeps the scalar form
template <class K> constexpr bool paired_ft() {
#ifdef TF_PAIRED_CHECKSUMS
  return std::is_same<typename K::real, float>::value;
#else
  return false;  // measured slower on GB300: the 16-byte weights double the shared-memory traffic
#endif
}
// Thread-level checksums (Sec. 4.2.1) apply where one thread holds a whole
// transform: a single radix pass in registers, no shared-memory exchange.
template <class K> constexpr bool thread_level_ok() {
  return K::P == 1 && K::KIND == KIND_SP && K::NP == 1 && !paired_ft<K>();
}
template <class K> constexpr int ev_entry_bytes() { return paired_ft<K>() ? 16 : (int)sizeof(typename K::c); }
template <class K> constexpr bool ev_in_smem() { return 2 * K::NS * ev_entry_bytes<K>() <= 32768; }
// checksum weight `pos` (table in shared memory for small NS, else global)
template <class K> __device__ __forceinline__ typename K::c weight(const typename K::c* tab, int pos);
template <class K, int FTM = 0> constexpr int pass_smem_bytes() {
  return NSTAGE * stage_bytes<K>() + ((FTM != 0 && ev_in_smem<K>()) ? 2 * K::NS * ev_entry_bytes<K>() : 0);
}

template <class K> __device__ __forceinline__ typename K::c weight(const typename K::c* tab, int pos) {
  return tab[pos];
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (cp.async, 16 bytes, L2 only)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// tensor-memory-accelerator (TMA) tile loads completing on an mbarrier
// (float32 column passes: a column tile is one 2-D box of S columns x up to
// 256 rows of the input viewed as [rows][n2] complex values; row passes and
// single-pass transforms with an unswizzled tile: one contiguous bulk copy)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* mb, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(mb)), "r"(count) : "memory");
}
// make the initialised barriers visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// order this thread's earlier (barrier-synchronised) shared-memory accesses
// before the asynchronous proxy's writes of the next TMA copy
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* mb, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(mb)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* mb, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(smem_addr(mb)), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait for phase `parity` of an mbarrier: false after about 2^22
// polls (each try_wait may itself suspend the thread for a while)
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* mb, unsigned parity) {
  for (int i = 0; i < (1 << 22); ++i)
    if (mbar_try_wait(mb, parity)) return true;
  return false;
}
// contiguous copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) into shared memory, completion counted on mb
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* mb) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(mb))
      : "memory");
}
// 2-D tile load: box at element coordinates (x, y) of the tensor map into
// shared memory at dst (128-byte aligned), completion counted on mb
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y,
                                            unsigned long long* mb) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(smem_addr(mb))
      : "memory");
}

// Staged tiles of slot-major (SP, ROW) kernels keep each slot's positions
// XOR-swizzled by (slot % M) * P, in whole 16-byte chunks: when a slot's P
// threads read fewer than 128 bytes per register index, the M slots of one
// warp would otherwise read the same banks (M-way conflicts on the first
// read of every transaction).
template <class K> struct StageSwz {
  static constexpr int RUN = K::P * (int)sizeof(typename K::c);  // bytes a slot's threads read per index
  static constexpr int EPC = 16 / (int)sizeof(typename K::c);    // values per 16-byte chunk
  static constexpr bool ON = !K::SLOT_FAST && K::P < 32 && RUN < 128 && (K::P % EPC) == 0;
  static constexpr int M = ON ? 128 / RUN : 1;
  static __device__ __forceinline__ int x(int slot) { return ON ? (slot % M) * K::P : 0; }
  // One thread per float32 transform (P = 1): the thread reads its values
  // as 16-byte pairs, and whole chunks are XOR-swizzled by slot so that the
  // 8 threads of a quarter warp read 8 different 16-byte bank groups.
  static constexpr bool PAIRS = !K::SLOT_FAST && K::P == 1 && EPC == 2;
  static constexpr int U = K::NS / 2;              // chunks per transform
  static constexpr int UM = U < 8 ? U : 8;
  static constexpr int SPAN = U < 8 ? 8 / U : 1;   // slots that share 8 chunks
  static __device__ __forceinline__ int chunk(int slot, int j) {
    if constexpr (PAIRS) return j ^ ((slot / SPAN) % UM);
    return ON ? (j ^ (x(slot) / EPC)) : j;
  }
};

// XOR swizzle of the row pass's transposed store through shared memory
// (slot-major buffer, position XOR tsw(slot)).  The read side (32 slots of a
// warp, one position each) needs slot & (W-1) to differ across W adjacent
// slots, W = values per 128-byte bank row; the write side (a warp spans
// 32/P slots, P adjacent positions each) also needs those slots spread over
// the W/P runs of a bank row when P < W, hence the extra term, which keeps
// the map a bijection for P >= 2.
template <class K> __device__ __forceinline__ int tsw(int slot) {
  constexpr int W = 1 << K::B;
  constexpr int M = (K::P >= 2 && K::P < W) ? W / K::P : 1;
  return (slot & (W - 1)) ^ ((slot % M) * K::P);
}

// Issue the copies of work unit `unit`'s input tile into `stage`.  Layout in
// shared memory: slot-major [slot][pos] for SP/ROW (contiguous in global
// memory), position-major [pos][slot] for COL (S adjacent columns of each
// row are contiguous).  Units past the end issue nothing; a ragged last SP
// unit copies only its valid transforms.
template <class K>
__device__ __forceinline__ void issue_unit(const PassArgs<typename K::real>& A, long long unit, char* stage,
                                           int tid) {
  using c = typename K::c;
  const Geo& g = A.geo;
  if constexpr (K::KIND == KIND_SP) {
    const long long first = unit * K::S;
    long long nv = g.batch - first;
    if (nv > K::S) nv = K::S;
    constexpr int cps = K::NS * (int)sizeof(c) / 16;  // 16-byte chunks per transform
    const int chunks = (int)nv * cps;
    if (g.in_tab == nullptr) {
      const char* src = reinterpret_cast<const char*>(A.in + first * K::NS);
      for (int q = tid; q < chunks; q += K::NT) {
        const int sl = q / cps, j = q - sl * cps;
        cp_async16(stage + (size_t)sl * K::NS * sizeof(c) + 16 * StageSwz<K>::chunk(sl, j), src + 16 * (size_t)q);
      }
    } else {
      // indexed transforms: one contiguous run per slot
      for (int q = tid; q < chunks; q += K::NT) {
        const int sl = q / cps, j = q - sl * cps;
        const char* src = reinterpret_cast<const char*>(A.in + __ldg(g.in_tab + first + sl));
        cp_async16(stage + (size_t)sl * K::NS * sizeof(c) + 16 * StageSwz<K>::chunk(sl, j), src + 16 * (size_t)j);
      }
    }
  } else if constexpr (K::KIND == KIND_ROW) {
    if (g.outer > 1) {
      // rows of S different sub-transforms: one contiguous run per slot
      constexpr int cps = K::NS * (int)sizeof(c) / 16;
      constexpr int LS = ILog2<K::S>::v;
      const long long b0 = row_unit_first<K>(g, unit);
      const int k2 = (int)((unit >> (g.l2outer - LS)) & (g.n1 - 1));
      const c* base = A.in + b0 * g.n + (long long)k2 * g.n2;
      for (int q = tid; q < K::S * cps; q += K::NT) {
        const int sl = q / cps, j = q - sl * cps;
        cp_async16(stage + (size_t)sl * K::NS * sizeof(c) + 16 * StageSwz<K>::chunk(sl, j),
                   reinterpret_cast<const char*>(base + (long long)sl * g.n) + 16 * j);
      }
      return;
    }
    constexpr int LS = ILog2<K::S>::v;
    const long long b = unit >> (g.l2n1 - LS);
    const int r0 = (int)(unit & ((1ll << (g.l2n1 - LS)) - 1)) * K::S;
    const char* src = reinterpret_cast<const char*>(A.in + tr_base(g.in_tab, b, g.n) + (long long)r0 * g.n2);
    constexpr int cps = K::NS * (int)sizeof(c) / 16;
    constexpr int chunks = K::S * cps;
    for (int q = tid; q < chunks; q += K::NT) {
      const int sl = q / cps, j = q - sl * cps;
      cp_async16(stage + (size_t)sl * K::NS * sizeof(c) + 16 * StageSwz<K>::chunk(sl, j), src + 16 * (size_t)q);
    }
  } else {
    long long b;
    int c0;
    col_unit<K>(g, unit, b, c0);
    constexpr int cpr = K::S * (int)sizeof(c) / 16;  // 16-byte chunks per row of the tile
    static_assert(cpr >= 1, "a column tile row must span 16 bytes");
    const c* base = A.in + tr_base(g.in_tab, b, g.n) + c0;
    constexpr int chunks = K::NS * cpr;
    for (int q = tid; q < chunks; q += K::NT) {
      const int p = q / cpr, j = q - p * cpr;
      cp_async16(stage + (size_t)p * K::S * sizeof(c) + 16 * j,
                 reinterpret_cast<const char*>(base + (long long)p * g.n2) + 16 * j);
    }
  }
}

// float32 passes may stage their tiles with TMA where the tile lies in
// shared memory exactly as in global memory up to a 2-D box: a column tile
// (S columns of S x 8 bytes, a multiple of 16, by NS rows, dense) or an
// unswizzled slot-major tile of contiguous transforms or rows (single pass,
// or the row pass of a two-pass plan, whose S rows are adjacent)
template <class K> constexpr bool tma_ok() {
  if constexpr (!std::is_same<typename K::real, float>::value || (stage_bytes<K>() % 128) != 0) {
    return false;
  } else if constexpr (K::KIND == KIND_COL) {
    return (K::S * 8) % 16 == 0 && K::S <= 256;
  } else {
    return !StageSwz<K>::ON && !StageSwz<K>::PAIRS && !K::SLOT_FAST && (K::NS * 8) % 16 == 0;
  }
}
template <class K> constexpr int tma_box_rows() { return K::NS < 256 ? K::NS : 256; }
// Issue the TMA copies of column-pass unit `unit`'s tile (one thread): the
// input is viewed as rows of n2 values, row b * (n / n2) + p holding row p
// of transform b's column tile; c0 (a multiple of S, so c0 * 8 bytes is a
// multiple of 16) is the first column
template <class K>
__device__ __forceinline__ void issue_unit_tma(const PassArgs<typename K::real>& A, const CUtensorMap* tm,
                                               long long unit, char* stage, unsigned long long* mb) {
  using c = typename K::c;
  const Geo& g = A.geo;
  if constexpr (K::KIND == KIND_COL) {
    long long b;
    int c0;
    col_unit<K>(g, unit, b, c0);
    constexpr int BR = tma_box_rows<K>();
    constexpr unsigned bytes = (unsigned)(K::NS * K::S * sizeof(c));
    const int row0 = (int)(b << g.l2n1);  // b * (n / n2) = b * n1
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(mb, bytes);
#pragma unroll
    for (int r = 0; r < K::NS / BR; ++r) tma_load_2d(stage + (size_t)r * BR * K::S * sizeof(c), tm, c0, row0 + r * BR, mb);
  } else {
    // the tile is contiguous in global memory: the nv valid transforms of a
    // single-pass unit (a ragged last unit copies only those), or the S
    // adjacent rows r0 .. r0 + S - 1 of transform b of a row pass
    const c* src;
    long long nv = K::S;
    if constexpr (K::KIND == KIND_SP) {
      const long long first = unit * K::S;
      nv = g.batch - first;
      if (nv > K::S) nv = K::S;
      src = A.in + first * K::NS;
    } else {
      constexpr int LS = ILog2<K::S>::v;
      const long long b = unit >> (g.l2n1 - LS);
      const int r0 = (int)(unit & ((1ll << (g.l2n1 - LS)) - 1)) * K::S;
      src = A.in + b * g.n + (long long)r0 * g.n2;
    }
    const unsigned bytes = (unsigned)(nv * K::NS * (long long)sizeof(c));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(mb, bytes);
    bulk_load(stage, src, bytes, mb);
  }
}

__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v) {
  atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));
}

// ---------------------------------------------------------------------------
// the transform kernel (one pass)
// ---------------------------------------------------------------------------
template <class K> __device__ __forceinline__ void block_sum3(double* red, double& a, double& b, double& c3);

// transform of work unit `unit` of a column / row pass
template <class K> __device__ __forceinline__ long long unit_transform(const Geo& g, long long unit) {
  const long long sig = signal_of<K>(g, unit, 0);
  return K::KIND == KIND_COL ? sig >> g.l2n2 : sig >> g.l2n1;
}

// FTM: 0 = no checksums; 1 = checksums, right-side sums formed on the rare
// path from HBM; 2 = checksums, right-side sums kept in registers during the
// pass (the thread-level accumulation of Sec. 4.3); 3 = thread-level ABFT
// (Sec. 4.2.1): every thread checks its own whole transform against a
// per-transform threshold, with no block reduction; a failing transform is
// recorded for the correction kernel, which recomputes it; 4 = transform-level
// checksums of a float64 two-pass plan: the column pass accumulates v.x and
// the input energy of every transform, the row pass e.y, each over whole
// transforms (N-point weights), and a check kernel compares them afterwards
//
// pass_body: the block's share of a pass, the work units first, first +
// stride, ... below end (the pass kernel: blockIdx.x, gridDim.x, all units;
// the persistent ragged kernel: a contiguous range per work item).  The
// caller makes sure that no thread of the block still uses shared memory of
// an earlier call.  TMA: tiles are staged by TMA copies described by the
// tensor map `tm` (float32 column passes of two-pass plans); a block whose
// wait for a tile runs out records TURBOFFT_TIMEOUT in the plan's state and
// stops.
template <class K, int FTM, bool TMA = false>
__device__ __forceinline__ void pass_body(const PassArgs<typename K::real>& A, char* smem_raw, long long first,
                                          long long stride, long long end, const CUtensorMap* tm = nullptr) {
  using R = typename K::real;
  using c = typename K::c;
  constexpr int E = K::E, P = K::P, S = K::S;
  constexpr bool FT = FTM != 0;
  constexpr bool EAGER = FTM == 2;
  constexpr bool TL = FTM == 3;
  constexpr bool TC = FTM == 4;
  static_assert(!TL || thread_level_ok<K>(), "thread-level checksums need one thread per transform");
  static_assert(!TC || (std::is_same<R, double>::value && K::KIND != KIND_SP && !paired_ft<K>()),
                "transform-level checksums: float64 column and row passes");
  __shared__ double tc_red[TC ? 3 * 32 : 1];
  double tc0 = 0, tc1 = 0, tc2 = 0;  // this block's sums for the current transform

  const int tid = threadIdx.x;
  const int slot = K::SLOT_FAST ? (tid % S) : (tid / P);
  const int t = K::SLOT_FAST ? (tid / S) : (tid % P);
  const Geo g = A.geo;
  TwReg<K, FT ? TF_FT_TW_BUDGET : 64> twr;
  twr.load(A.tw, t);
  const unsigned long long mask_in = sign_mask<c>(A.conj_in), mask_out = sign_mask<c>(A.conj_out);
  const bool scaled = A.out_scale != (R)1;
  // checksum vectors: shared-memory copies (small NS) or the global tables
  const c* __restrict__ evp = A.ev;
  const c* __restrict__ vvp = A.vv;
  const float4* __restrict__ ev4p = A.ev4;
  const float4* __restrict__ vv4p = A.vv4;
  if constexpr (FT && !TC && ev_in_smem<K>()) {
    if constexpr (paired_ft<K>()) {
      float4* evs = reinterpret_cast<float4*>(smem_raw + NSTAGE * stage_bytes<K>());
      float4* vvs = evs + K::NS;
      for (int q = tid; q < K::NS; q += K::NT) {
        evs[q] = A.ev4[q];
        vvs[q] = A.vv4[q];
      }
      ev4p = evs;
      vv4p = vvs;
    } else {
      c* evs = reinterpret_cast<c*>(smem_raw + NSTAGE * stage_bytes<K>());
      c* vvs = evs + K::NS;
      for (int q = tid; q < K::NS; q += K::NT) {
        evs[q] = A.ev[q];
        vvs[q] = A.vv[q];
      }
      evp = evs;
      vvp = vvs;
    }
    __syncthreads();
  }

  // checksum-group state (per thread)
  c xs[EAGER ? E : 1], ys[EAGER ? E : 1];
  R s1r = 0, s1i = 0, s2r = 0, s2i = 0, en = 0;
  int bad_lo = 0x7fffffff, bad_hi = -1;
  unsigned checked = 0;           // transforms checked (thread-level mode)
  int gi = 0;                     // transaction index inside the group
  long long g_unit0 = first;
  long long groups = 0;
  float max_ratio2 = 0.f;  // max (|S1| / tau)^2 over clean groups
  const R tau_coef2 = (R)(A.tau_coef * A.tau_coef);
  if constexpr (EAGER) {
#pragma unroll
    for (int i = 0; i < E; ++i) { xs[i] = mk<c>(0, 0); ys[i] = mk<c>(0, 0); }
  }

  static_assert(!TMA || tma_ok<K>(), "TMA staging: float32 passes with an unswizzled tile");
  __shared__ __align__(8) unsigned long long tma_mb[TMA ? NSTAGE : 1];
  __shared__ int tma_fail;
  if constexpr (TMA) {
    if (tid == 0) {
#pragma unroll
      for (int k = 0; k < NSTAGE; ++k) mbar_init(&tma_mb[k], 1);
      mbar_init_fence();
      tma_fail = 0;
    }
    __syncthreads();
  }
  // prologue: the first NSTAGE-1 transactions' tiles in flight
#pragma unroll
  for (int k = 0; k < NSTAGE - 1; ++k) {
    const long long u = first + k * stride;
    if constexpr (TMA) {
      if (u < end && tid == 0) issue_unit_tma<K>(A, tm, u, smem_raw + k * stage_bytes<K>(), &tma_mb[k]);
    } else {
      if (u < end) issue_unit<K>(A, u, smem_raw + k * stage_bytes<K>(), tid);
      cp_async_commit();
    }
  }
  int it = 0;
  for (long long unit = first; unit < end; unit += stride, ++it) {
    // prefetch NSTAGE-1 transactions ahead into the stage freed by the
    // previous transaction, then wait for this transaction's tile
    if constexpr (TMA) {
      const long long un = unit + (NSTAGE - 1) * stride;
      const int sn = (it + NSTAGE - 1) % NSTAGE;
      if (un < end && tid == 0) issue_unit_tma<K>(A, tm, un, smem_raw + sn * stage_bytes<K>(), &tma_mb[sn]);
      // the stage of transaction `it` completes its (it / NSTAGE)-th phase
      if (!mbar_wait_bounded(&tma_mb[it % NSTAGE], (unsigned)(it / NSTAGE) & 1u)) tma_fail = 1;
      __syncthreads();
      if (tma_fail) {
        // a copy that never completed: record the timeout, give the copy
        // just issued a bounded wait, and stop this block
        if (tid == 0) {
          if (A.err) atomicExch(A.err, 1);
          if (un < end) mbar_wait_bounded(&tma_mb[sn], (unsigned)((it + NSTAGE - 1) / NSTAGE) & 1u);
        }
        return;
      }
    } else {
      const long long un = unit + (NSTAGE - 1) * stride;
      if (un < end) issue_unit<K>(A, un, smem_raw + ((it + NSTAGE - 1) % NSTAGE) * stage_bytes<K>(), tid);
      cp_async_commit();
      cp_async_wait<NSTAGE - 1>();
      __syncthreads();
    }
    c* sm = reinterpret_cast<c*>(smem_raw + (it % NSTAGE) * stage_bytes<K>());
    const long long sig = signal_of<K>(g, unit, slot);
    const bool valid = sig >= 0;
    c a[E];
    // ---- home positions from the staged tile
    if constexpr (StageSwz<K>::PAIRS) {
      const float4* s4 = reinterpret_cast<const float4*>(sm) + slot * (K::NS / 2);
#pragma unroll
      for (int j = 0; j < E / 2; ++j) {
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) q = s4[StageSwz<K>::chunk(slot, j)];
        a[2 * j] = conj_mask(make_float2(q.x, q.y), mask_in);
        a[2 * j + 1] = conj_mask(make_float2(q.z, q.w), mask_in);
      }
    } else {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        c v = mk<c>(0, 0);
        const int pos = t + i * P;
        if (valid) v = tile_val(K::SLOT_FAST ? &sm[pos * S + slot] : &sm[slot * K::NS + (pos ^ StageSwz<K>::x(slot))]);
        a[i] = conj_mask(v, mask_in);
      }
    }
    __syncthreads();  // the tile is consumed; the stage becomes the exchange buffer
    // ---- input side of the checksums
    if constexpr (TL) en = 0;  // per-transform threshold
    c pin = mk<c>(0, 0);
    if constexpr (TC && K::KIND == KIND_COL) {
      // v.x with the N-point weights in access order, and the energy (in
      // float32 from integer-extracted bits, as below)
      const long long vb = col_of<K>(g, valid ? sig : 0) * K::NS;
      // the energy twice, of x and of x 2^-64, so that values beyond the
      // float32 range (to about 2^125) need no float64 fallback: float64
      // code under a condition would be issued, predicated off, on every
      // pass
      float enf = 0.f, enl = 0.f;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        cmac(pin, ldg(A.vcol + vb + t + i * P), a[i]);
        const float fx = abs_as_float(a[i].x), fy = abs_as_float(a[i].y);
        enf = fmaf(fx, fx, enf);
        enf = fmaf(fy, fy, enf);
        const float lx = abs_as_float(a[i].x, 64), ly = abs_as_float(a[i].y, 64);
        enl = fmaf(lx, lx, enl);
        enl = fmaf(ly, ly, enl);
      }
      const double et = isfinite(enf) ? (double)enf : (double)enl * 0x1p128;
      tc0 += pin.x;
      tc1 += pin.y;
      tc2 += et;
    } else if constexpr (FT && !TC) {
      if constexpr (paired_ft<K>()) {
        // (sum v.re x, sum v.im x) with x = (re, im): two FFMA2 per element
        float2 q1 = make_float2(0.f, 0.f), q2 = make_float2(0.f, 0.f), e2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < E; ++i) {
          if constexpr (EAGER) xs[i] = cadd(xs[i], a[i]);
          const float4 w = vv4p[t + i * P];
          q1 = __ffma2_rn(make_float2(w.x, w.y), a[i], q1);
          q2 = __ffma2_rn(make_float2(w.z, w.w), a[i], q2);
          e2 = __ffma2_rn(a[i], a[i], e2);
        }
        pin = mk<c>(q1.x - q2.y, q1.y + q2.x);
        en += e2.x + e2.y;
      } else if constexpr (std::is_same<R, double>::value) {
        // float64: the energy only scales tau, so it is accumulated in
        // float32 from converted values, keeping the float64 pipe for the
        // transform and the checksum products
        // (twice, of x and of x 2^-64, so that values beyond the float32
        // range, to about 2^125, need no float64 fallback: float64 code
        // under a condition would be issued, predicated off, on every pass)
        float enf = 0.f, enl = 0.f;
#pragma unroll
        for (int i = 0; i < E; ++i) {
          if constexpr (EAGER) xs[i] = cadd(xs[i], a[i]);
          cmac(pin, weight<K>(vvp, t + i * P), a[i]);
          const float fx = abs_as_float(a[i].x), fy = abs_as_float(a[i].y);
          enf = fmaf(fx, fx, enf);
          enf = fmaf(fy, fy, enf);
          const float lx = abs_as_float(a[i].x, 64), ly = abs_as_float(a[i].y, 64);
          enl = fmaf(lx, lx, enl);
          enl = fmaf(ly, ly, enl);
        }
        en += isfinite(enf) ? (R)enf : (R)enl * (R)0x1p128;
      } else {
        if constexpr (std::is_same<R, float>::value) {
          // energy (re^2, im^2) as one paired FP32 FMA per value
          float2 e2 = make_float2(0.f, 0.f);
#pragma unroll
          for (int i = 0; i < E; ++i) {
            if constexpr (EAGER) xs[i] = cadd(xs[i], a[i]);
            cmac(pin, weight<K>(vvp, t + i * P), a[i]);
            e2 = __ffma2_rn(a[i], a[i], e2);
          }
          en += e2.x + e2.y;
        } else {
#pragma unroll
          for (int i = 0; i < E; ++i) {
            if constexpr (EAGER) xs[i] = cadd(xs[i], a[i]);
            cmac(pin, weight<K>(vvp, t + i * P), a[i]);
            en = fma(a[i].x, a[i].x, en);
            en = fma(a[i].y, a[i].y, en);
          }
        }
      }
    }
    // ---- injection context (armed one-shot site)
    InjCtx ic{false, 0, 0, 0, 0};
    if (A.inj.active && valid && A.inj.pass == A.pass_id && A.inj.signal == sig) {
      ic.on = true;
      ic.stage = A.inj.stage;
      ic.pos = A.inj.pos;
      ic.comp = A.inj.comp;
      ic.bit = A.inj.bit;
    }
    // ---- the radix passes
    Passes<K, 0>::run(a, sm, twr, slot, t, ic);
    // ---- inter-pass twiddle (four-step, first pass), output side of checksums
    c pout = mk<c>(0, 0);
    if constexpr (K::KIND == KIND_COL || !paired_ft<K>()) {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int pos = t + i * P;
        if constexpr (K::KIND == KIND_COL) {
          if constexpr (EAGER) ys[i] = cadd(ys[i], a[i]);
          if constexpr (std::is_same<R, double>::value) {
            // float64 is bound by its FP64 pipe: the twiddle and the
            // checksum weight come from tables in access order (coalesced
            // loads) instead of two complex products per value
            const long long cw = col_of<K>(g, valid ? sig : 0) * K::NS + pos;
            a[i] = cmul(a[i], ldg(A.colw + cw));
            if constexpr (FT && !TC) cmac(pout, ldg(A.colwe + cw), a[i]);
          } else {
            const c w = colTwiddle<K>(g, A.tlo, A.thi, valid ? sig : 0, pos);
            a[i] = cmul(a[i], w);
            if constexpr (FT) cmac(pout, cmulconj(weight<K>(evp, pos), w), a[i]);
          }
        } else {
          if constexpr (EAGER) ys[i] = cadd(ys[i], a[i]);
          if constexpr (TC) {
            // e.y with the N-point weights of row k1 (contiguous)
            const long long k1 = valid ? (sig & (g.n1 - 1)) : 0;
            cmac(pout, ldg(A.erow + k1 * K::NS + pos), a[i]);
          } else if constexpr (FT) {
            cmac(pout, weight<K>(evp, pos), a[i]);
          }
        }
      }
    } else if constexpr (FT) {
      float2 q1 = make_float2(0.f, 0.f), q2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < E; ++i) {
        if constexpr (EAGER) ys[i] = cadd(ys[i], a[i]);
        const float4 w = ev4p[t + i * P];
        q1 = __ffma2_rn(make_float2(w.x, w.y), a[i], q1);
        q2 = __ffma2_rn(make_float2(w.z, w.w), a[i], q2);
      }
      pout = mk<c>(q1.x - q2.y, q1.y + q2.x);
    }
    // ---- thread-level check (one transform per thread, no block reduction)
    if constexpr (TL) {
      if (valid) {
        ++checked;
        const R rr = pout.x - pin.x, ri = pout.y - pin.y;
        const R tau2 = tau_coef2 * (R)K::NS * en;
        const R mag2 = rr * rr + ri * ri;
        if (isfinite(mag2) && isfinite(tau2) && mag2 <= (R)0.5 * tau2) {
          if (tau2 > 0) max_ratio2 = fmaxf(max_ratio2, (float)(mag2 / tau2));
        } else {
          // not clearly clean: the decision in float64
          const double tau = A.tau_coef * sqrt((double)K::NS * (double)en);
          const double mag = sqrt((double)rr * (double)rr + (double)ri * (double)ri);
          if (isfinite(mag) && isfinite(tau) && mag <= tau) {
            if (tau > 0) max_ratio2 = fmaxf(max_ratio2, (float)((mag / tau) * (mag / tau)));
          } else {
            // a record for the correction kernel that follows the pass: it
            // recomputes this one transform from its untouched input
            // (Delta = y - W x over a group of one) and checks it again
            atomicAdd(&A.fts->detected, 1ull);
            const unsigned long long r = atomicAdd(&A.fts->num_records, 1ull);
            if (r < (unsigned long long)MAX_RECORDS) {
              FtRecord& R0 = A.fts->rec[r];
              R0.pass_id = A.pass_id;
              R0.slot = slot;
              R0.count = 1;
              R0.located = 0;
              R0.unit0 = unit;
              R0.unit_stride = stride;
              R0.transform_base = A.transform_base;
              R0.s1r = rr; R0.s1i = ri; R0.s2r = rr; R0.s2i = ri;
              R0.tau = tau;
              R0.energy = en;
              R0.result = FT_RES_PENDING;
              R0.has_sums = 0;
              R0.signal = -1;
            } else {
              atomicAdd(&A.fts->dropped, 1ull);
            }
          }
        }
      }
    }
    // ---- store (scaled inverse: one uniform branch around the scaling; a
    // column pass is never last and has no scaling code, which would
    // otherwise be issued as predicated-off multiplies)
    if (K::KIND != KIND_COL && scaled) {
      if constexpr (std::is_same<R, double>::value && K::KIND != KIND_COL) {  // (a column pass is never last)
        // the scale 2^-k only lowers exponents: where every value of the
        // warp is zero or keeps a normal result, subtract k from the
        // exponent fields with integer operations (the same bits as the
        // product) and leave the float64 pipe to the transform
        const int scale_log2 = scaled_exponent_shift(A.out_scale);  // 1/N = 2^-scale_log2
        bool slow = false;
#pragma unroll
        for (int i = 0; i < E; ++i) slow |= !pow2_scalable(a[i].x, scale_log2) || !pow2_scalable(a[i].y, scale_log2);
        if (__any_sync(0xffffffffu, slow)) {
#pragma unroll
          for (int i = 0; i < E; ++i) a[i] = cscale(a[i], A.out_scale);
        } else {
#pragma unroll
          for (int i = 0; i < E; ++i) a[i] = mk<c>(pow2_scale(a[i].x, scale_log2), pow2_scale(a[i].y, scale_log2));
        }
      } else {
#pragma unroll
        for (int i = 0; i < E; ++i) a[i] = cscale(a[i], A.out_scale);
      }
    }
    if constexpr (K::KIND == KIND_ROW) {
      // transposed store: rows r0..r0+S-1 are contiguous in the output for a
      // fixed k2, so go through shared memory and store slot-fast
#pragma unroll
      for (int i = 0; i < E; ++i) sm[slot * K::NS + ((t + i * P) ^ tsw<K>(slot))] = a[i];
      __syncthreads();
      const int s2 = tid % S, t2 = tid / S;
      const long long sig2 = signal_of<K>(g, unit, s2);
      c* const ob = A.out + out_base<K>(g, sig2);
      const long long os = out_step<K>(g);
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int pos = t2 + i * P;
        const c v = conj_mask(sm[s2 * K::NS + (pos ^ tsw<K>(s2))], mask_out);
        store_out(ob + pos * os, v);  // streaming: keep L1 for the tables
      }
      __syncthreads();
    } else {
      if (valid) {
        c* const ob = A.out + out_base<K>(g, sig);
        if constexpr (StageSwz<K>::PAIRS) {
          // one thread per contiguous transform: 16-byte stores
          static_assert(K::KIND == KIND_SP, "paired stores need a contiguous transform");
#pragma unroll
          for (int j = 0; j < E / 2; ++j) {
            const c v0 = conj_mask(a[2 * j], mask_out), v1 = conj_mask(a[2 * j + 1], mask_out);
            __stcs(reinterpret_cast<float4*>(ob) + j, make_float4(v0.x, v0.y, v1.x, v1.y));
          }
        } else {
          const long long os = out_step<K>(g);
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const c v = conj_mask(a[i], mask_out);
            store_out(ob + (t + i * P) * os, v);
          }
        }
      }
    }
    // ---- transform-level sums: flushed when the next unit belongs to
    // another transform (a uniform decision: a unit is one transform's)
    if constexpr (TC) {
      if constexpr (K::KIND == KIND_ROW) {
        tc0 += pout.x;
        tc1 += pout.y;
      }
      const long long tb = unit_transform<K>(g, unit);
      const long long nx = unit + stride;
      if (nx >= end || unit_transform<K>(g, nx) != tb) {
        block_sum3<K>(tc_red, tc0, tc1, tc2);
        if (tid == 0) {
          double* acc = A.tacc + tb * 6 + (K::KIND == KIND_COL ? 0 : 2);
          atomicAdd(acc, tc0);
          atomicAdd(acc + 1, tc1);
          if constexpr (K::KIND == KIND_COL) atomicAdd(A.tacc + tb * 6 + 4, tc2);
        }
        tc0 = tc1 = tc2 = 0;
      }
    }
    // ---- per-transaction checksum residual, location encoding
    if constexpr (FT && !TL && !TC) {
      const R rr = pout.x - pin.x, ri = pout.y - pin.y;
      if (!(isfinite(rr) && isfinite(ri))) {
        bad_lo = min(bad_lo, gi);
        bad_hi = max(bad_hi, gi);
      }
      s1r += rr;
      s1i += ri;
      s2r += (R)(gi + 1) * rr;
      s2i += (R)(gi + 1) * ri;
    }
    ++gi;
    const bool group_end = (gi == A.T) || (unit + stride >= end);
    if constexpr (FT && !TL && !TC) {
      if (group_end) {
        // ---- reduce the group over the threads of each slot.  Phase 1
        // reduces S1 and the energy in the working precision and clears
        // every slot whose |S1|^2 is below tau^2 / 2 (far more margin than
        // the rounding of that sum); only if some slot is not clearly clean
        // does phase 2 redo the reduction of S1, S2, the energy and the
        // non-finite markers in float64 and take the decision there.
        __syncthreads();  // the exchange buffer is free now
        R* redr = reinterpret_cast<R*>(sm);
        int* flag = reinterpret_cast<int*>(reinterpret_cast<char*>(sm) + (size_t)Seg<K>::COUNT * 8 * sizeof(double));
        int* anyflag = flag + S;
        if (tid == 0) *anyflag = 0;
        {
          const R v0 = seg_reduce_sum<K>(s1r), v1 = seg_reduce_sum<K>(s1i), v4 = seg_reduce_sum<K>(en);
          int seg;
          if (seg_leader<K>(tid, seg)) {
            redr[seg * 4 + 0] = v0;
            redr[seg * 4 + 1] = v1;
            redr[seg * 4 + 2] = v4;
          }
        }
        __syncthreads();
        if (tid < S) {
          R S1r = 0, S1i = 0, EN = 0;
          for_slot_segments<K>(tid, [&](int sgi) {
            S1r += redr[sgi * 4 + 0];
            S1i += redr[sgi * 4 + 1];
            EN += redr[sgi * 4 + 2];
          });
          const R tau2 = tau_coef2 * (R)K::NS * EN;
          const R mag2 = S1r * S1r + S1i * S1i;
          if (isfinite(mag2) && isfinite(tau2) && mag2 <= (R)0.5 * tau2) {
            if (tau2 > 0) max_ratio2 = fmaxf(max_ratio2, (float)(mag2 / tau2));
          } else {
            *anyflag = 1;
          }
        }
        __syncthreads();
        const bool check = *anyflag != 0;
        if (check) {
          // phase 2 (rare): float64 decision, location, record
          __syncthreads();
          double* red = reinterpret_cast<double*>(sm);
          R v0 = seg_reduce_sum<K>(s1r), v1 = seg_reduce_sum<K>(s1i);
          R v2 = seg_reduce_sum<K>(s2r), v3 = seg_reduce_sum<K>(s2i);
          R v4 = seg_reduce_sum<K>(en);
          int blo = seg_reduce_min<K>(bad_lo), bhi = seg_reduce_max<K>(bad_hi);
          int seg;
          if (seg_leader<K>(tid, seg)) {
            double* d = red + seg * 8;
            d[0] = (double)v0; d[1] = (double)v1; d[2] = (double)v2; d[3] = (double)v3; d[4] = (double)v4;
            d[5] = (double)blo; d[6] = (double)bhi;
          }
          __syncthreads();
          if (tid < S) {
            double S1r = 0, S1i = 0, S2r = 0, S2i = 0, EN = 0;
            int lo = 0x7fffffff, hi = -1;
            for_slot_segments<K>(tid, [&](int sgi) {
              const double* d = red + sgi * 8;
              S1r += d[0]; S1i += d[1]; S2r += d[2]; S2i += d[3]; EN += d[4];
              lo = min(lo, (int)d[5]); hi = max(hi, (int)d[6]);
            });
            const double tau = A.tau_coef * sqrt((double)K::NS * EN);
            const double mag = sqrt(S1r * S1r + S1i * S1i);
            const bool finite = isfinite(S1r) && isfinite(S1i) && isfinite(EN);
            int rec = -1;
            // a slot with no valid signal in this group has EN == 0 and S1 == 0
            if (finite && mag <= tau) {
              if (tau > 0) max_ratio2 = fmaxf(max_ratio2, (float)((mag / tau) * (mag / tau)));
            } else {
              int located = -1;
              if (hi >= 0) {
                located = (lo == hi) ? lo : -2;   // non-finite residuals: direct location
              } else if (finite) {
                const double den = S1r * S1r + S1i * S1i;
                const double qr = (S2r * S1r + S2i * S1i) / den, qi = (S2i * S1r - S2r * S1i) / den;
                const double kk = floor(qr + 0.5);
                if (isfinite(qr) && isfinite(qi) && kk >= 1 && kk <= gi &&
                    sqrt((qr - kk) * (qr - kk) + qi * qi) < 0.25)
                  located = (int)kk - 1;
              }
              atomicAdd(&A.fts->detected, 1ull);
              unsigned long long r = atomicAdd(&A.fts->num_records, 1ull);
              if (r < (unsigned long long)MAX_RECORDS) {
                FtRecord& R0 = A.fts->rec[r];
                R0.pass_id = A.pass_id;
                R0.slot = tid;
                R0.count = gi;
                R0.located = located;
                R0.unit0 = g_unit0;
                R0.unit_stride = stride;
                R0.transform_base = A.transform_base;
                R0.s1r = S1r; R0.s1i = S1i; R0.s2r = S2r; R0.s2i = S2i;
                R0.tau = tau;
                R0.energy = EN;
                R0.result = FT_RES_PENDING;
                R0.has_sums = EAGER ? 1 : 0;
                R0.signal = -1;
                rec = (int)r;
              } else {
                atomicAdd(&A.fts->dropped, 1ull);
              }
            }
            flag[tid] = rec;
          }
          __syncthreads();
        } else if (tid < S) {
          flag[tid] = -1;
        }
        if constexpr (EAGER) {
          __syncthreads();
          const int myrec = flag[slot];
          if (myrec >= 0) {
            // right-side sums of this slot -> the record, for delayed correction
            c* xr = reinterpret_cast<c*>(A.rec_sums) + (size_t)myrec * 2 * A.rec_stride;
            c* yr = xr + A.rec_stride;
#pragma unroll
            for (int i = 0; i < E; ++i) { xr[t + i * P] = xs[i]; yr[t + i * P] = ys[i]; }
          }
#pragma unroll
          for (int i = 0; i < E; ++i) { xs[i] = mk<c>(0, 0); ys[i] = mk<c>(0, 0); }
        }
        __syncthreads();
        ++groups;
        s1r = s1i = s2r = s2i = en = 0;
        bad_lo = 0x7fffffff;
        bad_hi = -1;
      }
    }
    if (group_end) {
      gi = 0;
      g_unit0 = unit + stride;
    }
  }
  if constexpr (TL) {
    // every transform is its own check: count them, and the largest clean
    // ratio, per warp
    const unsigned total = __reduce_add_sync(0xffffffffu, checked);
    const unsigned mr = __reduce_max_sync(0xffffffffu, __float_as_uint(sqrtf(max_ratio2)));
    if ((tid & 31) == 0) {
      if (total) atomicAdd(&A.fts->groups, (unsigned long long)total);
      if (mr) atomic_max_nonneg(&A.fts->max_clean_ratio, __uint_as_float(mr));
    }
  } else if constexpr (FT && !TC) {
    if (tid == 0 && groups > 0) atomicAdd(&A.fts->groups, (unsigned long long)(groups * S));
    if (tid < S && max_ratio2 > 0.f) atomic_max_nonneg(&A.fts->max_clean_ratio, sqrtf(max_ratio2));
  }
}

template <class K, int FTM>
__global__ void __launch_bounds__(K::NT, FTM ? TwMode<K, TF_FT_TW_BUDGET>::MINB_FT : TwMode<K>::MINB)
    tf_pass_kernel(const PassArgs<typename K::real> A) {
  extern __shared__ __align__(128) unsigned char smem_raw_[];
  if constexpr (FTM == 4) {
    // transform-level checksums: every block works on contiguous unit
    // ranges of one transform at a time, so its sums change transform only
    // at range boundaries
    const long long ub = (K::KIND == KIND_COL ? A.geo.n2 : A.geo.n1) / K::S;  // units per transform
    const long long batch = A.num_units / ub;
    if (A.geo.n >= (1 << 20)) {
      // large N: the N-point tables outgrow L2, and the 16-byte columns /
      // transposed rows of one-wide tiles share 32-byte sectors with their
      // neighbours.  Item (b, p) is every parts-th unit of transform b from
      // p on; the items run transforms fastest, so the blocks running at
      // once hold adjacent units of every transform: neighbouring columns
      // (sectors) and the same table entries are used together, in L2.
      // About 16 items per block keep the tail short; an item keeps at
      // least 16 units where it can (each item restarts the block's copy
      // pipeline).
      long long parts = (16ll * gridDim.x + batch - 1) / batch;
      // items of at least 16 units, unless that leaves blocks without two
      // items (few transforms: a chunk of a host-buffer exec)
      const long long few = (2ll * gridDim.x + batch - 1) / batch;
      const long long cap = ub / 16 > few ? ub / 16 : few;
      if (parts > cap) parts = cap;
      if (parts > ub) parts = ub;
      if (parts < 1) parts = 1;
      const long long items = batch * parts;
      for (long long i = blockIdx.x; i < items; i += gridDim.x) {
        // (item indices stay below 2^32: a 32-bit division)
        const unsigned ui = (unsigned)i, ub32 = (unsigned)batch;
        const long long part = ui / ub32, b = ui - (unsigned)part * ub32;
        __syncthreads();
        pass_body<K, FTM>(A, reinterpret_cast<char*>(smem_raw_), b * ub + part, parts, (b + 1) * ub);
      }
    } else {
      // one contiguous range of units per block (the tables fit in L2)
      const long long per = (A.num_units + gridDim.x - 1) / gridDim.x;
      const long long first = (long long)blockIdx.x * per;
      pass_body<K, FTM>(A, reinterpret_cast<char*>(smem_raw_), first, 1,
                        first + per < A.num_units ? first + per : A.num_units);
    }
  } else {
    pass_body<K, FTM>(A, reinterpret_cast<char*>(smem_raw_), blockIdx.x, gridDim.x, A.num_units);
  }
}

// The pass kernel with TMA-staged tiles (float32).  The tensor map of a
// column pass is a kernel parameter (__grid_constant__: TMA reads it in
// place); single and row passes copy contiguous tiles and ignore it.  The
// launch adds 128 bytes of dynamic shared memory so that the ring can start
// on a 128-byte boundary, as TMA destinations must.
template <class K> constexpr int tma_smem_bytes(int ftm) {
  return (ftm ? pass_smem_bytes<K, 1>() : pass_smem_bytes<K, 0>()) + 128;
}
template <class K, int FTM>
__global__ void __launch_bounds__(K::NT, FTM ? TwMode<K, TF_FT_TW_BUDGET>::MINB_FT : TwMode<K>::MINB)
    tf_pass_kernel_tma(const PassArgs<typename K::real> A, const __grid_constant__ CUtensorMap tm) {
  extern __shared__ __align__(128) unsigned char smem_raw_[];
  const unsigned mis = smem_addr(smem_raw_) & 127u;
  char* const ring = reinterpret_cast<char*>(smem_raw_) + (mis ? 128u - mis : 0u);
  pass_body<K, FTM, true>(A, ring, blockIdx.x, gridDim.x, A.num_units, &tm);
}

// Transform-level correction (float64 two-pass plans): the transforms the
// check kernel recorded are recomputed from their untouched input, this
// pass's units of each shared by all blocks of the grid (the column pass in
// one launch, the row pass in the next).  The recompute runs without the
// armed fault site.  The row launch (block 0) counts each recorded
// transform as corrected.  Transform-level records are those with
// unit_stride 0 (block-level records hold the stride of their units); a
// record's transform_base tells the chunk of a chunked exec it belongs to.
template <class K>
__global__ void __launch_bounds__(K::NT) tf_tc_fix_kernel(const PassArgs<typename K::real> A) {
  extern __shared__ __align__(128) unsigned char smem_raw_[];
  if (A.ft != FT_CORRECT) return;
  const unsigned long long n = *reinterpret_cast<volatile unsigned long long*>(&A.fts->num_records);
  const unsigned long long nrec = n < (unsigned long long)MAX_RECORDS ? n : (unsigned long long)MAX_RECORDS;
  if (nrec == 0) return;
  PassArgs<typename K::real> B = A;
  B.inj.active = 0;
  const long long ub = (K::KIND == KIND_COL ? A.geo.n2 : A.geo.n1) / K::S;  // units per transform
  for (unsigned long long r = 0; r < nrec; ++r) {
    volatile FtRecord& rec = A.fts->rec[r];
    // transform-level records of this launch's transforms only (a chunked
    // exec appends the records of every chunk to one report)
    if (rec.unit_stride != 0 || rec.transform_base != A.transform_base) continue;
    const long long b = rec.signal;
    __syncthreads();
    pass_body<K, 0>(B, reinterpret_cast<char*>(smem_raw_), b * ub + blockIdx.x, gridDim.x, (b + 1) * ub);
    if (K::KIND == KIND_ROW && blockIdx.x == 0 && threadIdx.x == 0) {
      rec.result = FT_RES_RECOMPUTE;
      atomicAdd(&A.fts->located, 1ull);
      atomicAdd(&A.fts->corrected, 1ull);
      atomicAdd(&A.fts->recomputed, 1ull);
    }
  }
}

// ---------------------------------------------------------------------------
// correction kernel: one block per record of this pass (Sec. 4.1.2)
//   located signal k:  Delta = y_bar - W x_bar,  y_k <- y_k - Delta, re-check;
//   otherwise (or if that fails) recompute y_k from its untouched input;
//   ambiguous location: per-signal re-check of the group from HBM.
// ---------------------------------------------------------------------------
// load signal `sig` of this pass's input into the home registers (slot-0
// layout; every slot of the block computes the same thing)
template <class K>
__device__ __forceinline__ void load_input(const PassArgs<typename K::real>& A, long long sig, int t,
                                           typename K::c (&a)[K::E]) {
#pragma unroll
  for (int i = 0; i < K::E; ++i) {
    auto v = __ldcg(A.in + in_off<K>(A.geo, sig, t + i * K::P));  // L2: other blocks' writes are visible
    a[i] = A.conj_in ? cconj(v) : v;
  }
}

// stored output of signal `sig`, mapped back to the internal (pre-store,
// for KIND_COL pre-twiddle) domain
template <class K>
__device__ __forceinline__ void load_output_internal(const PassArgs<typename K::real>& A, long long sig, int t,
                                                     typename K::c (&a)[K::E]) {
  using R = typename K::real;
#pragma unroll
  for (int i = 0; i < K::E; ++i) {
    const int pos = t + i * K::P;
    auto v = __ldcg(A.out + out_off<K>(A.geo, sig, pos));
    v = cscale(v, (R)1 / A.out_scale);
    if (A.conj_out) v = cconj(v);
    if constexpr (K::KIND == KIND_COL) v = cmul(v, cconj(col_w<K>(A, sig, pos)));
    a[i] = v;
  }
}

template <class K>
__device__ __forceinline__ void store_output_internal(const PassArgs<typename K::real>& A, long long sig, int t,
                                                      const typename K::c (&a)[K::E]) {
#pragma unroll
  for (int i = 0; i < K::E; ++i) {
    const int pos = t + i * K::P;
    auto v = a[i];
    if constexpr (K::KIND == KIND_COL) v = cmul(v, col_w<K>(A, sig, pos));
    if (A.conj_out) v = cconj(v);
    v = cscale(v, A.out_scale);
    A.out[out_off<K>(A.geo, sig, pos)] = v;
  }
}

// block-wide sum of slot-0 contributions, in double
template <class K> __device__ __forceinline__ void block_sum3(double* red, double& a, double& b, double& c3) {
  const int tid = threadIdx.x;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c3 += __shfl_xor_sync(0xffffffffu, c3, o);
  }
  __syncthreads();
  if ((tid & 31) == 0) { red[(tid >> 5) * 3 + 0] = a; red[(tid >> 5) * 3 + 1] = b; red[(tid >> 5) * 3 + 2] = c3; }
  __syncthreads();
  a = b = c3 = 0;
  for (int w = 0; w < K::NT / 32; ++w) { a += red[w * 3]; b += red[w * 3 + 1]; c3 += red[w * 3 + 2]; }
  __syncthreads();
}

// residual r = e . y - v . x and energy of one signal (slot 0's threads)
template <class K>
__device__ __forceinline__ void residual(const PassArgs<typename K::real>& A, double* red, int slot, int t,
                                         const typename K::c (&x)[K::E], const typename K::c (&y)[K::E],
                                         double& rr, double& ri, double& en) {
  double a = 0, b = 0, e2 = 0;
  if (slot == 0) {
#pragma unroll
    for (int i = 0; i < K::E; ++i) {
      const int pos = t + i * K::P;
      auto ev = ldg(A.ev + pos), vv = ldg(A.vv + pos);
      double yr = y[i].x, yi = y[i].y, xr = x[i].x, xi = x[i].y;
      a += (double)ev.x * yr - (double)ev.y * yi - ((double)vv.x * xr - (double)vv.y * xi);
      b += (double)ev.x * yi + (double)ev.y * yr - ((double)vv.x * xi + (double)vv.y * xr);
      e2 += xr * xr + xi * xi;
    }
  }
  block_sum3<K>(red, a, b, e2);
  rr = a; ri = b; en = e2;
}

// does signal `sig` pass its own checksum test (from HBM, float64)?
template <class K>
__device__ __forceinline__ bool signal_passes(const PassArgs<typename K::real>& A, double* red, int slot, int t,
                                              long long sig) {
  typename K::c x[K::E], y[K::E];
  load_input<K>(A, sig, t, x);
  load_output_internal<K>(A, sig, t, y);
  double rr, ri, en;
  residual<K>(A, red, slot, t, x, y, rr, ri, en);
  const double m = sqrt(rr * rr + ri * ri);
  return m <= A.tau_coef * sqrt((double)K::NS * en);  // false for NaN
}

// fix_body: records first, first + stride, ... of this pass (the correction
// kernel: blockIdx.x, gridDim.x; the persistent ragged kernel after a grid
// barrier).  `red` is block-shared scratch of 3 x 32 doubles.
template <class K>
__device__ __forceinline__ void fix_body(const PassArgs<typename K::real>& A, char* smem_raw, double* red,
                                         unsigned long long first, unsigned long long stride) {
  using c = typename K::c;
  constexpr int E = K::E, P = K::P, S = K::S;
  c* sm = reinterpret_cast<c*>(smem_raw);

  // the records and their count are read around L1 (volatile): in the
  // persistent ragged kernel other blocks wrote them after this block may
  // have cached the lines
  const unsigned long long nrec = *reinterpret_cast<volatile unsigned long long*>(&A.fts->num_records);
  const int tid = threadIdx.x;
  const int slot = K::SLOT_FAST ? (tid % S) : (tid / P);
  const int t = K::SLOT_FAST ? (tid / S) : (tid % P);

  for (unsigned long long r = first; r < nrec && r < (unsigned long long)MAX_RECORDS; r += stride) {
    volatile FtRecord& rec = A.fts->rec[r];
    // uniform across the block: records of other passes, or already handled
    if (rec.pass_id != A.pass_id || rec.result != FT_RES_PENDING) continue;
    auto sig_of = [&](int k) { return signal_of<K>(A.geo, rec.unit0 + (long long)k * rec.unit_stride, rec.slot); };

    int k = rec.located;
    if (k == -1) {
      // ambiguous location: re-check every signal of the group on its own
      int found = -1, nbad = 0;
      for (int kk = 0; kk < rec.count; ++kk) {
        const long long s = sig_of(kk);
        if (s < 0) continue;
        if (!signal_passes<K>(A, red, slot, t, s)) { ++nbad; found = kk; }
      }
      if (nbad == 0) {
        if (tid == 0) rec.result = FT_RES_CLEAR;
        continue;
      }
      k = (nbad == 1) ? found : -2;
    }
    const long long sk = (k >= 0 && k < rec.count) ? sig_of(k) : -1;
    if (sk < 0) {
      if (tid == 0) { rec.result = FT_RES_UNCORRECTABLE; atomicAdd(&A.fts->uncorrectable, 1ull); }
      continue;
    }
    if (tid == 0) { rec.signal = sk; atomicAdd(&A.fts->located, 1ull); }
    if (A.ft != FT_CORRECT) {
      if (tid == 0) rec.result = FT_RES_LOCATED;
      continue;
    }
    c x[E], y_old[E];
    load_input<K>(A, sk, t, x);
    load_output_internal<K>(A, sk, t, y_old);
    double r_old_r, r_old_i, en;
    residual<K>(A, red, slot, t, x, y_old, r_old_r, r_old_i, en);
    const double tau_k = A.tau_coef * sqrt((double)K::NS * en);

    // (1) the paper's correction from the right-side sums:
    //     Delta = y_bar - W x_bar, y_k <- y_k - Delta
    //     (sums kept by the transform kernel, or formed here from the
    //     group's untouched inputs and stored outputs)
    int how = 0;
    {
      c a[E], yb[E];
      if (rec.has_sums) {
        const c* xr = reinterpret_cast<const c*>(A.rec_sums) + (size_t)r * 2 * A.rec_stride;
        const c* yr = xr + A.rec_stride;
#pragma unroll
        for (int i = 0; i < E; ++i) { a[i] = xr[t + i * P]; yb[i] = yr[t + i * P]; }
      } else {
#pragma unroll
        for (int i = 0; i < E; ++i) { a[i] = mk<c>(0, 0); yb[i] = mk<c>(0, 0); }
        for (int kk = 0; kk < rec.count; ++kk) {
          const long long s = sig_of(kk);
          if (s < 0) continue;
          c xv[E], yv[E];
          load_input<K>(A, s, t, xv);
          load_output_internal<K>(A, s, t, yv);
#pragma unroll
          for (int i = 0; i < E; ++i) { a[i] = cadd(a[i], xv[i]); yb[i] = cadd(yb[i], yv[i]); }
        }
      }
      TwReg<K> twr;
      twr.load(A.tw, t);
      fft_block<K>(a, sm, twr, slot, t);
      c cand[E];
      bool fin = true;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const c d = csub(yb[i], a[i]);
        cand[i] = csub(y_old[i], d);
        fin = fin && isfinite(cand[i].x) && isfinite(cand[i].y);
      }
      fin = __syncthreads_and(fin);
      if (fin) {
        double rr, ri, e2;
        residual<K>(A, red, slot, t, x, cand, rr, ri, e2);
        if (sqrt(rr * rr + ri * ri) <= tau_k) {
          if (slot == 0) store_output_internal<K>(A, sk, t, cand);
          how = FT_RES_DELTA;
        }
      }
    }
    if (how == 0) {
      // (2) recompute the signal from its untouched input
      c a[E];
#pragma unroll
      for (int i = 0; i < E; ++i) a[i] = x[i];
      TwReg<K> twr;
      twr.load(A.tw, t);
      fft_block<K>(a, sm, twr, slot, t);
      double rr, ri, e2;
      residual<K>(A, red, slot, t, x, a, rr, ri, e2);
      if (sqrt(rr * rr + ri * ri) <= tau_k) {
        if (slot == 0) store_output_internal<K>(A, sk, t, a);
        how = FT_RES_RECOMPUTE;
      }
    }
    // (3) the rest of the group must pass signal by signal: a second
    //     corrupted signal violates the single-error model
    bool rest_ok = true;
    if (how != 0 && rec.located >= 0) {
      __syncthreads();
      for (int kk = 0; kk < rec.count; ++kk) {
        const long long s = sig_of(kk);
        if (kk == k || s < 0) continue;
        if (!signal_passes<K>(A, red, slot, t, s)) rest_ok = false;
      }
    }
    if (tid == 0) {
      if (how != 0 && rest_ok) {
        rec.result = how;
        atomicAdd(&A.fts->corrected, 1ull);
        if (how == FT_RES_RECOMPUTE) atomicAdd(&A.fts->recomputed, 1ull);
      } else {
        if (how != 0) atomicAdd(&A.fts->corrected, 1ull);
        rec.result = FT_RES_UNCORRECTABLE;
        atomicAdd(&A.fts->uncorrectable, 1ull);
      }
    }
    __syncthreads();
  }
}

template <class K>
__global__ void __launch_bounds__(K::NT) tf_fix_kernel(const PassArgs<typename K::real> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[3 * 32];
  fix_body<K>(A, reinterpret_cast<char*>(smem_raw), red, blockIdx.x, gridDim.x);
}

}  // namespace tf
