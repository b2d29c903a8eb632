// Host tables of the library (TurboFFT Sec. 5.1.2: twiddles precomputed
// instead of evaluating trigonometric functions on the device; Sec. 4.2.2:
// the left encoding vector e^T W precomputed outside the transform),
// evaluated in long double and rounded once to the plan's precision; the
// kernel registry; plan-owned device allocations.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <vector>
#include <stdint.h>
#include <string.h>

#include "tf_plan.h"

namespace tfh {

int g_num_sms = 0;

const Registry& registry() {
  static Registry r;
  return r;
}

namespace {
const ld kTwoPi = 6.283185307179586476925286766559005768394338798750L;

// SplitMix64 (Steele, Lea, Flood 2014): phase of the checksum vector
uint64_t splitmix_mix(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
}  // namespace

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

int ilog2_exact(int64_t n) {
  int l = 0;
  while (((int64_t)1 << l) < n) ++l;
  return (((int64_t)1 << l) == n) ? l : -1;
}

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

bool upload_pairs(turbofft_plan* p, void** dst, const std::vector<cld>& v) {
  // each component as hi = nearest float, lo = nearest float of the rest
  // (the long-double value rounded once into 48 significand bits)
  std::vector<float4> t(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    const ld re = v[i].real(), im = v[i].imag();
    const float rh = (float)re, ih = (float)im;
    t[i] = make_float4(rh, (float)(re - (ld)rh), ih, (float)(im - (ld)ih));
  }
  const size_t bytes = t.size() * sizeof(float4);
  if (!dev_alloc(p, dst, bytes)) return false;
  return cudaMemcpy(*dst, t.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
}

// float64 pass twiddles folded into radix-2 layers, w = c (1 + i t)
// (Linzer and Feig 1993): for each pass p > 0 of a sub-transform of ns
// points done in radix-8 passes (the last one of radix ns / 8^(NP-1)), with
// L = 8^p and omega = w_{L R}^k, k = 0 .. L-1, the R - 1 layer twiddles
//   R = 8: omega^4, omega^2, W_4 omega^2, omega, W_4 omega, W_8 omega, W_8^3 omega
//   R = 4: omega^2, omega, W_4 omega
//   R = 2: omega
// each stored as (c, t), c = Re w and t = Im w / Re w where |Re w| >= |Im w|,
// else c = Im w and t = -Re w / Im w (then applied to i b); the lowest
// mantissa bit of t says which (rounded to the nearer double with that bit).
static std::vector<double> folded_twiddles(int ns) {
  int lns = 0;
  while ((1 << lns) < ns) ++lns;
  const int np = (lns + 2) / 3;
  std::vector<double> t;
  auto put = [&](cld w) {
    const ld wr = w.real(), wi = w.imag();
    const bool sw = fabsl(wi) > fabsl(wr);
    const ld c = sw ? wi : wr;
    const ld tl = sw ? -wr / wi : wi / wr;
    double td = (double)tl;
    uint64_t bits;
    memcpy(&bits, &td, 8);
    if ((bits & 1u) != (uint64_t)sw) td = nextafter(td, ((ld)td < tl) ? (double)INFINITY : -(double)INFINITY);
    if (td == 0.0 && sw) td = nextafter(0.0, 1.0);  // +-0 carries no set bit
    t.push_back((double)c);
    t.push_back(td);
  };
  for (int q = 1; q < np; ++q) {
    const int lr = (q == np - 1) ? lns - 3 * (np - 1) : 3;
    const int r = 1 << lr;
    const int64_t l = (int64_t)1 << (3 * q);
    const int64_t n = l * r;  // omega = w_n^k; W_4 = w_n^(n/4), W_8 = w_n^(n/8)
    for (int64_t k = 0; k < l; ++k) {
      if (r == 8) {
        put(root(n, 4 * k));
        put(root(n, 2 * k));
        put(root(n, 2 * k + n / 4));
        put(root(n, k));
        put(root(n, k + n / 4));
        put(root(n, k + n / 8));
        put(root(n, k + 3 * n / 8));
      } else if (r == 4) {
        put(root(n, 2 * k));
        put(root(n, k));
        put(root(n, k + n / 4));
      } else {
        put(root(n, k));
      }
    }
  }
  if (t.empty()) t.assign(2, 0.0);  // one pass: no twiddles are read
  return t;
}

bool upload_tables(turbofft_plan* p, PassPlan& pp) {
  const int ns = pp.ns;
  std::vector<cld> tw(ns);
  for (int q = 0; q < ns; ++q) tw[q] = root(ns, q);
  if (p->pairs) return upload_pairs(p, &pp.d_tw, tw);  // no checksums
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
  const std::vector<double> lf = folded_twiddles(ns);
  return dev_alloc(p, &pp.d_tw, lf.size() * sizeof(double)) &&
         cudaMemcpy(pp.d_tw, lf.data(), lf.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         upload<double>(p, &pp.d_ev, e) && upload<double>(p, &pp.d_vv, v);
}

namespace {
// Double-double arithmetic on the host (Dekker / Knuth error-free
// transformations with FMA): about 106 significand bits, so that a product
// of two tables rounds once to float64.
struct D2 {
  double hi, lo;
};
D2 d2_of(ld v) {
  const double h = (double)v;
  return {h, (double)(v - (ld)h)};
}
D2 d2_add(D2 a, D2 b) {
  const double s = a.hi + b.hi;
  const double bb = s - a.hi;
  const double e = (a.hi - (s - bb)) + (b.hi - bb) + (a.lo + b.lo);
  const double h = s + e;
  return {h, e - (h - s)};
}
D2 d2_mul(D2 a, D2 b) {
  const double p = a.hi * b.hi;
  const double e = std::fma(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
  const double h = p + e;
  return {h, e - (h - p)};
}
D2 d2_neg(D2 a) { return {-a.hi, -a.lo}; }
double d2_round(D2 a) { return a.hi + a.lo; }
}  // namespace

// Inter-pass twiddles of a float64 column pass over length L = n1 * n2 in
// the pass's access order, computed on the host: colw[n2 * n1 + k1] =
// w_L^{k1 n2}, and colwe = e_k1 conj(colw), the output-side checksum weight
// of a value taken after its twiddle.  w_L^q = w_L^{4096 (q >> 12)} *
// w_L^{q & 4095} from two long-double tables, multiplied in double-double
// and rounded once to float64 (error below 0.5 ulp + 2^-100).
bool col_tables(turbofft_plan* p, PassPlan& pp, bool weights) {
  const int n1 = pp.g_n1;
  const long long L = (long long)pp.g_n1 * pp.g_n2;
  const size_t total = (size_t)L;
  std::vector<D2> lo_re(4096), lo_im(4096), hi_re((size_t)std::max<long long>(1, L / 4096)),
      hi_im(hi_re.size());
  for (int j = 0; j < 4096; ++j) {
    const cld w = root(L, j);
    lo_re[j] = d2_of(w.real());
    lo_im[j] = d2_of(w.imag());
  }
  for (size_t j = 0; j < hi_re.size(); ++j) {
    const cld w = root(L, (int64_t)j * 4096);
    hi_re[j] = d2_of(w.real());
    hi_im[j] = d2_of(w.imag());
  }
  std::vector<D2> e_re(n1), e_im(n1);
  if (weights) {
    const std::vector<cld> e = encoding_vector(n1);
    for (int k = 0; k < n1; ++k) {
      e_re[k] = d2_of(e[k].real());
      e_im[k] = d2_of(e[k].imag());
    }
  }
  std::vector<double2> w_tab(total), we_tab(weights ? total : 0);
  for (size_t i = 0; i < total; ++i) {
    const long long n2 = (long long)(i / (size_t)n1);
    const int k1 = (int)(i - (size_t)n2 * n1);
    const unsigned q = (unsigned)((long long)k1 * n2 % L);
    const size_t a = q >> 12, b = q & 4095u;
    const D2 wr = d2_add(d2_mul(hi_re[a], lo_re[b]), d2_neg(d2_mul(hi_im[a], lo_im[b])));
    const D2 wi = d2_add(d2_mul(hi_re[a], lo_im[b]), d2_mul(hi_im[a], lo_re[b]));
    w_tab[i] = make_double2(d2_round(wr), d2_round(wi));
    if (weights) {
      // e * conj(w) = (er wr + ei wi) + i (ei wr - er wi)
      const D2 cr = d2_add(d2_mul(e_re[k1], wr), d2_mul(e_im[k1], wi));
      const D2 ci = d2_add(d2_mul(e_im[k1], wr), d2_neg(d2_mul(e_re[k1], wi)));
      we_tab[i] = make_double2(d2_round(cr), d2_round(ci));
    }
  }
  const size_t bytes = total * sizeof(double2);
  if (!dev_alloc(p, &pp.d_colw, bytes) ||
      cudaMemcpy(pp.d_colw, w_tab.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  if (weights && (!dev_alloc(p, &pp.d_colwe, bytes) ||
                  cudaMemcpy(pp.d_colwe, we_tab.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess))
    return false;
  return true;
}

// N-point weights of transform-level checksums (float64 two-pass plans).
// e: N unit-modulus phases (SplitMix64 from the seed of the block-level
// vectors, in float64); v = W e by a float64 radix-2 FFT on the host whose
// twiddles w_N^j are double-double products of two long-double tables
// rounded once (v is only needed consistent with e to the float64
// transform's own rounding level).  Stored in the passes' access orders:
// vcol[n2 * N1 + p] = v[p * N2 + n2] (column pass), erow[k1 * N2 + k2] =
// e[k1 + N1 * k2] (row pass).
bool tc_tables(turbofft_plan* p) {
  const int64_t N = p->n;
  const int n1 = p->n1, n2 = p->n2;
  std::vector<double> er((size_t)N), ei((size_t)N), vr, vi;
  const uint64_t seed = 0x5EEDull;
  for (int64_t j = 0; j < N; ++j) {
    const uint64_t w = splitmix_mix(seed + (uint64_t)(j + 1) * 0x9E3779B97F4A7C15ull);
    const double theta = (double)(w >> 11) * 0x1p-53;
    er[(size_t)j] = std::cos(6.283185307179586476925 * theta);
    ei[(size_t)j] = std::sin(6.283185307179586476925 * theta);
  }
  // twiddles w_N^j, j < N/2
  const size_t half = (size_t)(N / 2);
  std::vector<double> twr(half), twi(half);
  {
    const size_t nhi = std::max<size_t>(1, half / 4096 + 1);
    std::vector<D2> lr(4096), li(4096), hr(nhi), hi(nhi);
    for (int j = 0; j < 4096; ++j) {
      const cld w = root(N, j);
      lr[j] = d2_of(w.real());
      li[j] = d2_of(w.imag());
    }
    for (size_t j = 0; j < nhi; ++j) {
      const cld w = root(N, (int64_t)j * 4096);
      hr[j] = d2_of(w.real());
      hi[j] = d2_of(w.imag());
    }
    for (size_t j = 0; j < half; ++j) {
      const size_t a = j >> 12, b = j & 4095u;
      twr[j] = d2_round(d2_add(d2_mul(hr[a], lr[b]), d2_neg(d2_mul(hi[a], li[b]))));
      twi[j] = d2_round(d2_add(d2_mul(hr[a], li[b]), d2_mul(hi[a], lr[b])));
    }
  }
  // v = W e: bit-reversed order, then radix-2 butterflies
  vr = er;
  vi = ei;
  for (size_t i = 1, j = 0; i < (size_t)N; ++i) {
    size_t bit = (size_t)N >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      std::swap(vr[i], vr[j]);
      std::swap(vi[i], vi[j]);
    }
  }
  for (size_t len = 2; len <= (size_t)N; len <<= 1) {
    const size_t h = len / 2, step = (size_t)N / len;
    for (size_t i = 0; i < (size_t)N; i += len)
      for (size_t k = 0; k < h; ++k) {
        const double wr = twr[k * step], wi = twi[k * step];
        const size_t q = i + k + h;
        const double tr = vr[q] * wr - vi[q] * wi, ti = vr[q] * wi + vi[q] * wr;
        vr[q] = vr[i + k] - tr;
        vi[q] = vi[i + k] - ti;
        vr[i + k] += tr;
        vi[i + k] += ti;
      }
  }
  std::vector<double2> vcol((size_t)N), erow((size_t)N);
  for (int c = 0; c < n2; ++c)
    for (int q = 0; q < n1; ++q) {
      const size_t src = (size_t)q * n2 + c;
      vcol[(size_t)c * n1 + q] = make_double2(vr[src], vi[src]);
    }
  for (int k1 = 0; k1 < n1; ++k1)
    for (int k2 = 0; k2 < n2; ++k2) {
      const size_t src = (size_t)k1 + (size_t)n1 * k2;
      erow[(size_t)k1 * n2 + k2] = make_double2(er[src], ei[src]);
    }
  const size_t bytes = (size_t)N * sizeof(double2);
  return dev_alloc(p, &p->d_vcol, bytes) &&
         cudaMemcpy(p->d_vcol, vcol.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
         dev_alloc(p, &p->d_erow, bytes) &&
         cudaMemcpy(p->d_erow, erow.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
}

}  // namespace tfh
