// Host tables of the library (TurboFFT Sec. 5.1.2: twiddles precomputed
// instead of evaluating trigonometric functions on the device; Sec. 4.2.2:
// the left encoding vector e^T W precomputed outside the transform),
// evaluated in long double and rounded once to the plan's precision; the
// kernel registry; plan-owned device allocations.
#include <cuda_runtime.h>
#include <math.h>
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
  return upload<double>(p, &pp.d_tw, tw) && upload<double>(p, &pp.d_ev, e) && upload<double>(p, &pp.d_vv, v);
}

namespace {
// Inter-pass twiddles of a float64 column pass over length L = n1 * n2 in
// the pass's access order: colw[n2 * n1 + k1] = w_L^{k1 n2}, the same
// product of the two small tables that float32 column passes form per value,
// and colwe = e_k1 conj(colw), the output-side checksum weight of a value
// taken after its twiddle.
__global__ void col_fill_kernel(double2* colw, double2* colwe, const double2* tlo, const double2* thi,
                                const double2* ev, int n1, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long n2 = i / n1;
    const int k1 = (int)(i - n2 * n1);
    const unsigned q = (unsigned)k1 * (unsigned)n2;
    const double2 a = thi[q >> 12], b = tlo[q & 4095u];
    const double2 w = make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
    colw[i] = w;
    if (colwe) {
      const double2 e = ev[k1];
      colwe[i] = make_double2(e.x * w.x + e.y * w.y, e.y * w.x - e.x * w.y);
    }
  }
}
}  // namespace

bool col_tables(turbofft_plan* p, PassPlan& pp, const void* tlo, const void* thi, bool weights) {
  const long long total = (long long)pp.g_n1 * pp.g_n2;
  const size_t bytes = (size_t)total * sizeof(double2);
  if (!dev_alloc(p, &pp.d_colw, bytes)) return false;
  if (weights && !dev_alloc(p, &pp.d_colwe, bytes)) return false;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int threads = 256;
  const long long want = (total + threads - 1) / threads;
  const int blocks = (int)(want < 8192 ? want : 8192);
  col_fill_kernel<<<blocks, threads, 0, st>>>(static_cast<double2*>(pp.d_colw), static_cast<double2*>(pp.d_colwe),
                                              static_cast<const double2*>(tlo), static_cast<const double2*>(thi),
                                              static_cast<const double2*>(pp.d_ev), pp.g_n1, total);
  const bool ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
  cudaStreamDestroy(st);
  return ok;
}

}  // namespace tfh
