/*
 * Reference (oracle) implementation of the batched 1-D complex DFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; it is used by tests/, by __graft_entry__.smoke() and by the
 * CPU-baseline leg of bench.py.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * What it computes (TurboFFT, Sec. 2.2.1, definition of the DFT):
 *     forward  y_j = sum_n x_n exp(-2 pi i j n / N)
 *     inverse  x_j = (1/N) sum_n y_n exp(+2 pi i j n / N)
 * Complex numbers are stored interleaved (re, im) as doubles.
 *
 * Two routines:
 *   oracle_dft_naive  O(N^2) sum of the definition, accumulated in long
 *                     double with the phase reduced exactly in integers
 *                     (j*n mod N) before the trigonometric call.
 *   oracle_fft        iterative radix-2 decimation-in-time FFT in double:
 *                     bit-reversal permutation, then log2(N) butterfly
 *                     stages; twiddles exp(sign 2 pi i k/N) evaluated once
 *                     per call in long double and rounded to double.
 *                     Transforms of a batch are independent and are spread
 *                     over OpenMP threads when available.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const long double ORACLE_TWO_PI =
    6.283185307179586476925286766559005768394338798750L;

/* Number of OpenMP threads the last oracle_fft call used (1 without OpenMP). */
static int g_last_threads = 1;

int oracle_last_threads(void) { return g_last_threads; }

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Definition of the DFT summed term by term.  sign = -1 forward, +1 inverse;
 * scale multiplies every output (1/N for the scaled inverse, 1 otherwise). */
void oracle_dft_naive(int64_t n, int sign, const double *in, double *out,
                      double scale) {
  for (int64_t j = 0; j < n; ++j) {
    long double acc_re = 0.0L, acc_im = 0.0L;
    for (int64_t k = 0; k < n; ++k) {
      int64_t q = (int64_t)(((__int128)j * k) % n);
      long double ang = (long double)sign * ORACLE_TWO_PI * (long double)q /
                        (long double)n;
      long double c = cosl(ang), s = sinl(ang);
      long double xr = in[2 * k], xi = in[2 * k + 1];
      acc_re += xr * c - xi * s;
      acc_im += xr * s + xi * c;
    }
    out[2 * j] = (double)(acc_re * scale);
    out[2 * j + 1] = (double)(acc_im * scale);
  }
}

static int ilog2_exact(int64_t n) {
  int l = 0;
  while (((int64_t)1 << l) < n) ++l;
  return (((int64_t)1 << l) == n) ? l : -1;
}

/* One radix-2 transform of length n = 2^logn, in place on a (interleaved). */
static void fft_one(int64_t n, int logn, const double *tw, double *a) {
  /* bit-reversal permutation */
  for (int64_t i = 0; i < n; ++i) {
    int64_t r = 0;
    for (int b = 0; b < logn; ++b) r |= ((i >> b) & 1) << (logn - 1 - b);
    if (r > i) {
      double t0 = a[2 * i], t1 = a[2 * i + 1];
      a[2 * i] = a[2 * r];
      a[2 * i + 1] = a[2 * r + 1];
      a[2 * r] = t0;
      a[2 * r + 1] = t1;
    }
  }
  /* butterfly stages: sub-transform length m doubles every stage */
  for (int64_t m = 2; m <= n; m <<= 1) {
    int64_t half = m >> 1, step = n / m;
    for (int64_t k = 0; k < n; k += m) {
      for (int64_t j = 0; j < half; ++j) {
        double wr = tw[2 * (j * step)], wi = tw[2 * (j * step) + 1];
        double *u = a + 2 * (k + j), *v = a + 2 * (k + j + half);
        double tr = wr * v[0] - wi * v[1];
        double ti = wr * v[1] + wi * v[0];
        v[0] = u[0] - tr;
        v[1] = u[1] - ti;
        u[0] = u[0] + tr;
        u[1] = u[1] + ti;
      }
    }
  }
}

/* Batched radix-2 FFT.  in/out: batch*n interleaved complex doubles, may
 * alias.  sign = -1 forward, +1 inverse; every output is multiplied by scale.
 * nthreads <= 0 uses the OpenMP default.  Returns 0, or -1 if n is not a
 * power of two >= 1. */
int oracle_fft(int64_t n, int64_t batch, int sign, const double *in,
               double *out, double scale, int nthreads) {
  int logn = ilog2_exact(n);
  if (logn < 0 || batch < 0) return -1;
  int64_t nh = n / 2 > 0 ? n / 2 : 1;
  double *tw = (double *)malloc(sizeof(double) * 2 * (size_t)nh);
  if (!tw) return -2;
  for (int64_t k = 0; k < nh; ++k) {
    long double ang = (long double)sign * ORACLE_TWO_PI * (long double)k /
                      (long double)n;
    tw[2 * k] = (double)cosl(ang);
    tw[2 * k + 1] = (double)sinl(ang);
  }
  if (in != out) memcpy(out, in, sizeof(double) * 2 * (size_t)(n * batch));
  int used = 1;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int64_t b = 0; b < batch; ++b) {
#ifdef _OPENMP
    if (b == 0) used = omp_get_num_threads();
#endif
    double *a = out + 2 * (size_t)(b * n);
    fft_one(n, logn, tw, a);
    if (scale != 1.0)
      for (int64_t i = 0; i < 2 * n; ++i) a[i] *= scale;
  }
  g_last_threads = used;
  free(tw);
  return 0;
}
