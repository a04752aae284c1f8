/*
 * fft.c -- oracle (test infrastructure only): the unitary discrete Fourier
 * transform F of Eq. (DFT), F_{jk} = n^{-1/2} exp(-2 pi i j k / n) (0-based).
 *
 * orc_dft_brute is the definition written out (O(n^2)); orc_dft is the same
 * transform by the radix-2 Cooley-Tukey FFT (powers of two) or, for any other
 * n, Bluestein's chirp-z identity j k = (j^2 + k^2 - (j-k)^2)/2, which turns the
 * length-n DFT into a circular convolution of power-of-two length L >= 2n-1.
 * Pinned by tests against the brute-force definition and numpy.fft.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

static const double TWO_PI = 6.283185307179586476925286766559;

/* exp(sign * 2 pi i * num / den) with the argument reduced exactly first */
static zc root(int64_t num, int64_t den, int sign) {
  int64_t r = num % den;
  if (r < 0) r += den;
  double a = TWO_PI * (double)r / (double)den;
  return cos(a) + I * (double)sign * sin(a);
}

/* unnormalised radix-2 transform: x[j] <- sum_k x[k] exp(sign 2 pi i j k / L) */
static void fft_pow2(zc *x, int64_t L, int sign) {
  if (L <= 1) return;
  /* bit-reversal permutation */
  for (int64_t i = 1, j = 0; i < L; ++i) {
    int64_t bit = L >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) { zc t = x[i]; x[i] = x[j]; x[j] = t; }
  }
  zc *w = (zc *)malloc(sizeof(zc) * (size_t)(L / 2));
  for (int64_t k = 0; k < L / 2; ++k) w[k] = root(k, L, sign);
  for (int64_t len = 2; len <= L; len <<= 1) {
    int64_t half = len / 2, stride = L / len;
    for (int64_t start = 0; start < L; start += len) {
      for (int64_t k = 0; k < half; ++k) {
        zc u = x[start + k];
        zc v = x[start + k + half] * w[k * stride];
        x[start + k] = u + v;
        x[start + k + half] = u - v;
      }
    }
  }
  free(w);
}

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

void orc_dft(zc *x, int64_t n, int sign) {
  const double scale = 1.0 / sqrt((double)n);
  if (is_pow2(n)) {
    fft_pow2(x, n, sign);
    for (int64_t j = 0; j < n; ++j) x[j] *= scale;
    return;
  }
  /* Bluestein: chirp c_k = exp(sign pi i k^2 / n) = exp(sign 2 pi i (k^2 mod 2n) / (2n)) */
  int64_t L = 1;
  while (L < 2 * n - 1) L <<= 1;
  zc *c = (zc *)malloc(sizeof(zc) * (size_t)n);
  zc *a = (zc *)calloc((size_t)L, sizeof(zc));
  zc *b = (zc *)calloc((size_t)L, sizeof(zc));
  for (int64_t k = 0; k < n; ++k) {
    int64_t k2 = (int64_t)(((unsigned __int128)k * (unsigned __int128)k) % (unsigned __int128)(2 * n));
    c[k] = root(k2, 2 * n, sign);
  }
  for (int64_t k = 0; k < n; ++k) a[k] = x[k] * c[k];
  b[0] = conj(c[0]);
  for (int64_t k = 1; k < n; ++k) { b[k] = conj(c[k]); b[L - k] = conj(c[k]); }
  fft_pow2(a, L, -1);
  fft_pow2(b, L, -1);
  for (int64_t j = 0; j < L; ++j) a[j] *= b[j];
  fft_pow2(a, L, +1);
  for (int64_t j = 0; j < n; ++j) x[j] = c[j] * a[j] / (double)L * scale;
  free(c); free(a); free(b);
}

void orc_dft_brute(const zc *x, zc *out, int64_t n, int sign) {
  const double scale = 1.0 / sqrt((double)n);
  for (int64_t j = 0; j < n; ++j) {
    zc acc = 0;
    for (int64_t k = 0; k < n; ++k)
      acc += x[k] * root((int64_t)(((unsigned __int128)j * (unsigned __int128)k) % (unsigned __int128)n), n, sign);
    out[j] = acc * scale;
  }
}
