/*
 * dd.c -- oracle (test infrastructure only): products with A whose sums are
 * accumulated in double-double.
 *
 * At condition numbers near 1e6 the minimal-norm solution of the stored A is
 * only determined to about kappa * 2^-53 ~ 1e-10 by FP64 arithmetic (the
 * kappa-normalised errors of Tables 2 and 4 are 1e-15, i.e. raw errors near
 * 1e-9). Residuals b - A A^* y therefore need more than FP64 to certify
 * 1e-12. Each real product a*b is split exactly by TwoProd (a*b = p + e via
 * one fused multiply-add) and accumulated by TwoSum into (s, c), the
 * compensated dot product "Dot2" of Ogita, Rump & Oishi (SIAM J. Sci. Comput.
 * 26(6), 2005). The library is built with -ffp-contract=off so that TwoSum is
 * evaluated as written. The summation order of every output is the order of
 * the definition (index 0 first).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

typedef struct { double s, c; } acc2;

static inline void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double bb = x - a;
  *e = (a - (x - bb)) + (b - bb);
  *s = x;
}

static inline void acc_prod(acc2 *a, double x, double y) {
  double p = x * y;
  double e = fma(x, y, -p);                 /* TwoProd: x*y = p + e exactly */
  double s, q;
  two_sum(a->s, p, &s, &q);
  a->s = s;
  a->c += q + e;
}

/* (hi, lo) = s + c normalised so that |lo| <= ulp(hi)/2 */
static inline void acc_round(const acc2 *a, double *hi, double *lo) {
  double h, l;
  two_sum(a->s, a->c, &h, &l);
  *hi = h; *lo = l;
}

void orc_adj_matvec_dd(int64_t m, int64_t n, const zc *A, int64_t lda,
                       const zc *y_hi, const zc *y_lo, zc *x_hi, zc *x_lo) {
  const int64_t B = 256;
#pragma omp parallel for schedule(dynamic)
  for (int64_t j0 = 0; j0 < n; j0 += B) {
    const int64_t j1 = j0 + B < n ? j0 + B : n;
    acc2 re[256], im[256];
    memset(re, 0, sizeof re); memset(im, 0, sizeof im);
    for (int64_t i = 0; i < m; ++i) {
      const double yr = creal(y_hi[i]), yi = cimag(y_hi[i]);
      const double lr = y_lo ? creal(y_lo[i]) : 0.0, li = y_lo ? cimag(y_lo[i]) : 0.0;
      for (int64_t j = j0; j < j1; ++j) {
        const double ar = creal(A[i * lda + j]), ai = cimag(A[i * lda + j]);
        /* conj(a) * y = (ar yr + ai yi) + i (ar yi - ai yr) */
        acc2 *R = &re[j - j0], *M = &im[j - j0];
        acc_prod(R, ar, yr); acc_prod(R, ai, yi);
        acc_prod(M, ar, yi); acc_prod(M, -ai, yr);
        R->c += ar * lr + ai * li;
        M->c += ar * li - ai * lr;
      }
    }
    for (int64_t j = j0; j < j1; ++j) {
      double rh, rl, ih, il;
      acc_round(&re[j - j0], &rh, &rl);
      acc_round(&im[j - j0], &ih, &il);
      x_hi[j] = rh + I * ih;
      if (x_lo) x_lo[j] = rl + I * il;
    }
  }
}

void orc_matvec_dd(int64_t m, int64_t n, const zc *A, int64_t lda,
                   const zc *x_hi, const zc *x_lo, zc *v_hi, zc *v_lo) {
#pragma omp parallel for schedule(dynamic)
  for (int64_t i = 0; i < m; ++i) {
    acc2 R = {0, 0}, M = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
      const double ar = creal(A[i * lda + j]), ai = cimag(A[i * lda + j]);
      const double xr = creal(x_hi[j]), xi = cimag(x_hi[j]);
      /* a * x = (ar xr - ai xi) + i (ar xi + ai xr) */
      acc_prod(&R, ar, xr); acc_prod(&R, -ai, xi);
      acc_prod(&M, ar, xi); acc_prod(&M, ai, xr);
      if (x_lo) {
        const double lr = creal(x_lo[j]), li = cimag(x_lo[j]);
        R.c += ar * lr - ai * li;
        M.c += ar * li + ai * lr;
      }
    }
    double rh, rl, ih, il;
    acc_round(&R, &rh, &rl);
    acc_round(&M, &ih, &il);
    v_hi[i] = rh + I * ih;
    if (v_lo) v_lo[i] = rl + I * il;
  }
}

void orc_residual_dd(int64_t m, int64_t n, const zc *A, int64_t lda,
                     const zc *y_hi, const zc *y_lo, const zc *b,
                     zc *r, zc *x_hi, zc *x_lo) {
  zc *vh = (zc *)malloc(sizeof(zc) * (size_t)m);
  zc *vl = (zc *)malloc(sizeof(zc) * (size_t)m);
  orc_adj_matvec_dd(m, n, A, lda, y_hi, y_lo, x_hi, x_lo);
  orc_matvec_dd(m, n, A, lda, x_hi, x_lo, vh, vl);
  for (int64_t i = 0; i < m; ++i) {
    double sr, er, si, ei;
    two_sum(creal(b[i]), -creal(vh[i]), &sr, &er);
    two_sum(cimag(b[i]), -cimag(vh[i]), &si, &ei);
    r[i] = (sr + (er - creal(vl[i]))) + I * (si + (ei - cimag(vl[i])));
  }
  free(vh); free(vl);
}

void orc_adj_matvec(int64_t m, int64_t n, const zc *A, int64_t lda, const zc *y, zc *x) {
  const int64_t B = 256;
#pragma omp parallel for schedule(static)
  for (int64_t j0 = 0; j0 < n; j0 += B) {            /* each x[j] summed over i = 0..m-1 in order */
    const int64_t j1 = j0 + B < n ? j0 + B : n;
    for (int64_t j = j0; j < j1; ++j) x[j] = 0;
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = j0; j < j1; ++j) x[j] += conj(A[i * lda + j]) * y[i];
  }
}

void orc_matvec(int64_t m, int64_t n, const zc *A, int64_t lda, const zc *x, zc *v) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    zc acc = 0;
    for (int64_t j = 0; j < n; ++j) acc += A[i * lda + j] * x[j];
    v[i] = acc;
  }
}
