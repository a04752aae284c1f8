/*
 * srft.c -- oracle (test infrastructure only): the subsampled randomized
 * Fourier transform of Section 3 and Step 1 of Section 4.
 *
 *   T = G H                                  (Eq. SRFT)
 *   G = S F D                                (Eq. SRFT2)
 *   H = Theta Pi Z Theta~ Pi~ Z~             (Eq. Rokhlin_trans)
 *   Theta = G_0 G_1 ... G_{n-2}              (Eq. big_def, 0-based)
 * applied right to left, so Z~ acts first and S last, and inside a chain
 * G_{n-2} acts first. G_k rotates coordinates (k, k+1) by the printed block
 * [[cos, sin], [-sin, cos]]. S keeps rows s_0 < s_1 < ... < s_{l-1} of F D H.
 * T^* = H^* D^* F^* S^T reverses the order with conjugate transposes.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

void orc_chain(zc *v, int64_t n, const double *theta) {
  for (int64_t k = n - 2; k >= 0; --k) {
    double c = cos(theta[k]), s = sin(theta[k]);
    zc a = v[k], b = v[k + 1];
    v[k] = c * a + s * b;
    v[k + 1] = -s * a + c * b;
  }
}

void orc_chain_adjoint(zc *v, int64_t n, const double *theta) {
  for (int64_t k = 0; k <= n - 2; ++k) {
    double c = cos(theta[k]), s = sin(theta[k]);
    zc a = v[k], b = v[k + 1];
    v[k] = c * a - s * b;
    v[k + 1] = s * a + c * b;
  }
}

void orc_apply_H(const orc_srft *P, zc *v, zc *w) {
  const int64_t n = P->n;
  for (int64_t j = 0; j < n; ++j) v[j] *= P->zeta_t[j];           /* Z~  */
  for (int64_t j = 0; j < n; ++j) w[j] = v[P->pi_t[j]];           /* Pi~ */
  orc_chain(w, n, P->theta_t);                                    /* Theta~ */
  for (int64_t j = 0; j < n; ++j) w[j] *= P->zeta[j];             /* Z   */
  for (int64_t j = 0; j < n; ++j) v[j] = w[P->pi[j]];             /* Pi  */
  orc_chain(v, n, P->theta);                                      /* Theta */
}

void orc_srft_apply(const orc_srft *P, const zc *v, zc *y, zc *work) {
  const int64_t n = P->n;
  zc *u = work, *w = work + n;
  memcpy(u, v, sizeof(zc) * (size_t)n);
  orc_apply_H(P, u, w);
  for (int64_t j = 0; j < n; ++j) u[j] *= P->d[j];                /* D */
  orc_dft(u, n, -1);                                              /* F */
  for (int64_t t = 0; t < P->l; ++t) y[t] = u[P->s[t]];           /* S */
}

void orc_srft_adjoint(const orc_srft *P, const zc *y, zc *v, zc *work) {
  const int64_t n = P->n;
  zc *w = work;
  memset(w, 0, sizeof(zc) * (size_t)n);
  for (int64_t t = 0; t < P->l; ++t) w[P->s[t]] = y[t];           /* S^T */
  orc_dft(w, n, +1);                                              /* F^* */
  for (int64_t j = 0; j < n; ++j) w[j] *= conj(P->d[j]);          /* D^* */
  orc_chain_adjoint(w, n, P->theta);                              /* Theta^T */
  for (int64_t j = 0; j < n; ++j) v[P->pi[j]] = w[j];             /* Pi^T */
  for (int64_t j = 0; j < n; ++j) v[j] *= conj(P->zeta[j]);       /* Z^* */
  orc_chain_adjoint(v, n, P->theta_t);                            /* Theta~^T */
  for (int64_t j = 0; j < n; ++j) w[P->pi_t[j]] = v[j];           /* Pi~^T */
  for (int64_t j = 0; j < n; ++j) v[j] = w[j] * conj(P->zeta_t[j]); /* Z~^* */
}

void orc_sketch(const orc_srft *P, int64_t m, const zc *A, int64_t lda, zc *Y, int64_t ldy) {
  const int64_t n = P->n;
#pragma omp parallel
  {
    zc *v = (zc *)malloc(sizeof(zc) * (size_t)n);
    zc *work = (zc *)malloc(sizeof(zc) * (size_t)(2 * n));
#pragma omp for schedule(dynamic)
    for (int64_t i = 0; i < m; ++i) {
      for (int64_t j = 0; j < n; ++j) v[j] = conj(A[i * lda + j]);   /* column i of A^* */
      orc_srft_apply(P, v, Y + i * ldy, work);
    }
    free(v); free(work);
  }
}
