/*
 * minnorm.c -- oracle (test infrastructure only): the minimal-norm solution p
 * of A p = b for a full-rank complex A (m x n, m < n), two ways.
 *
 * O1 (orc_minnorm_direct) is the reference p: the direct method of Section 7
 * (pivoted Householder QR of A^*) followed by refinement of y in
 * A A^* y = b with double-double residuals, p = A^* y evaluated in
 * double-double. y is kept as an unevaluated sum y_hi + y_lo: rounding y to
 * FP64 alone would move A^* y by about kappa * 2^-53 relative.
 *
 * O2 (orc_minnorm_randomized) is the paper's algorithm, Section 4, Steps 1-5,
 * written out literally in FP64.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static zc *zalloc(int64_t count) { return (zc *)calloc((size_t)(count > 0 ? count : 1), sizeof(zc)); }

static double norm2sq(const zc *x, int64_t len) {
  double acc = 0.0;
  for (int64_t i = 0; i < len; ++i) acc += creal(x[i]) * creal(x[i]) + cimag(x[i]) * cimag(x[i]);
  return acc;
}

/* out = P R^{-1} in   (P: (P v)[piv[k]] = v[k] ordering of the pivoted QR) */
static void apply_prinv(const zc *R, int64_t ldr, const int64_t *piv, int64_t m,
                        const zc *in, zc *out, zc *tmp) {
  memcpy(tmp, in, sizeof(zc) * (size_t)m);
  orc_solve_r(R, ldr, m, tmp);
  for (int64_t k = 0; k < m; ++k) out[piv[k]] = tmp[k];
}

/* out = R^{-*} P^T in */
static void apply_rhinv_pt(const zc *R, int64_t ldr, const int64_t *piv, int64_t m,
                           const zc *in, zc *out) {
  for (int64_t k = 0; k < m; ++k) out[k] = in[piv[k]];
  orc_solve_rh(R, ldr, m, out);
}

static int rank_ok(const zc *R, int64_t ldr, int64_t m) {
  const double r00 = cabs(R[0]);
  const double rmm = cabs(R[(m - 1) + (m - 1) * ldr]);
  return r00 > 0.0 && rmm > r00 * 0x1.0p-52 * (double)m;
}

int orc_minnorm_direct(int64_t m, int64_t n, const zc *A, int64_t lda, const zc *b,
                       int32_t steps, zc *p, zc *y_out, zc *x0, orc_info *info) {
  zc *C = zalloc(n * m);                       /* A^*, column-major n x m */
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < n; ++j) C[j + i * n] = conj(A[i * lda + j]);
  int64_t *piv = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  zc *tau = zalloc(m);
  orc_qrp(C, n, n, m, piv, tau);               /* A^* P = Q R */
  const int ok = rank_ok(C, n, m);
  if (info) { info->rank_ok = ok; info->iters = 0; }
  if (!ok) { free(C); free(piv); free(tau); return 1; }

  zc *t = zalloc(m), *tmp = zalloc(m);
  if (x0) {                                    /* classical: x0 = Q R^{-*} P^T b */
    apply_rhinv_pt(C, n, piv, m, b, t);
    memset(x0, 0, sizeof(zc) * (size_t)n);
    memcpy(x0, t, sizeof(zc) * (size_t)m);
    orc_apply_q(C, n, n, m, tau, x0, 0);
  }
  zc *yh = zalloc(m), *yl = zalloc(m), *r = zalloc(m), *d = zalloc(m);
  zc *xh = zalloc(n), *xl = zalloc(n);
  memcpy(r, b, sizeof(zc) * (size_t)m);        /* residual of y = 0 is b exactly */
  if (info) info->resid0 = sqrt(norm2sq(b, m));
  for (int32_t step = 0; step <= steps; ++step) {
    if (step > 0) orc_residual_dd(m, n, A, lda, yh, yl, b, r, xh, xl);
    apply_rhinv_pt(C, n, piv, m, r, t);        /* d = P R^{-1} R^{-*} P^T r */
    apply_prinv(C, n, piv, m, t, d, tmp);
    for (int64_t i = 0; i < m; ++i) {          /* (yh, yl) += d, componentwise TwoSum */
      double parts[2][2] = {{creal(yh[i]), creal(d[i])}, {cimag(yh[i]), cimag(d[i])}};
      double lo[2] = {creal(yl[i]), cimag(yl[i])}, hi[2];
      for (int c = 0; c < 2; ++c) {
        double s = parts[c][0] + parts[c][1];
        double bb = s - parts[c][0];
        double e = (parts[c][0] - (s - bb)) + (parts[c][1] - bb);
        double l2 = lo[c] + e;
        hi[c] = s + l2;
        lo[c] = l2 - (hi[c] - s);
      }
      yh[i] = hi[0] + I * hi[1];
      yl[i] = lo[0] + I * lo[1];
    }
    if (info) info->iters = step;
  }
  orc_residual_dd(m, n, A, lda, yh, yl, b, r, xh, xl);   /* final x = A^* y in dd */
  if (info) info->resid = sqrt(norm2sq(r, m));
  memcpy(p, xh, sizeof(zc) * (size_t)n);
  if (y_out) memcpy(y_out, yh, sizeof(zc) * (size_t)m);
  free(C); free(piv); free(tau); free(t); free(tmp);
  free(yh); free(yl); free(r); free(d); free(xh); free(xl);
  return 0;
}

int orc_minnorm_randomized(const orc_srft *P, int64_t m, const zc *A, int64_t lda,
                           const zc *b, double delta, int32_t maxit,
                           zc *x, zc *y_out, zc *z_out, zc *c_out, zc *u0_out, orc_info *info) {
  const int64_t n = P->n, l = P->l;
  zc *Y = zalloc(l * m);
  int64_t *piv = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  zc *tau = zalloc(m);
  /* Step 1: Y = T A^* */
  orc_sketch(P, m, A, lda, Y, l);
  /* Step 2: Y P = Q R; minimal-norm z with Y^* z = b is z = Q R^{-*} P^T b */
  orc_qrp(Y, l, l, m, piv, tau);
  const int ok = rank_ok(Y, l, m);
  if (info) { info->rank_ok = ok; info->iters = 0; }
  if (!ok) { free(Y); free(piv); free(tau); return 1; }
  zc *z = zalloc(l), *t = zalloc(m), *tmp = zalloc(m);
  apply_rhinv_pt(Y, l, piv, m, b, t);
  memcpy(z, t, sizeof(zc) * (size_t)m);
  orc_apply_q(Y, l, l, m, tau, z, 0);
  /* Step 3: c = T^* z */
  zc *c = zalloc(n), *work = zalloc(2 * n);
  orc_srft_adjoint(P, z, c, work);
  /* Step 4: min || A^* y - c || with y = P R^{-1} u, CG on the normal equations
     of min_u || M u - c ||, M = A^* P R^{-1}, from the sketched solution u0 = Q^* T c */
  zc *tc = zalloc(l), *u = zalloc(m);
  orc_srft_apply(P, c, tc, work);
  orc_apply_q(Y, l, l, m, tau, tc, 1);
  memcpy(u, tc, sizeof(zc) * (size_t)m);
  if (u0_out) memcpy(u0_out, u, sizeof(zc) * (size_t)m);
  zc *w = zalloc(m), *q = zalloc(n), *r = zalloc(n), *v = zalloc(m), *s = zalloc(m), *pd = zalloc(m);
  apply_prinv(Y, l, piv, m, u, w, tmp);
  orc_adj_matvec(m, n, A, lda, w, q);
  for (int64_t j = 0; j < n; ++j) r[j] = c[j] - q[j];          /* r = c - M u */
  orc_matvec(m, n, A, lda, r, v);
  apply_rhinv_pt(Y, l, piv, m, v, s);                          /* s = M^* r */
  memcpy(pd, s, sizeof(zc) * (size_t)m);
  double gamma = norm2sq(s, m);
  if (info) info->resid0 = sqrt(gamma);
  int32_t it = 0;
  for (; it < maxit; ++it) {
    if (gamma <= delta * (norm2sq(r, n) - gamma)) break;
    apply_prinv(Y, l, piv, m, pd, w, tmp);
    orc_adj_matvec(m, n, A, lda, w, q);                        /* q = M pd */
    const double alpha = gamma / norm2sq(q, n);
    for (int64_t k = 0; k < m; ++k) u[k] += alpha * pd[k];
    for (int64_t j = 0; j < n; ++j) r[j] -= alpha * q[j];
    orc_matvec(m, n, A, lda, r, v);
    apply_rhinv_pt(Y, l, piv, m, v, s);                        /* s = M^* r */
    const double gnew = norm2sq(s, m);
    const double beta = gnew / gamma;
    gamma = gnew;
    for (int64_t k = 0; k < m; ++k) pd[k] = s[k] + beta * pd[k];
  }
  if (info) { info->iters = it; info->resid = sqrt(gamma); }
  /* Step 5: x = A^* y */
  zc *y = zalloc(m);
  apply_prinv(Y, l, piv, m, u, y, tmp);
  orc_adj_matvec(m, n, A, lda, y, x);
  if (y_out) memcpy(y_out, y, sizeof(zc) * (size_t)m);
  if (z_out) memcpy(z_out, z, sizeof(zc) * (size_t)l);
  if (c_out) memcpy(c_out, c, sizeof(zc) * (size_t)n);
  free(Y); free(piv); free(tau); free(z); free(t); free(tmp); free(c); free(work);
  free(tc); free(u); free(w); free(q); free(r); free(v); free(s); free(pd); free(y);
  return 0;
}

void orc_pcg_normal(int64_t m, int64_t n, const zc *A, int64_t lda, const zc *b,
                    const zc *R, int64_t ldr, const int64_t *piv,
                    const zc *u_start, int32_t iters, zc *u_hist, zc *y) {
  zc *u = zalloc(m), *s = zalloc(m), *pd = zalloc(m), *w = zalloc(m), *tmp = zalloc(m);
  zc *q = zalloc(n), *t = zalloc(m), *np = zalloc(m), *g = zalloc(m);
  if (u_start) memcpy(u, u_start, sizeof(zc) * (size_t)m);
  apply_rhinv_pt(R, ldr, piv, m, b, g);                        /* g = R^{-*} P^T b */
  /* s = g - N u,  N = R^{-*} P^T A A^* P R^{-1} */
  apply_prinv(R, ldr, piv, m, u, w, tmp);
  orc_adj_matvec(m, n, A, lda, w, q);
  orc_matvec(m, n, A, lda, q, t);
  apply_rhinv_pt(R, ldr, piv, m, t, np);
  for (int64_t k = 0; k < m; ++k) s[k] = g[k] - np[k];
  memcpy(pd, s, sizeof(zc) * (size_t)m);
  double gamma = norm2sq(s, m);
  for (int32_t it = 0; it < iters; ++it) {
    apply_prinv(R, ldr, piv, m, pd, w, tmp);
    orc_adj_matvec(m, n, A, lda, w, q);                        /* q = A^* P R^{-1} pd */
    orc_matvec(m, n, A, lda, q, t);
    apply_rhinv_pt(R, ldr, piv, m, t, np);                     /* np = N pd */
    const double alpha = gamma / norm2sq(q, n);                /* <pd, N pd> = ||q||^2 */
    for (int64_t k = 0; k < m; ++k) { u[k] += alpha * pd[k]; s[k] -= alpha * np[k]; }
    const double gnew = norm2sq(s, m);
    const double beta = gnew / gamma;
    gamma = gnew;
    for (int64_t k = 0; k < m; ++k) pd[k] = s[k] + beta * pd[k];
    if (u_hist) memcpy(u_hist + (int64_t)it * m, u, sizeof(zc) * (size_t)m);
  }
  apply_prinv(R, ldr, piv, m, u, y, tmp);
  free(u); free(s); free(pd); free(w); free(tmp); free(q); free(t); free(np); free(g);
}
