/*
 * qr.c -- oracle (test infrastructure only): Householder QR with column
 * pivoting, the "classical algorithm for pivoted QR-decompositions based on
 * plane (Householder) reflections" of Section 7 (Golub & Van Loan, ch. 5),
 * used in Step 2 (Eq. lineq, via GVL Algorithm 5.7.2) and by the direct
 * method of Section 7.
 *
 * Step i: pick the remaining column of largest partial norm (first one on a
 * tie), swap it to position i, build the reflector H_i = I - tau v v^* with
 * v_i = 1 and H_i^* y = (beta, 0, ..., 0), beta real, beta = -sign(Re y_i) ||y||
 * (the LAPACK zlarfg convention, so R has a real diagonal), apply H_i^* to the
 * trailing columns and downdate their partial norms, recomputing a norm from
 * scratch when the downdate has lost more than half the digits (the LAPACK
 * zlaqp2 safeguard of Drmac & Bujanovic 2008).
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

static double col_norm(const zc *x, int64_t len) {
  double acc = 0.0;
  for (int64_t r = 0; r < len; ++r) acc += creal(x[r]) * creal(x[r]) + cimag(x[r]) * cimag(x[r]);
  return sqrt(acc);
}

/* reflector annihilating x[1:len] below alpha = x[0]; returns tau, scales x[1:] to v */
static zc householder(zc *x, int64_t len) {
  double xnorm = col_norm(x + 1, len - 1);
  double ar = creal(x[0]), ai = cimag(x[0]);
  if (xnorm == 0.0 && ai == 0.0) return 0.0;
  double mag = sqrt(ar * ar + ai * ai + xnorm * xnorm);
  double beta = ar >= 0.0 ? -mag : mag;
  zc tau = (beta - ar) / beta - I * (ai / beta);
  zc scal = 1.0 / (x[0] - beta);
  for (int64_t r = 1; r < len; ++r) x[r] *= scal;
  x[0] = beta;
  return tau;
}

void orc_qrp(zc *Y, int64_t ldy, int64_t rows, int64_t cols, int64_t *piv, zc *tau) {
  const int64_t k = rows < cols ? rows : cols;
  const double tol3z = sqrt(0x1.0p-53);
  double *vn1 = (double *)malloc(sizeof(double) * (size_t)cols);
  double *vn2 = (double *)malloc(sizeof(double) * (size_t)cols);
  for (int64_t j = 0; j < cols; ++j) {
    vn1[j] = vn2[j] = col_norm(Y + j * ldy, rows);
    piv[j] = j;
  }
  for (int64_t i = 0; i < k; ++i) {
    int64_t p = i;
    for (int64_t j = i + 1; j < cols; ++j) if (vn1[j] > vn1[p]) p = j;
    if (p != i) {
      for (int64_t r = 0; r < rows; ++r) {
        zc t = Y[r + p * ldy]; Y[r + p * ldy] = Y[r + i * ldy]; Y[r + i * ldy] = t;
      }
      int64_t tp = piv[p]; piv[p] = piv[i]; piv[i] = tp;
      vn1[p] = vn1[i]; vn2[p] = vn2[i];
    }
    zc *v = Y + i + i * ldy;                       /* v[0] = 1 implicitly */
    const int64_t len = rows - i;
    tau[i] = householder(v, len);
    const zc beta = v[0];
    v[0] = 1.0;
#pragma omp parallel for schedule(static)
    for (int64_t j = i + 1; j < cols; ++j) {
      zc *y = Y + i + j * ldy;
      zc w = 0;
      for (int64_t r = 0; r < len; ++r) w += conj(v[r]) * y[r];
      zc f = conj(tau[i]) * w;
      for (int64_t r = 0; r < len; ++r) y[r] -= f * v[r];
    }
    v[0] = beta;
    for (int64_t j = i + 1; j < cols; ++j) {
      if (vn1[j] == 0.0) continue;
      double t = cabs(Y[i + j * ldy]) / vn1[j];
      double temp = 1.0 - t * t;
      if (temp < 0.0) temp = 0.0;
      double ratio = vn1[j] / vn2[j];
      double temp2 = temp * ratio * ratio;
      if (temp2 <= tol3z) {
        if (i < rows - 1) {
          vn1[j] = col_norm(Y + (i + 1) + j * ldy, rows - i - 1);
          vn2[j] = vn1[j];
        } else {
          vn1[j] = vn2[j] = 0.0;
        }
      } else {
        vn1[j] *= sqrt(temp);
      }
    }
  }
  free(vn1); free(vn2);
}

void orc_apply_q(const zc *Y, int64_t ldy, int64_t rows, int64_t k, const zc *tau,
                 zc *x, int conj_) {
  for (int64_t step = 0; step < k; ++step) {
    const int64_t j = conj_ ? step : k - 1 - step;
    const zc *v = Y + j + j * ldy;
    const int64_t len = rows - j;
    zc w = x[j];                                  /* v[0] = 1 */
    for (int64_t r = 1; r < len; ++r) w += conj(v[r]) * x[j + r];
    zc f = (conj_ ? conj(tau[j]) : tau[j]) * w;
    x[j] -= f;
    for (int64_t r = 1; r < len; ++r) x[j + r] -= f * v[r];
  }
}

void orc_solve_r(const zc *R, int64_t ldr, int64_t k, zc *x) {
  for (int64_t i = k - 1; i >= 0; --i) {
    zc acc = x[i];
    for (int64_t j = i + 1; j < k; ++j) acc -= R[i + j * ldr] * x[j];
    x[i] = acc / R[i + i * ldr];
  }
}

void orc_solve_rh(const zc *R, int64_t ldr, int64_t k, zc *x) {
  for (int64_t i = 0; i < k; ++i) {
    zc acc = x[i];
    for (int64_t j = 0; j < i; ++j) acc -= conj(R[j + i * ldr]) * x[j];
    x[i] = acc / conj(R[i + i * ldr]);
  }
}
