/*
 * oracle.h -- plain CPU FP64 oracle for Tygert's randomized minimal-norm solver
 * (arXiv:0905.4745, "A fast algorithm for computing minimal-norm solutions to
 * underdetermined systems of linear equations").
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load this library. The product path (the CUDA library
 * under paper_0905_4745_gb300/) shares no code, header, table or constant with
 * it, and never calls it.
 *
 * Conventions (all 0-based):
 *   - complex values are C99 `double complex`;
 *   - A is row-major m x n (row i contiguous, leading dimension lda >= n);
 *   - the sketch Y (the paper's S_{l x m}, Eq. randmat) is column-major l x m;
 *   - a permutation array p acts by gathering: (P v)[j] = v[p[j]].
 *
 * Functions whose result is not pinned by an independent check say so in their
 * comment ("parity unpinned"); every other function is pinned by tests/test_oracle_*.py.
 */
#ifndef MINNORM_ORACLE_H
#define MINNORM_ORACLE_H

#include <complex.h>
#include <stdint.h>

typedef double complex zc;

/* ---------------------------------------------------------------- rng.c --- */
/* SplitMix64 (Steele, Lea, Flood 2014) as a counter-based stream:
 *   draw(seed, kind, j) = mix64(seed + G*(kind*2^40 + j + 1)),  G = 0x9E3779B97F4A7C15.
 * For kind 0 this is exactly the j-th output of the published sequential
 * generator seeded with state `seed`. */
uint64_t orc_mix64(uint64_t z);
uint64_t orc_draw(uint64_t seed, uint64_t kind, uint64_t j);

/* The random parameters of one SRFT realization (Section 3, Eqs. SRFT, SRFT2,
 * Rokhlin_trans, big_def), drawn from kinds 0..7 in the order
 * zeta~, pi~, theta~, zeta, pi, theta, d, s. */
void orc_draw_params(uint64_t seed, int64_t n, int64_t l,
                     zc *zeta_t, int64_t *pi_t, double *theta_t,
                     zc *zeta, int64_t *pi, double *theta,
                     zc *d, int64_t *s);

/* ---------------------------------------------------------------- fft.c --- */
/* Unitary DFT of Eq. (DFT): out[j] = n^{-1/2} sum_k x[k] e^{sign*2 pi i j k/n}
 * (sign = -1 is F, sign = +1 is F^*), in place. Radix-2 for powers of two,
 * Bluestein's chirp-z reduction to radix-2 otherwise. */
void orc_dft(zc *x, int64_t n, int sign);
/* Same transform by the O(n^2) definition (reference for small n). */
void orc_dft_brute(const zc *x, zc *out, int64_t n, int sign);

/* --------------------------------------------------------------- srft.c --- */
typedef struct {
  int64_t n, l;
  const zc *zeta_t; const int64_t *pi_t; const double *theta_t;
  const zc *zeta;   const int64_t *pi;   const double *theta;
  const zc *d;      const int64_t *s;
} orc_srft;

/* Givens chain Theta = G_0 G_1 ... G_{n-2} of Eq. big_def applied to v in place
 * (G_{n-2} acts first); G_k rotates coordinates (k, k+1) by
 * [[cos t_k, sin t_k], [-sin t_k, cos t_k]]. */
void orc_chain(zc *v, int64_t n, const double *theta);
/* Theta^T (= Theta^*, the chain is real) applied to v in place. */
void orc_chain_adjoint(zc *v, int64_t n, const double *theta);
/* H v (Eq. Rokhlin_trans), in place, using work[n]. */
void orc_apply_H(const orc_srft *P, zc *v, zc *work);
/* y[l] = T v = S F D H v (Eqs. SRFT, SRFT2); v is not modified; work[2n]. */
void orc_srft_apply(const orc_srft *P, const zc *v, zc *y, zc *work);
/* v[n] = T^* y; work[n]. */
void orc_srft_adjoint(const orc_srft *P, const zc *y, zc *v, zc *work);
/* Step 1 (Eq. randmat): Y[:, i] = T conj(A[i, :]) for every row i. */
void orc_sketch(const orc_srft *P, int64_t m, const zc *A, int64_t lda, zc *Y, int64_t ldy);

/* ----------------------------------------------------------------- qr.c --- */
/* Householder QR with column pivoting (Golub & Van Loan ch. 5, the "classical
 * pivoted QR based on Householder reflections" of Section 7), in the LAPACK
 * zgeqp3/zlaqp2 conventions: on exit Y[:, 0:k] holds R (upper triangle, real
 * diagonal) and the Householder vectors (below the diagonal, unit leading entry
 * implicit), tau[k] the scalar factors, piv[k] the original index of the k-th
 * column, so that Y_in[:, piv] = Q R with Q = H_0 H_1 ... H_{k-1},
 * H_j = I - tau_j v_j v_j^*. k = min(rows, cols). */
void orc_qrp(zc *Y, int64_t ldy, int64_t rows, int64_t cols, int64_t *piv, zc *tau);
/* x[rows] <- Q x (apply H_{k-1} first) or Q^* x (conj = 1; H_0 first). */
void orc_apply_q(const zc *Y, int64_t ldy, int64_t rows, int64_t k, const zc *tau,
                 zc *x, int conj);
/* Triangular solves with the k x k upper triangle R stored in Y. */
void orc_solve_r(const zc *R, int64_t ldr, int64_t k, zc *x);       /* x <- R^{-1} x  */
void orc_solve_rh(const zc *R, int64_t ldr, int64_t k, zc *x);      /* x <- R^{-*} x  */

/* ----------------------------------------------------------------- dd.c --- */
/* Matrix-vector products with A treated exactly and sums accumulated in
 * double-double (Ogita, Rump, Oishi 2005, "Accurate sum and dot product",
 * Algorithm Dot2 with complex terms split into real products).
 * The vector operands may carry a low part (pass NULL for none). */
void orc_adj_matvec_dd(int64_t m, int64_t n, const zc *A, int64_t lda,
                       const zc *y_hi, const zc *y_lo, zc *x_hi, zc *x_lo);   /* x = A^* y */
void orc_matvec_dd(int64_t m, int64_t n, const zc *A, int64_t lda,
                   const zc *x_hi, const zc *x_lo, zc *v_hi, zc *v_lo);       /* v = A x   */
/* r = b - A (A^* y) with both products in double-double; r rounded to FP64,
 * x = A^* y returned as (x_hi, x_lo). */
void orc_residual_dd(int64_t m, int64_t n, const zc *A, int64_t lda,
                     const zc *y_hi, const zc *y_lo, const zc *b,
                     zc *r, zc *x_hi, zc *x_lo);
/* Plain FP64 products, loop order of the definition (no blocking). */
void orc_adj_matvec(int64_t m, int64_t n, const zc *A, int64_t lda, const zc *y, zc *x);
void orc_matvec(int64_t m, int64_t n, const zc *A, int64_t lda, const zc *x, zc *v);

/* ------------------------------------------------------------ minnorm.c --- */
typedef struct {
  int32_t iters;          /* CG iterations (O2) or refinement steps (O1)       */
  int32_t rank_ok;        /* 0 when a zero pivot made R singular               */
  double  resid0;         /* ||s_0|| (O2) / ||b - A x0|| (O1)                   */
  double  resid;          /* final ||s|| (O2) / final ||r|| (O1)                */
} orc_info;

/* O1: the classical direct method (Section 7): pivoted Householder QR of A^*,
 * A^* P = Q R, so A A^* = P R^* R P^T. x0 = Q R^{-*} P^T b (the direct
 * minimal-norm solution, time t_0 of Tables 1 and 3); then `steps` steps of
 * y <- y + P R^{-1} R^{-*} P^T (b - A A^* y) with double-double residuals,
 * and p = A^* y in double-double, rounded to FP64. x0 may be NULL. */
int orc_minnorm_direct(int64_t m, int64_t n, const zc *A, int64_t lda, const zc *b,
                       int32_t steps, zc *p, zc *y_out, zc *x0, orc_info *info);

/* O2: the randomized algorithm of Section 4, Steps 1-5, literally, FP64:
 *  1. Y = T A^*                       (Eq. randmat)
 *  2. z = minimal-norm solution of Y^* z = b via Y P = Q R: z = Q R^{-*} P^T b (Eq. lineq)
 *  3. c = T^* z                       (Eq. nonminnorm)
 *  4. y minimizing ||A^* y - c|| by CG on the normal equations of
 *     min_u ||M u - c||, M = A^* P R^{-1}, y = P R^{-1} u, started from the
 *     sketched solution u_0 = Q^* T c, stopped when ||M^*(c - M u)||^2 <=
 *     delta (||c - M u||^2 - ||M^*(c - M u)||^2)   (Eq. overdet; delta is the
 *     relative precision of Step 4)
 *  5. x = A^* y                       (Eq. output)
 * Outputs z (l), c (n), u0 (m), y (m), x (n); any may be NULL except x. */
int orc_minnorm_randomized(const orc_srft *P, int64_t m, const zc *A, int64_t lda,
                           const zc *b, double delta, int32_t maxit,
                           zc *x, zc *y, zc *z, zc *c, zc *u0, orc_info *info);

/* The normal-equation form used by the GPU path (no z, no c): CG on
 * (R^{-*} P^T A A^* P R^{-1}) u = R^{-*} P^T b from u = u_start (NULL: zero),
 * running exactly `iters` iterations, returning u after each iteration in
 * u_hist (iters x m, may be NULL) and y = P R^{-1} u. Used to check that it
 * reproduces O2's iterates (Lemma 5.1: A c = b). */
void orc_pcg_normal(int64_t m, int64_t n, const zc *A, int64_t lda, const zc *b,
                    const zc *R, int64_t ldr, const int64_t *piv,
                    const zc *u_start, int32_t iters, zc *u_hist, zc *y);

#endif
