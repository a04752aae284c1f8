// qrblk.cu -- Step 2 (Eq. lineq) for tall sketches: Y = Q1 R1 by Householder QR
// WITHOUT pivoting, blocked by 32 columns, whose trailing updates (W = V^H C,
// Z = T^H W, C -= V Z; the compact WY form of Schreiber and Van Loan) are the
// FP64-accurate tensor-core products of ozaki.cu; then the pivoted Householder
// QR of the m x m triangle R1 (qr.cu) gives R and P.
//
// Why this is Step 2's factorization: Y P = Q1 (R1 P) = Q1 Q2 R for the pivoted
// QR R1 P = Q2 R, and Q1 Q2 has orthonormal columns; column pivoting looks only
// at the norms of the remaining columns' projections, which R1 and Y share
// (Y^H Y = R1^H R1), so P is the pivoting of Y itself and R is its R-factor up
// to a unit diagonal (the sign LAPACK's reflectors give each row). The costly
// l x m part runs as products on the tensor cores; only the m x m part is
// factored column by column.
#include "common.cuh"
#include "kernels.h"

namespace mn {

static int64_t qpad(int64_t v, int64_t q) { return (v + q - 1) / q * q; }

void qrblk_sizes(int64_t l, int64_t m, int sms, size_t (&b)[13]) {
  b[0] = oz_slice_bytes(m, 2 * l);          // sA: A rows from C's columns
  b[1] = oz_slice_bytes(kOzN, 2 * l);       // sB: the reflectors, adjoint form
  b[2] = oz_slice_bytes(2 * l, kOzK);       // sV: the reflectors, update form
  b[3] = oz_slice_bytes(m, kOzK);           // sZ
  b[4] = sizeof(int32_t) * (size_t)qpad(m, kOzM);
  b[5] = sizeof(int32_t) * (size_t)kOzM;
  b[6] = sizeof(int32_t) * (size_t)qpad(2 * l, kOzM);
  b[7] = sizeof(int32_t) * (size_t)qpad(m, kOzM);
  b[8] = oz_adj_partial_bytes(l, m, sms);
  b[9] = sizeof(zd) * 32 * (size_t)m;       // W
  b[10] = sizeof(zd) * 32 * (size_t)m;      // Z
  b[11] = sizeof(zd) * 32 * 32;             // T
  b[12] = sizeof(double) * 2 * (size_t)m;   // tau
}

cudaError_t launch_trailing_products(QrBlkWork &w, const void *V, int64_t ldv, void *C, int64_t ldc, int64_t rows,
                                     int64_t cols, const void *Z, int64_t ldz, void *W, int *err, uint64_t limit_ns,
                                     cudaStream_t st) {
  if (rows > w.l || cols > w.m) return cudaErrorInvalidValue;
  cudaError_t e;
  if (W) {
    OzOperand a{w.sA, w.eA, 0, 0, 0, 0}, b{w.sB, w.eB, 0, 0, 0, 0};
    if ((e = launch_oz_slice_cols(C, ldc, rows, cols, a, st)) != cudaSuccess) return e;
    if ((e = launch_oz_slice_v_adj(V, ldv, rows, b, st)) != cudaSuccess) return e;
    OzAdjArgs g{a, b, w.part, w.part_bytes, W, 32, cols, err, limit_ns};
    if ((e = launch_oz_adj(g, st)) != cudaSuccess) return e;
  }
  if (Z) {
    OzOperand a{w.sV, w.eV, 0, 0, 0, 0}, b{w.sZ, w.eZ, 0, 0, 0, 0};
    if ((e = launch_oz_slice_v_fwd(V, ldv, rows, a, st)) != cudaSuccess) return e;
    if ((e = launch_oz_slice_z(Z, ldz, cols, b, st)) != cudaSuccess) return e;
    OzFwdArgs g{a, b, C, ldc, rows, cols, err, limit_ns};
    if ((e = launch_oz_fwd(g, st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace mn
