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
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mn {

static int64_t qpad(int64_t v, int64_t q) { return (v + q - 1) / q * q; }

constexpr int kPanel = 32;           // columns per panel (the reflectors of one compact WY block)
constexpr int kPanelThreads = 256;   // 8 warps; lane = panel column
constexpr int kPanelWarps = kPanelThreads / 32;
constexpr int kPanelLd = kPanel + 1; // shared-memory row stride of the panel block (complex entries)

__device__ __forceinline__ zd shfl_zd(zd v, int src) {
  return {__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
}
__device__ __forceinline__ zd sel_zd(bool p, zd a, zd b) { return {p ? a.re : b.re, p ? a.im : b.im}; }

// Householder QR without pivoting of the panel P (L rows x jb <= 32 columns, column-major,
// ld), LAPACK's zgeqr2 conventions: for column j, beta = -sign(Re alpha) ||P[j:, j]||,
// tau = (beta - alpha) / beta, v = P[j:, j] / (alpha - beta) with v_j = 1, and H_j^H =
// I - conj(tau) v v^H applied to the columns right of j.
//
// The CTAs own contiguous row ranges, held in shared memory for the whole panel (warp w
// takes the rows w, w + 8, ..., lane c column c). One grid-wide sum per column: with
// x = P[j+1:, j] (the rows below the diagonal), each CTA posts over its own rows
//     slot j:      ||x||^2,
//     slot c > j:  g_c = x^H P[j+1:, c],
//     slot i < j:  h_i = V[j+1:, i]^H x,
// and the CTA that owns row j posts that row (alpha = P[j, j], P[j, c] for c > j, and
// V[j, i] for i < j). Every CTA then forms, from the same sums in the same order, with
// s = 1 / (alpha - beta) (v = (1, s x)):
//     d_c = v^H P[j:, c] = P[j, c] + conj(s) g_c          (c > j),
//     e_i = v_i^H v      = conj(V[j, i]) + s h_i          (i < j),
// updates its rows, and in the same pass forms its slots for column j + 1. CTA 0 records
// e (column j of E, the strictly upper part of V^H V) and tau_j, from which qr_t_kernel builds
// the compact WY factor T off the panel's critical path. The posted values are double-buffered
// by the parity of j, so one barrier per column separates every write from its reads.
// Outputs: R's entries and the reflectors in P (beta on the diagonal), V (L x 32, unit
// diagonal, zeros above; the columns past jb zero), E (32 x 32, column-major; entries i < j
// of column j), tau.
// Dynamic shared memory: kPanelLd * ceil(L / G) complex entries.
__global__ void __launch_bounds__(kPanelThreads)
qr_panel_kernel(zd *P, int64_t ld, int L, int jb, zd *__restrict__ V, int64_t ldv, zd *__restrict__ E,
                zd *__restrict__ tau, zd *__restrict__ part, zd *__restrict__ rowb, GridBarrier *bar, int *err,
                uint64_t limit_ns) {
  extern __shared__ zd s_P[];   // own rows, row-major with stride kPanelLd
  __shared__ zd s_acc[kPanelWarps][kPanel];
  __shared__ zd s_row[kPanel];
  __shared__ zd s_d[kPanel];
  __shared__ double s_scal[5];   // beta, Re/Im tau, Re/Im s
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int r0 = (int)((int64_t)L * b / G), r1 = (int)((int64_t)L * (b + 1) / G);
  const int nr = r1 - r0;
  unsigned int epoch = 0;
  for (int e = tid; e < nr * kPanel; e += kPanelThreads) {
    const int c = e / nr, r = e - c * nr;
    s_P[r * kPanelLd + c] = c < jb ? ldcg(P + (int64_t)c * ld + r0 + r) : zd{0.0, 0.0};
  }
  __syncthreads();
  // the slots of column jn over the own rows r > jn, from the block as it stands; lane c
  // forms its slot branch-free (conj(a) b with a, b chosen by the lane's side of jn)
  auto post = [&](int jn) {
    zd acc = {0.0, 0.0};
    for (int rr = max(r0, jn + 1) - r0 + wid; rr < nr; rr += kPanelWarps) {
      const zd p = s_P[rr * kPanelLd + lane];
      const zd pj = s_P[rr * kPanelLd + jn];
      macc(acc, sel_zd(lane >= jn, pj, p), sel_zd(lane > jn, p, pj));
    }
    s_acc[wid][lane] = acc;
    __syncthreads();
    if (wid == 0) {
      zd t = {0.0, 0.0};
      for (int w = 0; w < kPanelWarps; ++w) t = t + s_acc[w][lane];
      part[((int64_t)(jn & 1) * G + b) * kPanel + lane] = t;
      if (jn >= r0 && jn < r1) rowb[(jn & 1) * kPanel + lane] = s_P[(jn - r0) * kPanelLd + lane];
    }
  };
  post(0);
  for (int j = 0; j < jb; ++j) {
    const int par = j & 1;
    if (!grid_sync(bar, G, epoch, limit_ns)) { if (tid == 0) atomicExch(err, 1); return; }
    {
      // slots i < j (the dots e_i of the earlier reflectors) are needed by CTA 0 alone (for T)
      zd a = {0.0, 0.0};
      if (b == 0 || lane >= j)
        for (int q = wid; q < G; q += kPanelWarps) a = a + ldcg(part + ((int64_t)par * G + q) * kPanel + lane);
      s_acc[wid][lane] = a;
      if (wid == 0) s_row[lane] = ldcg(rowb + par * kPanel + lane);
    }
    __syncthreads();
    if (wid == 0) {
      zd t = {0.0, 0.0};
      for (int w = 0; w < kPanelWarps; ++w) t = t + s_acc[w][lane];
      // the reflector of column j (the same arithmetic in every CTA)
      const zd alpha = s_row[j];
      const double xn2 = __shfl_sync(0xffffffffu, t.re, j);
      double bt = alpha.re;
      zd tj = {0.0, 0.0}, sc = {0.0, 0.0};
      if (!(xn2 == 0.0 && alpha.im == 0.0)) {
        const double mag = sqrt(alpha.re * alpha.re + alpha.im * alpha.im + xn2);
        bt = alpha.re >= 0.0 ? -mag : mag;
        tj = {(bt - alpha.re) / bt, -alpha.im / bt};
        const double dr = alpha.re - bt, di = alpha.im, iden = 1.0 / (dr * dr + di * di);
        sc = {dr * iden, -di * iden};   // 1 / (alpha - beta)
      }
      zd dv = {0.0, 0.0};
      if (lane > j && lane < jb) dv = s_row[lane] + conjg(sc) * t;
      else if (lane < j) dv = conjg(s_row[lane]) + sc * t;
      s_d[lane] = dv;
      if (b == 0) {
        if (lane < j) E[j * kPanel + lane] = dv;   // e_lane = v_lane^H v_j
        if (lane == 0) tau[j] = tj;
      }
      if (lane == 0) {
        s_scal[0] = bt;
        s_scal[1] = tj.re;
        s_scal[2] = tj.im;
        s_scal[3] = sc.re;
        s_scal[4] = sc.im;
      }
    }
    __syncthreads();
    const zd tj = {s_scal[1], s_scal[2]};
    const zd sc = {s_scal[3], s_scal[4]};
    // the own rows r >= j: P[r, c] -= conj(tau) d_c v_r (c > j; the lanes past jb have d = 0),
    // column j becomes v (beta on the diagonal)
    const zd f = lane > j ? conjg(tj) * s_d[lane] : zd{0.0, 0.0};
    // the warp's rows in batches of 32: v_r = s x_r (1 on row j) is formed once per row, by the
    // lane of the row's place in the batch, and broadcast (an FP64 instruction holds the pipe
    // for the whole warp, whatever its active lanes)
    const int rs = max(r0, j) - r0 + wid;
    for (int rb = rs; rb < nr; rb += 32 * kPanelWarps) {
      const int rl = rb + kPanelWarps * lane;
      zd vl = {0.0, 0.0};
      if (rl < nr) vl = r0 + rl == j ? zd{1.0, 0.0} : s_P[rl * kPanelLd + j] * sc;
      const int cnt = min(32, (nr - rb + kPanelWarps - 1) / kPanelWarps);
      for (int t = 0; t < cnt; ++t) {
        const int rr = rb + kPanelWarps * t;
        const int r = r0 + rr;
        zd *row = s_P + rr * kPanelLd;
        const zd v = shfl_zd(vl, t);
        zd p = row[lane];
        p = p - f * v;
        if (lane == j) p = r == j ? zd{s_scal[0], 0.0} : v;
        row[lane] = p;
      }
    }
    __syncthreads();
    if (j + 1 < jb) post(j + 1);
  }
  __syncthreads();
  for (int e = tid; e < nr * kPanel; e += kPanelThreads) {
    const int c = e / nr, r = e - c * nr, gr = r0 + r;
    const zd p = s_P[r * kPanelLd + c];
    if (c < jb) P[(int64_t)c * ld + gr] = p;
    V[(int64_t)c * ldv + gr] = c >= jb ? zd{0.0, 0.0} : gr > c ? p : gr == c ? zd{1.0, 0.0} : zd{0.0, 0.0};
  }
}

// The compact WY factor T of a panel from its E and tau, in place (column j of E is read before
// column j of T is written; T 32 x 32 column-major, zero past jb): Schreiber and Van Loan's
// recurrence (LAPACK's zlarft, forward and columnwise) T[j, j] = tau_j,
// T[i, j] = -tau_j sum_{k=i..j-1} T[i, k] e_k. One warp, lane = row i.
__global__ void __launch_bounds__(32)
qr_t_kernel(zd *__restrict__ ET, const zd *__restrict__ tau, int jb) {
  __shared__ zd sT[kPanel][kPanel + 1];   // sT[k][i] = T[i, k]
  const int i = threadIdx.x;
  for (int k = 0; k < kPanel; ++k) sT[k][i] = {0.0, 0.0};
  __syncwarp();
  for (int j = 0; j < jb; ++j) {
    const zd tj = tau[j];
    const zd e = i < j ? ET[j * kPanel + i] : zd{0.0, 0.0};
    zd sum = {0.0, 0.0};
    for (int k = 0; k < j; ++k) {
      const zd ek = shfl_zd(e, k);
      if (k >= i) mac(sum, sT[k][i], ek);
    }
    if (i < j) sT[j][i] = {-(tj.re * sum.re - tj.im * sum.im), -(tj.re * sum.im + tj.im * sum.re)};
    else if (i == j) sT[j][i] = tj;
    __syncwarp();
  }
  for (int k = 0; k < kPanel; ++k) ET[k * kPanel + i] = sT[k][i];
}

// Z = T^H W: Z[:, c] = T^H W[:, c], T 32 x 32 upper triangular (one thread per (row k, column c))
__global__ void qr_tw_kernel(const zd *__restrict__ T, const zd *__restrict__ W, zd *__restrict__ Z, int64_t cols) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= cols * kPanel) return;
  const int64_t c = e / kPanel;
  const int k = (int)(e % kPanel);
  zd z = {0.0, 0.0};
  for (int i = 0; i <= k; ++i) macc(z, T[k * kPanel + i], W[c * kPanel + i]);   // conj(T[i, k]) W[i, c]
  Z[c * kPanel + k] = z;
}

// R1 = the upper triangle of Y[0:m, 0:m] (zeros below), m x m column-major
__global__ void qr_copy_r1_kernel(const zd *__restrict__ Y, int64_t ldy, int m, zd *__restrict__ R1) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)m * m) return;
  const int64_t j = e / m, i = e % m;
  R1[e] = i <= j ? Y[j * ldy + i] : zd{0.0, 0.0};
}

void qrblk_sizes(int64_t l, int64_t m, int sms, size_t (&b)[18]) {
  b[0] = oz_slice_bytes(m, 2 * l, kOzSlicesAdj);         // sA: A rows from C's columns
  b[1] = oz_slice_bytes(64, 2 * l, kOzSlicesAdj);        // sB: the reflectors, adjoint form
  b[2] = oz_slice_bytes(2 * l, kOzK, kOzSlicesFwd);      // sV: the reflectors, update form
  b[3] = oz_slice_bytes(m, kOzK, kOzSlicesFwd);          // sZ
  b[4] = sizeof(int32_t) * (size_t)qpad(m, kOzM);
  b[5] = sizeof(int32_t) * (size_t)kOzM;
  b[6] = sizeof(int32_t) * (size_t)qpad(2 * l, kOzM);
  b[7] = sizeof(int32_t) * (size_t)qpad(m, kOzM);
  b[8] = oz_adj_partial_bytes(l, m, sms);
  b[9] = sizeof(zd) * 32 * (size_t)m;       // W
  b[10] = sizeof(zd) * 32 * (size_t)m;      // Z
  b[11] = sizeof(zd) * 32 * 32;             // T
  b[12] = sizeof(double) * 2 * (size_t)m;   // tau
  b[13] = sizeof(zd) * 32 * (size_t)l;      // Vb
  b[14] = sizeof(zd) * (size_t)m * (size_t)m;  // R1
  b[15] = sizeof(zd) * 32 * 2 * (size_t)sms;  // ppart: the panel's posted slots, two parities
  b[16] = sizeof(zd) * 32 * 2;                // rowb: the posted rows, two parities
  b[17] = sizeof(GridBarrier);
}

cudaError_t launch_trailing_products(QrBlkWork &w, const void *V, int64_t ldv, void *C, int64_t ldc, int64_t rows,
                                     int64_t cols, const void *Z, int64_t ldz, void *W, int *err, uint64_t limit_ns,
                                     cudaStream_t st) {
  if (rows > w.l || cols > w.m) return cudaErrorInvalidValue;
  cudaError_t e;
  if (W) {
    OzOperand a{w.sA, w.eA, 0, 0, 0, 0, 0}, b{w.sB, w.eB, 0, 0, 0, 0, 0};
    if ((e = launch_oz_slice_cols(C, ldc, rows, cols, a, st)) != cudaSuccess) return e;
    if ((e = launch_oz_slice_v_adj(V, ldv, rows, b, st)) != cudaSuccess) return e;
    OzAdjArgs g{a, b, w.part, w.part_bytes, W, 32, cols, err, limit_ns};
    if ((e = launch_oz_adj(g, st)) != cudaSuccess) return e;
  }
  if (Z) {
    OzOperand a{w.sV, w.eV, 0, 0, 0, 0, 0}, b{w.sZ, w.eZ, 0, 0, 0, 0, 0};
    if ((e = launch_oz_slice_v_fwd(V, ldv, rows, a, st)) != cudaSuccess) return e;
    if ((e = launch_oz_slice_z(Z, ldz, cols, b, st)) != cudaSuccess) return e;
    OzFwdArgs g{a, b, C, ldc, rows, cols, err, limit_ns};
    if ((e = launch_oz_fwd(g, st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// CTAs of a panel of L rows: at most one per SM, at least 16 rows each, at most
// kPanelMaxRows rows each (the block held in shared memory); 0 when L needs more
int qrblk_panel_grid(int64_t L, int sms) {
  const int64_t g = std::min<int64_t>(sms, std::max<int64_t>(1, L / 16));
  return (L + g - 1) / g <= kPanelMaxRows ? (int)g : 0;
}

// Y = Q1 R1 for the l x m sketch Y (column-major, ld l, overwritten): blocked Householder QR
// of Y without pivoting (panels of 32 columns, trailing updates on the tensor cores); R1 (the
// upper triangle) into the workspace.
cudaError_t launch_qr_tall(QrBlkWork &w, const QrArgs &q, int sms, cudaStream_t st) {
  const int64_t l = q.l, m = q.m;
  if (l > w.l || m > w.m || l < m) return cudaErrorInvalidValue;
  zd *Y = static_cast<zd *>(q.Y);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(qr_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(zd) * kPanelLd * kPanelMaxRows))) != cudaSuccess)
    return e;
  for (int64_t k0 = 0; k0 < m; k0 += kPanel) {
    const int jb = (int)std::min<int64_t>(kPanel, m - k0);
    const int L = (int)(l - k0);
    zd *P = Y + k0 * l + k0;
    if ((e = cudaMemsetAsync(w.bar, 0, sizeof(GridBarrier), st)) != cudaSuccess) return e;
    const int G = qrblk_panel_grid(L, sms);
    if (G <= 0) return cudaErrorInvalidValue;
    const size_t smem = sizeof(zd) * kPanelLd * (size_t)((L + G - 1) / G);
    zd *tau = static_cast<zd *>(w.tau) + k0;
    void *args[] = {(void *)&P, (void *)&l, (void *)&L, (void *)&jb, (void *)&w.Vb, (void *)&l, (void *)&w.T,
                    (void *)&tau, (void *)&w.ppart, (void *)&w.rowb, (void *)&w.bar, (void *)&q.err,
                    (void *)&q.limit_ns};
    note_launch();
    if ((e = cudaLaunchCooperativeKernel((const void *)qr_panel_kernel, dim3(G), dim3(kPanelThreads), args, smem,
                                         st)) != cudaSuccess)
      return e;
    if (k0 + jb < m) {
      const int64_t cols = m - k0 - jb;
      zd *C = Y + (k0 + jb) * l + k0;
      // T on the side stream while the adjoint product runs; Z = T^H W waits for it
      if ((e = cudaEventRecord(w.ev_panel, st)) != cudaSuccess) return e;
      if ((e = cudaStreamWaitEvent(w.side, w.ev_panel, 0)) != cudaSuccess) return e;
      note_launch();
      qr_t_kernel<<<1, 32, 0, w.side>>>(static_cast<zd *>(w.T), tau, jb);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = cudaEventRecord(w.ev_t, w.side)) != cudaSuccess) return e;
      if ((e = launch_trailing_products(w, w.Vb, l, C, l, L, cols, nullptr, 0, w.W, q.err, q.limit_ns, st)) !=
          cudaSuccess)
        return e;
      if ((e = cudaStreamWaitEvent(st, w.ev_t, 0)) != cudaSuccess) return e;
      note_launch();
      qr_tw_kernel<<<(unsigned)((cols * kPanel + 255) / 256), 256, 0, st>>>(
          static_cast<const zd *>(w.T), static_cast<const zd *>(w.W), static_cast<zd *>(w.Z), cols);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if ((e = launch_trailing_products(w, w.Vb, l, C, l, L, cols, w.Z, kPanel, nullptr, q.err, q.limit_ns, st)) !=
          cudaSuccess)
        return e;
    }
  }
  note_launch();
  qr_copy_r1_kernel<<<(unsigned)((m * m + 255) / 256), 256, 0, st>>>(Y, l, (int)m, static_cast<zd *>(w.R1));
  return cudaGetLastError();
}

// R1 P = Q2 R: the pivoted QR of the m x m triangle with the arguments of q (its Y replaced by R1)
cudaError_t launch_qr_triangle(QrBlkWork &w, const QrArgs &q, cudaStream_t st) {
  QrArgs q2 = q;
  q2.Y = w.R1;
  q2.l = q.m;
  return launch_qrp(q2, st);
}

// Y P = Q R: launch_qr_tall, then launch_qr_triangle
cudaError_t launch_qr_blocked(QrBlkWork &w, const QrArgs &q, int sms, cudaStream_t st) {
  cudaError_t e = launch_qr_tall(w, q, sms, st);
  return e != cudaSuccess ? e : launch_qr_triangle(w, q, st);
}

// ---- P R^{-1} by blocks of rows (Step 4's preconditioner) ---------------------------
// X = R^{-1} (R upper triangular, real diagonal) by block rows of kPanel from the bottom, the
// top block taking the remainder, right-looking: with C = I,
//   X_J = R_JJ^{-1} C_J                (block row J of C; FP64 back substitution, one warp per column)
//   C[0:j0, j0:m] -= R[0:j0, J] X_J    (the K = 32 update C -= V Z on the tensor cores)
// then Wp = P X and WpH = Wp^*. Every update of a block row reads only block rows below it, so
// X overwrites C in place.
//
// Rounding. F = R X - I, block row I: F_I = delta_I + sum_{J > I} D_IJ, with delta_I the back
// substitution's residual, |delta_I| <= 4 (bw + 2) 2^-53 |R_II| |X_I| (bw <= 32), and D_IJ the
// error of update J on block row I. The update's bound per entry (the products' operands cut to
// 55 bits below their row's scale, the dropped slice levels, the product rounded once to FP64,
// then the subtraction), with max|V_i:| <= ||V_i:||, sum|Z_:c| <= sqrt 32 ||Z_:c|| and so on:
//   |D_ic| <= 2^-53 ((2 sqrt 32 + 4) ||V_i:|| ||Z_:c|| + |C_ic after the update|),
// and |C_ic| <= [i == c] + (|R| |X|)_ic at every stage (a factor sqrt 2 more on the first term
// for the real forms of complex entries). Summed over the NB = ceil(m / 32) blocks (Cauchy-Schwarz
// over J for the first term) and taken in the Frobenius norm:
//   ||F||_F <= 2^-53 ((136 + sqrt 2 (2 sqrt 32 + 4) + NB) ||R||_F ||X||_F + NB sqrt m)
//           <= 2^-53 (160 + 2 NB) ||R||_F ||X||_F   (sqrt m = ||I||_F <= ||R||_F ||X||_F (1 + ||F||_F)),
// below the column-by-column substitution's 4 m 2^-53 ||R||_F ||X||_F, which the certificate
// uses, for every m >= kPinvBlockedMinM.
constexpr int kPinvWarps = 8;

__global__ void __launch_bounds__(256)
prinv_ident_kernel(zd *__restrict__ X, int m) {
  const int64_t n = (int64_t)m * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    X[e] = {e % (m + 1) == 0 ? 1.0 : 0.0, 0.0};
}

// X[j0:j0+bw, c] = R_JJ^{-1} X[j0:j0+bw, c] for c = j0..m-1: lane i holds row j0 + i; the
// reciprocals of R's (real) diagonal formed once per CTA, as in prinv_kernel
__global__ void __launch_bounds__(32 * kPinvWarps)
prinv_diag_kernel(const zd *__restrict__ R, int m, zd *__restrict__ X, int j0, int bw) {
  __shared__ zd sR[kPanel][kPanel + 1];   // sR[k][i] = R[j0 + i, j0 + k]
  __shared__ double sinv[kPanel];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int e = tid; e < bw * bw; e += blockDim.x) {
    const int i = e % bw, k = e / bw;
    sR[k][i] = R[(int64_t)(j0 + i) + (int64_t)(j0 + k) * m];
  }
  if (tid < bw) sinv[tid] = 1.0 / R[(int64_t)(j0 + tid) * (m + 1)].re;
  __syncthreads();
  const int64_t c = (int64_t)j0 + (int64_t)blockIdx.x * kPinvWarps + w;
  if (c >= m) return;   // warp-uniform
  zd *col = X + c * m + j0;
  zd x = {0.0, 0.0};
  if (lane < bw) x = col[lane];
  for (int k = bw - 1; k >= 0; --k) {
    if (lane == k) {
      x.re *= sinv[k];
      x.im *= sinv[k];
    }
    const double xr = __shfl_sync(0xffffffffu, x.re, k), xi = __shfl_sync(0xffffffffu, x.im, k);
    if (lane < k) {
      const zd a = sR[k][lane];
      x.re = fma(-a.re, xr, fma(a.im, xi, x.re));
      x.im = fma(-a.re, xi, fma(-a.im, xr, x.im));
    }
  }
  if (lane < bw) col[lane] = x;
}

// Wp[piv[i], k] = X[i, k] and WpH[k, piv[i]] = conj(X[i, k]) for i <= k, zero below the diagonal
// (every entry of both written once; 32 x 32 tiles through shared memory for Wp's rows)
__global__ void __launch_bounds__(256)
prinv_scatter_kernel(const zd *__restrict__ X, const int32_t *__restrict__ piv, int m, zd *__restrict__ Wp,
                     zd *__restrict__ WpH) {
  __shared__ zd t[32][33];   // t[k - k0][i - i0]
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + tx, k = k0 + r;
    zd v = {0.0, 0.0};
    if (i < m && k < m) {
      if (i <= k) v = X[(int64_t)i + (int64_t)k * m];
      WpH[(int64_t)k * m + piv[i]] = conjg(v);
    }
    t[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r, k = k0 + tx;
    if (i < m && k < m) Wp[(int64_t)piv[i] * m + k] = t[tx][r];
  }
}

cudaError_t launch_prinv_blocked(QrBlkWork &w, const void *R, const int32_t *piv, int m, void *Wp, void *WpH,
                                 int *err, uint64_t limit_ns, cudaStream_t st) {
  if (m > w.m || m < 1) return cudaErrorInvalidValue;
  zd *X = static_cast<zd *>(w.R1);   // m x m, free once the triangle's pivoted QR has run
  const zd *Rz = static_cast<const zd *>(R);
  note_launch();
  prinv_ident_kernel<<<1024, 256, 0, st>>>(X, m);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int j1 = m; j1 > 0; j1 -= kPanel) {
    const int j0 = j1 > kPanel ? j1 - kPanel : 0, bw = j1 - j0;
    note_launch();
    prinv_diag_kernel<<<(unsigned)((m - j0 + kPinvWarps - 1) / kPinvWarps), 32 * kPinvWarps, 0, st>>>(Rz, m, X, j0,
                                                                                                      bw);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (j0 > 0 &&
        (e = launch_trailing_products(w, Rz + (int64_t)j0 * m, m, X + (int64_t)j0 * m, m, j0, m - j0,
                                      X + j0 + (int64_t)j0 * m, m, nullptr, err, limit_ns, st)) != cudaSuccess)
      return e;
  }
  const dim3 grid((unsigned)((m + 31) / 32), (unsigned)((m + 31) / 32));
  note_launch();
  prinv_scatter_kernel<<<grid, 256, 0, st>>>(X, piv, m, static_cast<zd *>(Wp), static_cast<zd *>(WpH));
  return cudaGetLastError();
}

}  // namespace mn
