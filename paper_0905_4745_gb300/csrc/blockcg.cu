// blockcg.cu -- Step 4 for a block of right-hand sides sharing one A, one T and
// one R: KB independent conjugate-gradient recurrences (one per column, each
// with its own alpha, beta and stopping test) whose products with A are taken
// together, so that A is read once per product for all columns instead of once
// per column:
//     W  = Wp P        (FP64, m x m times m x KB)          block_mm_kernel
//     Q  = A^* W       (complex FP32, n x KB)              block_adj_kernel
//     T  = A Q         (complex FP32, split over n)         block_fwd_kernel + reduce
//     Np = Wp^* T      (FP64)                              block_mm_kernel
// with Wp = P R^{-1}. Block vectors are row-major m x KB (column c of row i at
// i * KB + c). Columns that have met their stopping test (or are unused) carry
// active = 0 and are left unchanged; once no column is active the kernels of
// iterations already enqueued return at once.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mn {

// ---- OUT = M V: M m x m row-major complex128, V m x KB ---------------------------
// Tile of 32 rows x KB columns per CTA, 128 threads: thread (row group rg, column
// group cg) accumulates 4 rows x (KB / 16) columns. FP64 (the R solves stay FP64).
template <int KB>
__global__ void __launch_bounds__(128)
block_mm_kernel(const zd *__restrict__ M, int m, const zd *__restrict__ V, zd *__restrict__ out,
                zf *__restrict__ out32, const int *__restrict__ alldone) {
  if (alldone && *alldone) return;
  constexpr int CT = KB / 16;  // columns per thread
  __shared__ zd sM[32][33];
  __shared__ zd sV[32][KB];
  const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;  // rg 0..7 (4 rows each), cg 0..15
  const int i0 = blockIdx.x * 32;
  zd acc[4][CT];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < CT; ++c) acc[r][c] = {0.0, 0.0};
  for (int k0 = 0; k0 < m; k0 += 32) {
    __syncthreads();
    for (int e = tid; e < 32 * 32; e += 128) {
      const int r = e >> 5, k = e & 31;
      sM[r][k] = (i0 + r < m && k0 + k < m) ? M[(int64_t)(i0 + r) * m + k0 + k] : zd{0.0, 0.0};
    }
    for (int e = tid; e < 32 * KB; e += 128) {
      const int k = e / KB, c = e - k * KB;
      sV[k][c] = (k0 + k < m) ? V[(int64_t)(k0 + k) * KB + c] : zd{0.0, 0.0};
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < 32; ++k) {
      zd a[4], v[CT];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = sM[rg * 4 + r][k];
#pragma unroll
      for (int c = 0; c < CT; ++c) v[c] = sV[k][cg + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < CT; ++c) mac(acc[r][c], a[r], v[c]);
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + rg * 4 + r;
    if (i < m) {
#pragma unroll
      for (int c = 0; c < CT; ++c) {
        const int col = cg + 16 * c;
        if (out) out[(int64_t)i * KB + col] = acc[r][c];
        if (out32) out32[(int64_t)i * KB + col] = {(float)acc[r][c].re, (float)acc[r][c].im};
      }
    }
  }
}

// ---- Q = A^* W: A m x n complex64 row-major (lda), W m x KB complex64 ------------
// CTA: 64 columns j of A x KB; 128 threads, thread (jg, cg) holds 4 j x (KB / 16)
// columns. Rows of A in tiles of 32 through shared memory (coalesced along j).
// qqp[blockIdx.x * KB + c] = sum over the tile's j of |Q_jc|^2 (FP32).
template <int KB>
__global__ void __launch_bounds__(128)
block_adj_kernel(const zf *__restrict__ A, int64_t lda, int m, int64_t n, const zf *__restrict__ W,
                 zf *__restrict__ Q, float *__restrict__ qqp, const int *__restrict__ alldone) {
  if (*alldone) return;
  constexpr int CT = KB / 16;
  __shared__ zf sA[32][64 + 1];
  __shared__ zf sW[32][KB];
  __shared__ float sq[8][KB];
  const int tid = threadIdx.x, jg = tid >> 4, cg = tid & 15;  // jg 0..7 (4 j each... x 2 halves)
  const int64_t j0 = (int64_t)blockIdx.x * 64;
  zf acc[8][CT];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < CT; ++c) acc[r][c] = {0.f, 0.f};
  for (int i0 = 0; i0 < m; i0 += 32) {
    __syncthreads();
    for (int e = tid; e < 32 * 64; e += 128) {
      const int r = e >> 6, jj = e & 63;
      sA[r][jj] = (i0 + r < m && j0 + jj < n) ? A[(int64_t)(i0 + r) * lda + j0 + jj] : zf{0.f, 0.f};
    }
    for (int e = tid; e < 32 * KB; e += 128) {
      const int r = e / KB, c = e - r * KB;
      sW[r][c] = (i0 + r < m) ? W[(int64_t)(i0 + r) * KB + c] : zf{0.f, 0.f};
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
      zf a[8], w[CT];
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = sA[r][jg + 8 * q];
#pragma unroll
      for (int c = 0; c < CT; ++c) w[c] = sW[r][cg + 16 * c];
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int c = 0; c < CT; ++c) macc(acc[q][c], a[q], w[c]);
    }
  }
  float qq[CT];
#pragma unroll
  for (int c = 0; c < CT; ++c) qq[c] = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t j = j0 + jg + 8 * q;
    if (j < n) {
#pragma unroll
      for (int c = 0; c < CT; ++c) {
        Q[j * KB + cg + 16 * c] = acc[q][c];
        qq[c] = fmaf(acc[q][c].re, acc[q][c].re, fmaf(acc[q][c].im, acc[q][c].im, qq[c]));
      }
    }
  }
  // per column: sum over the 8 j-groups (threads with equal cg)
#pragma unroll
  for (int c = 0; c < CT; ++c) sq[jg][cg + 16 * c] = qq[c];
  __syncthreads();
  if (tid < KB) {
    float s = 0.f;
#pragma unroll
    for (int g = 0; g < 8; ++g) s += sq[g][tid];
    qqp[(int64_t)blockIdx.x * KB + tid] = s;
  }
}

// ---- Tpart[split] = A[:, chunk] Q[chunk]: 64 rows x KB per CTA, split over n -----
template <int KB>
__global__ void __launch_bounds__(128)
block_fwd_kernel(const zf *__restrict__ A, int64_t lda, int m, int64_t n, int64_t chunk, const zf *__restrict__ Q,
                 zf *__restrict__ tpart, const int *__restrict__ alldone) {
  if (*alldone) return;
  constexpr int CT = KB / 16;
  __shared__ zf sA[64][32 + 1];
  __shared__ zf sQ[32][KB];
  const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15;  // rg 0..7: rows rg + 8 q
  const int i0 = blockIdx.x * 64;
  const int64_t c0 = (int64_t)blockIdx.y * chunk, c1 = c0 + chunk < n ? c0 + chunk : n;
  zf acc[8][CT];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < CT; ++c) acc[r][c] = {0.f, 0.f};
  for (int64_t jt = c0; jt < c1; jt += 32) {
    __syncthreads();
    for (int e = tid; e < 64 * 32; e += 128) {
      const int r = e >> 5, jj = e & 31;
      sA[r][jj] = (i0 + r < m && jt + jj < c1) ? A[(int64_t)(i0 + r) * lda + jt + jj] : zf{0.f, 0.f};
    }
    for (int e = tid; e < 32 * KB; e += 128) {
      const int jj = e / KB, c = e - jj * KB;
      sQ[jj][c] = (jt + jj < c1) ? Q[(jt + jj) * KB + c] : zf{0.f, 0.f};
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < 32; ++jj) {
      zf a[8], q[CT];
#pragma unroll
      for (int r = 0; r < 8; ++r) a[r] = sA[rg + 8 * r][jj];
#pragma unroll
      for (int c = 0; c < CT; ++c) q[c] = sQ[jj][cg + 16 * c];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < CT; ++c) mac(acc[r][c], a[r], q[c]);
    }
  }
  zf *tp = tpart + (int64_t)blockIdx.y * m * KB;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = i0 + rg + 8 * r;
    if (i < m) {
#pragma unroll
      for (int c = 0; c < CT; ++c) tp[(int64_t)i * KB + cg + 16 * c] = acc[r][c];
    }
  }
}

template <int KB>
__global__ void block_fwd_reduce_kernel(const zf *__restrict__ tpart, int nsplit, int m, zd *__restrict__ T,
                                        const int *__restrict__ alldone) {
  if (*alldone) return;
  const int64_t total = (int64_t)m * KB;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int s = 0; s < nsplit; ++s) {
      const zf v = tpart[(int64_t)s * total + e];
      re += (double)v.re;
      im += (double)v.im;
    }
    T[e] = {re, im};
  }
}

// ---- per-column sums of |X_ic|^2 over row ranges: part[blockIdx.x * KB + c] -------
template <int KB>
__device__ __forceinline__ void col_sumsq_part(const zd *__restrict__ X, int m, double *__restrict__ part,
                                               double *red) {
  // 256 threads: thread (rr, c) with c = tid % KB; rows rr, rr + 256/KB, ... within this CTA's range
  constexpr int RS = 256 / KB;
  const int tid = threadIdx.x, c = tid % KB, rr = tid / KB;
  const int per = (m + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * per, r1 = min(m, r0 + per);
  double acc = 0.0;
  for (int i = r0 + rr; i < r1; i += RS) {
    const zd v = X[(int64_t)i * KB + c];
    acc = fma(v.re, v.re, fma(v.im, v.im, acc));
  }
  red[tid] = acc;
  __syncthreads();
  if (tid < KB) {
    double s = 0.0;
    for (int q = 0; q < RS; ++q) s += red[q * KB + tid];
    part[(int64_t)blockIdx.x * KB + tid] = s;
  }
}

// U = 0, S = P = G; partial ||G_c||^2
template <int KB>
__global__ void __launch_bounds__(256)
block_cg_init_kernel(int m, const zd *__restrict__ G, zd *__restrict__ U, zd *__restrict__ S, zd *__restrict__ P,
                     double *__restrict__ part) {
  __shared__ double red[256];
  const int64_t total = (int64_t)m * KB;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const zd g = G[e];
    S[e] = g;
    P[e] = g;
    U[e] = {0.0, 0.0};
  }
  col_sumsq_part<KB>(G, m, part, red);
}

// scalars after init: gamma = gamma0 = ||g_c||^2, active = (gamma > 0) and the column is in use
template <int KB>
__global__ void block_cg_start_kernel(const double *__restrict__ part, int nparts, const int *__restrict__ use,
                                      double *__restrict__ gam, double *__restrict__ gam0, int *__restrict__ active,
                                      int *__restrict__ alldone) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int c = threadIdx.x;
  if (c < KB) {
    double s = 0.0;
    for (int q = 0; q < nparts; ++q) s += part[(int64_t)q * KB + c];
    gam[c] = s;
    gam0[c] = s;
    const int a = (use[c] && s > 0.0) ? 1 : 0;
    active[c] = a;
    if (a) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *alldone = any ? 0 : 1;
}

// alpha_c = gamma_c / qq_c (active columns, else 0); qq from the adjoint kernel's partials
template <int KB>
__global__ void block_alpha_kernel(const float *__restrict__ qqp, int nparts, const double *__restrict__ gam,
                                   const int *__restrict__ active, double *__restrict__ alpha,
                                   const int *__restrict__ alldone) {
  if (*alldone) return;
  // KB warps: warp c sums column c's partials
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c >= KB) return;
  double s = 0.0;
  for (int q = lane; q < nparts; q += 32) s += (double)qqp[(int64_t)q * KB + c];
  s = warp_sum(s);
  if (lane == 0) alpha[c] = (active[c] && s > 0.0) ? gam[c] / s : 0.0;
}

// U += alpha P; S -= alpha Np (per column); partial ||S_c||^2. Each CTA updates exactly the
// rows it then sums (the same range as col_sumsq_part).
template <int KB>
__global__ void __launch_bounds__(256)
block_cg_step_kernel(int m, const double *__restrict__ alpha, const zd *__restrict__ P, const zd *__restrict__ Np,
                     zd *__restrict__ U, zd *__restrict__ S, double *__restrict__ part,
                     const int *__restrict__ alldone) {
  __shared__ double red[256];
  if (*alldone) return;
  const int per = (m + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * per, r1 = min(m, r0 + per);
  for (int64_t e = (int64_t)r0 * KB + threadIdx.x; e < (int64_t)r1 * KB; e += blockDim.x) {
    const double a = alpha[e % KB];
    const zd p = P[e], np = Np[e];
    zd u = U[e], s = S[e];
    u.re = fma(a, p.re, u.re);
    u.im = fma(a, p.im, u.im);
    s.re = fma(-a, np.re, s.re);
    s.im = fma(-a, np.im, s.im);
    U[e] = u;
    S[e] = s;
  }
  __syncthreads();
  col_sumsq_part<KB>(S, m, part, red);
}

// beta_c = gamma'_c / gamma_c; the stopping test per column; all columns done -> alldone
template <int KB>
__global__ void block_beta_kernel(const double *__restrict__ part, int nparts, double tol2, double *__restrict__ gam,
                                  const double *__restrict__ gam0, const double *__restrict__ alpha,
                                  int *__restrict__ active, double *__restrict__ beta, int *__restrict__ iters,
                                  int *__restrict__ alldone) {
  __shared__ int any;
  if (*alldone) return;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int c = threadIdx.x;
  if (c < KB) {
    double b = 0.0;
    if (active[c]) {
      double s = 0.0;
      for (int q = 0; q < nparts; ++q) s += part[(int64_t)q * KB + c];
      b = gam[c] > 0.0 ? s / gam[c] : 0.0;
      gam[c] = s;
      iters[c] += 1;
      if (s <= tol2 * gam0[c] || !(alpha[c] > 0.0)) active[c] = 0;
      else atomicOr(&any, 1);
    }
    beta[c] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0 && !any) *alldone = 1;
}

// P = S + beta P (columns active after the test)
template <int KB>
__global__ void __launch_bounds__(256)
block_cg_dir_kernel(int m, const double *__restrict__ beta, const int *__restrict__ active, const zd *__restrict__ S,
                    zd *__restrict__ P, const int *__restrict__ alldone) {
  if (*alldone) return;
  const int64_t total = (int64_t)m * KB;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % KB);
    if (!active[c]) continue;
    const double b = beta[c];
    const zd s = S[e];
    zd p = P[e];
    p.re = fma(b, p.re, s.re);
    p.im = fma(b, p.im, s.im);
    P[e] = p;
  }
}

// ---- host -----------------------------------------------------------------------
static_assert(kBlockRhs == 32, "the launchers below instantiate KB = 32");

int block_adj_parts(int64_t n) { return (int)((n + 63) / 64); }
int block_fwd_splits(int64_t m, int64_t n, int sms) {
  const int64_t rb = (m + 63) / 64;
  int s = 1;
  while (rb * s < 4 * sms && n / (2 * s) >= 256) s *= 2;
  return s;
}
int block_col_parts(int64_t m) { return (int)std::min<int64_t>(64, (m + 255) / 256); }

cudaError_t launch_block_mm(const void *M, int m, const void *V, void *out, void *out32, const int *alldone,
                            cudaStream_t st) {
  note_launch();
  block_mm_kernel<kBlockRhs><<<(m + 31) / 32, 128, 0, st>>>((const zd *)M, m, (const zd *)V, (zd *)out, (zf *)out32,
                                                             alldone);
  return cudaGetLastError();
}

cudaError_t launch_block_adj(const BlockProductArgs &a, cudaStream_t st) {
  cudaError_t e;
  if (a.Bsplit && tc_block_supported(a.m, a.n, a.lda, a.A)) {
    e = launch_tc_block_adj(a.A, a.m, a.n, a.lda, a.W32, a.Bsplit, a.Q, a.qqp, a.alldone, a.err, a.limit_ns, a.sms,
                            st);
  } else {
    note_launch();
    block_adj_kernel<kBlockRhs><<<block_adj_parts(a.n), 128, 0, st>>>((const zf *)a.A, a.lda, (int)a.m, a.n,
                                                                      (const zf *)a.W32, (zf *)a.Q, a.qqp,
                                                                      a.alldone);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  note_launch();
  block_alpha_kernel<kBlockRhs><<<1, 32 * kBlockRhs, 0, st>>>(a.qqp, block_adj_parts(a.n), a.gam, a.active, a.alpha,
                                                             a.alldone);
  return cudaGetLastError();
}

cudaError_t launch_block_fwd(const BlockProductArgs &a, cudaStream_t st) {
  int ns = a.nsplit;
  cudaError_t e;
  if (a.Bsplit2 && a.nsplit_tc > 0 && tc_block_supported(a.m, a.n, a.lda, a.A)) {
    ns = a.nsplit_tc;
    e = launch_tc_block_fwd(a.A, a.m, a.n, a.lda, a.Q, a.Bsplit2, a.tpart, ns, a.alldone, a.err, a.limit_ns, st);
  } else {
    const int64_t chunk = (a.n + ns - 1) / ns;
    note_launch();
    block_fwd_kernel<kBlockRhs><<<dim3((unsigned)((a.m + 63) / 64), (unsigned)ns), 128, 0, st>>>(
        (const zf *)a.A, a.lda, (int)a.m, a.n, chunk, (const zf *)a.Q, (zf *)a.tpart, a.alldone);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return e;
  note_launch();
  block_fwd_reduce_kernel<kBlockRhs><<<(unsigned)std::min<int64_t>(1024, (a.m * kBlockRhs + 255) / 256), 256, 0,
                                       st>>>((const zf *)a.tpart, ns, (int)a.m, (zd *)a.T, a.alldone);
  return cudaGetLastError();
}

// column c of a block (m x KB row-major) <-> a contiguous m-vector; dd accumulate per used column
__global__ void block_get_col_kernel(int m, const zd *__restrict__ Bk, int c, zd *__restrict__ v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) v[i] = Bk[(int64_t)i * kBlockRhs + c];
}
__global__ void block_set_col_kernel(int m, const zd *__restrict__ v, int c, zd *__restrict__ Bk) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) Bk[(int64_t)i * kBlockRhs + c] = v[i];
}
// R[:, c] = B column (j0 + c) for c < kc, 0 otherwise (B column-major, leading dimension ldb)
__global__ void block_load_rhs_kernel(int m, int kc, const zd *__restrict__ B, int64_t ldb, zd *__restrict__ R) {
  const int64_t total = (int64_t)m * kBlockRhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / kBlockRhs), c = (int)(e % kBlockRhs);
    R[e] = c < kc ? B[(int64_t)c * ldb + i] : zd{0.0, 0.0};
  }
}
// Yh + Yl += dY (double-double) on the columns with use[c]
__global__ void block_dd_acc_kernel(int m, const int *__restrict__ use, zd *__restrict__ Yh, zd *__restrict__ Yl,
                                    const zd *__restrict__ dY) {
  const int64_t total = (int64_t)m * kBlockRhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    if (!use[e % kBlockRhs]) continue;
    const zd d = dY[e];
    zd h = Yh[e], l = Yl[e];
    double s, q;
    two_sum(h.re, d.re, s, q);
    h.re = s;
    l.re = __dadd_rn(l.re, q);
    two_sum(h.im, d.im, s, q);
    h.im = s;
    l.im = __dadd_rn(l.im, q);
    two_sum(h.re, l.re, s, q);
    h.re = s;
    l.re = q;
    two_sum(h.im, l.im, s, q);
    h.im = s;
    l.im = q;
    Yh[e] = h;
    Yl[e] = l;
  }
}
// per-column sums of |X_ic|^2 into part (block_col_parts(m) x KB)
template <int KB>
__global__ void __launch_bounds__(256) block_colnorm_kernel(int m, const zd *__restrict__ X, double *__restrict__ part) {
  __shared__ double red[256];
  col_sumsq_part<KB>(X, m, part, red);
}

cudaError_t launch_block_get_col(int m, const void *Bk, int c, void *v, cudaStream_t st) {
  note_launch();
  block_get_col_kernel<<<(m + 255) / 256, 256, 0, st>>>(m, (const zd *)Bk, c, (zd *)v);
  return cudaGetLastError();
}
cudaError_t launch_block_set_col(int m, const void *v, int c, void *Bk, cudaStream_t st) {
  note_launch();
  block_set_col_kernel<<<(m + 255) / 256, 256, 0, st>>>(m, (const zd *)v, c, (zd *)Bk);
  return cudaGetLastError();
}
cudaError_t launch_block_load_rhs(int m, int kc, const void *B, int64_t ldb, void *R, cudaStream_t st) {
  note_launch();
  block_load_rhs_kernel<<<(unsigned)std::min<int64_t>(1024, ((int64_t)m * kBlockRhs + 255) / 256), 256, 0, st>>>(
      m, kc, (const zd *)B, ldb, (zd *)R);
  return cudaGetLastError();
}
cudaError_t launch_block_dd_acc(int m, const int *use, void *Yh, void *Yl, const void *dY, cudaStream_t st) {
  note_launch();
  block_dd_acc_kernel<<<(unsigned)std::min<int64_t>(1024, ((int64_t)m * kBlockRhs + 255) / 256), 256, 0, st>>>(
      m, use, (zd *)Yh, (zd *)Yl, (const zd *)dY);
  return cudaGetLastError();
}
cudaError_t launch_block_colnorms(int m, const void *X, double *part, cudaStream_t st) {
  note_launch();
  block_colnorm_kernel<kBlockRhs><<<block_col_parts(m), 256, 0, st>>>(m, (const zd *)X, part);
  return cudaGetLastError();
}

cudaError_t launch_block_cg_init(int m, const void *G, void *U, void *S, void *P, double *part, const int *use,
                                 double *gam, double *gam0, int *active, int *alldone, cudaStream_t st) {
  const int np = block_col_parts(m);
  note_launch();
  block_cg_init_kernel<kBlockRhs><<<np, 256, 0, st>>>(m, (const zd *)G, (zd *)U, (zd *)S, (zd *)P, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launch();
  block_cg_start_kernel<kBlockRhs><<<1, kBlockRhs, 0, st>>>(part, np, use, gam, gam0, active, alldone);
  return cudaGetLastError();
}

cudaError_t launch_block_cg_update(int m, const double *alpha, void *P, const void *Np, void *U, void *S,
                                   double *part, double tol2, double *gam, const double *gam0, int *active,
                                   double *beta, int *iters, int *alldone, cudaStream_t st) {
  const int np = block_col_parts(m);
  note_launch();
  block_cg_step_kernel<kBlockRhs><<<np, 256, 0, st>>>(m, alpha, (const zd *)P, (const zd *)Np, (zd *)U, (zd *)S,
                                                      part, alldone);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launch();
  block_beta_kernel<kBlockRhs><<<1, kBlockRhs, 0, st>>>(part, np, tol2, gam, gam0, alpha, active, beta, iters,
                                                       alldone);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  note_launch();
  block_cg_dir_kernel<kBlockRhs><<<(unsigned)std::min<int64_t>(1024, ((int64_t)m * kBlockRhs + 255) / 256), 256, 0,
                                   st>>>(m, beta, active, (const zd *)S, (zd *)P, alldone);
  return cudaGetLastError();
}

}  // namespace mn
