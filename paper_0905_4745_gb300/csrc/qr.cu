// qr.cu -- Step 2 of the algorithm (Eq. lineq): Householder QR with column
// pivoting of the sketch, Y P = Q R (the "classical pivoted QR based on
// Householder reflections" of Section 7, Golub & Van Loan ch. 5), then the
// preconditioner P R^{-1} used by Step 4.
//
// qrp_bal_kernel is one cooperative grid (at most one CTA per SM). Per step k
// every CTA
//   1. picks the pivot p = the first column of largest partial norm among the
//      remaining ones, in the logical column order LAPACK's swaps produce,
//   2. in one block reduction forms ||Y[k+1:, p]||^2 and, for its share of the
//      trailing columns j, sum_r conj(Y[r,p]) Y[r,j] (the reflector's scale is
//      not needed for these sums, so all CTAs build the same reflector
//      H = I - tau v v^*, v = (1, Y[k+1:, p] / (Y[k,p] - beta)), beta real,
//      without waiting for each other),
//   3. applies H^* to its columns and downdates their partial norms (with
//      LAPACK's recomputation when the downdate loses half the digits),
//   4. meets the others at a grid barrier whose wait is bounded in time.
// The pivot column itself is left unscaled: only R and P are kept (Q is never
// needed: Steps 2-3 enter the solve through R alone, see solver.cu).
#include "common.cuh"
#include "kernels.h"

namespace mn {

constexpr int kQrThreads = 256;

__global__ void __launch_bounds__(kQrThreads)
qr_norms_kernel(const zd *__restrict__ Y, int l, double *__restrict__ vn1, double *__restrict__ vn2) {
  __shared__ double sc[kQrThreads / 32];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int r = threadIdx.x; r < l; r += blockDim.x) acc += abs2(Y[r + (int64_t)j * l]);
  const double t = block_sum(acc, sc);
  if (threadIdx.x == 0) { vn1[j] = sqrt(t); vn2[j] = sqrt(t); }
}

// Columns are assigned to CTAs afresh at every step: all CTAs keep the same
// logical order of the columns (a permutation updated by the same swaps
// LAPACK's zlaqp2 makes, so ties go to the same pivot as there), and CTA b
// takes the b-th equal share of the trailing positions k+1..m-1. Y stays in
// place in global memory (it is L2-resident for the sizes where the QR is
// latency-bound); partial norms are indexed by physical column and
// double-buffered across steps.
constexpr int kQrbThreads = 128;
// two CTAs per SM: one CTA's latency-bound scalar phases overlap the other's FP64 loops
constexpr int kQrCtasPerSm = 2;

// On GB300 every FP64 warp instruction occupies the SM's FP64 pipe for tens of
// cycles, so the per-step scalar work is arranged to issue few of them: the
// pivot search compares the norms' bit patterns as integers (they are
// non-negative), the block uses 4 warps so the reduction tree is short, and
// the factors of the own columns are computed by one lane each.
// The per-column loops are instantiated for the exact number of own columns
// (a predicated-off FP64 instruction still occupies the FP64 pipe).
template <int NC, int K>
__device__ __forceinline__ void qr_dots(const zd *__restrict__ yp, const zd *__restrict__ Y, const int *cols,
                                        int k, int l, double (&part)[K]) {
  const zd *cp[NC > 0 ? NC : 1];
#pragma unroll
  for (int c = 0; c < NC; ++c) cp[c] = Y + (int64_t)cols[c] * l;
  int r = k + 1 + threadIdx.x;
  const int stride = blockDim.x;
  // several rows per thread in flight (the columns live in L2), fewer for many columns
  constexpr int U = NC <= 2 ? 4 : (NC <= 4 ? 2 : 1);
  for (; r + (U - 1) * stride < l; r += U * stride) {
    zd a[U], y[U][NC > 0 ? NC : 1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a[u] = yp[r + u * stride];
#pragma unroll
      for (int c = 0; c < NC; ++c) y[u][c] = cp[c][r + u * stride];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      part[0] = fma(a[u].re, a[u].re, fma(a[u].im, a[u].im, part[0]));
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        part[1 + 2 * c] = fma(a[u].re, y[u][c].re, fma(a[u].im, y[u][c].im, part[1 + 2 * c]));
        part[2 + 2 * c] = fma(a[u].re, y[u][c].im, fma(-a[u].im, y[u][c].re, part[2 + 2 * c]));
      }
    }
  }
  for (; r < l; r += stride) {
    const zd a = yp[r];
    part[0] = fma(a.re, a.re, fma(a.im, a.im, part[0]));
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const zd y = cp[c][r];
      part[1 + 2 * c] = fma(a.re, y.re, fma(a.im, y.im, part[1 + 2 * c]));
      part[2 + 2 * c] = fma(a.re, y.im, fma(-a.im, y.re, part[2 + 2 * c]));
    }
  }
}

template <int NC>
__device__ __forceinline__ void qr_update(const zd *__restrict__ yp, zd *__restrict__ Y, const int *cols,
                                          const zd *g, int k, int l) {
  zd gg[NC > 0 ? NC : 1];
  zd *cp[NC > 0 ? NC : 1];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    gg[c] = g[c];
    cp[c] = Y + (int64_t)cols[c] * l;
  }
  int r = k + 1 + threadIdx.x;
  const int stride = blockDim.x;
  constexpr int U = NC <= 2 ? 4 : (NC <= 4 ? 2 : 1);
  for (; r + (U - 1) * stride < l; r += U * stride) {
    zd a[U], v[U][NC > 0 ? NC : 1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a[u] = yp[r + u * stride];
#pragma unroll
      for (int c = 0; c < NC; ++c) v[u][c] = cp[c][r + u * stride];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        zd t = v[u][c];
        t.re = fma(-gg[c].re, a[u].re, fma(gg[c].im, a[u].im, t.re));
        t.im = fma(-gg[c].re, a[u].im, fma(-gg[c].im, a[u].re, t.im));
        cp[c][r + u * stride] = t;
      }
    }
  }
  for (; r < l; r += stride) {
    const zd a = yp[r];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      zd v = cp[c][r];
      v.re = fma(-gg[c].re, a.re, fma(gg[c].im, a.im, v.re));
      v.im = fma(-gg[c].re, a.im, fma(-gg[c].im, a.re, v.im));
      cp[c][r] = v;
    }
  }
}

#define MN_QR_SWITCH(NACT, CALL0, CALLN)                      \
  switch (NACT) {                                             \
    case 0: CALL0; break;                                     \
    case 1: CALLN((MAXC >= 1 ? 1 : 0)); break;                \
    case 2: CALLN((MAXC >= 2 ? 2 : 0)); break;                \
    case 3: CALLN((MAXC >= 3 ? 3 : 0)); break;                \
    case 4: CALLN((MAXC >= 4 ? 4 : 0)); break;                \
    case 5: CALLN((MAXC >= 5 ? 5 : 0)); break;                \
    case 6: CALLN((MAXC >= 6 ? 6 : 0)); break;                \
    case 7: CALLN((MAXC >= 7 ? 7 : 0)); break;                \
    default: CALLN((MAXC >= 8 ? 8 : 0)); break;               \
  }

template <int MAXC>
__global__ void __launch_bounds__(kQrbThreads)
qrp_bal_kernel(zd *__restrict__ Y, int l, int m, double *__restrict__ vnA, double *__restrict__ vnB,
               double *__restrict__ vn2, double *__restrict__ beta, int32_t *__restrict__ piv,
               zd *__restrict__ Rout, GridBarrier *bar, int *err, uint64_t limit_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int *perm = reinterpret_cast<int *>(smem_raw);  // logical position -> physical column
  constexpr int K = 1 + 2 * MAXC;
  constexpr int NW = kQrbThreads / 32;
  __shared__ double red_scratch[NW * K];
  __shared__ double red_out[K];
  __shared__ long long s_val[NW];
  __shared__ int s_idx[NW];
  __shared__ int s_col[MAXC];
  __shared__ zd s_g[MAXC];
  __shared__ int s_rec[MAXC];
  __shared__ int s_nact, s_nrec;

  const int G = gridDim.x, b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const double tol3z = sqrt(0x1.0p-53);
  for (int j = tid; j < m; j += blockDim.x) perm[j] = j;
  __syncthreads();

  for (int k = 0; k < m; ++k) {
    const double *vn_cur = (k & 1) ? vnB : vnA;
    double *vn_nxt = (k & 1) ? vnA : vnB;
    // 1. pivot: first maximum over logical positions k..m-1 (integer compare of non-negative doubles)
    long long best = -1;
    int bpos = 0x7fffffff;
    for (int q = k + tid; q < m; q += blockDim.x) {
      const long long v = __double_as_longlong(vn_cur[perm[q]]);
      if (v > best) { best = v; bpos = q; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oq = __shfl_xor_sync(0xffffffffu, bpos, o);
      if (ov > best || (ov == best && oq < bpos)) { best = ov; bpos = oq; }
    }
    if (lane == 0) { s_val[wid] = best; s_idx[wid] = bpos; }
    __syncthreads();
    if (tid == 0) {
      long long bv = s_val[0];
      int bq = s_idx[0];
      for (int w = 1; w < NW; ++w)
        if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bq)) { bv = s_val[w]; bq = s_idx[w]; }
      const int tmp = perm[k];
      perm[k] = perm[bq];
      perm[bq] = tmp;
      if (b == 0) piv[k] = perm[k];
      const int T = m - k - 1;
      const int q0 = k + 1 + (int)(((long long)T * b) / G), q1 = k + 1 + (int)(((long long)T * (b + 1)) / G);
      int na = 0;
      for (int q = q0; q < q1; ++q) s_col[na++] = perm[q];
      s_nact = na;
    }
    __syncthreads();
    const int p = perm[k];
    const int nact = s_nact;
    const zd *yp = Y + (int64_t)p * l;

    // 2. one reduction: ||Y[k+1:,p]||^2 and conj(Y[k+1:,p])^T Y[k+1:,j] for own columns
    double part[K];
#pragma unroll
    for (int c = 0; c < K; ++c) part[c] = 0.0;
#define MN_DOTS(NC) qr_dots<NC, K>(yp, Y, s_col, k, l, part)
    if (MAXC <= 8) {
      MN_QR_SWITCH(nact, MN_DOTS(0), MN_DOTS)
    } else {
      for (int r = k + 1 + tid; r < l; r += blockDim.x) {
        const zd a = yp[r];
        part[0] = fma(a.re, a.re, fma(a.im, a.im, part[0]));
#pragma unroll
        for (int c = 0; c < MAXC; ++c) {
          if (c < nact) {
            const zd y = Y[r + (int64_t)s_col[c] * l];
            part[1 + 2 * c] = fma(a.re, y.re, fma(a.im, y.im, part[1 + 2 * c]));
            part[2 + 2 * c] = fma(a.re, y.im, fma(-a.im, y.re, part[2 + 2 * c]));
          }
        }
      }
    }
#undef MN_DOTS
    block_sum_k<double, K>(part, red_scratch, red_out);

    // 3. reflector H = I - tau v v^*, identical in every CTA (LAPACK zlarfg convention),
    //    computed by each lane that owns a column (and lane 0 of CTA 0 for beta), then that
    //    column's factor and partial-norm downdate
    if (tid == 0) s_nrec = 0;
    if (tid < (nact > 0 ? nact : 1)) {
      const zd alpha = yp[k];
      const double xn2 = red_out[0];
      zd tau = {0.0, 0.0}, scale = {0.0, 0.0};
      double bt;
      if (xn2 == 0.0 && alpha.im == 0.0) {
        bt = alpha.re;
      } else {
        const double mag = sqrt(alpha.re * alpha.re + alpha.im * alpha.im + xn2);
        bt = alpha.re >= 0.0 ? -mag : mag;
        const double ib = 1.0 / bt;
        tau = {(bt - alpha.re) * ib, -alpha.im * ib};
        const double dr = alpha.re - bt, di = alpha.im;
        const double iden = 1.0 / (dr * dr + di * di);
        scale = {dr * iden, -di * iden};
      }
      if (b == 0 && tid == 0) beta[k] = bt;
      if (tid < nact) {
        const int c = tid;
        const int j = s_col[c];
        zd *yj = Y + (int64_t)j * l;
        const zd d = {red_out[1 + 2 * c], red_out[2 + 2 * c]};
        zd w = yj[k];
        macc(w, scale, d);                      // w = y_k + conj(scale) d
        const zd f = conjg(tau) * w;            // H^* = I - conj(tau) v v^*
        s_g[c] = f * scale;
        const zd rk = yj[k] - f;
        yj[k] = rk;
        // LAPACK zlaqp2 downdate: vn1 *= sqrt(1 - (|r_k|/vn1)^2) unless that loses half the digits
        const double v1 = vn_cur[j];
        double nv = v1;
        if (v1 != 0.0) {
          const double iv = 1.0 / v1;
          const double t = sqrt(abs2(rk)) * iv;
          double temp = 1.0 - t * t;
          temp = temp < 0.0 ? 0.0 : temp;
          const double ratio = v1 / vn2[j];
          if (temp * ratio * ratio <= tol3z) s_rec[atomicAdd(&s_nrec, 1)] = c;
          else nv = v1 * sqrt(temp);
        }
        vn_nxt[j] = nv;
      }
    }
    __syncthreads();

    // 4. apply H^* to the own columns, rows k+1..l-1
#define MN_UPD(NC) qr_update<NC>(yp, Y, s_col, s_g, k, l)
    if (MAXC <= 8) {
      MN_QR_SWITCH(nact, (void)0, MN_UPD)
    } else {
      for (int r = k + 1 + tid; r < l; r += blockDim.x) {
        const zd a = yp[r];
#pragma unroll
        for (int c = 0; c < MAXC; ++c) {
          if (c < nact) {
            zd *y = Y + r + (int64_t)s_col[c] * l;
            zd v = *y;
            const zd g = s_g[c];
            v.re = fma(-g.re, a.re, fma(g.im, a.im, v.re));
            v.im = fma(-g.re, a.im, fma(-g.im, a.re, v.im));
            *y = v;
          }
        }
      }
    }
#undef MN_UPD
    const int nrec = s_nrec;
    for (int q = 0; q < nrec; ++q) {  // rare: recompute a partial norm from scratch
      __syncthreads();
      const int j = s_col[s_rec[q]];
      double acc = 0.0;
      for (int r = k + 1 + tid; r < l; r += blockDim.x) acc += abs2(Y[r + (int64_t)j * l]);
      const double t = sqrt(block_sum(acc, red_scratch));
      if (tid == 0) {
        const double v = (k < l - 1) ? t : 0.0;
        vn_nxt[j] = v;
        vn2[j] = v;
      }
    }
    if (!grid_sync(bar, G, limit_ns)) {
      if (tid == 0) atomicExch(err, 1);
      return;
    }
  }

  // R in pivot order: R[i, k] = Y[i, perm[k]] above the diagonal, beta_k on it
  for (int k = b; k < m; k += G) {
    const int pk = perm[k];
    for (int i = tid; i < m; i += blockDim.x) {
      zd v = {0.0, 0.0};
      if (i < k) v = Y[i + (int64_t)pk * l];
      else if (i == k) v = {beta[k], 0.0};
      Rout[i + (int64_t)k * m] = v;
    }
  }
}

template <int MAXC>
static cudaError_t launch_qrp_bal_t(const QrArgs &a, int G, cudaStream_t st) {
  auto kern = qrp_bal_kernel<MAXC>;
  const size_t smem = sizeof(int) * (size_t)a.m;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  zd *Y = (zd *)a.Y;
  double *vnB = a.vn1 + a.m;  // the vn1 buffer holds 2m doubles
  int l = a.l, m = a.m;
  zd *R = (zd *)a.R;
  uint64_t lim = a.limit_ns;
  void *args[] = {&Y, &l, &m, (void *)&a.vn1, &vnB, (void *)&a.vn2, (void *)&a.beta, (void *)&a.piv,
                  &R, (void *)&a.bar, (void *)&a.err, &lim};
  note_launch();
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(kQrbThreads), args, smem, st);
}

cudaError_t launch_qrp(const QrArgs &a, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int G = a.m < kQrCtasPerSm * sms ? a.m : kQrCtasPerSm * sms;
  const int per = (a.m - 1 + G - 1) / G;  // most own columns at step 0
  note_launch();
  qr_norms_kernel<<<a.m, kQrThreads, 0, st>>>((const zd *)a.Y, a.l, a.vn1, a.vn2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (per <= 2) return launch_qrp_bal_t<2>(a, G, st);
  if (per <= 4) return launch_qrp_bal_t<4>(a, G, st);
  if (per <= 8) return launch_qrp_bal_t<8>(a, G, st);
  if (per <= 16) return launch_qrp_bal_t<16>(a, G, st);
  if (per <= 32) return launch_qrp_bal_t<32>(a, G, st);
  return cudaErrorInvalidValue;
}

// ---- P R^{-1} ---------------------------------------------------------------
// One CTA per column k of R^{-1}: back substitution R w = e_k, column-oriented
// (after w_j is final, subtract w_j R[0:j, j] from the entries above). Writes
// Wp = P R^{-1} (row piv[i] of Wp is row i of R^{-1}) and WpH = Wp^*, both
// row-major; the caller zeroes them first.
__global__ void __launch_bounds__(128)
prinv_kernel(const zd *__restrict__ R, const int32_t *__restrict__ piv, int m, zd *__restrict__ Wp,
             zd *__restrict__ WpH) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zd *w = reinterpret_cast<zd *>(smem_raw);
  zd *wout = w + m;
  const int k = m - 1 - blockIdx.x;  // longest columns first: they bound the kernel's duration
  for (int i = threadIdx.x; i <= k; i += blockDim.x) w[i] = {i == k ? 1.0 : 0.0, 0.0};
  for (int j = k; j >= 0; --j) {
    __syncthreads();
    const double rjj = R[j + (int64_t)j * m].re;  // real diagonal
    const zd wj = {w[j].re / rjj, w[j].im / rjj};
    if (threadIdx.x == 0) wout[j] = wj;
    const zd *rj = R + (int64_t)j * m;
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      zd v = w[i];
      const zd a = rj[i];
      v.re = fma(-a.re, wj.re, fma(a.im, wj.im, v.re));
      v.im = fma(-a.re, wj.im, fma(-a.im, wj.re, v.im));
      w[i] = v;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= k; i += blockDim.x) {
    const zd v = wout[i];
    const int pi = piv[i];
    Wp[(int64_t)pi * m + k] = v;
    WpH[(int64_t)k * m + pi] = conjg(v);
  }
}

cudaError_t launch_prinv(const void *R, const int32_t *piv, int m, void *Wp, void *WpH, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(Wp, 0, sizeof(zd) * (size_t)m * m, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(WpH, 0, sizeof(zd) * (size_t)m * m, st);
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(zd) * 2 * (size_t)m;
  e = cudaFuncSetAttribute(prinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  note_launch();
  prinv_kernel<<<m, 128, smem, st>>>((const zd *)R, piv, m, (zd *)Wp, (zd *)WpH);
  return cudaGetLastError();
}

}  // namespace mn
