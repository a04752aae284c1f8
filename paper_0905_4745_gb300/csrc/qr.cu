// qr.cu -- Step 2 of the algorithm (Eq. lineq): Householder QR with column
// pivoting of the sketch, Y P = Q R (the "classical pivoted QR based on
// Householder reflections" of Section 7, Golub & Van Loan ch. 5), then the
// preconditioner P R^{-1} used by Step 4.
//
// qrp_kernel is one cooperative grid (at most one CTA per SM). Column j of Y
// belongs to CTA j mod G and never moves: the pivot list records which
// physical column is the k-th. Per step k every CTA
//   1. picks the pivot p = argmax of the partial norms (first index on ties),
//   2. in one block reduction forms ||Y[k+1:, p]||^2 and, for each of its own
//      trailing columns j, sum_r conj(Y[r,p]) Y[r,j] (the reflector's scale is
//      not needed for these sums, so all CTAs build the same reflector
//      H = I - tau v v^*, v = (1, Y[k+1:, p] / (Y[k,p] - beta)), beta real,
//      without waiting for each other),
//   3. applies H^* to its own columns and downdates their partial norms (with
//      LAPACK's recomputation when the downdate loses half the digits),
//   4. meets the others at a grid barrier whose wait is bounded in time.
// Partial norms are double-buffered so a CTA still choosing step k's pivot
// never sees step k+1's values. The pivot column itself is left unscaled:
// only R and P are kept (Q is never needed: Steps 2-3 enter the solve through
// R alone, see solver.cu).
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

template <int MAXC>
__global__ void __launch_bounds__(kQrThreads)
qrp_kernel(zd *__restrict__ Y, int l, int m, double *__restrict__ vnA, double *__restrict__ vnB,
           double *__restrict__ vn2, double *__restrict__ beta, int32_t *__restrict__ piv,
           zd *__restrict__ Rout, GridBarrier *bar, int *err, uint64_t limit_ns) {
  constexpr int K = 1 + 2 * MAXC;
  __shared__ double red_scratch[(kQrThreads / 32) * K];
  __shared__ double red_out[K];
  __shared__ double s_val[kQrThreads / 32];
  __shared__ int s_idx[kQrThreads / 32];
  __shared__ int s_p;
  __shared__ int s_col[MAXC];
  __shared__ int s_nact;
  __shared__ zd s_g[MAXC];
  __shared__ int s_recompute[MAXC];
  __shared__ int s_nrec;
  __shared__ double s_beta;

  const int G = gridDim.x, b = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double tol3z = sqrt(0x1.0p-53);

  for (int k = 0; k < m; ++k) {
    double *vn_cur = (k & 1) ? vnB : vnA;
    double *vn_nxt = (k & 1) ? vnA : vnB;
    // 1. pivot
    double best = -2.0;
    int bi = 0x7fffffff;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const double v = vn_cur[j];
      if (v > best) { best = v; bi = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { s_val[wid] = best; s_idx[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bv = s_val[0];
      int bx = s_idx[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (s_val[w] > bv || (s_val[w] == bv && s_idx[w] < bx)) { bv = s_val[w]; bx = s_idx[w]; }
      s_p = bx;
      int na = 0;
      for (int j = b; j < m; j += G) {
        if (j != bx && vn_cur[j] >= 0.0) s_col[na++] = j;
        else vn_nxt[j] = -1.0;  // chosen now or earlier
      }
      s_nact = na;
      if (bx % G == b) { piv[k] = bx; }
    }
    __syncthreads();
    const int p = s_p;
    const int nact = s_nact;
    const zd *yp = Y + (int64_t)p * l;

    // 2. combined reduction: ||Y[k+1:,p]||^2 and conj(Y[k+1:,p])^T Y[k+1:,j]
    double part[K];
#pragma unroll
    for (int c = 0; c < K; ++c) part[c] = 0.0;
    for (int r = k + 1 + threadIdx.x; r < l; r += blockDim.x) {
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
    block_sum_k<double, K>(part, red_scratch, red_out);

    // 3. reflector (identical in every CTA) and the per-column factors
    if (threadIdx.x == 0) {
      const zd alpha = yp[k];
      const double xn2 = red_out[0];
      zd tau = {0.0, 0.0}, scale = {0.0, 0.0};
      double bt;
      if (xn2 == 0.0 && alpha.im == 0.0) {
        bt = alpha.re;
      } else {
        const double mag = sqrt(alpha.re * alpha.re + alpha.im * alpha.im + xn2);
        bt = alpha.re >= 0.0 ? -mag : mag;
        tau = {(bt - alpha.re) / bt, -alpha.im / bt};
        const double dr = alpha.re - bt, di = alpha.im;
        const double den = dr * dr + di * di;
        scale = {dr / den, -di / den};
      }
      s_beta = bt;
      if (p % G == b) beta[k] = bt;
      int nrec = 0;
      for (int c = 0; c < nact; ++c) {
        const int j = s_col[c];
        zd *yj = Y + (int64_t)j * l;
        const zd d = {red_out[1 + 2 * c], red_out[2 + 2 * c]};
        zd w = yj[k];
        macc(w, scale, d);                      // w = y_k + conj(scale) d
        const zd f = conjg(tau) * w;            // H^* = I - conj(tau) v v^*
        s_g[c] = f * scale;
        const zd rk = yj[k] - f;
        yj[k] = rk;
        // partial-norm downdate (LAPACK zlaqp2)
        const double v1 = vn_cur[j];
        double nv = v1;
        if (v1 != 0.0) {
          const double t = sqrt(abs2(rk)) / v1;
          double temp = 1.0 - t * t;
          temp = temp < 0.0 ? 0.0 : temp;
          const double ratio = v1 / vn2[j];
          if (temp * ratio * ratio <= tol3z) {
            s_recompute[nrec++] = c;
            nv = -2.0;  // filled below
          } else {
            nv = v1 * sqrt(temp);
          }
        }
        vn_nxt[j] = nv;
      }
      s_nrec = nrec;
    }
    __syncthreads();

    // 4. apply the reflector to the owned trailing columns, rows k+1..l-1
    for (int r = k + 1 + threadIdx.x; r < l; r += blockDim.x) {
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
    const int nrec = s_nrec;
    for (int q = 0; q < nrec; ++q) {           // rare: recompute a partial norm
      __syncthreads();
      const int c = s_recompute[q];
      const int j = s_col[c];
      double acc = 0.0;
      for (int r = k + 1 + threadIdx.x; r < l; r += blockDim.x) acc += abs2(Y[r + (int64_t)j * l]);
      const double t = sqrt(block_sum(acc, red_scratch));
      if (threadIdx.x == 0) {
        const double v = (k < l - 1) ? t : 0.0;
        vn_nxt[j] = v;
        vn2[j] = v;
      }
    }
    if (!grid_sync(bar, G, limit_ns)) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      return;
    }
  }

  // R in pivot order: R[i, k] = Y[i, piv[k]] above the diagonal, beta_k on it
  for (int k = b; k < m; k += G) {
    const int pk = piv[k];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      zd v = {0.0, 0.0};
      if (i < k) v = Y[i + (int64_t)pk * l];
      else if (i == k) v = {beta[k], 0.0};
      Rout[i + (int64_t)k * m] = v;
    }
  }
}

// ---- shared-memory variant ---------------------------------------------------
// Same algorithm, for sizes where every CTA's own columns fit in shared
// memory (ceil(m/G) + 1 columns of l entries). The columns never leave the
// SM until R is written. Each CTA publishes, at the end of a step, its own
// best remaining column (partial norm, index and rows k+1..l-1) in a
// double-buffered candidate slot; after the grid barrier every CTA takes the
// global maximum over the G candidates (first index on ties) and reads the
// winning rows from L2, so one barrier per step suffices.
constexpr int kQr2Threads = 512;

template <int MAXC>
__global__ void __launch_bounds__(kQr2Threads)
qrp_smem_kernel(const zd *__restrict__ Y, int l, int m, double *__restrict__ cand_val,
                int32_t *__restrict__ cand_col, zd *__restrict__ cand_data, double *__restrict__ beta,
                int32_t *__restrict__ piv, zd *__restrict__ Rout, GridBarrier *bar, int *err,
                uint64_t limit_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int K = 1 + 2 * MAXC;
  constexpr int NW = kQr2Threads / 32;
  __shared__ double red_scratch[NW * K];
  __shared__ double red_out[K];
  __shared__ double s_vn1[MAXC], s_vn2[MAXC], s_beta[MAXC];
  __shared__ int s_step[MAXC];
  __shared__ zd s_g[MAXC];
  __shared__ int s_rec[MAXC];
  __shared__ int s_nrec, s_w, s_p, s_cand;

  const int G = gridDim.x, b = blockIdx.x;
  const int nc = (m - b + G - 1) / G;  // own columns j = b + c G, c < nc
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  zd *cols = reinterpret_cast<zd *>(smem_raw);
  zd *pbuf = cols + (size_t)nc * l;
  const double tol3z = sqrt(0x1.0p-53);

  for (int c = 0; c < nc; ++c) {
    const zd *src = Y + (int64_t)(b + c * G) * l;
    for (int r = tid; r < l; r += blockDim.x) cols[(size_t)c * l + r] = src[r];
  }
  if (tid < MAXC) s_step[tid] = -1;
  __syncthreads();
  {
    double part[K];
#pragma unroll
    for (int c = 0; c < K; ++c) part[c] = 0.0;
    for (int r = tid; r < l; r += blockDim.x) {
#pragma unroll
      for (int c = 0; c < MAXC; ++c)
        if (c < nc) part[c] += abs2(cols[(size_t)c * l + r]);
    }
    block_sum_k<double, K>(part, red_scratch, red_out);
    if (tid < nc) { s_vn1[tid] = sqrt(red_out[tid]); s_vn2[tid] = s_vn1[tid]; }
    __syncthreads();
  }

  // publish this CTA's best remaining column (rows row0..l-1) into `slot`
  auto publish = [&](int slot, int row0) {
    if (tid == 0) {
      int best = -1;
      double bv = -1.0;
      for (int c = 0; c < nc; ++c)
        if (s_step[c] < 0 && s_vn1[c] > bv) { bv = s_vn1[c]; best = c; }
      s_cand = best;
      cand_val[slot * G + b] = best >= 0 ? bv : -1.0;
      cand_col[slot * G + b] = best >= 0 ? b + best * G : 0x7fffffff;
    }
    __syncthreads();
    const int c = s_cand;
    if (c >= 0) {
      zd *dst = cand_data + (size_t)(slot * G + b) * l;
      for (int r = row0 + tid; r < l; r += blockDim.x) dst[r] = cols[(size_t)c * l + r];
    }
  };

  publish(0, 0);
  if (!grid_sync(bar, G, limit_ns)) { if (tid == 0) atomicExch(err, 1); return; }

  for (int k = 0; k < m; ++k) {
    const int slot = k & 1;
    // 1. global pivot among the published candidates
    if (wid == 0) {
      double bv = -2.0;
      int bc = 0x7fffffff, bw = -1;
      for (int gi = lane; gi < G; gi += 32) {
        const double v = cand_val[slot * G + gi];
        const int cc = cand_col[slot * G + gi];
        if (v > bv || (v == bv && cc < bc)) { bv = v; bc = cc; bw = gi; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
        const int ow = __shfl_xor_sync(0xffffffffu, bw, o);
        if (ov > bv || (ov == bv && oc < bc)) { bv = ov; bc = oc; bw = ow; }
      }
      if (lane == 0) { s_w = bw; s_p = bc; }
    }
    __syncthreads();
    const int w = s_w, p = s_p;
    {
      const zd *src = cand_data + (size_t)(slot * G + w) * l;
      for (int r = k + tid; r < l; r += blockDim.x) pbuf[r] = src[r];
    }
    if (b == w && tid == 0) {
      const int c = (p - b) / G;
      s_step[c] = k;
      piv[k] = p;
    }
    __syncthreads();

    // 2. ||pbuf[k+1:]||^2 and conj(pbuf[k+1:])^T col_c[k+1:] in one reduction
    double part[K];
#pragma unroll
    for (int c = 0; c < K; ++c) part[c] = 0.0;
    for (int r = k + 1 + tid; r < l; r += blockDim.x) {
      const zd a = pbuf[r];
      part[0] = fma(a.re, a.re, fma(a.im, a.im, part[0]));
#pragma unroll
      for (int c = 0; c < MAXC; ++c) {
        if (c < nc && s_step[c] < 0) {
          const zd y = cols[(size_t)c * l + r];
          part[1 + 2 * c] = fma(a.re, y.re, fma(a.im, y.im, part[1 + 2 * c]));
          part[2 + 2 * c] = fma(a.re, y.im, fma(-a.im, y.re, part[2 + 2 * c]));
        }
      }
    }
    block_sum_k<double, K>(part, red_scratch, red_out);

    // 3. reflector and per-column factors (identical in every CTA)
    if (tid == 0) {
      const zd alpha = pbuf[k];
      const double xn2 = red_out[0];
      zd tau = {0.0, 0.0}, scale = {0.0, 0.0};
      double bt;
      if (xn2 == 0.0 && alpha.im == 0.0) {
        bt = alpha.re;
      } else {
        const double mag = sqrt(alpha.re * alpha.re + alpha.im * alpha.im + xn2);
        bt = alpha.re >= 0.0 ? -mag : mag;
        tau = {(bt - alpha.re) / bt, -alpha.im / bt};
        const double dr = alpha.re - bt, di = alpha.im;
        const double den = dr * dr + di * di;
        scale = {dr / den, -di / den};
      }
      if (b == w) {
        beta[k] = bt;
        s_beta[(p - b) / G] = bt;
      }
      int nrec = 0;
      for (int c = 0; c < nc; ++c) {
        if (s_step[c] >= 0) continue;
        const zd d = {red_out[1 + 2 * c], red_out[2 + 2 * c]};
        zd wv = cols[(size_t)c * l + k];
        macc(wv, scale, d);
        const zd f = conjg(tau) * wv;
        s_g[c] = f * scale;
        const zd rk = cols[(size_t)c * l + k] - f;
        cols[(size_t)c * l + k] = rk;
        const double v1 = s_vn1[c];
        if (v1 != 0.0) {
          const double t = sqrt(abs2(rk)) / v1;
          double temp = 1.0 - t * t;
          temp = temp < 0.0 ? 0.0 : temp;
          const double ratio = v1 / s_vn2[c];
          if (temp * ratio * ratio <= tol3z) s_rec[nrec++] = c;
          else s_vn1[c] = v1 * sqrt(temp);
        }
      }
      s_nrec = nrec;
    }
    __syncthreads();

    // 4. apply H^* to the own trailing columns
    for (int r = k + 1 + tid; r < l; r += blockDim.x) {
      const zd a = pbuf[r];
#pragma unroll
      for (int c = 0; c < MAXC; ++c) {
        if (c < nc && s_step[c] < 0) {
          zd v = cols[(size_t)c * l + r];
          const zd g = s_g[c];
          v.re = fma(-g.re, a.re, fma(g.im, a.im, v.re));
          v.im = fma(-g.re, a.im, fma(-g.im, a.re, v.im));
          cols[(size_t)c * l + r] = v;
        }
      }
    }
    __syncthreads();
    const int nrec = s_nrec;
    for (int q = 0; q < nrec; ++q) {
      const int c = s_rec[q];
      double acc = 0.0;
      for (int r = k + 1 + tid; r < l; r += blockDim.x) acc += abs2(cols[(size_t)c * l + r]);
      const double t = sqrt(block_sum(acc, red_scratch));
      if (tid == 0) {
        const double v = (k < l - 1) ? t : 0.0;
        s_vn1[c] = v;
        s_vn2[c] = v;
      }
      __syncthreads();
    }
    if (k + 1 < m) publish((k + 1) & 1, k + 1);
    if (!grid_sync(bar, G, limit_ns)) { if (tid == 0) atomicExch(err, 1); return; }
  }

  // R in pivot order, from the columns still in shared memory
  for (int c = 0; c < nc; ++c) {
    const int kc = s_step[c];
    const double bt = s_beta[c];
    for (int i = tid; i < m; i += blockDim.x) {
      zd v = {0.0, 0.0};
      if (i < kc) v = cols[(size_t)c * l + i];
      else if (i == kc) v = {bt, 0.0};
      Rout[i + (int64_t)kc * m] = v;
    }
  }
}

template <int MAXC>
static cudaError_t launch_qrp_smem_t(const QrArgs &a, int G, size_t smem, cudaStream_t st) {
  auto kern = qrp_smem_kernel<MAXC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const zd *Y = (const zd *)a.Y;
  int l = a.l, m = a.m;
  zd *R = (zd *)a.R;
  zd *cd = (zd *)a.cand_data;
  uint64_t lim = a.limit_ns;
  void *args[] = {(void *)&Y, &l, &m, (void *)&a.cand_val, (void *)&a.cand_col, &cd, (void *)&a.beta,
                  (void *)&a.piv, &R, (void *)&a.bar, (void *)&a.err, &lim};
  note_launch();
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(kQr2Threads), args, smem, st);
}

size_t qrp_smem_bytes(int l, int m, int sms) {
  const int G = m < sms ? m : sms;
  const int per = (m + G - 1) / G;
  return sizeof(zd) * (size_t)(per + 1) * l;
}

template <int MAXC>
static cudaError_t launch_qrp_t(const QrArgs &a, int G, cudaStream_t st) {
  auto kern = qrp_kernel<MAXC>;
  zd *Y = (zd *)a.Y;
  double *vnB = a.vn1 + a.m;  // second half of the vn1 buffer (2m doubles)
  int l = a.l, m = a.m;
  zd *R = (zd *)a.R;
  uint64_t lim = a.limit_ns;
  void *args[] = {&Y, &l, &m, (void *)&a.vn1, &vnB, (void *)&a.vn2, (void *)&a.beta, (void *)&a.piv,
                  &R, (void *)&a.bar, (void *)&a.err, &lim};
  note_launch();
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3(kQrThreads), args, 0, st);
}

cudaError_t launch_qrp(const QrArgs &a, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int G = a.m < sms ? a.m : sms;
  const int per = (a.m + G - 1) / G;
  const size_t smem = qrp_smem_bytes(a.l, a.m, sms);
  if (a.cand_data && per <= 8 && smem <= kQrSmemLimit) {
    if (per <= 2) return launch_qrp_smem_t<2>(a, G, smem, st);
    if (per <= 4) return launch_qrp_smem_t<4>(a, G, smem, st);
    return launch_qrp_smem_t<8>(a, G, smem, st);
  }
  note_launch();
  qr_norms_kernel<<<a.m, kQrThreads, 0, st>>>((const zd *)a.Y, a.l, a.vn1, a.vn2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (per <= 4) return launch_qrp_t<4>(a, G, st);
  if (per <= 8) return launch_qrp_t<8>(a, G, st);
  if (per <= 16) return launch_qrp_t<16>(a, G, st);
  if (per <= 32) return launch_qrp_t<32>(a, G, st);
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
  const int k = blockIdx.x;
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
