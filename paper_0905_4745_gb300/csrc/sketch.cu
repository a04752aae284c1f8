// sketch.cu -- Step 1 of the algorithm (Eq. randmat): Y = T A^*, column i of Y
// being T applied to the conjugated row i of A, with
//   T = S F D Theta Pi Z Theta~ Pi~ Z~        (Eqs. SRFT, SRFT2, Rokhlin_trans)
// applied right to left. Per row the work is split into three stages:
//
//   chain_kernel (twice)  gather through a permutation, multiply by a unit
//                         phase, run a Givens chain (Eq. big_def), optionally
//                         multiply by D; one CTA per (row, 2048-element segment)
//   fft kernels           the unitary DFT F of Eq. (DFT) by radix-2 FFTs in
//                         shared memory (one pass for n <= 4096/8192, otherwise
//                         the four-step factorisation n = N1 N2), with the row
//                         sample S applied while storing into Y. A length n
//                         that is not a power of two takes Bluestein's chirp
//                         convolution: two FFTs of length L >= 2n - 1, the
//                         first with the chirp applied on load and conj(X bh)
//                         stored in full, the second sampled with the chirp and
//                         1/sqrt(n) folded into a per-row factor
//
// The chain Theta = G_0 G_1 ... G_{n-2} (G_{n-2} acting first) is the reverse
// affine recurrence
//     C_{n-1} = v_{n-1},   C_k = cos(t_k) v_k + sin(t_k) C_{k+1},
//     out_{k+1} = -sin(t_k) v_k + cos(t_k) C_{k+1},   out_0 = C_0,
// with real coefficients. Inside a CTA it is evaluated exactly as a parallel
// scan of the affine maps C -> s C + c v. Segments are independent: a segment
// is extended to the right by a precomputed halo over which the product of
// |sin t_k| falls below 2^-72 / sqrt(n) (FP64) or 2^-60 / sqrt(n) (double-word),
// so starting the recurrence at the halo's end with a zero carry changes the
// segment's outputs by less than that fraction of the row norm.
//
// Every kernel is instantiated for complex FP64 and for complex double-word
// arithmetic (dw.cuh: pairs of floats on the FP32 pipe, ~2^-46 per operation),
// the sketch of the mixed-precision path.
#include "common.cuh"
#include "dw.cuh"
#include "kernels.h"

namespace mn {

constexpr int kChainThreads = 256;

// Reverse (right-to-left) inclusive scan of affine maps x -> P x + Q across the
// block; returns for each thread the carry entering its chunk from the right,
// i.e. the composition of all maps to its right applied to 0.
template <typename R>
__device__ __forceinline__ cx<R> block_reverse_carry(R P, cx<R> Q, R *sP, cx<R> *sQ) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const R P2 = __shfl_down_sync(0xffffffffu, P, off);
    const R Q2r = __shfl_down_sync(0xffffffffu, Q.re, off);
    const R Q2i = __shfl_down_sync(0xffffffffu, Q.im, off);
    if (lane + off < 32) {
      Q.re = fma(P, Q2r, Q.re);
      Q.im = fma(P, Q2i, Q.im);
      P = P * P2;
    }
  }
  // lane holds F_lane o ... o F_31 (within the warp)
  if (lane == 0) { sP[wid] = P; sQ[wid] = Q; }
  __syncthreads();
  if (threadIdx.x == 0) {
    cx<R> c = {R(0), R(0)};
    for (int w = nw - 1; w >= 0; --w) {
      const cx<R> q = sQ[w];
      const R p = sP[w];
      sQ[w] = c;  // carry entering warp w from the right
      c = {fma(p, c.re, q.re), fma(p, c.im, q.im)};
    }
  }
  __syncthreads();
  const cx<R> wc = sQ[wid];
  const R Pn = __shfl_down_sync(0xffffffffu, P, 1);
  const R Qnr = __shfl_down_sync(0xffffffffu, Q.re, 1);
  const R Qni = __shfl_down_sync(0xffffffffu, Q.im, 1);
  cx<R> carry;
  if (lane == 31) {
    carry = wc;
  } else {
    carry = {fma(Pn, wc.re, Qnr), fma(Pn, wc.im, Qni)};
  }
  __syncthreads();  // sP/sQ may be reused by the caller
  return carry;
}

// One Givens-chain stage for rows [row0, row0 + gridDim.y):
//   v_j = phase[j] * (conj?) src[row, idx[j]]           (gather Pi and phase Z)
//   out = Theta v                                          (chain of Eq. big_def)
//   dst[row, j] = (post ? post[j] : 1) * out_j
template <typename R, typename S, bool CONJ, bool POST>
__global__ void __launch_bounds__(kChainThreads, 3)
chain_kernel(const S *__restrict__ src, int64_t ld_src, cx<R> *__restrict__ dst, int64_t ld_dst,
             const int32_t *__restrict__ idx, const cx<R> *__restrict__ phase,
             const cx<R> *__restrict__ cs, const cx<R> *__restrict__ post,
             const int32_t *__restrict__ halo, int n, int seg, int cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // V holds the gathered inputs, then (second scan pass, in place) the outputs: output o of the
  // segment at V[o - off], off = 1 for the first segment (whose out_0 is kept in s_out0)
  cx<R> *V = reinterpret_cast<cx<R> *>(smem_raw);
  cx<R> *CS = V + cap;
  __shared__ R sP[kChainThreads / 32];
  __shared__ cx<R> sQ[kChainThreads / 32];
  __shared__ cx<R> s_out0;

  const int g = blockIdx.x;
  const int64_t row = blockIdx.y;
  const int j0 = g * seg;
  const int len = min(seg, n - j0);
  const int lo = j0 > 0 ? j0 - 1 : 0;
  const int E = j0 + len + halo[g];
  const int cnt = E - lo;
  const S *srow = src + row * ld_src;

  // the gather is latency-bound: issue the index loads, then the gathered loads, of several
  // elements per thread before using any of them
  // (the phase and rotation loads do not depend on the gather: they go with the index loads)
  constexpr int kG = 4;
  for (int t0 = threadIdx.x; t0 < cnt; t0 += kG * blockDim.x) {
    int ix[kG];
    cx<R> ph[kG], rc[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      const int t = t0 + g * blockDim.x;
      const int j = lo + (t < cnt ? t : 0);
      ix[g] = idx[j];
      ph[g] = phase[j];
      rc[g] = cs[j];
    }
    S a[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) a[g] = srow[ix[g]];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      const int t = t0 + g * blockDim.x;
      if (t < cnt) {
        const cx<R> v = {R(a[g].re), CONJ ? -R(a[g].im) : R(a[g].im)};
        V[t] = v * ph[g];
        CS[t] = rc[g];
      }
    }
  }
  __syncthreads();

  const int per = (cnt + blockDim.x - 1) / blockDim.x;
  const int a0 = min(threadIdx.x * per, cnt);
  const int a1 = min(a0 + per, cnt);
  R P = R(1);
  cx<R> Q = {R(0), R(0)};
  for (int t = a1 - 1; t >= a0; --t) {
    const cx<R> c = CS[t];  // (cos, sin)
    const cx<R> v = V[t];
    Q = {fma(c.im, Q.re, c.re * v.re), fma(c.im, Q.im, c.re * v.im)};
    P *= c.im;
  }
  cx<R> C = block_reverse_carry<R>(P, Q, sP, sQ);
  const int off = lo + 1 - j0;  // 1 for the first segment, else 0
  for (int t = a1 - 1; t >= a0; --t) {
    const cx<R> c = CS[t];
    const cx<R> v = V[t];
    // element k = lo + t; C holds C_{k+1}; output o = k + 1 - j0 = t + off goes to V[t] (this
    // thread has just read V[t]; no other thread touches its run of V in this pass)
    if (t < len - off) V[t] = {fma(c.re, C.re, -c.im * v.re), fma(c.re, C.im, -c.im * v.im)};
    C = {fma(c.im, C.re, c.re * v.re), fma(c.im, C.im, c.re * v.im)};
  }
  if (j0 == 0 && a0 == 0 && a1 > a0) s_out0 = C;  // out_0 = C_0
  __syncthreads();

  cx<R> *drow = dst + row * ld_dst;
  for (int t = threadIdx.x; t < len; t += blockDim.x) {
    cx<R> o = (off == 1 && t == 0) ? s_out0 : V[t - off];
    if (POST) o = o * post[j0 + t];
    drow[j0 + t] = o;
  }
}

// ---- FFT ----------------------------------------------------------------
__device__ __forceinline__ int bitrev(int j, int logL) {
  return logL == 0 ? 0 : (int)(__brev((unsigned)j) >> (32 - logL));
}

// The twiddles of every butterfly stage, stage by stage: stw[h + k] = e^{-2 pi i k / (2h)} for
// h = 1, 2, 4, ..., L/2 and k < h (L entries, stw[0] unused), copied from the table tw (NT
// entries, e^{-2 pi i j / NT}, L divides NT) into shared memory. A stage's twiddles are then
// consecutive words (a warp's reads are conflict-free), and each is the table entry of the
// plain layout, so the transform is unchanged.
template <typename R>
__device__ __forceinline__ void load_twiddles(cx<R> *stw, int logL, const cx<R> *__restrict__ tw, int logNT) {
  for (int idx = threadIdx.x + 1; idx < (1 << logL); idx += blockDim.x) {
    const int lh = 31 - __clz(idx);
    const int k = idx - (1 << lh);
    stw[idx] = tw[(int64_t)k << (logNT - lh - 1)];
  }
}

// In-place radix-2 DIT FFT (forward, e^{-2 pi i jk/L}) of B sequences of length
// L = 2^logL, `stride` elements apart, stored in bit-reversed order; twiddles
// from stw (see load_twiddles).
template <typename R>
__device__ __forceinline__ void smem_fft(cx<R> *data, int B, int logL, int stride, const cx<R> *stw) {
  const int L = 1 << logL;
  const int halfL = L >> 1;
  const int total = B * halfL;
  for (int lh = 0; lh < logL; ++lh) {
    const int h = 1 << lh;
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
      const int seqi = b >> (logL - 1);
      const int bb = b & (halfL - 1);
      const int k = bb & (h - 1);
      const int pos = ((bb >> lh) << (lh + 1)) + k;
      cx<R> *d = data + seqi * stride;
      const cx<R> w = stw[h + k];
      const cx<R> u = d[pos];
      const cx<R> v = d[pos + h] * w;
      d[pos] = u + v;
      d[pos + h] = u - v;
    }
    __syncthreads();
  }
}

// input element j of a row: plain, or (Bluestein) x_j c_j zero-padded past nin
template <typename R>
__device__ __forceinline__ cx<R> fft_in(const cx<R> *__restrict__ s, int64_t j, const cx<R> *__restrict__ chirp,
                                        int nin) {
  if (!chirp) return s[j];
  return j < nin ? s[j] * chirp[j] : cx<R>{R(0), R(0)};
}

// sampled output t: X / sqrt(L), or (Bluestein) conj(X) * fac[t]
template <typename R>
__device__ __forceinline__ zd fft_out(cx<R> v, int t, const double *__restrict__ fac, double scale) {
  if (!fac) return {double(v.re) * scale, double(v.im) * scale};
  const double fr = fac[2 * t], fi = fac[2 * t + 1];
  const double vr = double(v.re), vi = -double(v.im);
  return {vr * fr - vi * fi, vr * fi + vi * fr};
}

// Whole-row FFT (L <= smem capacity) + sample: Y[t, row] = X[s_t] / sqrt(L),
// or the Bluestein stages (see FftArgs).
template <typename R>
__global__ void __launch_bounds__(256)
fft_row_kernel(const cx<R> *__restrict__ src, int64_t ld_src, int logn, const cx<R> *__restrict__ tw,
               const int32_t *__restrict__ samp_t, const int32_t *__restrict__ samp_loc, int l,
               zd *__restrict__ Y, int64_t ldy, int row_offset, double scale, const cx<R> *__restrict__ chirp,
               int nin, cx<R> *__restrict__ full, const cx<R> *__restrict__ bh, int64_t ldf,
               const double *__restrict__ fac) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R> *data = reinterpret_cast<cx<R> *>(smem_raw);
  const int n = 1 << logn;
  cx<R> *stw = data + n;  // n twiddle slots (stage by stage)
  const int64_t row = blockIdx.y;
  const cx<R> *s = src + row * ld_src;
  load_twiddles<R>(stw, logn, tw, logn);
  for (int j0 = threadIdx.x; j0 < n; j0 += 8 * blockDim.x) {  // eight loads in flight per thread
    cx<R> v[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int j = j0 + g * blockDim.x;
      v[g] = j < n ? fft_in(s, j, chirp, nin) : cx<R>{R(0), R(0)};
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int j = j0 + g * blockDim.x;
      if (j < n) data[bitrev(j, logn)] = v[g];
    }
  }
  __syncthreads();
  smem_fft<R>(data, 1, logn, n, stw);
  if (full) {
    cx<R> *f = full + row * ldf;
    for (int k = threadIdx.x; k < n; k += blockDim.x) f[k] = conjg(data[k] * bh[k]);
    return;
  }
  zd *y = Y + (row + row_offset) * ldy;
  for (int e = threadIdx.x; e < l; e += blockDim.x) {
    const int t = samp_t[e];
    y[t] = fft_out(data[samp_loc[e]], t, fac, scale);
  }
}

// Four-step pass A: for each j1 in this CTA's tile, the length-N2 FFT over j2 of
// v[j1 + N1 j2], times e^{-2 pi i j1 k2 / n}, stored at W[k2 N1 + j1].
template <typename R>
__global__ void __launch_bounds__(256)
fft_pass_a_kernel(const cx<R> *__restrict__ src, int64_t ld, cx<R> *__restrict__ W, int64_t ldw, int logn,
                  int logN1, int tj, const cx<R> *__restrict__ tw, const cx<R> *__restrict__ chirp, int nin) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R> *data = reinterpret_cast<cx<R> *>(smem_raw);
  const int n = 1 << logn, N1 = 1 << logN1, logN2 = logn - logN1, N2 = 1 << logN2;
  const int j1_0 = blockIdx.x * tj;
  const int64_t row = blockIdx.y;
  const cx<R> *s = src + row * ld;
  const int total = tj * N2;
  cx<R> *stw = data + tj * (N2 + 1);  // N2 twiddle slots (stage by stage)
  load_twiddles<R>(stw, logN2, tw, logn);
  for (int e0 = threadIdx.x; e0 < total; e0 += 8 * blockDim.x) {  // eight loads in flight per thread
    cx<R> v[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int e = e0 + g * blockDim.x;
      const int jj = e % tj, j2 = e / tj;
      v[g] = e < total ? fft_in(s, (j1_0 + jj) + (int64_t)N1 * j2, chirp, nin) : cx<R>{R(0), R(0)};
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int e = e0 + g * blockDim.x;
      if (e < total) data[(e % tj) * (N2 + 1) + bitrev(e / tj, logN2)] = v[g];
    }
  }
  __syncthreads();
  smem_fft<R>(data, tj, logN2, N2 + 1, stw);
  cx<R> *w = W + row * ldw;
  for (int e0 = threadIdx.x; e0 < total; e0 += 8 * blockDim.x) {
    cx<R> t8[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int e = e0 + g * blockDim.x;
      const int jj = e % tj, k2 = e / tj;
      t8[g] = e < total ? tw[((int64_t)(j1_0 + jj) * k2) & (n - 1)] : cx<R>{R(0), R(0)};
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int e = e0 + g * blockDim.x;
      if (e < total) {
        const int jj = e % tj, k2 = e / tj;
        w[(int64_t)k2 * N1 + j1_0 + jj] = data[jj * (N2 + 1) + k2] * t8[g];
      }
    }
  }
}

// Four-step pass B: for each k2 in the tile, the length-N1 FFT over j1 of
// W[k2 N1 + j1] gives X[N2 k1 + k2]; the sampled ones go to Y.
template <typename R>
__global__ void __launch_bounds__(256)
fft_pass_b_kernel(const cx<R> *__restrict__ W, int64_t ldw, int logn, int logN1, int tk,
                  const cx<R> *__restrict__ tw, const int32_t *__restrict__ samp_off,
                  const int32_t *__restrict__ samp_t, const int32_t *__restrict__ samp_loc,
                  zd *__restrict__ Y, int64_t ldy, int row_offset, double scale, cx<R> *__restrict__ full,
                  const cx<R> *__restrict__ bh, int64_t ldf, const double *__restrict__ fac) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R> *data = reinterpret_cast<cx<R> *>(smem_raw);
  const int N1 = 1 << logN1;
  const int k2_0 = blockIdx.x * tk;
  const int64_t row = blockIdx.y;
  const cx<R> *w = W + row * ldw + (int64_t)k2_0 * N1;
  const int total = tk * N1;
  cx<R> *stw = data + tk * (N1 + 1);  // N1 twiddle slots (stage by stage)
  load_twiddles<R>(stw, logN1, tw, logn);
  for (int e0 = threadIdx.x; e0 < total; e0 += 8 * blockDim.x) {  // eight loads in flight per thread
    cx<R> v[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int e = e0 + g * blockDim.x;
      v[g] = e < total ? w[e] : cx<R>{R(0), R(0)};
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int e = e0 + g * blockDim.x;
      if (e < total) data[(e >> logN1) * (N1 + 1) + bitrev(e & (N1 - 1), logN1)] = v[g];
    }
  }
  __syncthreads();
  smem_fft<R>(data, tk, logN1, N1 + 1, stw);
  if (full) {
    // X[N2 k1 + k2] for k2 = k2_0 + kk sits at data[kk (N1 + 1) + k1]; runs of tk consecutive outputs
    const int N2 = 1 << (logn - logN1);
    cx<R> *f = full + row * ldf;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int k1 = e / tk, kk = e - k1 * tk;
      const int64_t K = (int64_t)N2 * k1 + k2_0 + kk;
      f[K] = conjg(data[kk * (N1 + 1) + k1] * bh[K]);
    }
    return;
  }
  zd *y = Y + (row + row_offset) * ldy;
  const int b0 = samp_off[blockIdx.x], b1 = samp_off[blockIdx.x + 1];
  for (int e = b0 + threadIdx.x; e < b1; e += blockDim.x) {
    const int t = samp_t[e];
    y[t] = fft_out(data[samp_loc[e]], t, fac, scale);
  }
}

__global__ void to_c64_kernel(const zd *__restrict__ A, int64_t lda, zf *__restrict__ B, int64_t ldb,
                              int64_t cols) {
  const int64_t i = blockIdx.y;
  const zd *a = A + i * lda;
  zf *b = B + i * ldb;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols; j += (int64_t)gridDim.x * blockDim.x) {
    const zd v = a[j];
    b[j] = {float(v.re), float(v.im)};
  }
}

__global__ void widen_kernel(int64_t len, const zf *__restrict__ src, zd *__restrict__ dst) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < len; j += (int64_t)gridDim.x * blockDim.x) {
    const zf v = src[j];
    dst[j] = {double(v.re), double(v.im)};
  }
}

// ---- host launchers -----------------------------------------------------
template <typename R, typename S, bool CONJ, bool POST>
static cudaError_t launch_chain_t(const ChainArgs &a, cudaStream_t st) {
  const size_t smem = sizeof(cx<R>) * (size_t)(2 * a.cap);
  cudaError_t e = cudaFuncSetAttribute(chain_kernel<R, S, CONJ, POST>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nseg = (a.n + a.seg - 1) / a.seg;
  dim3 grid(nseg, a.rows);
  note_launch();
  chain_kernel<R, S, CONJ, POST><<<grid, kChainThreads, smem, st>>>(
      (const S *)a.src, a.ld_src, (cx<R> *)a.dst, a.ld_dst, a.idx, (const cx<R> *)a.phase,
      (const cx<R> *)a.cs, (const cx<R> *)a.post, a.halo, a.n, a.seg, a.cap);
  return cudaGetLastError();
}

cudaError_t launch_chain(const ChainArgs &a, cudaStream_t st) {
  // arithmetic: complex FP64 or complex double-word; sources: complex128, complex64, or the
  // previous chain's double-word output
  if (a.arith == kArithDW) {
    if (a.src_kind == kSrcDW) {
      if (a.conj) return a.post ? launch_chain_t<df, zw, true, true>(a, st) : launch_chain_t<df, zw, true, false>(a, st);
      return a.post ? launch_chain_t<df, zw, false, true>(a, st) : launch_chain_t<df, zw, false, false>(a, st);
    }
    if (a.src_kind == kSrcC64) {
      if (a.conj) return a.post ? launch_chain_t<df, zf, true, true>(a, st) : launch_chain_t<df, zf, true, false>(a, st);
      return a.post ? launch_chain_t<df, zf, false, true>(a, st) : launch_chain_t<df, zf, false, false>(a, st);
    }
    if (a.conj) return a.post ? launch_chain_t<df, zd, true, true>(a, st) : launch_chain_t<df, zd, true, false>(a, st);
    return a.post ? launch_chain_t<df, zd, false, true>(a, st) : launch_chain_t<df, zd, false, false>(a, st);
  }
  if (a.arith != kArithF64 || a.src_kind == kSrcDW) return cudaErrorInvalidValue;
  if (a.src_kind == kSrcC64) {
    if (a.conj) return a.post ? launch_chain_t<double, zf, true, true>(a, st) : launch_chain_t<double, zf, true, false>(a, st);
    return a.post ? launch_chain_t<double, zf, false, true>(a, st) : launch_chain_t<double, zf, false, false>(a, st);
  }
  if (a.conj) return a.post ? launch_chain_t<double, zd, true, true>(a, st) : launch_chain_t<double, zd, true, false>(a, st);
  return a.post ? launch_chain_t<double, zd, false, true>(a, st) : launch_chain_t<double, zd, false, false>(a, st);
}

template <typename R>
static cudaError_t launch_fft_t(const FftArgs &a, cudaStream_t st) {
  const double scale = 1.0 / sqrt((double)(1LL << a.logn));
  cudaError_t e;
  if (a.logN1 == 0) {
    const size_t smem = (sizeof(cx<R>) << a.logn) * 2;  // data + twiddles
    e = cudaFuncSetAttribute(fft_row_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    note_launch();
    fft_row_kernel<R><<<dim3(1, a.rows), 256, smem, st>>>(
        (const cx<R> *)a.src, a.ld, a.logn, (const cx<R> *)a.tw, a.samp_t, a.samp_loc, a.l, (zd *)a.Y,
        a.ldy, a.row_offset, scale, (const cx<R> *)a.chirp, a.nin, (cx<R> *)a.full, (const cx<R> *)a.bh, a.ldf,
        a.fac);
    return cudaGetLastError();
  }
  const int N1 = 1 << a.logN1, N2 = 1 << (a.logn - a.logN1);
  // sequences padded by one element: the strided transposes into and out of shared memory
  // then touch distinct banks
  const size_t smemA = sizeof(cx<R>) * ((size_t)a.tj * (N2 + 1) + N2);
  const size_t smemB = sizeof(cx<R>) * ((size_t)a.tk * (N1 + 1) + N1);
  e = cudaFuncSetAttribute(fft_pass_a_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemA);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fft_pass_b_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemB);
  if (e != cudaSuccess) return e;
  note_launch();
  fft_pass_a_kernel<R><<<dim3(N1 / a.tj, a.rows), 256, smemA, st>>>(
      (const cx<R> *)a.src, a.ld, (cx<R> *)a.work, a.ldw, a.logn, a.logN1, a.tj, (const cx<R> *)a.tw,
      (const cx<R> *)a.chirp, a.nin);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launch();
  fft_pass_b_kernel<R><<<dim3(N2 / a.tk, a.rows), 256, smemB, st>>>(
      (const cx<R> *)a.work, a.ldw, a.logn, a.logN1, a.tk, (const cx<R> *)a.tw, a.samp_off, a.samp_t,
      a.samp_loc, (zd *)a.Y, a.ldy, a.row_offset, scale, (cx<R> *)a.full, (const cx<R> *)a.bh, a.ldf, a.fac);
  return cudaGetLastError();
}

cudaError_t launch_fft(const FftArgs &a, cudaStream_t st) {
  if (a.arith == kArithDW) return launch_fft_t<df>(a, st);
  if (a.arith == kArithF64) return launch_fft_t<double>(a, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_to_c64(const void *A, int64_t lda, void *B, int64_t ldb, int64_t rows, int64_t cols,
                          cudaStream_t st) {
  int64_t bx = (cols + 255) / 256;
  if (bx > 64) bx = 64;
  note_launch();
  to_c64_kernel<<<dim3((unsigned)bx, (unsigned)rows), 256, 0, st>>>((const zd *)A, lda, (zf *)B, ldb, cols);
  return cudaGetLastError();
}

cudaError_t launch_narrow(int64_t len, const void *src, void *dst, cudaStream_t st) {
  return launch_to_c64(src, len, dst, len, 1, len, st);
}

cudaError_t launch_widen(int64_t len, const void *src, void *dst, cudaStream_t st) {
  int64_t b = (len + 255) / 256;
  if (b > 1024) b = 1024;
  note_launch();
  widen_kernel<<<(unsigned)b, 256, 0, st>>>(len, (const zf *)src, (zd *)dst);
  return cudaGetLastError();
}

}  // namespace mn
