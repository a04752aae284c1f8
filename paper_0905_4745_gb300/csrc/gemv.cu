// gemv.cu -- the passes over A of Step 4 (one A^* w and one A q per CG
// iteration, Eq. overdet), of Step 5 (x = A^* y, Eq. output) and of the
// refinement residuals, for a row-major A (row i contiguous).
//
//   adjoint  out[j] = sum_i conj(A[i,j]) v[i]: a CTA owns 512 consecutive
//            columns and streams a range of rows, each row segment read as
//            one contiguous 4 or 8 KiB span; row ranges are split across CTAs
//            (adj_split) so that the grid covers the GPU, and a second kernel
//            adds the splits (also forming ||out||^2 per CTA).
//   forward  out[i] = sum_j A[i,j] v[j]: a CTA owns kFwdRows rows and a
//            column chunk; each thread keeps one accumulator per row, so the
//            chunk of v is read once per CTA; chunk partials are added by a
//            second kernel in FP64. Complex64 rows are read two entries per
//            16-byte load when the layout allows it (even ld and column count,
//            16-byte aligned A and v), and the chunks are sized for about 12
//            CTAs per SM: at 2048 x 262144 this reads A at 7.3 TB/s, against
//            3.9 TB/s with 16 rows per CTA, 8-byte loads and 3 CTAs per SM.
//   (the refinement's accurate products are in xprod.cu)
//
// Modes: 0 = complex128 A, FP64 arithmetic; 1 = complex64 A, FP32 arithmetic
// (mixed precision); 2 = complex64 A, FP64 arithmetic.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace mn {

constexpr int kAdjThreads = 256;
constexpr int kAdjVpt = 2;                       // columns per thread
constexpr int kAdjCols = kAdjThreads * kAdjVpt;  // columns per CTA
constexpr int kFwdThreads = 256;
constexpr int kFwdRows = 8;

template <typename T> struct ComputeOf;
template <> struct ComputeOf<zd> { using R = double; };
template <> struct ComputeOf<zf> { using R = float; };

// ---- adjoint ------------------------------------------------------------
template <typename T, typename R>
__global__ void __launch_bounds__(kAdjThreads)
adj_kernel(const T *__restrict__ A, int64_t rows, int64_t cols, int64_t ld, const cx<R> *__restrict__ v,
           cx<R> *__restrict__ out, int split, const int *__restrict__ skip) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R> *sv = reinterpret_cast<cx<R> *>(smem_raw);
  if (skip && *skip) return;
  const int s = blockIdx.y;
  const int64_t r0 = rows * s / split, r1 = rows * (s + 1) / split;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) sv[i - r0] = v[i];
  __syncthreads();
  const int64_t c = (int64_t)blockIdx.x * kAdjCols + (int64_t)threadIdx.x * kAdjVpt;
  cx<R> acc[kAdjVpt];
#pragma unroll
  for (int q = 0; q < kAdjVpt; ++q) acc[q] = {R(0), R(0)};
  if (c + kAdjVpt <= cols) {
    const T *a = A + r0 * ld + c;
    int64_t i = r0;
    for (; i + 4 <= r1; i += 4) {
      T x[4][kAdjVpt];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < kAdjVpt; ++q) x[u][q] = a[u * ld + q];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const cx<R> w = sv[i - r0 + u];
#pragma unroll
        for (int q = 0; q < kAdjVpt; ++q) macc(acc[q], cvt<R>(x[u][q]), w);
      }
      a += 4 * ld;
    }
    for (; i < r1; ++i) {
      const cx<R> w = sv[i - r0];
#pragma unroll
      for (int q = 0; q < kAdjVpt; ++q) macc(acc[q], cvt<R>(a[q]), w);
      a += ld;
    }
  } else {
    for (int64_t i = r0; i < r1; ++i) {
      const cx<R> w = sv[i - r0];
#pragma unroll
      for (int q = 0; q < kAdjVpt; ++q)
        if (c + q < cols) macc(acc[q], cvt<R>(A[i * ld + c + q]), w);
    }
  }
  cx<R> *o = out + (int64_t)s * cols;
#pragma unroll
  for (int q = 0; q < kAdjVpt; ++q)
    if (c + q < cols) o[c + q] = acc[q];
}

// out[j] = sum_s partial[s][j] (in FP64), written as OutT; qq[block] = sum |out|^2
template <typename R, typename OutT>
__global__ void __launch_bounds__(256)
adj_reduce_kernel(const cx<R> *__restrict__ partial, int split, int64_t cols, OutT *__restrict__ out,
                  double *__restrict__ qq, const int *__restrict__ skip) {
  __shared__ double sc[8];
  if (skip && *skip) return;
  double loc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols; j += (int64_t)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int s = 0; s < split; ++s) {
      const cx<R> p = partial[(int64_t)s * cols + j];
      re += (double)p.re;
      im += (double)p.im;
    }
    OutT o;
    o.re = re;
    o.im = im;
    out[j] = o;
    const double ore = (double)o.re, oim = (double)o.im;
    loc = fma(ore, ore, fma(oim, oim, loc));
  }
  const double t = block_sum(loc, sc);
  if (qq && threadIdx.x == 0) qq[blockIdx.x] = t;
}

// ---- forward ------------------------------------------------------------
// PAIR: complex64 A read two entries per 16-byte load (c0 and the chunk even; v likewise when
// it is complex64)
template <typename T, typename R, int ROWS, bool PAIR>
__global__ void __launch_bounds__(kFwdThreads)
fwd_kernel(const T *__restrict__ A, int64_t rows, int64_t cols, int64_t ld, const cx<R> *__restrict__ v,
           int64_t chunk, cx<R> *__restrict__ partial, const int *__restrict__ skip) {
  __shared__ R scratch[(kFwdThreads / 32) * 2 * ROWS];
  __shared__ R red[2 * ROWS];
  if (skip && *skip) return;
  const int64_t i0 = (int64_t)blockIdx.y * ROWS;
  const int64_t c0 = (int64_t)blockIdx.x * chunk;
  const int64_t c1 = c0 + chunk < cols ? c0 + chunk : cols;
  R acc[2 * ROWS];
#pragma unroll
  for (int r = 0; r < 2 * ROWS; ++r) acc[r] = R(0);
  if constexpr (PAIR) {
    for (int64_t c = c0 + 2 * threadIdx.x; c < c1; c += 2 * kFwdThreads) {
      cx<R> x0, x1;   // v[c], v[c + 1]
      if constexpr (std::is_same<R, float>::value) {
        const float4 t = *reinterpret_cast<const float4 *>(v + c);
        x0 = {t.x, t.y};
        x1 = {t.z, t.w};
      } else {
        x0 = v[c];
        x1 = v[c + 1];
      }
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        if (i0 + r < rows) {
          const float4 a = __ldcs(reinterpret_cast<const float4 *>(A + (i0 + r) * ld + c));
          R re = acc[2 * r], im = acc[2 * r + 1];
          re = fma((R)a.x, x0.re, fma(-(R)a.y, x0.im, re));
          im = fma((R)a.x, x0.im, fma((R)a.y, x0.re, im));
          re = fma((R)a.z, x1.re, fma(-(R)a.w, x1.im, re));
          im = fma((R)a.z, x1.im, fma((R)a.w, x1.re, im));
          acc[2 * r] = re;
          acc[2 * r + 1] = im;
        }
      }
    }
  } else {
    for (int64_t c = c0 + threadIdx.x; c < c1; c += kFwdThreads) {
      const cx<R> x = v[c];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        if (i0 + r < rows) {
          const cx<R> a = cvt<R>(A[(i0 + r) * ld + c]);
          acc[2 * r] = fma(a.re, x.re, fma(-a.im, x.im, acc[2 * r]));
          acc[2 * r + 1] = fma(a.re, x.im, fma(a.im, x.re, acc[2 * r + 1]));
        }
      }
    }
  }
  block_sum_k<R, 2 * ROWS>(acc, scratch, red);
  if (threadIdx.x < ROWS && i0 + threadIdx.x < rows) {
    partial[(int64_t)blockIdx.x * rows + i0 + threadIdx.x] = {red[2 * threadIdx.x], red[2 * threadIdx.x + 1]};
  }
}

template <typename R>
__global__ void __launch_bounds__(256)
fwd_reduce_kernel(const cx<R> *__restrict__ partial, int nchunk, int64_t rows, zd *__restrict__ out,
                  const int *__restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      const cx<R> p = partial[(int64_t)c * rows + i];
      re += (double)p.re;
      im += (double)p.im;
    }
    out[i] = {re, im};
  }
}

// ---- small dense m x m products (the preconditioner P R^{-1}) ------------
__global__ void __launch_bounds__(256)
small_gemv_kernel(const zd *__restrict__ M, int m, const zd *__restrict__ v, zd *__restrict__ out,
                  zf *__restrict__ out32, const int *__restrict__ skip) {
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= m) return;
  const zd *row = M + (int64_t)i * m;
  double re = 0.0, im = 0.0;
  for (int k = lane; k < m; k += 32) {
    const zd a = row[k], x = v[k];
    re = fma(a.re, x.re, fma(-a.im, x.im, re));
    im = fma(a.re, x.im, fma(a.im, x.re, im));
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if (lane == 0) {
    out[i] = {re, im};
    if (out32) out32[i] = {(float)re, (float)im};
  }
}

// ---- configuration and launchers ------------------------------------------
void gemv_configure(GemvPlan &g, int64_t rows, int64_t cols, int64_t ld, int mode, int num_sms) {
  g.rows = rows;
  g.cols = cols;
  g.ld = ld;
  g.mode = mode;
  const int64_t col_blocks = (cols + kAdjCols - 1) / kAdjCols;
  int split = 1;
  while (col_blocks * split < 2 * num_sms && split * 2 <= rows && split < 64) split *= 2;
  g.adj_split = split;
  g.fwd_rows = kFwdRows;
  const int64_t row_blocks = (rows + g.fwd_rows - 1) / g.fwd_rows;
  int64_t nchunk = 1;
  while (row_blocks * nchunk < 12 * num_sms && cols / (nchunk * 2) >= 1024) nchunk *= 2;
  g.fwd_nchunk = (int)nchunk;
  // an even chunk keeps every chunk's first column on a 16-byte boundary for paired loads
  const int64_t chunk = (cols + nchunk - 1) / nchunk;
  g.fwd_chunk = (int)(chunk + (chunk & 1));
}

size_t gemv_adj_partial_elems(const GemvPlan &g) { return (size_t)g.adj_split * g.cols; }
size_t gemv_fwd_partial_elems(const GemvPlan &g) { return (size_t)g.fwd_nchunk * g.rows; }

static int reduce_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1024 ? (b < 1 ? 1 : b) : 1024);
}

template <typename T, typename R, typename OutT>
static cudaError_t adj_t(const GemvPlan &g, const void *A, const void *v, void *out, void *partial,
                         double *qq, const int *skip, cudaStream_t st) {
  const int64_t rows_per = (g.rows + g.adj_split - 1) / g.adj_split + 1;
  const size_t smem = sizeof(cx<R>) * (size_t)rows_per;
  cudaError_t e = cudaFuncSetAttribute(adj_kernel<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((g.cols + kAdjCols - 1) / kAdjCols), g.adj_split);
  note_launch();
  adj_kernel<T, R><<<grid, kAdjThreads, smem, st>>>((const T *)A, g.rows, g.cols, g.ld, (const cx<R> *)v,
                                                     (cx<R> *)partial, g.adj_split, skip);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launch();
  adj_reduce_kernel<R, OutT><<<reduce_blocks(g.cols), 256, 0, st>>>((const cx<R> *)partial, g.adj_split,
                                                                     g.cols, (OutT *)out, qq, skip);
  return cudaGetLastError();
}

template <typename T, typename R>
static cudaError_t fwd_t(const GemvPlan &g, const void *A, const void *v, void *out, void *partial,
                         const int *skip, cudaStream_t st) {
  dim3 grid(g.fwd_nchunk, (unsigned)((g.rows + kFwdRows - 1) / kFwdRows));
  note_launch();
  bool pair = false;
  if constexpr (std::is_same<T, zf>::value) {
    pair = g.ld % 2 == 0 && g.cols % 2 == 0 && reinterpret_cast<uintptr_t>(A) % 16 == 0 &&
           reinterpret_cast<uintptr_t>(v) % 16 == 0;   // (complex128 v: 16-byte entries)
    if (pair)
      fwd_kernel<T, R, kFwdRows, true><<<grid, kFwdThreads, 0, st>>>((const T *)A, g.rows, g.cols, g.ld,
                                                                     (const cx<R> *)v, g.fwd_chunk,
                                                                     (cx<R> *)partial, skip);
  }
  if (!pair)
    fwd_kernel<T, R, kFwdRows, false><<<grid, kFwdThreads, 0, st>>>((const T *)A, g.rows, g.cols, g.ld,
                                                                    (const cx<R> *)v, g.fwd_chunk, (cx<R> *)partial,
                                                                    skip);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launch();
  fwd_reduce_kernel<R><<<reduce_blocks(g.rows), 256, 0, st>>>((const cx<R> *)partial, g.fwd_nchunk, g.rows,
                                                              (zd *)out, skip);
  return cudaGetLastError();
}

cudaError_t launch_gemv_adj(const GemvPlan &g, const void *A, const void *v, void *out, void *partial,
                            double *qq, const int *skip, cudaStream_t st) {
  if (g.mode == 0) return adj_t<zd, double, zd>(g, A, v, out, partial, qq, skip, st);
  if (g.mode == 2) return adj_t<zf, double, zd>(g, A, v, out, partial, qq, skip, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_gemv_fwd(const GemvPlan &g, const void *A, const void *v, void *out, void *partial,
                            const int *skip, cudaStream_t st) {
  if (g.mode == 0) return fwd_t<zd, double>(g, A, v, out, partial, skip, st);
  if (g.mode == 2) return fwd_t<zf, double>(g, A, v, out, partial, skip, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_gemv_adj_f32(const GemvPlan &g, const void *A, const void *v32, void *out32,
                                void *partial, double *qq, const int *skip, cudaStream_t st) {
  return adj_t<zf, float, zf>(g, A, v32, out32, partial, qq, skip, st);
}

cudaError_t launch_gemv_fwd_f32(const GemvPlan &g, const void *A, const void *v32, void *out64,
                                void *partial, const int *skip, cudaStream_t st) {
  return fwd_t<zf, float>(g, A, v32, out64, partial, skip, st);
}

cudaError_t launch_small_gemv(const void *M, int m, const void *v, void *out, void *out32, const int *skip,
                              cudaStream_t st) {
  note_launch();
  small_gemv_kernel<<<(m + 7) / 8, 256, 0, st>>>((const zd *)M, m, (const zd *)v, (zd *)out, (zf *)out32, skip);
  return cudaGetLastError();
}

}  // namespace mn
