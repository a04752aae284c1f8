// xprod.cu -- the refinement's accurate products x = A^* y and r = b - A x on
// the integer pipe.
//
// At kappa(A) ~ 1e6 the residual b - A A^* y and x = A^* y must be formed to
// roughly twice FP64 precision (their terms cancel by a factor kappa). On
// GB300 FP64 arithmetic runs at 1.2 TFLOP/s while 32-bit integer multiply-add
// runs at ~19 Tops/s, so these products are computed exactly in fixed point:
//
//   A      each row i scaled by 2^(62 - E_i), E_i the exponent of the row's
//          largest component, rounded to int64 (|a| < 2^62). Exact for
//          complex64 storage; for complex128, components more than 2^9 below
//          their row's largest are rounded at 2^(E_i - 62), a relative
//          perturbation of A below 2^-63.
//   y      y' = y 2^(E_i) as one 128-bit fixed-point vector, |y'| < 2^Wy,
//          Wy = 124 - ceil(log2 m); built from the double-double y exactly up
//          to one unit.
//   x      accumulated exactly in __int128 (products taken as
//          floor(a y' / 2^64), error < 1 unit each), returned as a
//          double-double vector, then re-scaled into 128-bit fixed point,
//          |x'| < 2^Wx, Wx = 124 - ceil(log2 n), for the forward product.
//   r      sum_j a_ij x'_j exact per CTA and across CTAs, converted to
//          double-double, r = b - t rounded to FP64.
// The bounds on |a|, |y'|, |x'| keep every partial and total sum below 2^127.
#include "common.cuh"
#include "kernels.h"

namespace mn {

typedef __int128 i128;

// |v| < 2^expo(v) for finite v != 0 (and a very small value for 0)
__device__ __forceinline__ int expo(double v) {
  const long long bits = __double_as_longlong(v);
  return (int)((bits >> 52) & 0x7FF) - 1022;
}

// round(v * 2^k) as a 128-bit integer; requires |v 2^k| < 2^126
__device__ __forceinline__ i128 d2fix(double v, int k) {
  const long long bits = __double_as_longlong(v);
  int ex = (int)((bits >> 52) & 0x7FF);
  unsigned long long mant = (unsigned long long)bits & 0xFFFFFFFFFFFFFULL;
  if (mant == 0 && ex == 0) return 0;
  if (ex == 0) ex = 1;
  else mant |= (1ULL << 52);
  const int sh = ex - 1075 + k;  // v 2^k = mant 2^sh
  i128 r;
  if (sh >= 0) {
    r = ((i128)mant) << sh;
  } else if (sh > -64) {
    const unsigned long long half = 1ULL << (-sh - 1);
    r = (i128)((mant + half) >> (-sh));
  } else {
    r = 0;
  }
  return bits < 0 ? -r : r;
}

// v * 2^scale as a double-double (hi, lo), v split in three exactly convertible pieces
__device__ __forceinline__ void fix2dd(i128 v, int scale, double &hi, double &lo) {
  const unsigned long long mask = (1ULL << 53) - 1;
  const unsigned long long c0 = (unsigned long long)v & mask;
  const unsigned long long c1 = (unsigned long long)(v >> 53) & mask;
  const long long c2 = (long long)(v >> 106);
  const double p2 = scalbn((double)c2, 106 + scale);
  const double p1 = scalbn((double)c1, 53 + scale);
  const double p0 = scalbn((double)c0, scale);
  double s, e;
  two_sum(p2, p1, s, e);
  double s2, e2;
  two_sum(s, p0, s2, e2);
  const double l = __dadd_rn(e, e2);
  two_sum(s2, l, hi, lo);
}

// floor(a y / 2^64) for |a| < 2^63
__device__ __forceinline__ i128 mulP(long long a, i128 y) {
  const long long yh = (long long)(y >> 64);
  const unsigned long long yl = (unsigned long long)y;
  const i128 p1 = (i128)a * (i128)yh;
  const unsigned long long h = __umul64hi((unsigned long long)a, yl);
  const long long hs = (long long)(h - (a < 0 ? yl : 0ULL));
  return p1 + (i128)hs;
}

struct fixc {
  long long re, im;
};
struct alignas(16) i128c {
  i128 re, im;
};

// ---- A -> fixed point (and the complex64 copy for mixed precision) -----------
template <typename T>
__global__ void __launch_bounds__(512)
fix_prep_kernel(const T *__restrict__ A, int64_t lda, int64_t cols, fixc *__restrict__ afix,
                int32_t *__restrict__ E, zf *__restrict__ A32, double *__restrict__ rown2) {
  __shared__ int red[16];
  __shared__ double red2[16];
  const int64_t i = blockIdx.x;
  const T *a = A + i * lda;
  int mx = -100000;
  float ss = 0.0f;  // this thread's sum of |a_ij|^2 over its <= k = ceil(cols / blockDim) entries
  for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) {
    const T v = a[j];
    const double re = (double)v.re, im = (double)v.im;
    if (re != 0.0) mx = max(mx, expo(re));
    if (im != 0.0) mx = max(mx, expo(im));
    const float fr = (float)v.re, fi = (float)v.im;
    ss = __fmaf_rn(fr, fr, __fmaf_rn(fi, fi, ss));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  double ssd = (double)ss;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ssd += __shfl_xor_sync(0xffffffffu, ssd, o);
  if ((threadIdx.x & 31) == 0) red2[threadIdx.x >> 5] = ssd;
  __syncthreads();
  int e = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) e = max(e, red[w]);
  if (e < -99999) e = 0;  // a zero row
  if (threadIdx.x == 0) {
    E[i] = e;
    if (rown2) {
      // an upper bound of ||a_i||^2: each float term carries at most one rounding of 2^-24 from
      // the FMA that adds it and, for complex128 entries, 2^-23 from squaring the rounded
      // components; a float sum of k nonnegative terms exceeds none of them by more than
      // (1 + 2^-24)^k; the double sums of the partials add 2^-40 at most
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red2[w];
      const double k = (double)((cols + blockDim.x - 1) / blockDim.x);
      rown2[i] = t * (1.0 + (k + 4.0) * 0x1.0p-23 + 0x1.0p-40) + (double)cols * 0x1.0p-140;  // + underflow
    }
  }
  const int k = 62 - e;
  fixc *o = afix + i * cols;
  for (int64_t j = threadIdx.x; j < cols; j += blockDim.x) {
    const T v = a[j];
    o[j] = {(long long)d2fix((double)v.re, k), (long long)d2fix((double)v.im, k)};
    if (A32) A32[i * cols + j] = {(float)v.re, (float)v.im};
  }
}

// ---- y' = (yh + yl) 2^E_i as 128-bit fixed point ------------------------------
__global__ void __launch_bounds__(1024)
fix_y_kernel(int m, const zd *__restrict__ yh, const zd *__restrict__ yl, const int32_t *__restrict__ E,
             int Wy, i128c *__restrict__ yfix, int *__restrict__ Fy_out, const int *__restrict__ skip) {
  __shared__ int red[32];
  if (skip && *skip) return;  // an asynchronous solve that has stopped
  int mx = -100000;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const zd h = yh[i];
    if (h.re != 0.0) mx = max(mx, expo(h.re) + E[i]);
    if (h.im != 0.0) mx = max(mx, expo(h.im) + E[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  int F = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) F = max(F, red[w]);
  if (F < -99999) F = 0;
  F += 1;  // margin for the low parts
  if (threadIdx.x == 0) *Fy_out = F;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int k = E[i] + Wy - F;
    const zd h = yh[i];
    const zd l = yl ? yl[i] : zd{0.0, 0.0};
    yfix[i] = {d2fix(h.re, k) + d2fix(l.re, k), d2fix(h.im, k) + d2fix(l.im, k)};
  }
}

// ---- x = A^* y' exactly; output as double-double, max exponent to Fx -------------
constexpr int kXadjThreads = 128;
constexpr int kXadjUnroll = 8;

// Complex products use Gauss's three multiplications, exact in integers up to
// the floor of each product:  conj(a) y = (t1 + t2) + i (t3 - t1 + t2) with
// t1 = a_r y_r, t2 = a_i y_i, t3 = (a_r - a_i)(y_r + y_i).
// The rows are split over gridDim.y CTAs (more resident warps to hide the
// loads' latency); each writes its exact partial sums, added by xadj_finish.
__global__ void __launch_bounds__(kXadjThreads)
xadj_kernel(const fixc *__restrict__ afix, int64_t rows, int64_t cols, const i128c *__restrict__ yfix,
            i128c *__restrict__ xpart, const int *__restrict__ skip) {
  __shared__ i128c sy[kXadjThreads];
  __shared__ i128 ss[kXadjThreads];
  if (skip && *skip) return;  // an asynchronous solve that has stopped
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (rows + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = (int64_t)blockIdx.y * per, r1 = r0 + per < rows ? r0 + per : rows;
  i128 are = 0, aim = 0;
  for (int64_t i0 = r0; i0 < r1; i0 += kXadjThreads) {
    __syncthreads();
    if (i0 + threadIdx.x < r1) {
      const i128c y = yfix[i0 + threadIdx.x];
      sy[threadIdx.x] = y;
      ss[threadIdx.x] = y.re + y.im;
    }
    __syncthreads();
    if (j < cols) {
      const int ie = (int)((i0 + kXadjThreads < r1 ? i0 + kXadjThreads : r1) - i0);
      const fixc *a = afix + i0 * cols + j;
      int u = 0;
      for (; u + kXadjUnroll <= ie; u += kXadjUnroll) {
        fixc av[kXadjUnroll];
#pragma unroll
        for (int q = 0; q < kXadjUnroll; ++q) av[q] = a[(int64_t)(u + q) * cols];
#pragma unroll
        for (int q = 0; q < kXadjUnroll; ++q) {
          const i128c y = sy[u + q];
          const i128 t1 = mulP(av[q].re, y.re), t2 = mulP(av[q].im, y.im);
          const i128 t3 = mulP(av[q].re - av[q].im, ss[u + q]);
          are += t1 + t2;
          aim += t3 - t1 + t2;
        }
      }
      for (; u < ie; ++u) {
        const fixc av = a[(int64_t)u * cols];
        const i128c y = sy[u];
        const i128 t1 = mulP(av.re, y.re), t2 = mulP(av.im, y.im);
        const i128 t3 = mulP(av.re - av.im, ss[u]);
        are += t1 + t2;
        aim += t3 - t1 + t2;
      }
    }
  }
  if (j < cols) xpart[(int64_t)blockIdx.y * cols + j] = {are, aim};
}

// x_j = sum of the row splits' partials, as double-double; max exponent to Fx
__global__ void __launch_bounds__(256)
xadj_finish_kernel(const i128c *__restrict__ xpart, int nsplit, int64_t cols, const int *__restrict__ Fy, int Wy,
                   zd *__restrict__ xh, zd *__restrict__ xl, int *__restrict__ Fx, const int *__restrict__ skip) {
  __shared__ int red[8];
  if (skip && *skip) return;  // an asynchronous solve that has stopped
  int mx = -100000;
  const int scale = 2 + *Fy - Wy;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols; j += (int64_t)gridDim.x * blockDim.x) {
    i128 are = 0, aim = 0;
    for (int q = 0; q < nsplit; ++q) {
      const i128c v = xpart[(int64_t)q * cols + j];
      are += v.re;
      aim += v.im;
    }
    double h1, l1, h2, l2;
    fix2dd(are, scale, h1, l1);
    fix2dd(aim, scale, h2, l2);
    xh[j] = {h1, h2};
    xl[j] = {l1, l2};
    if (h1 != 0.0) mx = max(mx, expo(h1));
    if (h2 != 0.0) mx = max(mx, expo(h2));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    int e = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) e = max(e, red[w]);
    if (e > -99999) atomicMax(Fx, e + 1);
  }
}

// x' = (xh + xl) 2^(Wx - Fx) as 128-bit fixed point, once per column for the forward pass
__global__ void __launch_bounds__(256)
xfix_kernel(int64_t cols, const zd *__restrict__ xh, const zd *__restrict__ xl, const int *__restrict__ Fx, int Wx,
            i128c *__restrict__ xfix, const int *__restrict__ skip) {
  if (skip && *skip) return;  // an asynchronous solve that has stopped
  const int k = Wx - *Fx;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols; j += (int64_t)gridDim.x * blockDim.x) {
    const zd h = xh[j], l = xl[j];
    xfix[j] = {d2fix(h.re, k) + d2fix(l.re, k), d2fix(h.im, k) + d2fix(l.im, k)};
  }
}

// ---- t = A x' exactly, per (column chunk, row) partial sums ---------------------
constexpr int kXfwdThreads = 256;
constexpr int kXfwdRows = 8;

__device__ __forceinline__ i128 shfl_xor_i128(i128 v, int o) {
  const long long hi = __shfl_xor_sync(0xffffffffu, (long long)(v >> 64), o);
  const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
  return ((i128)hi << 64) | (i128)lo;
}

__global__ void __launch_bounds__(kXfwdThreads)
xfwd_kernel(const fixc *__restrict__ afix, int64_t rows, int64_t cols, const i128c *__restrict__ xfix,
            int64_t chunk, i128c *__restrict__ partial, const int *__restrict__ skip) {
  __shared__ i128c sred[(kXfwdThreads / 32) * kXfwdRows];
  if (skip && *skip) return;  // an asynchronous solve that has stopped
  const int64_t i0 = (int64_t)blockIdx.y * kXfwdRows;
  const int64_t c0 = (int64_t)blockIdx.x * chunk;
  const int64_t c1 = c0 + chunk < cols ? c0 + chunk : cols;
  i128 acc_re[kXfwdRows], acc_im[kXfwdRows];
#pragma unroll
  for (int r = 0; r < kXfwdRows; ++r) { acc_re[r] = 0; acc_im[r] = 0; }
  const int nr = rows - i0 < kXfwdRows ? (int)(rows - i0) : kXfwdRows;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const i128c xv = xfix[c];
    fixc av[kXfwdRows];
#pragma unroll
    for (int r = 0; r < kXfwdRows; ++r) av[r] = r < nr ? afix[(i0 + r) * cols + c] : fixc{0, 0};
    const i128 xr = xv.re, xi = xv.im;
    const i128 xs = xr + xi;
#pragma unroll
    for (int r = 0; r < kXfwdRows; ++r) {
      // a x = (t1 - t2) + i (t3 - t1 - t2), t1 = ar xr, t2 = ai xi, t3 = (ar + ai)(xr + xi)
      const i128 t1 = mulP(av[r].re, xr), t2 = mulP(av[r].im, xi);
      const i128 t3 = mulP(av[r].re + av[r].im, xs);
      acc_re[r] += t1 - t2;
      acc_im[r] += t3 - t1 - t2;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < kXfwdRows; ++r) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc_re[r] += shfl_xor_i128(acc_re[r], o);
      acc_im[r] += shfl_xor_i128(acc_im[r], o);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int r = 0; r < kXfwdRows; ++r) sred[wid * kXfwdRows + r] = {acc_re[r], acc_im[r]};
  }
  __syncthreads();
  if (threadIdx.x < kXfwdRows && i0 + threadIdx.x < rows) {
    const int r = threadIdx.x;
    i128 sr = 0, si = 0;
    for (int w = 0; w < kXfwdThreads / 32; ++w) {
      sr += sred[w * kXfwdRows + r].re;
      si += sred[w * kXfwdRows + r].im;
    }
    partial[(int64_t)blockIdx.x * rows + i0 + r] = {sr, si};
  }
}

// r_i = b_i - t_i, t_i = (sum of chunk partials) 2^(E_i - 62 + Fx - Wx + 64), in double-double
__global__ void xfwd_finish_kernel(const i128c *__restrict__ partial, int nchunk, int64_t rows,
                                   const int32_t *__restrict__ E, const int *__restrict__ Fx, int Wx,
                                   const zd *__restrict__ b, zd *__restrict__ r, zd *__restrict__ th,
                                   zd *__restrict__ tl, const int *__restrict__ skip) {
  if (skip && *skip) return;  // an asynchronous solve that has stopped
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
    i128 sr = 0, si = 0;
    for (int c = 0; c < nchunk; ++c) {
      sr += partial[(int64_t)c * rows + i].re;
      si += partial[(int64_t)c * rows + i].im;
    }
    const int scale = E[i] - 62 + *Fx - Wx + 64;
    double h1, l1, h2, l2;
    fix2dd(sr, scale, h1, l1);
    fix2dd(si, scale, h2, l2);
    if (th) th[i] = {h1, h2};
    if (tl) tl[i] = {l1, l2};
    if (r) {
      const zd bi = b[i];
      double s1, e1, s2, e2;
      two_sum(bi.re, -h1, s1, e1);
      two_sum(bi.im, -h2, s2, e2);
      r[i] = {__dadd_rn(s1, __dsub_rn(e1, l1)), __dadd_rn(s2, __dsub_rn(e2, l2))};
    }
  }
}

// ---- host launchers ---------------------------------------------------------------
static int ceil_log2(int64_t v) {
  int k = 0;
  while ((int64_t(1) << k) < v) ++k;
  return k;
}

int xprod_wy(int64_t m) { return 126 - ceil_log2(m) - 2; }
int xprod_wx(int64_t n) { return 126 - ceil_log2(n) - 2; }

cudaError_t launch_fix_prep(const void *A, int64_t lda, bool c64, int64_t rows, int64_t cols, void *afix,
                            int32_t *E, void *A32, cudaStream_t st, double *rown2) {
  note_launch();
  if (c64)
    fix_prep_kernel<zf><<<(unsigned)rows, 512, 0, st>>>((const zf *)A, lda, cols, (fixc *)afix, E, (zf *)A32,
                                                         rown2);
  else
    fix_prep_kernel<zd><<<(unsigned)rows, 512, 0, st>>>((const zd *)A, lda, cols, (fixc *)afix, E, (zf *)A32,
                                                         rown2);
  return cudaGetLastError();
}

size_t xprod_partial_bytes(int64_t rows, int nchunk) { return sizeof(i128c) * (size_t)rows * nchunk; }

// row splits of x = A^* y: enough CTAs for several per SM while each split keeps >= 64 rows
int xadj_splits(int64_t rows, int64_t cols) {
  const int64_t nbx = (cols + kXadjThreads - 1) / kXadjThreads;
  int s = 1;
  while (s < 8 && nbx * s < 4096 && rows / (2 * s) >= 64) s *= 2;
  return s;
}
// largest row split the partial buffer is sized for: up to 8, each split >= 64 rows
int xadj_max_splits(int64_t rows) {
  int s = 1;
  while (s < 8 && rows / (2 * s) >= 64) s *= 2;
  return s;
}
size_t xadj_partial_bytes(int64_t rows, int64_t cols) {
  return sizeof(i128c) * (size_t)cols * xadj_max_splits(rows);
}
size_t xfix_bytes(int64_t cols) { return sizeof(i128c) * (size_t)cols; }

cudaError_t launch_xresidual(const XprodArgs &a, cudaStream_t st) {
  const int Wy = xprod_wy(a.rows), Wx = xprod_wx(a.cols);
  cudaError_t e = cudaMemsetAsync(a.Fx, 0x80, sizeof(int), st);  // very negative start for atomicMax
  if (e != cudaSuccess) return e;
  note_launch();
  fix_y_kernel<<<1, 1024, 0, st>>>((int)a.rows, (const zd *)a.yh, (const zd *)a.yl, a.E, Wy, (i128c *)a.yfix,
                                   a.Fy, a.skip);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    const int64_t nbx = (a.cols + kXadjThreads - 1) / kXadjThreads;
    const int nsplit = a.xsplit > 0 ? a.xsplit : xadj_splits(a.rows, a.cols);
    note_launch();
    xadj_kernel<<<dim3((unsigned)nbx, (unsigned)nsplit), kXadjThreads, 0, st>>>(
        (const fixc *)a.afix, a.rows, a.cols, (const i128c *)a.yfix, (i128c *)a.xpart, a.skip);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int64_t nb = (a.cols + 255) / 256;
    if (nb > 2048) nb = 2048;
    note_launch();
    xadj_finish_kernel<<<(unsigned)nb, 256, 0, st>>>((const i128c *)a.xpart, nsplit, a.cols, a.Fy, Wy,
                                                     (zd *)a.xh, (zd *)a.xl, a.Fx, a.skip);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (!a.b) return cudaSuccess;  // x only
  {
    int64_t nb = (a.cols + 255) / 256;
    if (nb > 2048) nb = 2048;
    note_launch();
    xfix_kernel<<<(unsigned)nb, 256, 0, st>>>(a.cols, (const zd *)a.xh, (const zd *)a.xl, a.Fx, Wx,
                                              (i128c *)a.xfix, a.skip);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  dim3 grid(a.nchunk, (unsigned)((a.rows + kXfwdRows - 1) / kXfwdRows));
  note_launch();
  xfwd_kernel<<<grid, kXfwdThreads, 0, st>>>((const fixc *)a.afix, a.rows, a.cols, (const i128c *)a.xfix, a.chunk,
                                             (i128c *)a.partial, a.skip);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int64_t nb = (a.rows + 255) / 256;
  if (nb > 1024) nb = 1024;
  note_launch();
  xfwd_finish_kernel<<<(unsigned)nb, 256, 0, st>>>((const i128c *)a.partial, a.nchunk, a.rows, a.E, a.Fx, Wx,
                                                   (const zd *)a.b, (zd *)a.r, (zd *)a.th, (zd *)a.tl, a.skip);
  return cudaGetLastError();
}

}  // namespace mn
