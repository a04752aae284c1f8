// common.cuh -- device helpers shared by the sm_103a kernels of the minimal-norm
// solver: an interleaved complex type, block reductions, double-double steps and
// a grid barrier whose wait is bounded in time.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mn {

template <typename R>
struct alignas(2 * sizeof(R)) cx {
  R re, im;
};
using zd = cx<double>;
using zf = cx<float>;

template <typename R>
__host__ __device__ __forceinline__ cx<R> mk(R a, R b) { return cx<R>{a, b}; }

template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
template <typename R>
__device__ __forceinline__ cx<R> scal(R s, cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__device__ __forceinline__ cx<R> conjg(cx<R> a) { return {a.re, -a.im}; }
template <typename R>
__device__ __forceinline__ R abs2(cx<R> a) { return fma(a.re, a.re, a.im * a.im); }

// acc += a * b
template <typename R>
__device__ __forceinline__ void mac(cx<R> &acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R>
__device__ __forceinline__ void macc(cx<R> &acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

template <typename D, typename S>
__device__ __forceinline__ cx<D> cvt(cx<S> a) { return {(D)a.re, (D)a.im}; }

// loads and stores through L2 only (ld/st.global.cg): for data other CTAs
// rewrite while the kernel runs
template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }
template <typename T>
__device__ __forceinline__ void stcg(T *p, T v) { __stcg(p, v); }
__device__ __forceinline__ zd ldcg(const zd *p) {
  const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ void stcg(zd *p, zd v) { __stcg(reinterpret_cast<double2 *>(p), make_double2(v.re, v.im)); }
__device__ __forceinline__ zf ldcg(const zf *p) {
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
  return {v.x, v.y};
}

// ---- reductions ---------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of `v` over the block; every thread gets the result. `scratch` holds
// blockDim.x/32 values. Contains __syncthreads.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  T t = (T)0;
  for (int w = 0; w < nw; ++w) t += scratch[w];
  return t;
}

// Sum of K values per thread over the block, into out[K] (visible to all
// threads after return). scratch: (blockDim.x/32) * K values.
template <typename T, int K>
__device__ __forceinline__ void block_sum_k(T (&v)[K], T *scratch, T *out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) scratch[wid * K + k] = v[k];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    T t = (T)0;
    for (int w = 0; w < nw; ++w) t += scratch[w * K + k];
    out[k] = t;
  }
  __syncthreads();
}

// ---- double-double (error-free transformations with explicit rounding so
// that the compiler cannot contract them) -----------------------------------
struct dd_acc {
  double s, c;
};
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
  s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}
// acc += x * y with the product split exactly (TwoProd) and summed by TwoSum
__device__ __forceinline__ void dd_prod(dd_acc &a, double x, double y) {
  double p = __dmul_rn(x, y);
  double e = __fma_rn(x, y, -p);
  double s, q;
  two_sum(a.s, p, s, q);
  a.s = s;
  a.c = __dadd_rn(a.c, __dadd_rn(q, e));
}
// acc += t with t a small correction (no error term kept for it)
__device__ __forceinline__ void dd_small(dd_acc &a, double t) { a.c = __dadd_rn(a.c, t); }
// acc += (s2 + c2)
__device__ __forceinline__ void dd_add(dd_acc &a, dd_acc b) {
  double s, q;
  two_sum(a.s, b.s, s, q);
  a.s = s;
  a.c = __dadd_rn(a.c, __dadd_rn(q, b.c));
}
__device__ __forceinline__ void dd_round(dd_acc a, double &hi, double &lo) { two_sum(a.s, a.c, hi, lo); }

// ---- grid barrier with a bounded wait ------------------------------------
struct GridBarrier {
  unsigned int count;  // arrivals since launch
  unsigned int gen;    // unused
  int err;  // set to 1 when a wait expired (or by a caller to stop the grid)
  int pad;
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int *p) {
  return *((const volatile int *)p);
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void red_release_add_u32(unsigned int *p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// All blocks of a co-resident (cooperative) grid meet here. Returns false,
// on every thread of the block, if the barrier gave up: after `limit_ns` of
// waiting, or when another block already reported a failure. The arrival
// counter only grows: the e-th barrier of a launch is complete once it reaches
// e * nblocks, so one atomic per block and a poll of the same word suffice
// (`epoch` counts this block's barriers; it starts at 0 and the counter must be
// zero at launch). The arrival is a release reduction (no returned value to wait
// for) and the poll an acquire load, which order the block's writes before, and
// the other blocks' writes after, the barrier; the clock is read every 64 polls.
__device__ __forceinline__ bool grid_sync(GridBarrier *b, unsigned int nblocks, unsigned int &epoch,
                                          uint64_t limit_ns) {
  __shared__ int s_ok;
  epoch += 1u;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int target = epoch * nblocks;
    red_release_add_u32(&b->count, 1u);
    if ((int)(target - ld_acquire_u32(&b->count)) > 0) {
      const uint64_t t0 = global_ns();
      unsigned int polls = 0;
      while ((int)(target - ld_acquire_u32(&b->count)) > 0) {
        if ((++polls & 63u) == 0) {
          if (ld_volatile_i32(&b->err)) { ok = 0; break; }
          if (global_ns() - t0 > limit_ns) { atomicExch(&b->err, 1); ok = 0; break; }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace mn
