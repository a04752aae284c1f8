// ozaki.cu -- FP64-accurate complex products on the tensor cores, for the
// trailing updates of the blocked Householder QR of Step 2 (qrblk.cu):
//     W^H = C^H V      (the adjoint product, K = the rows of the trailing block)
//     C  -= V Z        (the update, K = 32 reflectors)
// with C, V, Z complex FP64.
//
// The error-free splitting of Ozaki, Ogita, Oishi and Rump ("Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012), with
// integer slices: every entry x of an operand row with exponent e (all of the
// row's entries below 2^e in magnitude) is written exactly (to 2^-56 of 2^e) as
//     x = 2^e / 16 * sum_{s=0}^{13} sigma_s,   sigma_s = +-d_s 16^-s,
// d_s in 0..15 the base-16 digits of |x| 2^(56-e), read off the FP64 bit pattern
// with integer shifts (no FP64 instruction; entries within 2^3 of the row's
// scale keep every bit). Each sigma_s is exact in BF16. A product of two rows
// is then 2^(e + f) / 256 times the sum over the levels L = s + t of
// sum_k sigma_s sigma_t. The levels L <= 15 are kept (130 pairs; the dropped
// ones add at most 14 * 15 * 16^-15 of 2^(e+f)/256 per term, the order of the
// 56-bit truncation of the entries themselves). A level's sum is an integer
// multiple of 16^-L whose integer part stays below 14 * 225 * 4096 < 2^24 for
// K <= 4096 per CTA, so the tensor cores' FP32 accumulation of every kept level
// (one accumulator each, 16 x 32 = all 512 columns of tensor memory) is EXACT. (A shared FP32 accumulator for the trailing levels is not enough: its
// rounding grows with the number of terms, and the tensor cores' accumulation
// truncates.) The levels are combined exactly in two int64 halves and rounded
// once to FP64; K splits across CTAs are added in FP64. The only other errors
// are the truncation of each entry to 52 bits below its row's scale: the
// product is as accurate as an FP64 dot product, at the tensor cores' BF16 rate
// divided by the 130 slice pairs.
//
// Real forms of the complex products (interleaved re/im along K):
//   adjoint: A row c = (Re C[r,c], Im C[r,c])_r, B row j < 32 = (Re V[r,j], Im V[r,j])_r,
//            B row 32 + j = (Im V[r,j], -Re V[r,j])_r: D[c][j] = Re (C^H V)[c,j],
//            D[c][32 + j] = Im (C^H V)[c,j].
//   update:  A row 2i = (Re V[i,j], -Im V[i,j])_j, A row 2i+1 = (Im V[i,j], Re V[i,j])_j,
//            B row c = (Re Z[j,c], Im Z[j,c])_j: D[2i][c] = Re (V Z)[i,c], D[2i+1][c] = Im.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

#include <algorithm>

namespace mn {

namespace {

constexpr int kOzThreads = 256;
constexpr int kOzRing = 6;                        // A slice tiles in flight
constexpr int kOzATile = kOzM * kOzK * 2;         // 16 KB: 128 rows x 64 BF16
constexpr int kOzBTile = kOzN * kOzK * 2;         // 4 KB: 32 rows x 64 BF16
constexpr int kOzKept = kOzSlices + 2;            // levels 0..15 (pairs s + t <= 15), one accumulator each
constexpr int kOzTmemCols = kOzKept * kOzN;       // 512
constexpr int kOzOffB = kOzRing * kOzATile;       // 96 KB
constexpr int kOzOffBar = kOzOffB + kOzSlices * kOzBTile;  // 148 KB
constexpr int kOzSmem = kOzOffBar + 512 + 1024;   // barriers + alignment slack

// exponent of a row: the least e with every |x| < 2^e (the FP64 exponent field of the
// largest entry, plus one); -2000 for a zero row
__device__ __forceinline__ int oz_expo_of(double x) {
  const long long b = __double_as_longlong(x);
  const int f = (int)((b >> 52) & 0x7ff);
  return f == 0 ? -2000 : f - 1023 + 1;
}

// the 14 signed slices sigma_s = +-d_s 16^-s of x for row exponent e, as BF16
__device__ __forceinline__ void oz_slices(double x, int e, __nv_bfloat16 (&q)[kOzSlices]) {
  const long long b = __double_as_longlong(x);
  const int f = (int)((b >> 52) & 0x7ff);
  unsigned long long N = 0;
  if (f != 0 && e > -2000) {
    const unsigned long long mant = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = e - (f - 1023);  // >= 1: |x| < 2^e
    // floor(|x| 2^(56 - e)) = mant 2^(4 - sh), 56 bits
    N = sh <= 4 ? (mant << (4 - sh)) : (sh - 4 < 64 ? (mant >> (sh - 4)) : 0ull);
  }
  const float sgn = b < 0 ? -1.0f : 1.0f;
#pragma unroll
  for (int s = 0; s < kOzSlices; ++s) {
    const int d = (int)((N >> (4 * (kOzSlices - 1 - s))) & 15ull);
    q[s] = __float2bfloat16_rn(sgn * (float)d * __int_as_float((127 - 4 * s) << 23));  // d 16^-s, exact
  }
}

__device__ __forceinline__ int oz_block_max(int v, int *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int m = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
  return m;
}

// store the slices of one K position pair (k, k+1) of row `row`
__device__ __forceinline__ void oz_put2(__nv_bfloat16 *S, int64_t sstride, int64_t kpad, int64_t row, int64_t k,
                                        const __nv_bfloat16 (&a)[kOzSlices], const __nv_bfloat16 (&b)[kOzSlices]) {
#pragma unroll
  for (int s = 0; s < kOzSlices; ++s) {
    __nv_bfloat162 v;
    v.x = a[s];
    v.y = b[s];
    *reinterpret_cast<__nv_bfloat162 *>(S + s * sstride + row * kpad + k) = v;
  }
}

// A rows of the adjoint product: one CTA per column c of C
__global__ void __launch_bounds__(256)
oz_slice_cols_kernel(const zd *__restrict__ C, int64_t ldc, int64_t rows, int64_t cols, __nv_bfloat16 *__restrict__ S,
                     int32_t *__restrict__ expo, int64_t rows_pad, int64_t kpad) {
  __shared__ int red[8];
  const int64_t c = blockIdx.x;
  const zd *col = C + c * ldc;
  int e = -2000;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
    const zd v = col[r];
    e = max(e, max(oz_expo_of(v.re), oz_expo_of(v.im)));
  }
  e = oz_block_max(e, red);
  if (threadIdx.x == 0) expo[c] = e;
  const int64_t ss = rows_pad * kpad;
  for (int64_t r = threadIdx.x; 2 * r < kpad; r += blockDim.x) {
    __nv_bfloat16 a[kOzSlices], b[kOzSlices];
    const zd v = r < rows ? col[r] : zd{0.0, 0.0};
    oz_slices(v.re, e, a);
    oz_slices(v.im, e, b);
    oz_put2(S, ss, kpad, c, 2 * r, a, b);
  }
}

// B rows of the adjoint product from the 32 reflectors: one CTA per reflector j (two rows)
__global__ void __launch_bounds__(256)
oz_slice_v_adj_kernel(const zd *__restrict__ V, int64_t ldv, int64_t rows, __nv_bfloat16 *__restrict__ S,
                      int32_t *__restrict__ expo, int64_t kpad) {
  __shared__ int red[8];
  const int j = blockIdx.x;
  const zd *col = V + (int64_t)j * ldv;
  int e = -2000;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
    const zd v = col[r];
    e = max(e, max(oz_expo_of(v.re), oz_expo_of(v.im)));
  }
  e = oz_block_max(e, red);
  if (threadIdx.x == 0) { expo[j] = e; expo[32 + j] = e; }
  const int64_t ss = (int64_t)64 * kpad;
  for (int64_t r = threadIdx.x; 2 * r < kpad; r += blockDim.x) {
    __nv_bfloat16 a[kOzSlices], b[kOzSlices], na[kOzSlices];
    const zd v = r < rows ? col[r] : zd{0.0, 0.0};
    oz_slices(v.re, e, a);
    oz_slices(v.im, e, b);
    oz_slices(-v.re, e, na);
    oz_put2(S, ss, kpad, j, 2 * r, a, b);         // (Re, Im)
    oz_put2(S, ss, kpad, 32 + j, 2 * r, b, na);   // (Im, -Re)
  }
}

// A rows of the update: one thread per row i of V (two rows 2i, 2i+1, K = 64)
__global__ void __launch_bounds__(128)
oz_slice_v_fwd_kernel(const zd *__restrict__ V, int64_t ldv, int64_t rows, __nv_bfloat16 *__restrict__ S,
                      int32_t *__restrict__ expo, int64_t rows_pad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (2 * i >= rows_pad) return;
  const int64_t ss = rows_pad * kOzK;
  zd v[32];
  int e = -2000;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    v[j] = i < rows ? V[(int64_t)j * ldv + i] : zd{0.0, 0.0};
    e = max(e, max(oz_expo_of(v[j].re), oz_expo_of(v[j].im)));
  }
  expo[2 * i] = e;
  expo[2 * i + 1] = e;
#pragma unroll 1
  for (int j = 0; j < 32; ++j) {
    __nv_bfloat16 re[kOzSlices], im[kOzSlices], nim[kOzSlices];
    oz_slices(v[j].re, e, re);
    oz_slices(v[j].im, e, im);
    oz_slices(-v[j].im, e, nim);
    oz_put2(S, ss, kOzK, 2 * i, 2 * j, re, nim);    // (Re V, -Im V)
    oz_put2(S, ss, kOzK, 2 * i + 1, 2 * j, im, re); // (Im V, Re V)
  }
}

// B rows of the update: one thread per column c of Z (32 x cols, column-major)
__global__ void __launch_bounds__(128)
oz_slice_z_kernel(const zd *__restrict__ Z, int64_t ldz, int64_t cols, __nv_bfloat16 *__restrict__ S,
                  int32_t *__restrict__ expo, int64_t rows_pad) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= rows_pad) return;
  const int64_t ss = rows_pad * kOzK;
  zd z[32];
  int e = -2000;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    z[j] = c < cols ? Z[c * ldz + j] : zd{0.0, 0.0};
    e = max(e, max(oz_expo_of(z[j].re), oz_expo_of(z[j].im)));
  }
  expo[c] = e;
#pragma unroll 1
  for (int j = 0; j < 32; ++j) {
    __nv_bfloat16 re[kOzSlices], im[kOzSlices];
    oz_slices(z[j].re, e, re);
    oz_slices(z[j].im, e, im);
    oz_put2(S, ss, kOzK, c, 2 * j, re, im);
  }
}

}  // namespace

namespace {

struct OzParams {
  int a_rows_pad, b_rows_pad;    // rows of one slice in the tensor maps
  int kb0_stride;                // adjoint: K-blocks per split
  int nkb;                       // K-blocks of the whole K
  const int32_t *ea, *eb;        // row exponents
  // adjoint: partial sums part[split][row][64]
  double *part;
  int part_rows;
  // update: C[i, c] -= D for i < rows, c < cols
  zd *C;
  int64_t ldc;
  int rows, cols;
  int *err;
  uint64_t limit_ns;
};

// Tile: A rows [128 ma, +128), B rows [64 nb, +64), K-blocks [kb0, kb1). Adjoint: grid
// (A tiles, K splits), nb = 0; update: grid (A tiles, B tiles), one K-block.
// Roles: warp 0 lane 0 issues the TMA loads (the 13 B slice tiles of a K-block stay resident;
// the A slice tiles stream through a 4-deep ring), warp 1 lane 0 issues the MMAs and commits
// them to the barriers that free the tiles, warp 2 owns the tensor memory, warps 4-7 read the
// eight accumulators (TMEM lanes 32 (w & 3) + lane = tile rows) and write the result.
template <bool FWD>
__global__ void __launch_bounds__(kOzThreads, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
               const OzParams P) {
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;
  unsigned char *sB = base + kOzOffB;
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + kOzOffBar);
  uint64_t *a_full = bars;                     // kOzRing
  uint64_t *a_empty = bars + kOzRing;          // kOzRing
  uint64_t *b_full = bars + 2 * kOzRing;       // kOzSlices
  uint64_t *b_empty = b_full + kOzSlices;      // kOzSlices
  uint64_t *acc_full = b_empty + kOzSlices;    // 1
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_full + 1);
  __shared__ int s_abort;
  __shared__ int s_a_issued, s_a_used, s_b_issued, s_b_used;

  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int ma = blockIdx.x;
  const int nb = FWD ? blockIdx.y : blockIdx.z;
  const int kb0 = FWD ? 0 : blockIdx.y * P.kb0_stride;
  const int kb1 = FWD ? 1 : min(P.nkb, kb0 + P.kb0_stride);
  const int nkb = kb1 - kb0;

  if (tid == 0) {
    for (int q = 0; q < kOzRing; ++q) { bar_init(&a_full[q], 1); bar_init(&a_empty[q], 1); }
    for (int t = 0; t < kOzSlices; ++t) { bar_init(&b_full[t], 1); bar_init(&b_empty[t], 1); }
    bar_init(acc_full, 1);
    s_abort = 0;
    s_a_issued = s_a_used = s_b_issued = s_b_used = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (wid == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tmem_slot)),
                 "r"(kOzTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (nkb > 0 && wid == 0 && lane == 0) {
    // producer: per K-block A_0..A_3, then B_12..B_0 (freed in that order by the previous
    // K-block's products), then A_4..A_12; every wait for a free tile is bounded
    int ai = 0, bi = 0;
    bool ok = true;
    auto load_a = [&](int kb, int s) -> bool {
      const int slot = ai % kOzRing;
      if (ai >= kOzRing && !bar_wait(&a_empty[slot], (uint32_t)(((ai / kOzRing) - 1) & 1), P.limit_ns)) return false;
      bar_expect(&a_full[slot], kOzATile);
      tma2d(sA + slot * kOzATile, &amap, kb * kOzK, s * P.a_rows_pad + ma * kOzM, &a_full[slot]);
      ++ai;
      return true;
    };
    auto load_b = [&](int kb, int t, int kk) -> bool {
      if (kk > 0 && !bar_wait(&b_empty[t], (uint32_t)((kk - 1) & 1), P.limit_ns)) return false;
      bar_expect(&b_full[t], kOzBTile);
      tma2d(sB + t * kOzBTile, &bmap, kb * kOzK, t * P.b_rows_pad + nb * kOzN, &b_full[t]);
      ++bi;
      return true;
    };
    for (int kk = 0; kk < nkb && ok; ++kk) {
      const int kb = kb0 + kk;
      for (int s = 0; s < kOzRing && ok; ++s) ok = load_a(kb, s) && !*(volatile int *)&s_abort;
      for (int t = kOzSlices - 1; t >= 0 && ok; --t) ok = load_b(kb, t, kk) && !*(volatile int *)&s_abort;
      for (int s = kOzRing; s < kOzSlices && ok; ++s) ok = load_a(kb, s) && !*(volatile int *)&s_abort;
    }
    if (!ok) atomicExch(&s_abort, 1);
    s_a_issued = ai;
    s_b_issued = bi;
  } else if (nkb > 0 && wid == 1 && lane == 0) {
    // products: pair (s, t), s + t <= 15, into accumulator s + t (exact); the first product
    // into an accumulator (pair (0, t), or (1, 13) and (2, 13) for levels 14 and 15, of the
    // first K-block) overwrites it. B_t has its last pair at s = 15 - t (B_0 and B_1 at s = 13).
    int ai = 0, bu = 0;
    bool ok = true;
    const uint32_t id = idesc(kOzN);
    for (int kk = 0; kk < nkb && ok; ++kk) {
      for (int s = 0; s < kOzSlices && ok; ++s) {
        const int slot = ai % kOzRing;
        ok = bar_wait(&a_full[slot], (uint32_t)((ai / kOzRing) & 1), P.limit_ns);
        if (ok && s == 0) {
          for (int t = 0; t < kOzSlices && ok; ++t) ok = bar_wait(&b_full[t], (uint32_t)(kk & 1), P.limit_ns);
          bu += ok ? kOzSlices : 0;
        }
        if (!ok || *(volatile int *)&s_abort) { ok = false; break; }
        tc_fence_after();
        const uint32_t a0 = sa(sA + slot * kOzATile);
        for (int t = 0; t < kOzSlices && s + t < kOzKept; ++t) {
          const uint32_t d = tmem + (uint32_t)((s + t) * kOzN);
          const uint32_t b0 = sa(sB + t * kOzBTile);
          const bool first = kk == 0 && (s == 0 || (s <= 2 && t == kOzSlices - 1));
#pragma unroll
          for (int k16 = 0; k16 < kOzK / 16; ++k16) {
            const uint32_t accum = (first && k16 == 0) ? 0u : 1u;
            mma_bf16(d, sdesc(a0 + k16 * 32), sdesc(b0 + k16 * 32), id, accum);
          }
        }
        mma_commit(&a_empty[slot]);                   // A_s read
        if (s >= 2) mma_commit(&b_empty[kOzKept - 1 - s]);   // B_{15 - s} has had its last pair
        if (s == kOzSlices - 1) {                             // and B_1, B_0 at s = 13
          mma_commit(&b_empty[1]);
          mma_commit(&b_empty[0]);
        }
        ++ai;
      }
    }
    if (ok) mma_commit(acc_full);
    else atomicExch(&s_abort, 1);
    s_a_used = ai;
    s_b_used = bu;
  }

  // epilogue: warps 4-7
  bool good = true;
  if (wid >= 4) {
    if (nkb > 0) {
      good = false;
      const uint64_t t0 = global_ns();
      while (!good && !*(volatile int *)&s_abort) {
        good = bar_try(acc_full, 0u);
        if (!good && global_ns() - t0 > P.limit_ns) break;
      }
      good = __all_sync(0xffffffffu, good);
    }
    if (good) {
      tc_fence_after();
      const int row = 32 * (wid & 3) + lane;           // tile row (TMEM lane)
      const int ga = ma * kOzM + row;                   // A row
      const int ea = P.ea[ga];
      {
        // levels 0..7 into Ih = sum I_L 16^(7-L), levels 8..15 into Il = sum I_L 16^(15-L), each
        // level's sum an exact integer I_L times 16^-L below 2^24 (both halves below 2^53)
        long long Ih[32], Il[32];
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) { Ih[k] = 0; Il[k] = 0; }
        if (nkb > 0) {
#pragma unroll 1
          for (int L = 0; L < kOzKept; ++L) {
            tmem_ld32(tmem + ((uint32_t)(32 * (wid & 3)) << 16) + (uint32_t)(L * kOzN), v);
            const float up = __int_as_float((127 + 4 * L) << 23);  // 16^L
            if (L < 8) {
#pragma unroll
              for (int k = 0; k < 32; ++k) Ih[k] += (long long)__float2int_rn(v[k] * up) << (4 * (7 - L));
            } else {
#pragma unroll
              for (int k = 0; k < 32; ++k) Il[k] += (long long)__float2int_rn(v[k] * up) << (4 * (15 - L));
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const int col = k;
          const int eb = P.eb[nb * kOzN + col];
          // the levels' sum Ih 16^-7 + Il 16^-15 (one rounding), times 2^(ea + eb) / 256
          double r = fma((double)Il[k], 0x1.0p-60, (double)Ih[k] * 0x1.0p-28);
          const int sc = ea + eb - 8;
          if (ea <= -2000 || eb <= -2000) r = 0.0;
          else if (sc >= -1022 && sc <= 1023) r *= __longlong_as_double((long long)(sc + 1023) << 52);  // 2^sc
          else r = ldexp(r, sc);
          if (FWD) {
            const int c = nb * kOzN + col;
            const int i = ga >> 1, p = ga & 1;
            if (i < P.rows && c < P.cols) {
              double *dst = reinterpret_cast<double *>(P.C + (int64_t)c * P.ldc + i) + p;
              *dst -= r;
            }
          } else {
            P.part[((int64_t)blockIdx.y * P.part_rows + ga) * 64 + nb * kOzN + col] = r;
          }
        }
      }
      tc_fence_before();
    }
    if (!good) atomicExch(&s_abort, 1);
  }
  __syncthreads();
  if (s_abort && tid == 0) {
    atomicExch(P.err, 1);
    // loads still in flight: the A tiles issued but not taken, the B tiles likewise (bounded)
    for (int q = s_a_used; q < s_a_issued; ++q) bar_wait(&a_full[q % kOzRing], (uint32_t)((q / kOzRing) & 1), P.limit_ns);
    const int kk_b = s_b_used / kOzSlices;
    for (int q = s_b_used; q < s_b_issued; ++q) bar_wait(&b_full[q % kOzSlices], (uint32_t)(kk_b & 1), P.limit_ns);
    // products in flight: the last A tile's commit
    if (s_a_used > 0) {
      const int q = s_a_used - 1;
      bar_wait(&a_empty[q % kOzRing], (uint32_t)((q / kOzRing) & 1), P.limit_ns);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (wid == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzTmemCols) : "memory");
  }
}

}  // namespace

// ---- host ---------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 oz_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// the slices of an operand as a 2-D BF16 array (k_pad wide, kOzSlices rows_pad rows) read in
// boxes of 64 (K) x box_rows, 128-byte swizzle: the K-major layout the MMA descriptors expect
cudaError_t oz_map(const OzOperand &o, uint32_t box_rows, CUtensorMap *map) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = oz_encode();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t gdim[2] = {(cuuint64_t)o.k_pad, (cuuint64_t)(kOzSlices * o.rows_pad)};
  const cuuint64_t gstride[1] = {(cuuint64_t)(o.k_pad * sizeof(__nv_bfloat16))};
  const cuuint32_t box[2] = {kOzK, box_rows};
  const cuuint32_t es[2] = {1, 1};
  if (enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, o.slices, gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
      CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

int64_t pad_to(int64_t v, int64_t q) { return (v + q - 1) / q * q; }

}  // namespace

size_t oz_slice_bytes(int64_t rows, int64_t k) {
  return (size_t)kOzSlices * (size_t)pad_to(rows, kOzM) * (size_t)pad_to(k, kOzK) * sizeof(__nv_bfloat16);
}

cudaError_t launch_oz_slice_cols(const void *C, int64_t ldc, int64_t rows, int64_t cols, OzOperand &out,
                                 cudaStream_t st) {
  out.rows = cols;
  out.rows_pad = pad_to(cols, kOzM);
  out.k = 2 * rows;
  out.k_pad = pad_to(2 * rows, kOzK);
  if (cols < 1) return cudaSuccess;
  note_launch();
  oz_slice_cols_kernel<<<(unsigned)cols, 256, 0, st>>>((const zd *)C, ldc, rows, cols, (__nv_bfloat16 *)out.slices,
                                                       out.expo, out.rows_pad, out.k_pad);
  return cudaGetLastError();
}

cudaError_t launch_oz_slice_v_adj(const void *V, int64_t ldv, int64_t rows, OzOperand &out, cudaStream_t st) {
  out.rows = 64;
  out.rows_pad = 64;
  out.k = 2 * rows;
  out.k_pad = pad_to(2 * rows, kOzK);
  note_launch();
  oz_slice_v_adj_kernel<<<32, 256, 0, st>>>((const zd *)V, ldv, rows, (__nv_bfloat16 *)out.slices, out.expo,
                                            out.k_pad);
  return cudaGetLastError();
}

cudaError_t launch_oz_slice_v_fwd(const void *V, int64_t ldv, int64_t rows, OzOperand &out, cudaStream_t st) {
  out.rows = 2 * rows;
  out.rows_pad = pad_to(2 * rows, kOzM);
  out.k = kOzK;
  out.k_pad = kOzK;
  const int64_t th = out.rows_pad / 2;
  note_launch();
  oz_slice_v_fwd_kernel<<<(unsigned)((th + 127) / 128), 128, 0, st>>>((const zd *)V, ldv, rows,
                                                                      (__nv_bfloat16 *)out.slices, out.expo,
                                                                      out.rows_pad);
  return cudaGetLastError();
}

cudaError_t launch_oz_slice_z(const void *Z, int64_t ldz, int64_t cols, OzOperand &out, cudaStream_t st) {
  out.rows = cols;
  out.rows_pad = pad_to(cols, kOzN);
  out.k = kOzK;
  out.k_pad = kOzK;
  note_launch();
  oz_slice_z_kernel<<<(unsigned)((out.rows_pad + 127) / 128), 128, 0, st>>>((const zd *)Z, ldz, cols,
                                                                            (__nv_bfloat16 *)out.slices, out.expo,
                                                                            out.rows_pad);
  return cudaGetLastError();
}

// K splits of the adjoint product: at most kOzKMax real K per CTA (the exact levels), and
// enough splits for about two CTAs per SM
static int oz_adj_splits(int64_t rows, int64_t cols, int sms, int *kb_per) {
  const int64_t nkb = pad_to(2 * rows, kOzK) / kOzK;
  const int64_t mt = pad_to(cols, kOzM) / kOzM;
  int64_t per = kOzKMax / kOzK;                       // K-blocks per split, at most
  int64_t splits = (nkb + per - 1) / per;
  while (mt * splits < 2 * sms && splits < nkb) ++splits;
  per = (nkb + splits - 1) / splits;
  splits = (nkb + per - 1) / per;
  *kb_per = (int)per;
  return (int)splits;
}

// splits x padded rows of the partial sums, bounded for every rows <= l, cols <= m: the split
// loop stops once splits x M-tiles reaches 2 sms (so at most 2 sms + mt - 1), or starts above it
// at ceil(K-blocks / 128) splits
size_t oz_adj_partial_bytes(int64_t l, int64_t m, int sms) {
  const int64_t mt = pad_to(m, kOzM) / kOzM, nkb = pad_to(2 * l, kOzK) / kOzK;
  const int64_t tiles = std::max<int64_t>(2 * (int64_t)sms + mt, (nkb / (kOzKMax / kOzK) + 1) * mt);
  return sizeof(double) * (size_t)tiles * kOzM * 64;
}

__global__ void oz_adj_reduce_kernel(const double *__restrict__ part, int splits, int64_t rows_pad, int64_t cols,
                                     zd *__restrict__ W, int64_t ldw) {
  // W[j, c] = conj(D[c][j] + i D[c][32 + j]) summed over the splits
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= cols * 32) return;
  const int64_t c = e / 32;
  const int j = (int)(e % 32);
  double re = 0.0, im = 0.0;
  for (int s = 0; s < splits; ++s) {
    const double *d = part + ((int64_t)s * rows_pad + c) * 64;
    re += d[j];
    im += d[32 + j];
  }
  W[c * ldw + j] = {re, -im};
}

cudaError_t launch_oz_adj(const OzAdjArgs &a, cudaStream_t st) {
  if (a.cols < 1) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  CUtensorMap amap, bmap;
  if ((e = oz_map(a.a, kOzM, &amap)) != cudaSuccess) return e;
  if ((e = oz_map(a.b, kOzN, &bmap)) != cudaSuccess) return e;
  int per = 0;
  const int splits = oz_adj_splits(a.a.k / 2, a.cols, sms, &per);
  if (sizeof(double) * (size_t)splits * (size_t)a.a.rows_pad * 64 > a.part_bytes) return cudaErrorInvalidValue;
  OzParams P{};
  P.a_rows_pad = (int)a.a.rows_pad;
  P.b_rows_pad = (int)a.b.rows_pad;
  P.kb0_stride = per;
  P.nkb = (int)(a.a.k_pad / kOzK);
  P.ea = a.a.expo;
  P.eb = a.b.expo;
  P.part = a.part;
  P.part_rows = (int)a.a.rows_pad;
  P.err = a.err;
  P.limit_ns = a.limit_ns;
  if ((e = cudaFuncSetAttribute(oz_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem)) !=
      cudaSuccess)
    return e;
  note_launch();
  oz_gemm_kernel<false><<<dim3((unsigned)(a.a.rows_pad / kOzM), (unsigned)splits, 2u), kOzThreads, kOzSmem, st>>>(
      amap, bmap, P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  note_launch();
  oz_adj_reduce_kernel<<<(unsigned)((a.cols * 32 + 255) / 256), 256, 0, st>>>(a.part, splits, a.a.rows_pad, a.cols,
                                                                              (zd *)a.W, a.ldw);
  return cudaGetLastError();
}

cudaError_t launch_oz_fwd(const OzFwdArgs &a, cudaStream_t st) {
  if (a.rows < 1 || a.cols < 1) return cudaSuccess;
  cudaError_t e;
  CUtensorMap amap, bmap;
  if ((e = oz_map(a.a, kOzM, &amap)) != cudaSuccess) return e;
  if ((e = oz_map(a.b, kOzN, &bmap)) != cudaSuccess) return e;
  OzParams P{};
  P.a_rows_pad = (int)a.a.rows_pad;
  P.b_rows_pad = (int)a.b.rows_pad;
  P.nkb = 1;
  P.ea = a.a.expo;
  P.eb = a.b.expo;
  P.C = (zd *)a.C;
  P.ldc = a.ldc;
  P.rows = (int)a.rows;
  P.cols = (int)a.cols;
  P.err = a.err;
  P.limit_ns = a.limit_ns;
  if ((e = cudaFuncSetAttribute(oz_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem)) !=
      cudaSuccess)
    return e;
  note_launch();
  oz_gemm_kernel<true><<<dim3((unsigned)(a.a.rows_pad / kOzM), (unsigned)(a.b.rows_pad / kOzN)), kOzThreads, kOzSmem,
                         st>>>(amap, bmap, P);
  return cudaGetLastError();
}

}  // namespace mn
