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
// row's entries below 2^e in magnitude) is truncated to N = floor(|x| 2^(55-e))
// < 2^55 (read off the FP64 bit pattern with integer shifts; no FP64
// instruction) and written in balanced base 256,
//     x ~ sign(x) 2^(e-7) sum_{s=0}^{6} d_s 256^-s,   d_0 in [0, 128], d_s in [-128, 127],
// an error below 2^(e-55) <= 2^-54 max|row|. Each d_s is an integer of at most
// 8 bits, exact in BF16. A product of two rows is then 2^(e+f-14) times the sum
// over the levels L = s + t of 256^-L I_L, I_L = sum_k sum_{s+t=L} d_s d'_t. The
// levels L <= 7 are kept (34 pairs; the dropped ones add at most K 2^(e+f) 5.02
// 2^-64 <= K 2^-59.3 max|a| max|b|). A level has at most 7 pairs and every
// product is an integer of magnitude <= 2^14, so over 128 real terms (two
// K-blocks) a level's sum is an integer below 7 2^21 < 2^24 and the tensor
// cores' FP32 accumulation of it is EXACT (one accumulator per level: 8 x 64 =
// all 512 columns of tensor memory). Every two K-blocks the epilogue warps move
// the levels into exact int64 sums, Ih = sum_{L<=3} I_L 256^(3-L) and Il =
// sum_{L>=4} I_L 256^(7-L); at the end Ih + Il 2^-32 is rounded once to FP64.
// K splits across CTAs are added in FP64. The product is as accurate as an FP64
// dot product (normwise), at the tensor cores' BF16 rate divided by 34.
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

constexpr int kOzEpiWarps = 16;                   // epilogue: 4 lane quarters x 4 column quarters
constexpr int kOzThreads = 32 * (4 + kOzEpiWarps);
constexpr int kOzRing = 6;                        // A slice tiles in flight
constexpr int kOzATile = kOzM * kOzK * 2;         // 16 KB: 128 rows x 64 BF16
constexpr int kOzBTile = kOzN * kOzK * 2;         // 8 KB: 64 rows x 64 BF16
constexpr int kOzTmemCols = kOzLevels * kOzN;     // 512
constexpr int kOzOffB = kOzRing * kOzATile;       // 96 KB
constexpr int kOzOffBar = kOzOffB + 2 * kOzSlices * kOzBTile;  // + 112 KB: two sets of B slices
constexpr int kOzSmem = kOzOffBar + 512 + 1024;   // barriers + alignment slack

// exponent of a row: the least e with every |x| < 2^e (the FP64 exponent field of the
// largest entry, plus one); -2000 for a zero row
__device__ __forceinline__ int oz_expo_of(double x) {
  const long long b = __double_as_longlong(x);
  const int f = (int)((b >> 52) & 0x7ff);
  return f == 0 ? -2000 : f - 1023 + 1;
}

// the 7 balanced base-256 digits of x for row exponent e, signed, as BF16
__device__ __forceinline__ void oz_slices(double x, int e, __nv_bfloat16 (&q)[kOzSlices]) {
  const long long b = __double_as_longlong(x);
  const int f = (int)((b >> 52) & 0x7ff);
  unsigned long long N = 0;
  if (f != 0 && e > -2000) {
    const unsigned long long mant = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = e - (f - 1023);  // >= 1: |x| < 2^e
    // floor(|x| 2^(55 - e)) = floor(mant 2^(3 - sh)) < 2^55
    N = sh <= 3 ? (mant << (3 - sh)) : (sh - 3 < 64 ? (mant >> (sh - 3)) : 0ull);
  }
  const float sgn = b < 0 ? -1.0f : 1.0f;
  int carry = 0;
#pragma unroll
  for (int s = kOzSlices - 1; s >= 1; --s) {
    const int r = (int)((N >> (8 * (kOzSlices - 1 - s))) & 255ull) + carry;   // 0..256
    carry = r >= 128 ? 1 : 0;
    q[s] = __float2bfloat16_rn(sgn * (float)(r - (carry << 8)));            // -128..127, exact
  }
  q[0] = __float2bfloat16_rn(sgn * (float)((int)(N >> 48) + carry));        // 0..128, exact
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

__device__ __forceinline__ bool elect_one() {
  uint32_t p = 0;
  asm volatile("{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n selp.u32 %0, 1, 0, e;\n}\n" : "=r"(p));
  return p != 0;
}
__device__ __forceinline__ void bar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
// 16 consecutive 32-bit columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// Tile: A rows [128 ma, +128), B rows [64 nb, +64), K-blocks [kb0, kb1). Adjoint: grid
// (A tiles, K splits), nb = 0; update: grid (A tiles, B tiles), one K-block.
// Roles: warp 0 lane 0 issues the TMA loads (the 7 B slice tiles of a K-block into one of two
// sets, the A slice tiles through a 6-deep ring); warp 1 runs the product loop converged, one
// elected lane issuing the MMAs and the commits that free the tiles; warp 2 owns the tensor
// memory; warps 4-19 drain the 8 level accumulators every kOzDrain K-blocks (warp w reads TMEM
// lanes 32 (w & 3) + lane = tile rows, columns 16 ((w - 4) >> 2) + 0..15) and write the result.
template <bool FWD>
__global__ void __launch_bounds__(kOzThreads, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
               const OzParams P) {
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;
  unsigned char *sB = base + kOzOffB;              // [2][kOzSlices] tiles
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + kOzOffBar);
  uint64_t *a_full = bars;                         // kOzRing
  uint64_t *a_empty = bars + kOzRing;              // kOzRing
  uint64_t *b_full = bars + 2 * kOzRing;           // 2 x kOzSlices
  uint64_t *b_empty = b_full + 2 * kOzSlices;      // 2 x kOzSlices
  uint64_t *acc_full = b_empty + 2 * kOzSlices;    // 1
  uint64_t *acc_empty = acc_full + 1;              // 1
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 1);
  __shared__ int s_abort;
  __shared__ int s_a_issued, s_a_used, s_b_issued, s_b_used;

  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int ma = blockIdx.x;
  const int nb = FWD ? blockIdx.y : 0;
  const int kb0 = FWD ? 0 : blockIdx.y * P.kb0_stride;
  const int kb1 = FWD ? 1 : min(P.nkb, kb0 + P.kb0_stride);
  const int nkb = kb1 - kb0;
  const int ndrain = (nkb + kOzDrain - 1) / kOzDrain;

  if (tid == 0) {
    for (int q = 0; q < kOzRing; ++q) { bar_init(&a_full[q], 1); bar_init(&a_empty[q], 1); }
    for (int t = 0; t < 2 * kOzSlices; ++t) { bar_init(&b_full[t], 1); bar_init(&b_empty[t], 1); }
    bar_init(acc_full, 1);
    bar_init(acc_empty, kOzEpiWarps);
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
    // producer: per K-block its 7 B tiles (set kk & 1, free once K-block kk - 2's products
    // are done with it), then its 7 A tiles through the ring; every wait is bounded
    int ai = 0, bi = 0;
    bool ok = true;
    for (int kk = 0; kk < nkb && ok; ++kk) {
      const int kb = kb0 + kk, set = kk & 1, use = kk >> 1;
      for (int t = 0; t < kOzSlices && ok; ++t) {
        uint64_t *fb = &b_full[set * kOzSlices + t];
        if (use > 0 && !bar_wait(&b_empty[set * kOzSlices + t], (uint32_t)((use - 1) & 1), P.limit_ns)) ok = false;
        if (!ok || *(volatile int *)&s_abort) { ok = false; break; }
        bar_expect(fb, kOzBTile);
        tma2d(sB + (set * kOzSlices + t) * kOzBTile, &bmap, kb * kOzK, t * P.b_rows_pad + nb * kOzN, fb);
        ++bi;
      }
      for (int s = 0; s < kOzSlices && ok; ++s) {
        const int slot = ai % kOzRing;
        if (ai >= kOzRing && !bar_wait(&a_empty[slot], (uint32_t)(((ai / kOzRing) - 1) & 1), P.limit_ns)) ok = false;
        if (!ok || *(volatile int *)&s_abort) { ok = false; break; }
        bar_expect(&a_full[slot], kOzATile);
        tma2d(sA + slot * kOzATile, &amap, kb * kOzK, s * P.a_rows_pad + ma * kOzM, &a_full[slot]);
        ++ai;
      }
    }
    if (!ok) atomicExch(&s_abort, 1);
    s_a_issued = ai;
    s_b_issued = bi;
  } else if (nkb > 0 && wid == 1) {
    // products: pair (s, t), s + t <= 7, t <= 6, into the accumulator of level s + t; the first
    // pair of a level in an accumulation period ((0, L), or (1, 6) for level 7) overwrites it.
    // B_t has its last pair at s = 7 - t (B_1 and B_0 at s = 6).
    int ai = 0, bu = 0;
    bool ok = true;
    constexpr uint32_t id = idesc(kOzN);
    const uint64_t a_desc0 = sdesc(sa(sA)), b_desc0 = sdesc(sa(sB));
    for (int kk = 0; kk < nkb && ok; ++kk) {
      const int set = kk & 1, use = kk >> 1, per = kk % kOzDrain;
      // every wait's outcome is made warp-uniform: the lanes stay converged for elect.sync
      if (per == 0 && kk > 0)
        ok = __all_sync(0xffffffffu, bar_wait(acc_empty, (uint32_t)(((kk / kOzDrain) - 1) & 1), P.limit_ns));
      for (int t = 0; t < kOzSlices && ok; ++t)
        ok = __all_sync(0xffffffffu, bar_wait(&b_full[set * kOzSlices + t], (uint32_t)(use & 1), P.limit_ns));
      if (ok) bu += kOzSlices;
      const uint64_t bset = b_desc0 + (uint64_t)((set * kOzSlices * kOzBTile) >> 4);
#pragma unroll
      for (int s = 0; s < kOzSlices; ++s) {
        const int slot = ai % kOzRing;
        if (ok) ok = __all_sync(0xffffffffu, bar_wait(&a_full[slot], (uint32_t)((ai / kOzRing) & 1), P.limit_ns));
        if (!ok || __any_sync(0xffffffffu, *(volatile int *)&s_abort != 0)) { ok = false; break; }
        tc_fence_after();
        const uint64_t ad = a_desc0 + (uint64_t)((slot * kOzATile) >> 4);
        if (elect_one()) {
#pragma unroll
          for (int t = 0; t < kOzSlices; ++t) {
            if (s + t < kOzLevels) {
              const uint32_t d = tmem + (uint32_t)((s + t) * kOzN);
              const uint64_t bd = bset + (uint64_t)((t * kOzBTile) >> 4);
              const bool first = per == 0 && (s == 0 || (s == 1 && t == kOzSlices - 1));
#pragma unroll
              for (int k16 = 0; k16 < kOzK / 16; ++k16)
                mma_bf16(d, ad + 2 * k16, bd + 2 * k16, id, (first && k16 == 0) ? 0u : 1u);
            }
          }
          mma_commit(&a_empty[slot]);                                   // A_s read
          if (s >= 1) mma_commit(&b_empty[set * kOzSlices + kOzLevels - 1 - s]);   // B_{7-s}: its last pair
          if (s == kOzSlices - 1) mma_commit(&b_empty[set * kOzSlices]);             // and B_0 at s = 6
        }
        __syncwarp();
        ++ai;
      }
      if (ok && (per == kOzDrain - 1 || kk == nkb - 1)) {
        if (elect_one()) mma_commit(acc_full);
        __syncwarp();
      }
    }
    if (!ok && lane == 0) atomicExch(&s_abort, 1);
    if (lane == 0) {
      s_a_used = ai;
      s_b_used = bu;
    }
  }

  // epilogue: warps 4-19
  bool good = true;
  if (wid >= 4) {
    const int q = wid & 3, h = (wid - 4) >> 2;
    const int row = 32 * q + lane;                    // tile row (TMEM lane)
    const int ga = ma * kOzM + row;                   // A row
    long long Ih[16], Il[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) { Ih[k] = 0; Il[k] = 0; }
    for (int dr = 0; dr < ndrain && good; ++dr) {
      bool ready = false;
      const uint64_t t0 = global_ns();
      while (!ready && !*(volatile int *)&s_abort) {
        ready = bar_try(acc_full, (uint32_t)(dr & 1));
        if (!ready && global_ns() - t0 > P.limit_ns) break;
      }
      good = __all_sync(0xffffffffu, ready);
      if (!good) break;
      tc_fence_after();
      float v[16];
#pragma unroll
      for (int L = 0; L < kOzLevels; ++L) {
        tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(L * kOzN + 16 * h), v);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const long long I = (long long)__float2int_rn(v[k]);   // an integer below 2^24: exact
          if (L < 4) Ih[k] += I * (long long)(1 << (8 * (3 - L)));
          else Il[k] += I * (long long)(1 << (8 * (7 - L)));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) bar_arrive(acc_empty);
    }
    if (good) {
      const int ea = P.ea[ga];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int col = 16 * h + k;
        const int eb = P.eb[nb * kOzN + col];
        // sum_L I_L 256^-L = 2^-24 (Ih + 2^-32 Il): carry Il's high part into Ih (exact), then
        // one rounding; the product is 2^(ea + eb - 14) times that sum
        const long long hi = Ih[k] + (Il[k] >> 32);
        const long long lo = Il[k] & 0xFFFFFFFFll;
        double r = fma((double)lo, 0x1.0p-32, (double)hi);
        const int sc = ea + eb - 38;
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
          P.part[((int64_t)blockIdx.y * P.part_rows + ga) * kOzN + col] = r;
        }
      }
    } else if (!good) {
      atomicExch(&s_abort, 1);
    }
  }
  __syncthreads();
  if (s_abort && tid == 0) {
    atomicExch(P.err, 1);
    // loads still in flight: the A tiles issued but not taken, the B tiles likewise (bounded)
    for (int q = s_a_used; q < s_a_issued; ++q) bar_wait(&a_full[q % kOzRing], (uint32_t)((q / kOzRing) & 1), P.limit_ns);
    for (int q = s_b_used; q < s_b_issued; ++q) {
      const int kk = q / kOzSlices, t = q % kOzSlices;
      bar_wait(&b_full[(kk & 1) * kOzSlices + t], (uint32_t)((kk >> 1) & 1), P.limit_ns);
    }
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

// K splits of the adjoint product: at most kOzKbMax K-blocks per CTA (the int64 level sums
// stay exact in FP64), and as many splits as fit one wave of CTAs (one per SM) beside the
// M-tiles, at least one K-block each
static int oz_adj_splits(int64_t rows, int64_t cols, int sms, int *kb_per) {
  const int64_t nkb = pad_to(2 * rows, kOzK) / kOzK;
  const int64_t mt = pad_to(cols, kOzM) / kOzM;
  int64_t splits = std::max<int64_t>(1, sms / mt);
  splits = std::max<int64_t>(splits, (nkb + kOzKbMax - 1) / kOzKbMax);
  splits = std::min<int64_t>(splits, nkb);
  const int64_t per = (nkb + splits - 1) / splits;
  *kb_per = (int)per;
  return (int)((nkb + per - 1) / per);
}

// splits x padded rows of the partial sums, bounded for every rows <= l, cols <= m: the splits
// are at most max(sms / mt, ceil(K-blocks / kOzKbMax)), so splits x mt <= max(sms, (K-blocks /
// kOzKbMax + 1) mt)
size_t oz_adj_partial_bytes(int64_t l, int64_t m, int sms) {
  const int64_t mt = pad_to(m, kOzM) / kOzM, nkb = pad_to(2 * l, kOzK) / kOzK;
  const int64_t tiles = std::max<int64_t>((int64_t)sms + mt, (nkb / kOzKbMax + 1) * mt);
  return sizeof(double) * (size_t)tiles * kOzM * kOzN;
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
    const double *d = part + ((int64_t)s * rows_pad + c) * kOzN;
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
  if (sizeof(double) * (size_t)splits * (size_t)a.a.rows_pad * kOzN > a.part_bytes) return cudaErrorInvalidValue;
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
  oz_gemm_kernel<false><<<dim3((unsigned)(a.a.rows_pad / kOzM), (unsigned)splits), kOzThreads, kOzSmem, st>>>(
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
