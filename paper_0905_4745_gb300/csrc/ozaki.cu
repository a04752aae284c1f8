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
// row's entries below 2^e in magnitude) is truncated to N = floor(|x| 2^(8S-1-e))
// < 2^(8S-1) (read off the FP64 bit pattern with integer shifts; no FP64
// instruction) and written in balanced base 256,
//     x ~ sign(x) 2^(e-7) sum_{s<S} d_s 256^-s,   d_0 in [0, 128], d_s in [-128, 127],
// an error below 2^(e-8S+1) <= 2^(-8S+2) max|row|. Each d_s is an integer of at
// most 8 bits, exact in BF16. A product of two rows is then 2^(e+f-14) times the
// sum over the levels L = s + t of 256^-L I_L, I_L = sum_k sum_{s+t=L} d_s d'_t;
// the levels L < NL are kept. A level has at most 8 pairs and every product is an
// integer of magnitude <= 2^14, so over 128 real terms (two K-blocks) a level's
// sum is an integer of magnitude <= 2^24 and the tensor cores' FP32 accumulation
// of it is EXACT (one accumulator per level in tensor memory). Every two
// K-blocks the epilogue warps move the levels into exact int64 sums; at the end
// the sum is rounded once to FP64. K splits across CTAs are added with a
// compensated sum (one rounding in all). Two shapes:
//   adjoint (K up to the sketch's l): S = 8 (63 bits), NL = 9 (43 pairs), 32-column
//     tiles; dropped levels <= K 2^-67.4 max|a| max|b|: within a few units of
//     2^-53 |a|^T |b| at any K, as accurate as an FP64 dot product
//   update (K = 64 real): S = 7 (55 bits), NL = 8 (34 pairs), 64-column tiles;
//     dropped levels <= K 2^-59.6 max|a| max|b|
// at the tensor cores' BF16 rate divided by the pair count.
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
constexpr int kOzTmemCols = 512;

template <int S, int NT>
struct OzShape {
  static constexpr int kBTile = NT * kOzK * 2;                  // NT rows x 64 BF16
  static constexpr int kOffB = kOzRing * kOzATile;              // 96 KB of A ring
  static constexpr int kOffBar = kOffB + 2 * S * kBTile;        // two sets of B slices
  static constexpr int kSmem = kOffBar + 512 + 1024;            // barriers + alignment slack
};

// exponent of a row: the least e with every |x| < 2^e (the FP64 exponent field of the
// largest entry, plus one); -2000 for a zero row
__device__ __forceinline__ int oz_expo_of(double x) {
  const long long b = __double_as_longlong(x);
  const int f = (int)((b >> 52) & 0x7ff);
  return f == 0 ? -2000 : f - 1023 + 1;
}

// the S balanced base-256 digits of x for row exponent e (N = floor(|x| 2^(8S - 1 - e)) <
// 2^(8S - 1)), signed, as BF16
template <int S>
__device__ __forceinline__ void oz_slices(double x, int e, __nv_bfloat16 (&q)[S]) {
  static_assert(S == 7 || S == 8, "7 or 8 slices");
  constexpr int kb = 8 * S - 1;   // bits kept below 2^e
  const long long b = __double_as_longlong(x);
  const int f = (int)((b >> 52) & 0x7ff);
  unsigned long long N = 0;
  if (f != 0 && e > -2000) {
    const unsigned long long mant = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = e - (f - 1023);  // >= 1: |x| < 2^e
    // floor(|x| 2^(kb - e)) = floor(mant 2^(kb - 52 - sh)) < 2^kb
    N = sh <= kb - 52 ? (mant << (kb - 52 - sh)) : (sh - (kb - 52) < 64 ? (mant >> (sh - (kb - 52))) : 0ull);
  }
  const float sgn = b < 0 ? -1.0f : 1.0f;
  int carry = 0;
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const int r = (int)((N >> (8 * (S - 1 - s))) & 255ull) + carry;   // 0..256
    carry = r >= 128 ? 1 : 0;
    q[s] = __float2bfloat16_rn(sgn * (float)(r - (carry << 8)));      // -128..127, exact
  }
  q[0] = __float2bfloat16_rn(sgn * (float)((int)(N >> (8 * (S - 1))) + carry));   // 0..128, exact
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
template <int NS>
__device__ __forceinline__ void oz_put2(__nv_bfloat16 *S, int64_t sstride, int64_t kpad, int64_t row, int64_t k,
                                        const __nv_bfloat16 (&a)[NS], const __nv_bfloat16 (&b)[NS]) {
#pragma unroll
  for (int s = 0; s < NS; ++s) {
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
    __nv_bfloat16 a[kOzSlicesAdj], b[kOzSlicesAdj];
    const zd v = r < rows ? col[r] : zd{0.0, 0.0};
    oz_slices<kOzSlicesAdj>(v.re, e, a);
    oz_slices<kOzSlicesAdj>(v.im, e, b);
    oz_put2<kOzSlicesAdj>(S, ss, kpad, c, 2 * r, a, b);
  }
}

// B rows of the adjoint product from the 32 reflectors: CTA (j, chunk) writes reflector j's two
// rows for its chunk of the K positions; every CTA of a reflector forms the same exponent from
// the whole column (read from L2), so the chunks need no second pass
constexpr int kOzVadjChunks = 8;
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
  if (threadIdx.x == 0 && blockIdx.y == 0) { expo[j] = e; expo[32 + j] = e; }
  const int64_t ss = (int64_t)64 * kpad;
  const int64_t np = kpad / 2, r0 = np * blockIdx.y / gridDim.y, r1 = np * (blockIdx.y + 1) / gridDim.y;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    __nv_bfloat16 a[kOzSlicesAdj], b[kOzSlicesAdj], na[kOzSlicesAdj];
    const zd v = r < rows ? col[r] : zd{0.0, 0.0};
    oz_slices<kOzSlicesAdj>(v.re, e, a);
    oz_slices<kOzSlicesAdj>(v.im, e, b);
    oz_slices<kOzSlicesAdj>(-v.re, e, na);
    oz_put2<kOzSlicesAdj>(S, ss, kpad, j, 2 * r, a, b);         // (Re, Im)
    oz_put2<kOzSlicesAdj>(S, ss, kpad, 32 + j, 2 * r, b, na);   // (Im, -Re)
  }
}

// A rows of the update: one warp per row i of V (two rows 2i, 2i+1, K = 64), lane j = column j;
// the row's exponent is the warp's maximum
__global__ void __launch_bounds__(256)
oz_slice_v_fwd_kernel(const zd *__restrict__ V, int64_t ldv, int64_t rows, __nv_bfloat16 *__restrict__ S,
                      int32_t *__restrict__ expo, int64_t rows_pad) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (2 * i >= rows_pad) return;   // warp-uniform
  const int64_t ss = rows_pad * kOzK;
  const zd v = i < rows ? V[(int64_t)lane * ldv + i] : zd{0.0, 0.0};
  int e = max(oz_expo_of(v.re), oz_expo_of(v.im));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (lane == 0) {
    expo[2 * i] = e;
    expo[2 * i + 1] = e;
  }
  __nv_bfloat16 re[kOzSlicesFwd], im[kOzSlicesFwd], nim[kOzSlicesFwd];
  oz_slices<kOzSlicesFwd>(v.re, e, re);
  oz_slices<kOzSlicesFwd>(v.im, e, im);
  oz_slices<kOzSlicesFwd>(-v.im, e, nim);
  oz_put2<kOzSlicesFwd>(S, ss, kOzK, 2 * i, 2 * lane, re, nim);    // (Re V, -Im V)
  oz_put2<kOzSlicesFwd>(S, ss, kOzK, 2 * i + 1, 2 * lane, im, re); // (Im V, Re V)
}

// B rows of the update: one warp per column c of Z (32 x cols, column-major), lane j = row j
__global__ void __launch_bounds__(256)
oz_slice_z_kernel(const zd *__restrict__ Z, int64_t ldz, int64_t cols, __nv_bfloat16 *__restrict__ S,
                  int32_t *__restrict__ expo, int64_t rows_pad) {
  const int lane = threadIdx.x & 31;
  const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (c >= rows_pad) return;   // warp-uniform
  const int64_t ss = rows_pad * kOzK;
  const zd z = c < cols ? Z[c * ldz + lane] : zd{0.0, 0.0};
  int e = max(oz_expo_of(z.re), oz_expo_of(z.im));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (lane == 0) expo[c] = e;
  __nv_bfloat16 re[kOzSlicesFwd], im[kOzSlicesFwd];
  oz_slices<kOzSlicesFwd>(z.re, e, re);
  oz_slices<kOzSlicesFwd>(z.im, e, im);
  oz_put2<kOzSlicesFwd>(S, ss, kOzK, c, 2 * lane, re, im);
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
  // update: C[i, c] -= (V Z)[i, c] for i < rows, c < cols
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
// C consecutive 32-bit columns (8 or 16) of this warp's 32 lanes
template <int C>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float (&v)[C]) {
  uint32_t r[C];
  if constexpr (C == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
  } else {
    static_assert(C == 8, "8 or 16 columns");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < C; ++k) v[k] = __uint_as_float(r[k]);
}

// The adjoint product W^H = C^H V. Tile: A rows [128 ma, +128), B rows [NT nb, +NT), K-blocks
// [kb0, kb1); grid (A tiles, K splits, B tiles). S slices, the levels s + t < NL kept; the FP64
// partial sums of a K split go to part[split][A row][64].
// Roles: warp 0 lane 0 issues the TMA loads (the S B slice tiles of a K-block into one of two
// sets, the A slice tiles through a 6-deep ring); warp 1 runs the product loop converged, one
// elected lane issuing the MMAs and the commits that free the tiles; warp 2 owns the tensor
// memory; warps 4-19 drain the NL level accumulators every kOzDrain K-blocks (warp w reads TMEM
// lanes 32 (w & 3) + lane = tile rows, columns NT/4 ((w - 4) >> 2) + 0..NT/4-1) and write the
// result.
template <int S, int NL, int NT>
__global__ void __launch_bounds__(kOzThreads, 1)
oz_adj_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
              const OzParams P) {
  using SH = OzShape<S, NT>;
  static_assert(NL * NT <= kOzTmemCols && NL <= 9 && NL >= S, "levels x columns within tensor memory");
  constexpr int CPT = NT / 4;                       // columns per epilogue thread
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;
  unsigned char *sB = base + SH::kOffB;            // [2][S] tiles
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + SH::kOffBar);
  uint64_t *a_full = bars;                         // kOzRing
  uint64_t *a_empty = bars + kOzRing;              // kOzRing
  uint64_t *b_full = bars + 2 * kOzRing;           // 2 x S
  uint64_t *b_empty = b_full + 2 * S;              // 2 x S
  uint64_t *acc_full = b_empty + 2 * S;            // 1
  uint64_t *acc_empty = acc_full + 1;              // 1
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 1);
  __shared__ int s_abort;
  __shared__ int s_a_issued, s_a_used, s_b_issued, s_b_used;

  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int ma = blockIdx.x;
  const int nb = blockIdx.z;
  const int kb0 = blockIdx.y * P.kb0_stride;
  const int kb1 = min(P.nkb, kb0 + P.kb0_stride);
  const int nkb = kb1 - kb0;
  const int ndrain = (nkb + kOzDrain - 1) / kOzDrain;

  if (tid == 0) {
    for (int q = 0; q < kOzRing; ++q) { bar_init(&a_full[q], 1); bar_init(&a_empty[q], 1); }
    for (int t = 0; t < 2 * S; ++t) { bar_init(&b_full[t], 1); bar_init(&b_empty[t], 1); }
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
    // producer: per K-block its S B tiles (set kk & 1, free once K-block kk - 2's products
    // are done with it), then its S A tiles through the ring; every wait is bounded
    int ai = 0, bi = 0;
    bool ok = true;
    for (int kk = 0; kk < nkb && ok; ++kk) {
      const int kb = kb0 + kk, set = kk & 1, use = kk >> 1;
      for (int t = 0; t < S && ok; ++t) {
        uint64_t *fb = &b_full[set * S + t];
        if (use > 0 && !bar_wait(&b_empty[set * S + t], (uint32_t)((use - 1) & 1), P.limit_ns)) ok = false;
        if (!ok || *(volatile int *)&s_abort) { ok = false; break; }
        bar_expect(fb, SH::kBTile);
        tma2d(sB + (set * S + t) * SH::kBTile, &bmap, kb * kOzK, t * P.b_rows_pad + nb * NT, fb);
        ++bi;
      }
      for (int s = 0; s < S && ok; ++s) {
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
    // products: pair (s, t), s + t < NL, into the accumulator of level s + t; the first pair of
    // a level in an accumulation period (the least s, t = L - s <= S - 1) overwrites it. B_t has
    // its last pair at s = min(S - 1, NL - 1 - t). Every wait's outcome is made warp-uniform:
    // the lanes stay converged for elect.sync.
    int ai = 0, bu = 0;
    bool ok = true;
    constexpr uint32_t id = idesc(NT);
    const uint64_t a_desc0 = sdesc(sa(sA)), b_desc0 = sdesc(sa(sB));
    for (int kk = 0; kk < nkb && ok; ++kk) {
      const int set = kk & 1, use = kk >> 1, per = kk % kOzDrain;
      if (per == 0 && kk > 0)
        ok = __all_sync(0xffffffffu, bar_wait(acc_empty, (uint32_t)(((kk / kOzDrain) - 1) & 1), P.limit_ns));
      for (int t = 0; t < S && ok; ++t)
        ok = __all_sync(0xffffffffu, bar_wait(&b_full[set * S + t], (uint32_t)(use & 1), P.limit_ns));
      if (ok) bu += S;
      const uint64_t bset = b_desc0 + (uint64_t)((set * S * SH::kBTile) >> 4);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int slot = ai % kOzRing;
        if (ok) ok = __all_sync(0xffffffffu, bar_wait(&a_full[slot], (uint32_t)((ai / kOzRing) & 1), P.limit_ns));
        if (!ok || __any_sync(0xffffffffu, *(volatile int *)&s_abort != 0)) { ok = false; break; }
        tc_fence_after();
        const uint64_t ad = a_desc0 + (uint64_t)((slot * kOzATile) >> 4);
        if (elect_one()) {
#pragma unroll
          for (int t = 0; t < S; ++t) {
            if (s + t < NL) {
              const int L = s + t;
              const uint32_t d = tmem + (uint32_t)(L * NT);
              const uint64_t bd = bset + (uint64_t)((t * SH::kBTile) >> 4);
              const bool first = per == 0 && s == (L > S - 1 ? L - (S - 1) : 0);
#pragma unroll
              for (int k16 = 0; k16 < kOzK / 16; ++k16)
                mma_bf16(d, ad + 2 * k16, bd + 2 * k16, id, (first && k16 == 0) ? 0u : 1u);
            }
          }
          mma_commit(&a_empty[slot]);                   // A_s read
#pragma unroll
          for (int t = 0; t < S; ++t)                   // the B tiles whose last pair this was
            if (s == (NL - 1 - t < S - 1 ? NL - 1 - t : S - 1)) mma_commit(&b_empty[set * S + t]);
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

  // epilogue: warps 4-19. Exact int64 sums of the levels: G0 = sum_{L<=3} I_L 256^(3-L),
  // G1 = sum_{4<=L<=7} I_L 256^(7-L), G2 = I_8, so that sum_L I_L 256^-L = 256^-3 (G0 +
  // 2^-32 G1 + 2^-40 G2)
  bool good = true;
  if (wid >= 4) {
    const int q = wid & 3, h = (wid - 4) >> 2;
    const int row = 32 * q + lane;                    // tile row (TMEM lane)
    const int ga = ma * kOzM + row;                   // A row
    long long G0[CPT], G1[CPT], G2[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) { G0[k] = 0; G1[k] = 0; G2[k] = 0; }
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
      float v[CPT];
#pragma unroll
      for (int L = 0; L < NL; ++L) {
        tmem_ld<CPT>(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(L * NT + CPT * h), v);
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
          const long long I = (long long)__float2int_rn(v[k]);   // an integer of magnitude <= 2^24: exact
          if (L < 4) G0[k] += I * (long long)(1 << (8 * (3 - L)));
          else if (L < 8) G1[k] += I * (long long)(1 << (8 * (7 - L)));
          else G2[k] += I;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) bar_arrive(acc_empty);
    }
    if (good) {
      const int ea = P.ea[ga];
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int col = CPT * h + k;
        const int eb = P.eb[nb * NT + col];
        // carry the low sums' high parts upwards (exact), then one rounding: G0 < 2^53,
        // G1 + 2^-8 G2 < 2^32 is exact in FP64; the product is 2^(ea + eb - 38) times the sum
        long long g1 = G1[k] + (G2[k] >> 8);
        const long long g2 = G2[k] & 255ll;
        const long long g0 = G0[k] + (g1 >> 32);
        g1 &= 0xFFFFFFFFll;
        double r = fma(fma((double)g2, 0x1.0p-8, (double)g1), 0x1.0p-32, (double)g0);
        const int sc = ea + eb - 38;
        if (ea <= -2000 || eb <= -2000) r = 0.0;
        else if (sc >= -1022 && sc <= 1023) r *= __longlong_as_double((long long)(sc + 1023) << 52);  // 2^sc
        else r = ldexp(r, sc);
        P.part[((int64_t)blockIdx.y * P.part_rows + ga) * 64 + nb * NT + col] = r;
      }
    } else {
      atomicExch(&s_abort, 1);
    }
  }
  __syncthreads();
  if (s_abort && tid == 0) {
    atomicExch(P.err, 1);
    // loads still in flight: the A tiles issued but not taken, the B tiles likewise (bounded)
    for (int q = s_a_used; q < s_a_issued; ++q) bar_wait(&a_full[q % kOzRing], (uint32_t)((q / kOzRing) & 1), P.limit_ns);
    for (int q = s_b_used; q < s_b_issued; ++q) {
      const int kk = q / S, t = q % S;
      bar_wait(&b_full[(kk & 1) * S + t], (uint32_t)((kk >> 1) & 1), P.limit_ns);
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

// The update C -= V Z as a persistent kernel. The (row tile, column tile) items (row tiles of 128
// rows of the real form of V, column tiles of 32 columns of Z; column tiles innermost) are dealt
// to the CTAs in equal contiguous shares, so every SM has work even when the update has fewer
// row tiles than SMs (short, wide updates). A CTA loads a row tile's S A slices when its share
// enters that row tile (at most a few times) and keeps them in shared memory while the column
// tiles of Z stream through two B buffers; the level accumulators of a column tile (8 levels x
// 32 TMEM columns) alternate between the two halves of tensor memory, so the epilogue of one
// column tile overlaps the products of the next. Roles as in oz_adj_kernel (warp 0 loads, warp
// 1 multiplies, warp 2 owns tensor memory, warps 4-19 drain and write).
constexpr int kOzFwdNT = 32;
struct OzFwdShape {
  static constexpr int kBTile = kOzFwdNT * kOzK * 2;                  // 4 KB
  static constexpr int kOffB = kOzSlicesFwd * kOzATile;               // 112 KB: the row tile's A slices
  static constexpr int kOffBar = kOffB + 2 * kOzSlicesFwd * kBTile;   // + 56 KB: two sets of B slices
  static constexpr int kSmem = kOffBar + 256 + 1024;
};

__global__ void __launch_bounds__(kOzThreads, 1)
oz_fwd_persistent_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                         const OzParams P, int n_row_tiles, int n_col_tiles) {
  constexpr int S = kOzSlicesFwd, NL = kOzLevelsFwd, NT = kOzFwdNT, CPT = NT / 4;
  static_assert(2 * NL * NT <= kOzTmemCols, "two accumulator sets in tensor memory");
  using SH = OzFwdShape;
  extern __shared__ unsigned char oz_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)oz_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base;
  unsigned char *sB = base + SH::kOffB;               // [2][S] tiles
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + SH::kOffBar);
  uint64_t *a_full = bars, *a_empty = bars + 1;
  uint64_t *b_full = bars + 2, *b_empty = bars + 4;   // 2 each
  uint64_t *acc_full = bars + 6, *acc_empty = bars + 8;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 10);
  __shared__ int s_abort;
  __shared__ int s_a_issued, s_a_used, s_b_issued, s_b_used;

  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int64_t n_items = (int64_t)n_row_tiles * n_col_tiles;
  const int64_t item0 = n_items * blockIdx.x / gridDim.x;
  const int ntiles = (int)(n_items * (blockIdx.x + 1) / gridDim.x - item0);   // this CTA's items

  if (tid == 0) {
    bar_init(a_full, 1);
    bar_init(a_empty, 1);
    for (int q = 0; q < 2; ++q) {
      bar_init(&b_full[q], 1);
      bar_init(&b_empty[q], 1);
      bar_init(&acc_full[q], 1);
      bar_init(&acc_empty[q], kOzEpiWarps);
    }
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

  if (ntiles > 0 && wid == 0 && lane == 0) {
    // producer: a row tile's A slices once the previous row tile's products are done with them,
    // then one B set per column tile once the products two tiles back have read it
    int ai = 0, bi = 0;
    bool ok = true;
    for (int it = 0; it < ntiles && ok; ++it) {
      const int64_t gi = item0 + it;
      const int rt = (int)(gi / n_col_tiles), ct = (int)(gi - (int64_t)rt * n_col_tiles);
      if (it == 0 || ct == 0) {   // the share enters row tile rt: its A slices, once the products
                                  // of the previous row tile are done with the buffer
        if (ai > 0 && !bar_wait(a_empty, (uint32_t)((ai - 1) & 1), P.limit_ns)) { ok = false; break; }
        bar_expect(a_full, S * kOzATile);
        for (int s = 0; s < S; ++s) tma2d(sA + s * kOzATile, &amap, 0, s * P.a_rows_pad + rt * kOzM, a_full);
        ++ai;
      }
      const int set = it & 1, use = it >> 1;
      if (use > 0 && !bar_wait(&b_empty[set], (uint32_t)((use - 1) & 1), P.limit_ns)) { ok = false; break; }
      if (*(volatile int *)&s_abort) { ok = false; break; }
      bar_expect(&b_full[set], S * SH::kBTile);
      for (int t = 0; t < S; ++t)
        tma2d(sB + (set * S + t) * SH::kBTile, &bmap, 0, t * P.b_rows_pad + ct * NT, &b_full[set]);
      ++bi;
    }
    if (!ok) atomicExch(&s_abort, 1);
    s_a_issued = ai;
    s_b_issued = bi;
  } else if (ntiles > 0 && wid == 1) {
    // products of a column tile: pair (s, t), s + t < NL, into the level accumulator s + t of the
    // tile's TMEM half (the first pair of each level overwrites it); the commits free the B set,
    // fill the accumulator half and, after a row tile's last column tile, free the A slices
    int au = 0, bu = 0;
    bool ok = true;
    constexpr uint32_t id = idesc(NT);
    const uint64_t a_desc0 = sdesc(sa(sA)), b_desc0 = sdesc(sa(sB));
    for (int it = 0; it < ntiles && ok; ++it) {
      const int64_t gi = item0 + it;
      const int ct = (int)(gi % n_col_tiles);
      const int set = it & 1, use = it >> 1;
      if (it == 0 || ct == 0) {
        ok = __all_sync(0xffffffffu, bar_wait(a_full, (uint32_t)(au & 1), P.limit_ns));
        if (!ok) break;
        ++au;
      }
      if (use > 0) ok = __all_sync(0xffffffffu, bar_wait(&acc_empty[set], (uint32_t)((use - 1) & 1), P.limit_ns));
      if (ok) ok = __all_sync(0xffffffffu, bar_wait(&b_full[set], (uint32_t)(use & 1), P.limit_ns));
      if (!ok || __any_sync(0xffffffffu, *(volatile int *)&s_abort != 0)) { ok = false; break; }
      ++bu;
      tc_fence_after();
      const uint64_t bset = b_desc0 + (uint64_t)((set * S * SH::kBTile) >> 4);
      const uint32_t dbase = tmem + (uint32_t)(set * NL * NT);
      if (elect_one()) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const uint64_t ad = a_desc0 + (uint64_t)((s * kOzATile) >> 4);
#pragma unroll
          for (int t = 0; t < S; ++t) {
            if (s + t < NL) {
              const int L = s + t;
              const uint32_t d = dbase + (uint32_t)(L * NT);
              const uint64_t bd = bset + (uint64_t)((t * SH::kBTile) >> 4);
              const bool first = s == (L > S - 1 ? L - (S - 1) : 0);
#pragma unroll
              for (int k16 = 0; k16 < kOzK / 16; ++k16)
                mma_bf16(d, ad + 2 * k16, bd + 2 * k16, id, (first && k16 == 0) ? 0u : 1u);
            }
          }
        }
        mma_commit(&b_empty[set]);
        mma_commit(&acc_full[set]);
        if (ct == n_col_tiles - 1 || it == ntiles - 1) mma_commit(a_empty);   // the row tile's last item
      }
      __syncwarp();
    }
    if (!ok && lane == 0) atomicExch(&s_abort, 1);
    if (lane == 0) {
      s_a_used = au;
      s_b_used = bu;
    }
  }

  // epilogue: warps 4-19; warp w reads TMEM lanes 32 (w & 3) + lane, columns CPT ((w - 4) >> 2) + 0..CPT-1
  if (wid >= 4) {
    const int q = wid & 3, h = (wid - 4) >> 2;
    const int row = 32 * q + lane;
    bool good = true;
    for (int it = 0; it < ntiles && good; ++it) {
      const int64_t gi = item0 + it;
      const int rt = (int)(gi / n_col_tiles), ct = (int)(gi - (int64_t)rt * n_col_tiles);
      const int set = it & 1, use = it >> 1;
      // the tile's entries of C first: their loads overlap the wait for the products and the drain
      const int ga = rt * kOzM + row;
      const int i = ga >> 1, p = ga & 1;
      double cv[CPT];
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int c = ct * NT + CPT * h + k;
        cv[k] = (i < P.rows && c < P.cols) ? reinterpret_cast<const double *>(P.C + (int64_t)c * P.ldc + i)[p] : 0.0;
      }
      bool ready = false;
      const uint64_t t0 = global_ns();
      while (!ready && !*(volatile int *)&s_abort) {
        ready = bar_try(&acc_full[set], (uint32_t)(use & 1));
        if (!ready && global_ns() - t0 > P.limit_ns) break;
      }
      good = __all_sync(0xffffffffu, ready);
      if (!good) break;
      tc_fence_after();
      long long G0[CPT], G1[CPT];
      float v[CPT];
#pragma unroll
      for (int k = 0; k < CPT; ++k) { G0[k] = 0; G1[k] = 0; }
#pragma unroll
      for (int L = 0; L < NL; ++L) {
        tmem_ld<CPT>(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(set * NL * NT + L * NT + CPT * h), v);
#pragma unroll
        for (int k = 0; k < CPT; ++k) {
          const long long I = (long long)__float2int_rn(v[k]);   // an integer of magnitude <= 2^24: exact
          if (L < 4) G0[k] += I * (long long)(1 << (8 * (3 - L)));
          else G1[k] += I * (long long)(1 << (8 * (7 - L)));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) bar_arrive(&acc_empty[set]);
      // C[i, c] -= 2^(ea + eb - 38) (G0 + 2^-32 G1)
      const int ea = P.ea[ga];
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        const int c = ct * NT + CPT * h + k;
        if (i < P.rows && c < P.cols) {
          const int eb = P.eb[c];
          // one K-block: |G0| <= 2^44.1 and |G1| <= 2^46.4, so G0 2^17 + G1 2^-15 fits an int64; the
          // dropped low 15 bits of G1 are below 2^(ea + eb - 55) <= 2^-53 max|v| max|z|. One
          // conversion, and the scale 2^(ea + eb - 55) added to the exponent field with an
          // integer add: two FP64-pipe instructions per output with the subtraction
          double r = 0.0;
          const long long comb = G0[k] * (1ll << 17) + (G1[k] >> 15);
          if (comb != 0 && ea > -2000 && eb > -2000) {
            r = (double)comb;
            const int sc = ea + eb - 55;
            const long long rb = __double_as_longlong(r);
            const int fe = (int)((rb >> 52) & 0x7ff) + sc;
            r = (fe >= 1 && fe <= 2046) ? __longlong_as_double(rb + ((long long)sc << 52)) : ldexp(r, sc);
          }
          reinterpret_cast<double *>(P.C + (int64_t)c * P.ldc + i)[p] = cv[k] - r;
        }
      }
    }
    if (!good) atomicExch(&s_abort, 1);
  }
  __syncthreads();
  if (s_abort && tid == 0) {
    atomicExch(P.err, 1);
    // loads still in flight (bounded waits): A row tiles and B sets issued but not taken
    for (int k = s_a_used; k < s_a_issued; ++k) bar_wait(a_full, (uint32_t)(k & 1), P.limit_ns);
    for (int k = s_b_used; k < s_b_issued; ++k) bar_wait(&b_full[k & 1], (uint32_t)((k >> 1) & 1), P.limit_ns);
    // products in flight: the last column tile's commit
    if (s_b_used > 0) {
      const int k = s_b_used - 1;
      bar_wait(&acc_full[k & 1], (uint32_t)((k >> 1) & 1), P.limit_ns);
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

// the slices of an operand as a 2-D BF16 array (k_pad wide, ns rows_pad rows) read in
// boxes of 64 (K) x box_rows, 128-byte swizzle: the K-major layout the MMA descriptors expect
cudaError_t oz_map(const OzOperand &o, uint32_t box_rows, CUtensorMap *map) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = oz_encode();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t gdim[2] = {(cuuint64_t)o.k_pad, (cuuint64_t)(o.ns * o.rows_pad)};
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

size_t oz_slice_bytes(int64_t rows, int64_t k, int ns) {
  return (size_t)ns * (size_t)pad_to(rows, kOzM) * (size_t)pad_to(k, kOzK) * sizeof(__nv_bfloat16);
}

cudaError_t launch_oz_slice_cols(const void *C, int64_t ldc, int64_t rows, int64_t cols, OzOperand &out,
                                 cudaStream_t st) {
  out.rows = cols;
  out.rows_pad = pad_to(cols, kOzM);
  out.k = 2 * rows;
  out.k_pad = pad_to(2 * rows, kOzK);
  out.ns = kOzSlicesAdj;
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
  out.ns = kOzSlicesAdj;
  note_launch();
  oz_slice_v_adj_kernel<<<dim3(32, kOzVadjChunks), 256, 0, st>>>((const zd *)V, ldv, rows, (__nv_bfloat16 *)out.slices,
                                                                 out.expo, out.k_pad);
  return cudaGetLastError();
}

cudaError_t launch_oz_slice_v_fwd(const void *V, int64_t ldv, int64_t rows, OzOperand &out, cudaStream_t st) {
  out.rows = 2 * rows;
  out.rows_pad = pad_to(2 * rows, kOzM);
  out.k = kOzK;
  out.k_pad = kOzK;
  out.ns = kOzSlicesFwd;
  const int64_t warps = out.rows_pad / 2;   // one per row of V, padding rows included
  note_launch();
  oz_slice_v_fwd_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>((const zd *)V, ldv, rows,
                                                                     (__nv_bfloat16 *)out.slices, out.expo,
                                                                     out.rows_pad);
  return cudaGetLastError();
}

cudaError_t launch_oz_slice_z(const void *Z, int64_t ldz, int64_t cols, OzOperand &out, cudaStream_t st) {
  out.rows = cols;
  out.rows_pad = pad_to(cols, kOzNFwd);
  out.k = kOzK;
  out.k_pad = kOzK;
  out.ns = kOzSlicesFwd;
  note_launch();
  oz_slice_z_kernel<<<(unsigned)((out.rows_pad + 7) / 8), 256, 0, st>>>((const zd *)Z, ldz, cols,
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
  int64_t splits = std::max<int64_t>(1, sms / (2 * mt));   // two CTAs (halves of B) per M-tile
  splits = std::max<int64_t>(splits, (nkb + kOzKbMax - 1) / kOzKbMax);
  splits = std::min<int64_t>(splits, nkb);
  const int64_t per = (nkb + splits - 1) / splits;
  *kb_per = (int)per;
  return (int)((nkb + per - 1) / per);
}

// splits x padded rows of the partial sums, bounded for every rows <= l, cols <= m: the splits
// are at most max(sms / (2 mt), ceil(K-blocks / kOzKbMax)), so splits x mt <= max(sms, (K-blocks /
// kOzKbMax + 1) mt)
size_t oz_adj_partial_bytes(int64_t l, int64_t m, int sms) {
  const int64_t mt = pad_to(m, kOzM) / kOzM, nkb = pad_to(2 * l, kOzK) / kOzK;
  const int64_t tiles = std::max<int64_t>((int64_t)sms + mt, (nkb / kOzKbMax + 1) * mt);
  return sizeof(double) * (size_t)tiles * kOzM * 64;
}

// W[j, c] = conj(D[c][j] + i D[c][32 + j]) summed over the splits with a compensated (TwoSum)
// sum: the result is the splits' exact sum rounded once, up to a second-order term, so the
// splits add one rounding in all rather than one per split
__device__ __forceinline__ void two_sum_acc(double &hi, double &lo, double x) {
  const double t = hi + x;
  const double z = t - hi;
  lo += (hi - (t - z)) + (x - z);
  hi = t;
}
__global__ void oz_adj_reduce_kernel(const double *__restrict__ part, int splits, int64_t rows_pad, int64_t cols,
                                     zd *__restrict__ W, int64_t ldw) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= cols * 32) return;
  const int64_t c = e / 32;
  const int j = (int)(e % 32);
  double re = 0.0, re_lo = 0.0, im = 0.0, im_lo = 0.0;
  for (int s = 0; s < splits; ++s) {
    const double *d = part + ((int64_t)s * rows_pad + c) * 64;
    two_sum_acc(re, re_lo, d[j]);
    two_sum_acc(im, im_lo, d[32 + j]);
  }
  W[c * ldw + j] = {re + re_lo, -(im + im_lo)};
}

cudaError_t launch_oz_adj(const OzAdjArgs &a, cudaStream_t st) {
  if (a.cols < 1) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  CUtensorMap amap, bmap;
  if ((e = oz_map(a.a, kOzM, &amap)) != cudaSuccess) return e;
  if ((e = oz_map(a.b, kOzNAdj, &bmap)) != cudaSuccess) return e;
  int per = 0;
  const int splits = oz_adj_splits(a.a.k / 2, a.cols, sms, &per);
  if (sizeof(double) * (size_t)splits * (size_t)a.a.rows_pad * 64 > a.part_bytes) return cudaErrorInvalidValue;
  if (a.a.ns != kOzSlicesAdj || a.b.ns != kOzSlicesAdj) return cudaErrorInvalidValue;
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
  auto kern = oz_adj_kernel<kOzSlicesAdj, kOzLevelsAdj, kOzNAdj>;
  constexpr int smem = OzShape<kOzSlicesAdj, kOzNAdj>::kSmem;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
  note_launch();
  kern<<<dim3((unsigned)(a.a.rows_pad / kOzM), (unsigned)splits, 64u / kOzNAdj), kOzThreads, smem, st>>>(amap, bmap,
                                                                                                      P);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  note_launch();
  oz_adj_reduce_kernel<<<(unsigned)((a.cols * 32 + 255) / 256), 256, 0, st>>>(a.part, splits, a.a.rows_pad, a.cols,
                                                                              (zd *)a.W, a.ldw);
  return cudaGetLastError();
}

cudaError_t launch_oz_fwd(const OzFwdArgs &a, cudaStream_t st) {
  if (a.rows < 1 || a.cols < 1) return cudaSuccess;
  if (a.a.ns != kOzSlicesFwd || a.b.ns != kOzSlicesFwd || a.a.k_pad != kOzK || a.b.k_pad != kOzK)
    return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  CUtensorMap amap, bmap;
  if ((e = oz_map(a.a, kOzM, &amap)) != cudaSuccess) return e;
  if ((e = oz_map(a.b, kOzFwdNT, &bmap)) != cudaSuccess) return e;
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
  const int n_row_tiles = (int)(a.a.rows_pad / kOzM);
  const int n_col_tiles = (int)((a.cols + kOzFwdNT - 1) / kOzFwdNT);
  // one CTA per SM, each with an equal share of the items (at least one)
  const int grid = (int)std::min<int64_t>((int64_t)n_row_tiles * n_col_tiles, sms);
  if ((int64_t)n_col_tiles * kOzFwdNT > a.b.rows_pad) return cudaErrorInvalidValue;
  if ((e = cudaFuncSetAttribute(oz_fwd_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                OzFwdShape::kSmem)) != cudaSuccess)
    return e;
  note_launch();
  oz_fwd_persistent_kernel<<<grid, kOzThreads, OzFwdShape::kSmem, st>>>(amap, bmap, P, n_row_tiles, n_col_tiles);
  return cudaGetLastError();
}

}  // namespace mn
