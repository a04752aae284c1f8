// tcblock.cu -- the two products of block CG on the tensor cores (tcgen05):
//     Q = A^* W     (A m x n complex64, W m x 32, Q n x 32)
//     T = A Q       (T m x 32)
// with FP32 accuracy from BF16 operands: every FP32 value x is split exactly
// into three BF16 pieces x = x1 + x2 + x3 (8 significant bits each), and the
// six products whose pieces sum to at most the third (x1y1, x1y2, x2y1, x1y3,
// x2y2, x3y1) are accumulated in FP32 in tensor memory; the dropped ones are
// below 2^-24 relative. (A single BF16 or TF32 product is too coarse for the
// refinement at condition numbers near 1e6: the inner operator must be about as
// accurate as FP32.)
//
// Complex arithmetic as real products over the floats of A's rows (f = 2 j + c,
// c = 0: Re, 1: Im):
//   Q: M = 128 floats of a row segment (64 columns j), K = rows i of A,
//      N = 64 = [Re W | Im W]; Re Q_jc = D[2j][c] + D[2j+1][32+c],
//      Im Q_jc = D[2j][32+c] - D[2j+1][c].
//   T: M = 128 rows i, K = the floats f of the rows, N = 64 = [Re T | Im T] against
//      B[f][c] = (Re Q_jc, -Im Q_jc) and B[f][32+c] = (Im Q_jc, Re Q_jc) for f = 2j, 2j+1.
//
// One CTA per SM; per K-block of 64:
//   * TMA brings the FP32 tile of A three steps ahead,
//   * the 256 threads split it into three BF16 operands in the K-major,
//     128-byte-swizzled layout the MMA reads (16-byte chunks of 8 K values),
//   * one thread issues three tcgen05.mma (N = 192, 128, 64 against the pieces of
//     the other operand stacked along N, fetched by TMA one step ahead) and
//     commits them to an mbarrier; the next K-block's split waits for it.
// Every 8 K-blocks (512 terms) warps 4-7 read the accumulator (128 lanes x 192
// columns) back with tcgen05.ld, sum its three 64-column blocks into FP32
// registers and leave the region to the chunk after next (two regions
// alternate): the FP32 accumulation error of the tensor cores grows with the
// number of terms summed in place. At the end of a tile: Q and its partial sums
// of |Q_jc|^2, or T's partial sums over the CTA's K range.
// Every wait is bounded in time; on expiry the kernel records an error, waits
// (bounded) for its copies and products in flight, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace mn {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcCols = 64;           // Q: complex columns of A per tile (M = 128 floats)
constexpr int kTcK = 64;              // K values per K-block (Q: rows of A; T: floats of A's rows)
constexpr int kTcAStages = 3;         // FP32 tiles in flight
constexpr int kTcAStage = kTcK * 2 * kTcCols * 4;  // 32 KB
constexpr int kTcPiece = 128 * kTcK * 2;           // one BF16 operand: 16 KB
constexpr int kTcBRows = 3 * 64;                   // three pieces of [Re W | Im W]
constexpr int kTcBStage = kTcBRows * kTcK * 2;     // 24 KB
constexpr int kTcTmemCols = 512;  // two accumulator regions of 192 columns, at 0 and 256
constexpr int kTcChunk = 8;        // K-blocks per accumulation in tensor memory (512 terms)
// shared memory: A pieces | 2 B stages | FP32 stages | |Q|^2 scratch | barriers
constexpr int kTcOffA = 0;
constexpr int kTcOffB = kTcOffA + 3 * kTcPiece;                 // 48 KB
constexpr int kTcOffF = kTcOffB + 2 * kTcBStage;                // 96 KB
constexpr int kTcOffQ = kTcOffF + kTcAStages * kTcAStage;       // 192 KB
constexpr int kTcOffBar = kTcOffQ + 64 * 32 * 4;                // 200 KB
constexpr int kTcSmem = kTcOffBar + 256 + 1024;                 // + barriers + alignment slack

// exact split of x into three BF16 pieces (round to nearest at each step; the
// remainders are exact in FP32)
__device__ __forceinline__ void split3(float x, __nv_bfloat16 &p1, __nv_bfloat16 &p2, __nv_bfloat16 &p3) {
  p1 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(p1);
  p2 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(p2);
  p3 = __float2bfloat16_rn(r2);
}
__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

struct TcParams {
  int m, nkb, ntiles;  // Q: K-blocks per tile (rows of A / 64) and tiles (n / 64); T: K-blocks in all, M tiles
  int nsplit;          // T: K ranges (CTAs per M tile)
  int64_t n;
  zf *Q;               // Q: n x 32
  float *qqp;          // Q: ntiles x 32
  zf *tpart;           // T: nsplit x m x 32
  const int *alldone;
  int *err;
  uint64_t limit_ns;
};

}  // namespace

template <bool FWD>
__global__ void __launch_bounds__(kTcThreads, 1)
tc_block_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                const TcParams P) {
  if (*P.alldone) return;
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = base + kTcOffA;
  unsigned char *sB = base + kTcOffB;
  float *sF = reinterpret_cast<float *>(base + kTcOffF);
  float *sQ = reinterpret_cast<float *>(base + kTcOffQ);
  uint64_t *bars = reinterpret_cast<uint64_t *>(base + kTcOffBar);
  uint64_t *a_full = bars;              // kTcAStages
  uint64_t *b_full = bars + 3;          // 2
  uint64_t *mma_bar = bars + 5;         // one phase per K-block
  uint64_t *acc_bar = bars + 6;         // 2: one phase per accumulation chunk in that region
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 8);
  __shared__ int s_abort;

  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int G = gridDim.x, b = blockIdx.x;
  // Q: tiles b, b + G, ..., each over all nkb K-blocks. T: one M tile (b % ntiles) over
  // the K-blocks [kb0, kb0 + nkb_u) of split b / ntiles.
  const int mt = FWD ? b % P.ntiles : 0, split = FWD ? b / P.ntiles : 0;
  const int kb0 = FWD ? (int)((int64_t)P.nkb * split / P.nsplit) : 0;
  const int nkb_u = FWD ? (int)((int64_t)P.nkb * (split + 1) / P.nsplit) - kb0 : P.nkb;
  const int my_tiles = FWD ? (nkb_u > 0 ? 1 : 0) : (P.ntiles > b ? (P.ntiles - b + G - 1) / G : 0);
  const int nsteps = my_tiles * nkb_u;

  if (tid == 0) {
    for (int s = 0; s < kTcAStages; ++s) bar_init(&a_full[s], 1);
    bar_init(&b_full[0], 1);
    bar_init(&b_full[1], 1);
    bar_init(mma_bar, 1);
    bar_init(&acc_bar[0], 1);
    bar_init(&acc_bar[1], 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (wid == 0) {  // tensor memory for the accumulator (one CTA per SM)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tmem_slot)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // step s <-> Q: (tile b + (s / nkb) G, K-block s % nkb); T: K-block kb0 + s of tile mt
  auto issue_a = [&](int s) {
    uint64_t *bar = &a_full[s % kTcAStages];
    bar_expect(bar, kTcAStage);
    float *dst = sF + (s % kTcAStages) * (kTcAStage / 4);
    if (FWD) {
      tma2d(dst, &amap, (kb0 + s) * kTcK, mt * 128, bar);  // 128 rows x 64 floats
    } else {
      const int t = b + (s / nkb_u) * G, kb = s % nkb_u;
      tma2d(dst, &amap, t * 2 * kTcCols, kb * kTcK, bar);   // 64 rows x 128 floats
    }
  };
  auto issue_b = [&](int s) {
    uint64_t *bar = &b_full[s & 1];
    bar_expect(bar, kTcBStage);
    tma2d(sB + (s & 1) * kTcBStage, &bmap, (FWD ? kb0 + s : s % nkb_u) * kTcK, 0, bar);
  };
  int a_issued = 0, b_issued = 0, mma_done = 0;  // thread 0's counters (steps issued / committed)
  if (tid == 0) {
    for (; a_issued < kTcAStages && a_issued < nsteps; ++a_issued) issue_a(a_issued);
    if (nsteps > 0) issue_b(b_issued++);
  }

  // The accumulator is emptied every kTcChunk K-blocks into FP32 registers of warps
  // 4-7 (a sum of at most 512 terms stays in tensor memory: its FP32 accumulation
  // error grows with the length), while the next chunk accumulates in the other
  // region. Chunk g (counted over the CTA's tiles) uses region g & 1.
  float acc[64];
#pragma unroll
  for (int k = 0; k < 64; ++k) acc[k] = 0.f;
  const int chunks_per_tile = (nkb_u + kTcChunk - 1) / kTcChunk;
  // warps 4-7: add chunk g's three 64-column blocks into acc (lanes 32 (w & 3) + lane)
  auto flush = [&](int g) -> bool {
    bool okw = bar_wait(&acc_bar[g & 1], (uint32_t)((g >> 1) & 1), P.limit_ns);
    okw = __all_sync(0xffffffffu, okw);
    if (!okw) return false;
    tc_fence_after();
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (wid & 3)) << 16) + 256u * (uint32_t)(g & 1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[32], x[32];
      tmem_ld32(lane_base + 32 * h, v);
#pragma unroll
      for (int blk = 1; blk < 3; ++blk) {
        tmem_ld32(lane_base + 64 * blk + 32 * h, x);
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] += x[k];
      }
#pragma unroll
      for (int k = 0; k < 32; ++k) acc[32 * h + k] += v[k];
    }
    tc_fence_before();
    return true;
  };

  bool ok = true, good = true;
  int s = 0;
  for (int lt = 0; lt < my_tiles && ok; ++lt) {
    const int t = FWD ? mt : b + lt * G;
    for (int kb = 0; kb < nkb_u; ++kb, ++s) {
      const int g = lt * chunks_per_tile + kb / kTcChunk;
      // (1) the FP32 tile of this step has landed; the products of the previous step
      //     have finished reading the BF16 operands
      bool w = bar_wait(&a_full[s % kTcAStages], (uint32_t)((s / kTcAStages) & 1), P.limit_ns);
      if (w && s > 0) w = bar_wait(mma_bar, (uint32_t)((s - 1) & 1), P.limit_ns);
      // (2) split into the three BF16 operands, one 16-byte chunk (8 K values of operand
      //     row f) at a time. Q: f = tid & 127 (column-wise reads of the 64 x 128 tile,
      //     consecutive lanes on consecutive floats); T: f = (tid >> 3) + 32 r, chunk
      //     tid & 7 (two 16-byte reads of a row of the 128 x 64 tile)
      if (w) {
        const float *F = sF + (s % kTcAStages) * (kTcAStage / 4);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int f = FWD ? (tid >> 3) + 32 * r : tid & 127;
          const int kc = FWD ? tid & 7 : (tid >> 7) + 2 * r;
          float x[8];
          if (FWD) {
            const float4 u0 = *reinterpret_cast<const float4 *>(F + f * 64 + 8 * kc);
            const float4 u1 = *reinterpret_cast<const float4 *>(F + f * 64 + 8 * kc + 4);
            x[0] = u0.x; x[1] = u0.y; x[2] = u0.z; x[3] = u0.w;
            x[4] = u1.x; x[5] = u1.y; x[6] = u1.z; x[7] = u1.w;
          } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = F[(8 * kc + k) * 128 + f];
          }
          uint32_t w1[4], w2[4], w3[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            __nv_bfloat16 a1, a2, a3, b1, b2, b3;
            split3(x[2 * e], a1, a2, a3);
            split3(x[2 * e + 1], b1, b2, b3);
            w1[e] = pack2(a1, b1);
            w2[e] = pack2(a2, b2);
            w3[e] = pack2(a3, b3);
          }
          const uint32_t off = (uint32_t)((f >> 3) * 1024 + (f & 7) * 128 + ((kc ^ (f & 7)) << 4));
          *reinterpret_cast<uint4 *>(sA + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
          *reinterpret_cast<uint4 *>(sA + kTcPiece + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
          *reinterpret_cast<uint4 *>(sA + 2 * kTcPiece + off) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      if (__syncthreads_or(!w || !good)) {
        ok = false;
        break;
      }
      // (3) thread 0: refill the FP32 stage just read, fetch the next pieces of the other
      //     operand, issue this step's products into region g & 1
      if (tid == 0) {
        if (a_issued < nsteps) issue_a(a_issued++);
        if (b_issued < nsteps) issue_b(b_issued++);
        bool wb = bar_wait(&b_full[s & 1], (uint32_t)((s >> 1) & 1), P.limit_ns);
        if (!wb) {
          s_abort = 1;
        } else {
          tc_fence_after();
          const uint32_t a0 = sa(sA), b0 = sa(sB + (s & 1) * kTcBStage);
          const uint32_t d = tmem + 256u * (uint32_t)(g & 1);
#pragma unroll
          for (int k16 = 0; k16 < kTcK / 16; ++k16) {
            const uint32_t accum = (kb % kTcChunk != 0 || k16 > 0) ? 1u : 0u;
            mma_bf16(d, sdesc(a0 + k16 * 32), sdesc(b0 + k16 * 32), idesc(192), accum);
            mma_bf16(d, sdesc(a0 + kTcPiece + k16 * 32), sdesc(b0 + k16 * 32), idesc(128), 1u);
            mma_bf16(d, sdesc(a0 + 2 * kTcPiece + k16 * 32), sdesc(b0 + k16 * 32), idesc(64), 1u);
          }
          mma_commit(mma_bar);
          mma_done = s + 1;
          if (kb % kTcChunk == kTcChunk - 1 || kb == nkb_u - 1) mma_commit(&acc_bar[g & 1]);
        }
      }
      // warps 4-7: at the start of a chunk, empty the previous chunk of this tile
      if (wid >= 4 && kb % kTcChunk == 0 && kb > 0 && good) good = flush(g - 1);
      // the W wait of thread 0 decides for all before the next step
      if (kb == nkb_u - 1 || (s & 7) == 7) {
        __syncthreads();
        if (s_abort) {
          ok = false;
          break;
        }
      }
    }
    if (!ok) break;
    // (4) epilogue (warps 4-7, TMEM lanes 32 (w & 3) .. + 31 = operand rows): the last
    //     chunk into acc, then T's partial or Q and |Q|^2
    if (wid >= 4 && good) good = flush(lt * chunks_per_tile + chunks_per_tile - 1);
    if (__syncthreads_or(!good)) {
      ok = false;
      break;
    }
    if (wid >= 4) {
      const int f = 32 * (wid & 3) + lane;
      if (FWD) {  // row i = 128 mt + f: T partial = (acc[c], acc[32 + c])
        const int i = 128 * mt + f;
        if (i < P.m) {
          float4 *dst = reinterpret_cast<float4 *>(P.tpart + ((int64_t)split * P.m + i) * 32);
#pragma unroll
          for (int c = 0; c < 32; c += 2)
            dst[c / 2] = make_float4(acc[c], acc[32 + c], acc[c + 1], acc[33 + c]);
        }
      } else {
        // even f holds the Re A terms of column jl = f / 2, odd f the Im terms
        const int jl = f >> 1;
        const int64_t j = (int64_t)t * kTcCols + jl;
        float qr[32], qi[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const float p_lo = __shfl_down_sync(0xffffffffu, acc[c], 1);       // odd row: Re W part
          const float p_hi = __shfl_down_sync(0xffffffffu, acc[32 + c], 1);  // odd row: Im W part
          qr[c] = acc[c] + p_hi;
          qi[c] = acc[32 + c] - p_lo;
        }
        if (!(f & 1)) {
          if (j < P.n) {
#pragma unroll
            for (int c = 0; c < 32; ++c) sQ[jl * 32 + c] = qr[c] * qr[c] + qi[c] * qi[c];
            float4 *dst = reinterpret_cast<float4 *>(P.Q + j * 32);
#pragma unroll
            for (int c = 0; c < 32; c += 2) dst[c / 2] = make_float4(qr[c], qi[c], qr[c + 1], qi[c + 1]);
          } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) sQ[jl * 32 + c] = 0.f;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 64; ++k) acc[k] = 0.f;
    }
    __syncthreads();
    if (!FWD && tid < 32) {  // partial |Q_jc|^2 of this tile, columns j in a fixed order
      float q2 = 0.f;
      for (int jl = 0; jl < kTcCols; ++jl) q2 += sQ[jl * 32 + tid];
      P.qqp[(int64_t)t * 32 + tid] = q2;
    }
  }
  if (!ok) {
    if (tid == 0) {
      atomicExch(P.err, 1);
      // copies still in flight: A steps [s, a_issued), W steps [s, b_issued); bounded waits
      for (int q = s; q < a_issued; ++q) bar_wait(&a_full[q % kTcAStages], (uint32_t)((q / kTcAStages) & 1), P.limit_ns);
      for (int q = s; q < b_issued; ++q) bar_wait(&b_full[q & 1], (uint32_t)((q >> 1) & 1), P.limit_ns);
      // products in flight: the last commit
      if (mma_done > 0) bar_wait(mma_bar, (uint32_t)((mma_done - 1) & 1), P.limit_ns);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (wid == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
  }
}

// Bs[p * 64 + nn][i] = piece p of (nn < 32 ? Re W[i][nn] : Im W[i][nn - 32]), BF16, row length ldb
__global__ void tc_split_w_kernel(const zf *__restrict__ W, int m, int64_t ldb, __nv_bfloat16 *__restrict__ Bs) {
  const int64_t total = (int64_t)64 * ldb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int nn = (int)(e / ldb);
    const int64_t i = e - (int64_t)nn * ldb;
    float x = 0.f;
    if (i < m) {
      const zf w = W[i * 32 + (nn & 31)];
      x = nn < 32 ? w.re : w.im;
    }
    __nv_bfloat16 p1, p2, p3;
    split3(x, p1, p2, p3);
    Bs[(int64_t)nn * ldb + i] = p1;
    Bs[(int64_t)(64 + nn) * ldb + i] = p2;
    Bs[(int64_t)(128 + nn) * ldb + i] = p3;
  }
}

// Bs[p * 64 + nn][2j + c] = piece p of B[f][nn] for the product T = A Q (row length
// ld2 >= 2n, even): nn < 32: (Re Q_j,nn, -Im Q_j,nn); nn >= 32: (Im Q_j,nn-32, Re Q_j,nn-32)
__global__ void tc_split_q_kernel(const zf *__restrict__ Q, int64_t n, int64_t ld2, __nv_bfloat16 *__restrict__ Bs) {
  const int64_t nj = ld2 / 2, total = 64 * nj;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int nn = (int)(e / nj);
    const int64_t j = e - (int64_t)nn * nj;
    float x0 = 0.f, x1 = 0.f;
    if (j < n) {
      const zf q = Q[j * 32 + (nn & 31)];
      if (nn < 32) {
        x0 = q.re;
        x1 = -q.im;
      } else {
        x0 = q.im;
        x1 = q.re;
      }
    }
    __nv_bfloat16 a1, a2, a3, b1, b2, b3;
    split3(x0, a1, a2, a3);
    split3(x1, b1, b2, b3);
    uint32_t *row = reinterpret_cast<uint32_t *>(Bs + (int64_t)nn * ld2) + j;
    const int64_t piece = 64 * ld2 / 2;  // 32-bit words per piece
    row[0] = pack2(a1, b1);
    row[piece] = pack2(a2, b2);
    row[2 * piece] = pack2(a3, b3);
  }
}

// ---- host -------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tc_encode() {
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

int64_t tc_split_ld(int64_t m) { return (m + 7) / 8 * 8; }
size_t tc_split_bytes(int64_t m) { return (size_t)kTcBRows * (size_t)tc_split_ld(m) * sizeof(__nv_bfloat16); }
static int64_t tc_split2_ld(int64_t n) { return (2 * n + 7) / 8 * 8; }
size_t tc_split2_bytes(int64_t n) { return (size_t)kTcBRows * (size_t)tc_split2_ld(n) * sizeof(__nv_bfloat16); }
// K ranges per M tile of T = A Q: about one CTA per SM, at least one K-block per range
int tc_fwd_splits(int64_t m, int64_t n, int sms) {
  const int64_t mt = (m + 127) / 128, nkb = (2 * n + kTcK - 1) / kTcK;
  int64_t s = sms / mt;
  if (s > nkb) s = nkb;
  return (int)(s < 1 ? 1 : s);
}

bool tc_block_supported(int64_t m, int64_t n, int64_t lda, const void *A) {
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) !=
                                                cudaSuccess)
    return false;
  return major == 10 && m >= 1 && n >= 1 && (lda % 2) == 0 && (((uintptr_t)A) & 15) == 0 && tc_encode() != nullptr;
}

// A as rows of 2n floats with the given box; the other operand's pieces: 192 rows of ld BF16,
// box 64 (K) x 192 rows, 128-byte swizzle (the MMA's layout)
static cudaError_t tc_maps(const void *A, int64_t m, int64_t n, int64_t lda, uint32_t box_x, uint32_t box_y,
                           void *Bs, int64_t ld, CUtensorMap *amap, CUtensorMap *bmap) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tc_encode();
  if (!enc) return cudaErrorNotSupported;
  {
    const cuuint64_t gdim[2] = {(cuuint64_t)(2 * n), (cuuint64_t)m};
    const cuuint64_t gstride[1] = {(cuuint64_t)(lda * sizeof(zf))};
    const cuuint32_t box[2] = {box_x, box_y};
    const cuuint32_t es[2] = {1, 1};
    if (enc(amap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(A), gdim, gstride, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    const cuuint64_t gdim[2] = {(cuuint64_t)ld, (cuuint64_t)kTcBRows};
    const cuuint64_t gstride[1] = {(cuuint64_t)(ld * sizeof(__nv_bfloat16))};
    const cuuint32_t box[2] = {kTcK, kTcBRows};
    const cuuint32_t es[2] = {1, 1};
    if (enc(bmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Bs, gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t launch_tc_block_adj(const void *A, int64_t m, int64_t n, int64_t lda, const void *W32, void *Bsplit,
                                void *Q, float *qqp, const int *alldone, int *err, uint64_t limit_ns, int sms,
                                cudaStream_t st) {
  const int64_t ldb = tc_split_ld(m);
  note_launch();
  tc_split_w_kernel<<<(unsigned)std::min<int64_t>(2048, (64 * ldb + 255) / 256), 256, 0, st>>>(
      (const zf *)W32, (int)m, ldb, (__nv_bfloat16 *)Bsplit);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap amap, bmap;
  e = tc_maps(A, m, n, lda, 2 * kTcCols, kTcK, Bsplit, ldb, &amap, &bmap);
  if (e != cudaSuccess) return e;
  TcParams P{};
  P.m = (int)m;
  P.n = n;
  P.nkb = (int)((m + kTcK - 1) / kTcK);
  P.ntiles = (int)((n + kTcCols - 1) / kTcCols);
  P.nsplit = 1;
  P.Q = (zf *)Q;
  P.qqp = qqp;
  P.alldone = alldone;
  P.err = err;
  P.limit_ns = limit_ns;
  e = cudaFuncSetAttribute(tc_block_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e != cudaSuccess) return e;
  const int G = P.ntiles < sms ? P.ntiles : sms;
  note_launch();
  tc_block_kernel<false><<<G, kTcThreads, kTcSmem, st>>>(amap, bmap, P);
  return cudaGetLastError();
}

cudaError_t launch_tc_block_fwd(const void *A, int64_t m, int64_t n, int64_t lda, const void *Q32, void *Bsplit2,
                                void *tpart, int nsplit, const int *alldone, int *err, uint64_t limit_ns,
                                cudaStream_t st) {
  const int64_t ld2 = tc_split2_ld(n);
  note_launch();
  tc_split_q_kernel<<<(unsigned)std::min<int64_t>(8192, (64 * (ld2 / 2) + 255) / 256), 256, 0, st>>>(
      (const zf *)Q32, n, ld2, (__nv_bfloat16 *)Bsplit2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap amap, bmap;
  e = tc_maps(A, m, n, lda, kTcK, 128, Bsplit2, ld2, &amap, &bmap);
  if (e != cudaSuccess) return e;
  TcParams P{};
  P.m = (int)m;
  P.n = n;
  P.nkb = (int)((2 * n + kTcK - 1) / kTcK);
  P.ntiles = (int)((m + 127) / 128);
  P.nsplit = nsplit;
  P.tpart = (zf *)tpart;
  P.alldone = alldone;
  P.err = err;
  P.limit_ns = limit_ns;
  e = cudaFuncSetAttribute(tc_block_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e != cudaSuccess) return e;
  note_launch();
  tc_block_kernel<true><<<P.ntiles * nsplit, kTcThreads, kTcSmem, st>>>(amap, bmap, P);
  return cudaGetLastError();
}

}  // namespace mn
