// cgfused.cu -- Step 4 (Eq. overdet) as one persistent cooperative kernel for
// the mixed-precision path: conjugate gradients on
//     (Wp^* A A^* Wp) du = g,   Wp = P R^{-1},
// with every iteration reading A (complex64) from HBM exactly once.
//
// Each CTA owns every G-th 16-column sub-panel of A (m <= 512 rows). A sub-panel (m x 16 complex64, 128 bytes per row) is brought into
// shared memory by 2-D TMA loads (cp.async.bulk.tensor, 128-byte swizzle)
// through a three-stage mbarrier pipeline, and used twice while resident:
//     q_j  = sum_i conj(A_ij) w_i      for the sub-panel's 16 columns
//     t_i += sum_j A_ij q_j            for all m rows (per-thread accumulators)
// so A^* w and A (A^* w) cost one pass. Successive iterations walk the own
// sub-panels in opposite directions: the last kStages sub-panels of one
// iteration are still in shared memory when the next begins (no reload), and
// the ones read just before them were loaded with an L2 evict-last hint, so
// the next iteration finds its first stretch of A in L2. The FP64 parts (w = Wp p,
// Np = Wp^* t, the CG scalars) are spread over the CTAs by rows, between four
// grid barriers per iteration (bounded waits, see common.cuh). The search
// direction p is kept, identically, in every CTA's shared memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.h"
#include "vec.h"

namespace mn {

constexpr int kCgThreads = 512;
constexpr int kPanel = 16;      // columns per sub-panel: 16 complex64 = 128 bytes
constexpr int kBoxRows = 256;   // rows per TMA box
constexpr int kMaxFusedRows = 512;
constexpr int kStages = 3;      // TMA ring depth

struct CgFusedParams {
  int m, n, nbox;
  int keep;         // sub-panels per CTA at the end of each sweep loaded with an L2 evict-last hint
  const zd *Wp, *WpH;
  const zd *g;
  zd *u, *s, *w, *t, *dy;
  zf *tpart;        // G x m
  double *qq_part;  // G
  double *gg_part;  // G
  CgScalars *sc;
  double tol2;
  int maxit;
  GridBarrier *bar;
  int *err;
  uint64_t limit_ns;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the phase with the given parity, at most limit_ns
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// 2-D tile load with an L2 cache policy (createpolicy: evict_first or evict_last)
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;"
      ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// warp sums of 32 floats, transposed: afterwards v[0] of lane L holds the sum over
// the warp of v[L] (a butterfly: at offset o each lane keeps the half of its
// remaining values selected by its bit o and receives the partner's partial sums)
__device__ __forceinline__ void warp_transpose_sum32(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool lo = !(lane & o);
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const float send = lo ? v[k + o] : v[k];
      const float keep = lo ? v[k] : v[k + o];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

// warp sums of 4 floats, transposed: lane 0 gets v[0], lane 8 v[1], lane 16 v[2], lane 24 v[3]
__device__ __forceinline__ float warp_sum_t4(const float (&v)[4], int lane) {
  const bool lo = !(lane & 16);
  const float w0 = (lo ? v[0] : v[2]) + __shfl_xor_sync(0xffffffffu, lo ? v[2] : v[0], 16);
  const float w1 = (lo ? v[1] : v[3]) + __shfl_xor_sync(0xffffffffu, lo ? v[3] : v[1], 16);
  const bool lo2 = !(lane & 8);
  float z = (lo2 ? w0 : w1) + __shfl_xor_sync(0xffffffffu, lo2 ? w1 : w0, 8);
  z += __shfl_xor_sync(0xffffffffu, z, 4);
  z += __shfl_xor_sync(0xffffffffu, z, 2);
  z += __shfl_xor_sync(0xffffffffu, z, 1);
  return z;
}

// out[i] = sum_k M[i][k] v[k] for i in [r0, r1): one warp per row (FP64)
__device__ __forceinline__ void rows_dot(const zd *__restrict__ M, const zd *v, int m, int r0, int r1,
                                         zd *out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = r0 + wid; i < r1; i += nw) {
    const zd *row = M + (int64_t)i * m;
    double re = 0.0, im = 0.0;
    for (int k = lane; k < m; k += 32) {
      const zd a = row[k], x = v[k];
      re = fma(a.re, x.re, fma(-a.im, x.im, re));
      im = fma(a.re, x.im, fma(a.im, x.re, im));
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) out[i] = {re, im};
  }
}

__global__ void __launch_bounds__(kCgThreads, 1)
cg_fused_kernel(const __grid_constant__ CUtensorMap amap, const CgFusedParams P) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int m = P.m, nbox = P.nbox;
  const int rows_pad = nbox * kBoxRows;
  const int stage_bytes = rows_pad * 128;
  auto stage = [&](int q) { return base + q * stage_bytes; };
  zd *p_s = reinterpret_cast<zd *>(base + kStages * stage_bytes);  // m: search direction
  zd *v_s = p_s + m;                                               // m: t, then u
  float *q_f = reinterpret_cast<float *>(v_s + m);                 // 32: q of the current sub-panel
  uint64_t *mbar = reinterpret_cast<uint64_t *>(q_f + 2 * kPanel); // kStages
  __shared__ double red[32];
  __shared__ double s_scal[4];
  __shared__ double s_qq[kCgThreads / 32];
  __shared__ float s_red[kCgThreads / 32][32];

  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int r0 = (int)((long long)m * b / G), r1 = (int)((long long)m * (b + 1) / G);
  // sub-panels b, b + G, b + 2G, ...: at any moment the grid reads one contiguous
  // stretch of every row (DRAM page locality), not G scattered 128-byte pieces
  const int NP = (P.n + kPanel - 1) / kPanel;
  const int nsp = NP > b ? (NP - b + G - 1) / G : 0;
  unsigned int epoch = 0;
  const uint32_t stage_tx = (uint32_t)stage_bytes;

  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) mbar_init(&mbar[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // start: u = 0, s = p = g
  double loc = 0.0;
  for (int i = tid; i < m; i += blockDim.x) {
    const zd gi = P.g[i];
    p_s[i] = gi;
    loc = fma(gi.re, gi.re, fma(gi.im, gi.im, loc));
  }
  for (int i = r0 + tid; i < r1; i += blockDim.x) {
    P.s[i] = P.g[i];
    P.u[i] = {0.0, 0.0};
  }
  double gamma = block_sum(loc, red);
  const double gamma0 = gamma;
  bool done = !(gamma > 0.0);
  uint32_t parity[kStages] = {};
  const uint64_t pol_first = policy_evict_first(), pol_last = policy_evict_last();
  int it = 0;
  bool ok = true;

  while (!done && it < P.maxit) {
    // P1: w = Wp p (own rows)
    rows_dot(P.Wp, p_s, m, r0, r1, P.w);
    if (!grid_sync(P.bar, G, epoch, P.limit_ns)) { ok = false; break; }

    // P2: q = A^* w and t = A q over the own sub-panels, A read once
    // thread i holds w_i and, per sub-panel, row i of the sub-panel in registers
    const zf wreg = tid < m ? cvt<float>(P.w[tid]) : zf{0.f, 0.f};
    zf tacc = {0.f, 0.f};
    // |q|^2 in FP32 inside the loop (an FP64 instruction costs ~76 cycles of the SM
    // sub-partition's FP64 pipe on GB300), widened once at the end
    float qq_loc = 0.f;
    // sweep direction alternates; the first nres positions of this sweep are the
    // last ones of the previous sweep, still resident in their stages
    const bool fwd = (it & 1) == 0;
    const int nres = it > 0 ? (nsp < kStages ? nsp : kStages) : 0;
    // stage of a sub-panel = its own index mod kStages: a load issued after position e
    // is consumed (position e + kStages, in either direction) reuses e's stage
    auto issue = [&](int e) {
      const int ipn = fwd ? e : nsp - 1 - e;
      const int sl = ipn % kStages;
      const uint64_t pol = e >= nsp - P.keep ? pol_last : pol_first;
      mbar_expect_tx(&mbar[sl], stage_tx);
      for (int bx = 0; bx < nbox; ++bx)
        tma_load_2d(stage(sl) + bx * kBoxRows * 128, &amap, (b + ipn * G) * 2 * kPanel, bx * kBoxRows, &mbar[sl],
                    pol);
    };
    if (tid == 0 && it == 0) {
      for (int e = 0; e < kStages && e < nsp; ++e) issue(e);
    }
    for (int e = 0; e < nsp; ++e) {
      const int ip = fwd ? e : nsp - 1 - e;
      const int st = ip % kStages;
      const int sp = b + ip * G;
      bool w_ok = true;
      if (e >= nres) {
        w_ok = mbar_wait(&mbar[st], parity[st], P.limit_ns);
        if (!w_ok) w_ok = mbar_wait(&mbar[st], parity[st], P.limit_ns);  // a second bounded wait
        parity[st] ^= 1u;
      }
      w_ok = __all_sync(0xffffffffu, w_ok);  // warp-uniform: the q step below uses full-warp shuffles
      const unsigned char *S = stage(st);
      // (a) row tid of the sub-panel into registers (eight 16-byte swizzled chunks), its
      //     terms conj(A_ij) w_i of the 16 q_j, summed over the warp's 32 rows by a butterfly
      float4 av[8];
      if (w_ok && tid < rows_pad) {
        const unsigned char *row = S + tid * 128;
#pragma unroll
        for (int kc = 0; kc < 8; ++kc) av[kc] = *reinterpret_cast<const float4 *>(row + ((kc ^ (tid & 7)) << 4));
      } else {
#pragma unroll
        for (int kc = 0; kc < 8; ++kc) av[kc] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      float c[32];
#pragma unroll
      for (int kc = 0; kc < 8; ++kc) {
        c[4 * kc + 0] = fmaf(av[kc].x, wreg.re, av[kc].y * wreg.im);
        c[4 * kc + 1] = fmaf(av[kc].x, wreg.im, -av[kc].y * wreg.re);
        c[4 * kc + 2] = fmaf(av[kc].z, wreg.re, av[kc].w * wreg.im);
        c[4 * kc + 3] = fmaf(av[kc].z, wreg.im, -av[kc].w * wreg.re);
      }
      warp_transpose_sum32(c, lane);
      s_red[wid][lane] = c[0];
      if (__syncthreads_or(!w_ok)) {
        // give up uniformly; later stages may still hold issued copies: wait for them (bounded)
        ok = false;
        for (int e2 = e + 1; e2 < e + kStages && e2 < nsp; ++e2) {
          if (e2 < nres) continue;  // resident, nothing in flight
          const int s2 = (fwd ? e2 : nsp - 1 - e2) % kStages;
          mbar_wait(&mbar[s2], parity[s2], P.limit_ns);
        }
        break;
      }
      // stage st is free (the sub-panel is in registers): refill it now
      if (tid == 0 && e + kStages < nsp) issue(e + kStages);
      // (b) q over the 16 warps (fixed order), and |q|^2 of the columns inside A
      if (wid == 0) {
        float qf = 0.f;
#pragma unroll
        for (int w2 = 0; w2 < kCgThreads / 32; ++w2) qf += s_red[w2][lane];
        q_f[lane] = qf;
        if (sp * kPanel + (lane >> 1) < P.n) qq_loc = fmaf(qf, qf, qq_loc);
      }
      __syncthreads();
      // (c) t_i += sum_j A_ij q_j from the registers
      if (tid < m) {
#pragma unroll
        for (int kc = 0; kc < 8; ++kc) {
          const float4 q4 = *reinterpret_cast<const float4 *>(q_f + 4 * kc);
          mac(tacc, zf{av[kc].x, av[kc].y}, zf{q4.x, q4.y});
          mac(tacc, zf{av[kc].z, av[kc].w}, zf{q4.z, q4.w});
        }
      }
    }
    if (!ok) break;
    if (tid < m) P.tpart[(int64_t)b * m + tid] = tacc;
    qq_loc = warp_sum(qq_loc);
    if (lane == 0) s_qq[wid] = (double)qq_loc;
    __syncthreads();
    if (tid == 0) {
      double qsum = 0.0;
      for (int w2 = 0; w2 < kCgThreads / 32; ++w2) qsum += s_qq[w2];
      P.qq_part[b] = qsum;
    }
    if (!grid_sync(P.bar, G, epoch, P.limit_ns)) { ok = false; break; }

    // P3a: t (own rows) = sum of the partials; qq = sum of the per-CTA |q|^2
    for (int i = r0 + wid; i < r1; i += blockDim.x >> 5) {
      double re = 0.0, im = 0.0;
      for (int c = lane; c < G; c += 32) {
        const zf v = P.tpart[(int64_t)c * m + i];
        re += (double)v.re;
        im += (double)v.im;
      }
      re = warp_sum(re);
      im = warp_sum(im);
      if (lane == 0) P.t[i] = {re, im};
    }
    if (wid == 0) {
      double qs = 0.0;
      for (int c = lane; c < G; c += 32) qs += P.qq_part[c];
      qs = warp_sum(qs);
      if (lane == 0) s_scal[0] = qs;
    }
    if (!grid_sync(P.bar, G, epoch, P.limit_ns)) { ok = false; break; }
    const double qq = s_scal[0];
    const double alpha = qq > 0.0 ? gamma / qq : 0.0;

    // P3b: Np = Wp^* t (own rows); s -= alpha Np; u += alpha p; partial ||s||^2
    for (int i = tid; i < m; i += blockDim.x) v_s[i] = P.t[i];
    __syncthreads();
    rows_dot(P.WpH, v_s, m, r0, r1, P.dy);   // dy holds Np for the own rows here
    __syncthreads();
    double gl = 0.0;
    for (int i = r0 + tid; i < r1; i += blockDim.x) {
      const zd np = P.dy[i], pi = p_s[i];
      zd si = P.s[i], ui = P.u[i];
      si.re = fma(-alpha, np.re, si.re);
      si.im = fma(-alpha, np.im, si.im);
      ui.re = fma(alpha, pi.re, ui.re);
      ui.im = fma(alpha, pi.im, ui.im);
      P.s[i] = si;
      P.u[i] = ui;
      gl = fma(si.re, si.re, fma(si.im, si.im, gl));
    }
    if (wid == 0) {
      const double gs = warp_sum(gl);
      if (lane == 0) P.gg_part[b] = gs;
    }
    if (!grid_sync(P.bar, G, epoch, P.limit_ns)) { ok = false; break; }

    // P4: gamma' and the new direction, identically in every CTA
    if (wid == 0) {
      double gs = 0.0;
      for (int c = lane; c < G; c += 32) gs += P.gg_part[c];
      gs = warp_sum(gs);
      if (lane == 0) s_scal[1] = gs;
    }
    __syncthreads();
    const double gnew = s_scal[1];
    const double beta = gamma > 0.0 ? gnew / gamma : 0.0;
    for (int i = tid; i < m; i += blockDim.x) {
      const zd si = P.s[i];
      zd pi = p_s[i];
      pi.re = fma(beta, pi.re, si.re);
      pi.im = fma(beta, pi.im, si.im);
      p_s[i] = pi;
    }
    gamma = gnew;
    ++it;
    if (gnew <= P.tol2 * gamma0 || !(qq > 0.0)) done = true;
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) atomicExch(P.err, 1);
    // no TMA load is left in flight: every issued stage was waited for above
    return;
  }
  // dy = Wp u (own rows)
  if (!grid_sync(P.bar, G, epoch, P.limit_ns)) {
    if (tid == 0) atomicExch(P.err, 1);
    return;
  }
  for (int i = tid; i < m; i += blockDim.x) v_s[i] = P.u[i];
  __syncthreads();
  rows_dot(P.Wp, v_s, m, r0, r1, P.dy);
  if (b == 0 && tid == 0) {
    P.sc->iters = it;
    P.sc->gamma = gamma;
    P.sc->gamma0 = gamma0;
    P.sc->done = done ? 1 : 0;
  }
}

// ---- host -------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
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

bool cg_fused_supported(int64_t m, int64_t n, int64_t lda, const void *A) {
  return m >= 1 && m <= kMaxFusedRows && n >= kPanel && (lda % 2) == 0 && (((uintptr_t)A) & 15) == 0 &&
         get_encode() != nullptr;
}

size_t cg_fused_smem(int64_t m) {
  const int nbox = (int)((m + kBoxRows - 1) / kBoxRows);
  const size_t rows_pad = (size_t)nbox * kBoxRows;
  return 1024 + kStages * rows_pad * 128 + 2 * (size_t)m * sizeof(zd) + 2 * kPanel * sizeof(float) +
         kStages * sizeof(uint64_t);
}

cudaError_t launch_cg_fused(const CgFusedArgs &a, cudaStream_t st) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  // A as a 2-D array of floats: dim0 = 2n (re, im interleaved), dim1 = m rows
  const cuuint64_t gdim[2] = {(cuuint64_t)(2 * a.n), (cuuint64_t)a.m};
  const cuuint64_t gstride[1] = {(cuuint64_t)(a.lda * sizeof(zf))};
  const cuuint32_t box[2] = {2 * kPanel, kBoxRows};
  const cuuint32_t estride[2] = {1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(a.A), gdim, gstride, box,
                   estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  CgFusedParams P;
  P.m = (int)a.m;
  P.n = (int)a.n;
  P.nbox = (int)((a.m + kBoxRows - 1) / kBoxRows);
  P.Wp = (const zd *)a.Wp;
  P.WpH = (const zd *)a.WpH;
  P.g = (const zd *)a.g;
  P.u = (zd *)a.u;
  P.s = (zd *)a.s;
  P.w = (zd *)a.w;
  P.t = (zd *)a.t;
  P.dy = (zd *)a.dy;
  P.tpart = (zf *)a.tpart;
  P.qq_part = a.qq_part;
  P.gg_part = a.gg_part;
  P.sc = a.sc;
  P.tol2 = a.tol2;
  P.maxit = a.maxit;
  P.bar = a.bar;
  P.err = a.err;
  P.limit_ns = a.limit_ns;
  const size_t smem = cg_fused_smem(a.m);
  cudaError_t e = cudaFuncSetAttribute(cg_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int NP = (int)((a.n + kPanel - 1) / kPanel);
  const int G = a.grid < NP ? a.grid : NP;
  // sub-panels per CTA kept in L2 between sweeps: about 60 % of L2
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
    l2 = 0;
  const double stage_bytes = (double)P.nbox * kBoxRows * 128;
  P.keep = (int)(0.6 * (double)l2 / ((double)G * stage_bytes));
  void *args[] = {(void *)&map, (void *)&P};
  note_launch();
  return cudaLaunchCooperativeKernel((const void *)cg_fused_kernel, dim3(G), dim3(kCgThreads), args, smem, st);
}

}  // namespace mn
