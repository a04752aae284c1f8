// cgfused.cu -- Step 4 (Eq. overdet) as one persistent cooperative kernel for
// the mixed-precision path: conjugate gradients on
//     (Wp^* A A^* Wp) du = g,   Wp = P R^{-1},
// with every iteration reading A (complex64) from HBM exactly once.
//
// Each CTA owns every G-th 16-column sub-panel of A (m <= 512 rows). A sub-panel
// (m x 16 complex64, 128 bytes per row) is brought into shared memory by 2-D TMA
// loads (cp.async.bulk.tensor, 128-byte swizzle) through a three-stage mbarrier
// pipeline. Each thread copies eight columns of two rows of it into registers (the
// stage is refilled at once) and uses them twice:
//     q_j  = sum_i conj(A_ij) w_i      (in-thread over its two rows, then a warp
//                                        butterfly and a fixed-order sum over warps)
//     t_i += sum_j A_ij q_j            (per-thread accumulators)
// so A^* w and A (A^* w) cost one pass. Successive iterations walk the own
// sub-panels in opposite directions: the last kStages sub-panels of one
// iteration are still in shared memory when the next begins (no reload), and
// the ones read just before them were loaded with an L2 evict-last hint. The
// FP64 parts (w = Wp p, Np = Wp^* t, the CG scalars) are spread over the CTAs by
// rows, between four grid barriers per iteration (bounded waits, see
// common.cuh); s and u of a CTA's rows stay in its registers, and dy = Wp u is
// accumulated as the sum of alpha_k w_k by the owners of the rows of w. The
// search direction p is kept, identically, in every CTA's shared memory.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

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
  const int *skip;
  int withhold;
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

// warp sums of 16 floats, transposed: afterwards v[0] of lane L holds the warp
// sum of v[L & 15] (a butterfly: at offset o each lane keeps the half of its
// remaining values selected by its bit o and receives the partner's partial sums;
// the last step adds the two half-warps)
__device__ __forceinline__ void warp_transpose_sum16(float (&v)[16], int lane) {
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool lo = !(lane & o);
#pragma unroll
    for (int k = 0; k < o; ++k) {
      const float send = lo ? v[k + o] : v[k];
      const float keep = lo ? v[k] : v[k + o];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// warp sums of re and im in one butterfly (lanes 0-15 carry re, 16-31 im: five
// FP64 additions instead of ten); the result is valid in lane 0
__device__ __forceinline__ zd warp_sum_pair(double re, double im, int lane) {
  const bool lo = lane < 16;
  double z = (lo ? re : im) + __shfl_xor_sync(0xffffffffu, lo ? im : re, 16);
  z += __shfl_xor_sync(0xffffffffu, z, 8);
  z += __shfl_xor_sync(0xffffffffu, z, 4);
  z += __shfl_xor_sync(0xffffffffu, z, 2);
  z += __shfl_xor_sync(0xffffffffu, z, 1);
  return {z, __shfl_sync(0xffffffffu, z, 16)};
}

// out[i] = sum_k M[i][k] v[k] for i in [r0, r1): one warp per row (FP64), v in
// shared memory; out is global (gout) or shared (sout[i - r0]). Returns, in lane 0,
// the warp's last row.
__device__ __forceinline__ zd rows_dot(const zd *__restrict__ M, const zd *v, int m, int r0, int r1, zd *gout,
                                       zd *sout) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  zd last = {0.0, 0.0};
  for (int i = r0 + wid; i < r1; i += nw) {
    const zd *row = M + (int64_t)i * m;
    double re = 0.0, im = 0.0;
    for (int k = lane; k < m; k += 32) {
      const zd a = row[k], x = v[k];
      re = fma(a.re, x.re, fma(-a.im, x.im, re));
      im = fma(a.re, x.im, fma(a.im, x.re, im));
    }
    const zd r = warp_sum_pair(re, im, lane);
    if (lane == 0) {
      if (gout) gout[i] = r;
      else sout[i - r0] = r;
    }
    last = r;
  }
  return last;
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
  zd *np_s = v_s + m;                                              // m: Np of the own u-space rows
  float *q_f = reinterpret_cast<float *>(np_s + m);                // 32: q of the current sub-panel
  uint64_t *mbar = reinterpret_cast<uint64_t *>(q_f + 2 * kPanel); // kStages
  __shared__ double red[32];
  __shared__ double s_scal[4];
  __shared__ double s_qq[kCgThreads / 32];
  __shared__ float s_red[kCgThreads / 32][32];
  // an asynchronous solve that has stopped: every CTA reads the same word (written by an
  // earlier kernel of the stream), so all return before the first grid barrier
  if (P.skip && *P.skip) return;
  // a test of the bounded waits: CTA 0 leaves before it issues any copy or arrives anywhere,
  // so the others' first grid barrier runs out after limit_ns and they report ETIMEOUT
  if (P.withhold && blockIdx.x == 0) return;

  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int r0 = (int)((long long)m * b / G), r1 = (int)((long long)m * (b + 1) / G);  // own rows
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
  // dy = Wp u = sum over the iterations of alpha_k Wp p_k = sum alpha_k w_k: when every warp
  // has at most one own row, lane 0 of warp w accumulates row r0 + w of it from the w_k it
  // computed (no product with Wp after the loop)
  const bool acc_dy = (m + G - 1) / G <= kCgThreads / 32;
  const bool dy_row = acc_dy && lane == 0 && r0 + wid < r1;
  zd w_mine = {0.0, 0.0}, dy_mine = {0.0, 0.0};
  // s and u of the own row r0 + tid live in registers (only this CTA updates them)
  const bool own_su = tid < r1 - r0;
  zd s_reg = own_su ? P.g[r0 + tid] : zd{0.0, 0.0};
  zd u_reg = {0.0, 0.0};
  double gamma = block_sum(loc, red);
  const double gamma0 = gamma;
  bool done = !(gamma > 0.0);
  uint32_t parity[kStages] = {};
  const uint64_t pol_first = policy_evict_first(), pol_last = policy_evict_last();
  int it = 0;
  bool ok = true;
  // the first sweep's first stages do not depend on w: start them now, under the set-up
  // and the first w = Wp p (until that sweep begins they are this thread's to wait for)
  const int nearly = nsp < kStages ? nsp : kStages;
  bool early_pending = !done && nearly > 0;
  if (tid == 0 && early_pending) {
    for (int e = 0; e < nearly; ++e) {
      mbar_expect_tx(&mbar[e], stage_tx);
      for (int bx = 0; bx < nbox; ++bx)
        tma_load_2d(stage(e) + bx * kBoxRows * 128, &amap, (b + e * G) * 2 * kPanel, bx * kBoxRows, &mbar[e],
                    e >= nsp - P.keep ? pol_last : pol_first);
    }
  }

  while (!done && it < P.maxit) {
    // P1: w = Wp p (own rows)
    w_mine = rows_dot(P.Wp, p_s, m, r0, r1, P.w, nullptr);
    if (!grid_sync(P.bar, G, epoch, P.limit_ns)) { ok = false; break; }

    // P2: q = A^* w and t = A q over the own sub-panels, A read once.
    // Thread (warp wid, lane) takes columns 8h..8h+7 (h = wid & 1) of rows ra and
    // ra + 256 (ra = 32 (wid >> 1) + lane) of every sub-panel into registers: its two
    // rows' terms of a q_j are added in the thread, so the warp reduces 16 values.
    const int h = wid & 1, ra = 32 * (wid >> 1) + lane, rb = ra + 256;
    const zf w0 = ra < m ? cvt<float>(P.w[ra]) : zf{0.f, 0.f};
    const zf w1 = rb < m ? cvt<float>(P.w[rb]) : zf{0.f, 0.f};
    zf t0 = {0.f, 0.f}, t1 = {0.f, 0.f};
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
    early_pending = false;  // issued before the loop; waited for below like any other stage
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
      // (a) the thread's two half rows (four 16-byte swizzled chunks each) into registers;
      //     their terms conj(A_ij) w_i of the 8 q_j, summed over the warp by a butterfly
      float4 a0[4], a1[4];
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        a0[kc] = make_float4(0.f, 0.f, 0.f, 0.f);
        a1[kc] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (w_ok) {
        const int ch = 4 * h;
        if (ra < rows_pad) {
#pragma unroll
          for (int kc = 0; kc < 4; ++kc)
            a0[kc] = *reinterpret_cast<const float4 *>(S + ra * 128 + (((ch + kc) ^ (ra & 7)) << 4));
        }
        if (rb < rows_pad) {
#pragma unroll
          for (int kc = 0; kc < 4; ++kc)
            a1[kc] = *reinterpret_cast<const float4 *>(S + rb * 128 + (((ch + kc) ^ (rb & 7)) << 4));
        }
      }
      float c[16];
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        c[4 * kc + 0] = fmaf(a0[kc].x, w0.re, fmaf(a0[kc].y, w0.im, fmaf(a1[kc].x, w1.re, a1[kc].y * w1.im)));
        c[4 * kc + 1] = fmaf(a0[kc].x, w0.im, fmaf(-a0[kc].y, w0.re, fmaf(a1[kc].x, w1.im, -a1[kc].y * w1.re)));
        c[4 * kc + 2] = fmaf(a0[kc].z, w0.re, fmaf(a0[kc].w, w0.im, fmaf(a1[kc].z, w1.re, a1[kc].w * w1.im)));
        c[4 * kc + 3] = fmaf(a0[kc].z, w0.im, fmaf(-a0[kc].w, w0.re, fmaf(a1[kc].z, w1.im, -a1[kc].w * w1.re)));
      }
      warp_transpose_sum16(c, lane);
      if (lane < 16) s_red[wid][lane] = c[0];
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
      if (wid == 0) {  // lane = 16 h' + v: value v of column half h', over the 8 warps of that half
        float qf = 0.f;
#pragma unroll
        for (int w2 = 0; w2 < kCgThreads / 64; ++w2) qf += s_red[2 * w2 + (lane >> 4)][lane & 15];
        q_f[lane] = qf;
        if (sp * kPanel + (lane >> 1) < P.n) qq_loc = fmaf(qf, qf, qq_loc);
      }
      __syncthreads();
      // (c) t_i += sum_j A_ij q_j over the thread's 8 columns, from the registers
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        const float4 q4 = *reinterpret_cast<const float4 *>(q_f + 16 * h + 4 * kc);
        mac(t0, zf{a0[kc].x, a0[kc].y}, zf{q4.x, q4.y});
        mac(t0, zf{a0[kc].z, a0[kc].w}, zf{q4.z, q4.w});
        mac(t1, zf{a1[kc].x, a1[kc].y}, zf{q4.x, q4.y});
        mac(t1, zf{a1[kc].z, a1[kc].w}, zf{q4.z, q4.w});
      }
    }
    if (!ok) break;
    {  // the two column halves of a row meet in shared memory (np_s is free here)
      zf *th = reinterpret_cast<zf *>(np_s);
      if (h == 1) {
        if (ra < m) th[ra] = t0;
        if (rb < m) th[rb] = t1;
      }
      __syncthreads();
      if (h == 0) {
        if (ra < m) P.tpart[(int64_t)b * m + ra] = t0 + th[ra];
        if (rb < m) P.tpart[(int64_t)b * m + rb] = t1 + th[rb];
      }
    }
    if (wid == 0) {  // only warp 0 accumulated |q|^2
      qq_loc = warp_sum(qq_loc);
      if (lane == 0) P.qq_part[b] = (double)qq_loc;
    }
    if (!grid_sync(P.bar, G, epoch, P.limit_ns)) { ok = false; break; }

    // P3a: t (own rows) = sum of the partials; qq = sum of the per-CTA |q|^2
    for (int i = r0 + wid - 1; wid > 0 && i < r1; i += (blockDim.x >> 5) - 1) {   // warps 1..15
      double re = 0.0, im = 0.0;
      for (int c = lane; c < G; c += 32) {
        const zf v = ldcg(P.tpart + (int64_t)c * m + i);
        re += (double)v.re;
        im += (double)v.im;
      }
      const zd ti = warp_sum_pair(re, im, lane);
      if (lane == 0) stcg(P.t + i, ti);
    }
    if (wid == 0) {  // the CG scalars are formed by one thread (an FP64 division is a
      double qs = 0.0;  // long chain of FP64 instructions) and read by all
      for (int c = lane; c < G; c += 32) qs += ldcg(P.qq_part + c);
      qs = warp_sum(qs);
      if (lane == 0) {
        s_scal[0] = qs;
        s_scal[2] = qs > 0.0 ? gamma / qs : 0.0;
      }
    }
    if (!grid_sync(P.bar, G, epoch, P.limit_ns)) { ok = false; break; }
    const double qq = s_scal[0];
    const double alpha = s_scal[2];
    if (dy_row) {
      dy_mine.re = fma(alpha, w_mine.re, dy_mine.re);
      dy_mine.im = fma(alpha, w_mine.im, dy_mine.im);
    }

    // P3b: Np = Wp^* t (own rows); s -= alpha Np; u += alpha p; partial ||s||^2
    for (int i = tid; i < m; i += blockDim.x) v_s[i] = ldcg(P.t + i);
    __syncthreads();
    rows_dot(P.WpH, v_s, m, r0, r1, nullptr, np_s);
    __syncthreads();
    double gl = 0.0;
    if (own_su) {
      const zd np = np_s[tid], pi = p_s[r0 + tid];
      s_reg.re = fma(-alpha, np.re, s_reg.re);
      s_reg.im = fma(-alpha, np.im, s_reg.im);
      u_reg.re = fma(alpha, pi.re, u_reg.re);
      u_reg.im = fma(alpha, pi.im, u_reg.im);
      stcg(P.s + r0 + tid, s_reg);
      gl = fma(s_reg.re, s_reg.re, s_reg.im * s_reg.im);
    }
    if (r1 - r0 <= 32) {  // the own rows are all in warp 0
      if (wid == 0) {
        gl = warp_sum(gl);
        if (lane == 0) P.gg_part[b] = gl;
      }
    } else {
      gl = warp_sum(gl);
      if (lane == 0) s_qq[wid] = gl;
      __syncthreads();
      if (tid == 0) {
        double gs = 0.0;
        for (int w2 = 0; w2 < kCgThreads / 32; ++w2) gs += s_qq[w2];
        P.gg_part[b] = gs;
      }
    }
    if (!grid_sync(P.bar, G, epoch, P.limit_ns)) { ok = false; break; }

    // P4: gamma' and the new direction, identically in every CTA (s loaded first)
    const zd s_all = tid < m ? ldcg(P.s + tid) : zd{0.0, 0.0};
    if (wid == 0) {
      double gs = 0.0;
      for (int c = lane; c < G; c += 32) gs += ldcg(P.gg_part + c);
      gs = warp_sum(gs);
      if (lane == 0) {
        s_scal[1] = gs;
        s_scal[3] = gamma > 0.0 ? gs / gamma : 0.0;
      }
    }
    __syncthreads();
    const double gnew = s_scal[1];
    const double beta = s_scal[3];
    if (tid < m) {
      zd pi = p_s[tid];
      pi.re = fma(beta, pi.re, s_all.re);
      pi.im = fma(beta, pi.im, s_all.im);
      p_s[tid] = pi;
    }
    gamma = gnew;
    ++it;
    if (gnew <= P.tol2 * gamma0 || !(qq > 0.0)) done = true;
    __syncthreads();
  }
  if (early_pending && tid == 0) {  // the loop ended before the first sweep: wait for its copies
    for (int e = 0; e < nearly; ++e) mbar_wait(&mbar[e], 0, P.limit_ns);
  }
  if (!ok) {
    if (tid == 0) atomicExch(P.err, 1);
    // no TMA load is left in flight: every issued stage was waited for above
    return;
  }
  // dy = Wp u
  if (own_su) stcg(P.u + r0 + tid, u_reg);
  if (acc_dy) {
    if (dy_row) P.dy[r0 + wid] = dy_mine;
  } else {
    if (!grid_sync(P.bar, G, epoch, P.limit_ns)) {
      if (tid == 0) atomicExch(P.err, 1);
      return;
    }
    for (int i = tid; i < m; i += blockDim.x) v_s[i] = ldcg(P.u + i);
    __syncthreads();
    rows_dot(P.Wp, v_s, m, r0, r1, P.dy, nullptr);
  }
  if (b == 0 && tid == 0) {
    P.sc->iters = it;
    P.sc->gamma = gamma;
    P.sc->gamma0 = gamma0;
    P.sc->done = done ? 1 : 0;
  }
}


// ---- one-pass CG product for 512 < m <= 4096 -------------------------------------
// t = A (A^* w) and ||A^* w||^2 for one mixed-precision CG iteration, reading A (complex64)
// from HBM once. A cluster of CL = ceil(m / 512) CTAs shares each 16-column sub-panel: CTA r
// holds rows 512 r .. 512 r + 511 of it (two rows and eight columns per thread, the register
// layout of cg_fused_kernel), brought into shared memory by 2-D TMA loads through a three-stage
// mbarrier ring. Per sub-panel every CTA forms the partial q_j = sum_i conj(A_ij) w_i over its
// rows, writes it into every CTA of the cluster (distributed shared memory, double-buffered by
// the sub-panel's parity), meets the others at one cluster barrier, adds the CL partials in rank
// order (so q is the same in every CTA) and accumulates t_i += sum_j A_ij q_j for its rows. The
// clusters take every NC-th sub-panel, so the grid's reads sweep every row front to back
// together; each cluster writes its partial t, added in FP64 by cg_pair_finish_kernel. Every
// CTA of a cluster runs the same number of cluster barriers whatever happens (a load that does
// not arrive within the wait limit turns the rest of the pass into zeros and reports the error),
// so no CTA can be left waiting at one.
// the cluster barrier in two halves (every thread of the cluster arrives, then waits)
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

constexpr int kPairRows = 2 * kBoxRows;   // rows per CTA
constexpr int kPairMaxCluster = 8;
constexpr int kPairStageBytes = kPairRows * 128;

struct CgPairParams {
  int m, n, nsub;        // rows, columns, 16-column sub-panels
  const zf *w;           // m
  zf *tpart;             // clusters x m
  double *qq_part;       // clusters
  int *err;
  uint64_t limit_ns;
  const int *skip;
};

__global__ void __launch_bounds__(kCgThreads, 1)
cg_pair_kernel(const __grid_constant__ CUtensorMap amap, const CgPairParams P) {
  namespace cgr = cooperative_groups;
  extern __shared__ unsigned char smem_raw[];
  __shared__ float xch[2][kPairMaxCluster][2 * kPanel];   // every rank's partial q, by parity
  __shared__ float s_red[kCgThreads / 32][32];
  __shared__ __align__(16) float q_f[2 * kPanel];
  __shared__ zf th[kPairRows];
  __shared__ uint64_t mbar[kStages];
  // an asynchronous or finished CG: every CTA reads the same word, so the whole grid returns
  if (P.skip && *P.skip) return;
  cgr::cluster_group cl = cgr::this_cluster();
  const int CL = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int NC = (int)(gridDim.x / CL), c = (int)(blockIdx.x / CL);
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  auto stage = [&](int q) { return base + q * kPairStageBytes; };
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int r0 = rank * kPairRows;
  const int nsp = P.nsub > c ? (P.nsub - c + NC - 1) / NC : 0;   // the same in every CTA of the cluster
  if (tid == 0) {
    for (int q = 0; q < kStages; ++q) mbar_init(&mbar[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const uint64_t pol = policy_evict_first();
  uint32_t pending = 0;   // thread 0: bit q set while a load issued into stage q is not waited for
  auto issue = [&](int e) {
    const int sl = e % kStages;
    mbar_expect_tx(&mbar[sl], (uint32_t)kPairStageBytes);
    for (int bx = 0; bx < kPairRows / kBoxRows; ++bx)
      tma_load_2d(stage(sl) + bx * kBoxRows * 128, &amap, (c + e * NC) * 2 * kPanel, r0 + bx * kBoxRows, &mbar[sl],
                  pol);
    pending |= 1u << sl;
  };
  if (tid == 0)
    for (int e = 0; e < kStages && e < nsp; ++e) issue(e);
  const int h = wid & 1, ra = 32 * (wid >> 1) + lane, rb = ra + kBoxRows;
  const int ga = r0 + ra, gb = r0 + rb;
  const zf w0 = ga < P.m ? P.w[ga] : zf{0.f, 0.f};
  const zf w1 = gb < P.m ? P.w[gb] : zf{0.f, 0.f};
  zf t0 = {0.f, 0.f}, t1 = {0.f, 0.f};
  float qq_loc = 0.f;
  uint32_t parity = 0;   // bit q: the parity of stage q's next phase, as this thread saw them complete
  bool ok = true;
  // Sub-panel e's partial q leaves for the peers before its t is formed: the cluster barrier of
  // e stays open while the CTA reads sub-panel e + 1 and forms its partial (its registers are
  // kept), and only then waits, adds the partials of e and updates t from e's registers.
  float4 p0[4], p1[4];   // the registers of the sub-panel whose q is in flight
  float pq = 0.f;        // warp 0: this CTA's partial q of the newest sub-panel
  // (a) sub-panel e into registers (a0, a1), its partial q into s_red and, in warp 0, pq
  auto take = [&](int e, float4 (&a0)[4], float4 (&a1)[4]) {
    const int st = e % kStages;
    bool w_ok = true;
    if (ok) {
      w_ok = mbar_wait(&mbar[st], (parity >> st) & 1u, P.limit_ns);
      if (w_ok) parity ^= 1u << st;
    }
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      a0[kc] = make_float4(0.f, 0.f, 0.f, 0.f);
      a1[kc] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (ok && w_ok) {
      const unsigned char *S = stage(st);
      const int ch = 4 * h;
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        a0[kc] = *reinterpret_cast<const float4 *>(S + ra * 128 + (((ch + kc) ^ (ra & 7)) << 4));
        a1[kc] = *reinterpret_cast<const float4 *>(S + rb * 128 + (((ch + kc) ^ (rb & 7)) << 4));
      }
    }
    float cq[16];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      cq[4 * kc + 0] = fmaf(a0[kc].x, w0.re, fmaf(a0[kc].y, w0.im, fmaf(a1[kc].x, w1.re, a1[kc].y * w1.im)));
      cq[4 * kc + 1] = fmaf(a0[kc].x, w0.im, fmaf(-a0[kc].y, w0.re, fmaf(a1[kc].x, w1.im, -a1[kc].y * w1.re)));
      cq[4 * kc + 2] = fmaf(a0[kc].z, w0.re, fmaf(a0[kc].w, w0.im, fmaf(a1[kc].z, w1.re, a1[kc].w * w1.im)));
      cq[4 * kc + 3] = fmaf(a0[kc].z, w0.im, fmaf(-a0[kc].w, w0.re, fmaf(a1[kc].z, w1.im, -a1[kc].w * w1.re)));
    }
    warp_transpose_sum16(cq, lane);
    if (lane < 16) s_red[wid][lane] = cq[0];
    // the stage is in registers everywhere and the warp sums are in place; a failed wait
    // anywhere in the CTA ends its loads (the cluster barriers still run)
    const bool was_ok = ok;
    if (__syncthreads_or(ok && !w_ok)) ok = false;
    if (tid == 0) {
      if (was_ok && w_ok) pending &= ~(1u << st);   // thread 0 saw this stage's copy arrive
      if (ok && e + kStages < nsp) issue(e + kStages);
    }
    if (wid == 0) {
      float qf = 0.f;
#pragma unroll
      for (int w2 = 0; w2 < kCgThreads / 64; ++w2) qf += s_red[2 * w2 + (lane >> 4)][lane & 15];
      pq = qf;
    }
  };
  // (b) the partial of sub-panel e into every CTA of the cluster (after the barrier of e - 1:
  // every peer has read that slot's previous contents, those of e - 2)
  auto send = [&](int e) {
    if (wid == 0)
      for (int r = 0; r < CL; ++r) *cl.map_shared_rank(&xch[e & 1][rank][lane], r) = pq;
  };
  // (c) the total q of sub-panel e (after its barrier) and t from its registers
  auto finish = [&](int e, const float4 (&a0)[4], const float4 (&a1)[4]) {
    if (wid == 0) {
      float qt = 0.f;
      for (int r = 0; r < CL; ++r) qt += xch[e & 1][r][lane];
      q_f[lane] = qt;
      if (rank == 0 && (c + e * NC) * kPanel + (lane >> 1) < P.n) qq_loc = fmaf(qt, qt, qq_loc);
    }
    __syncthreads();
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      const float4 q4 = *reinterpret_cast<const float4 *>(q_f + 16 * h + 4 * kc);
      mac(t0, zf{a0[kc].x, a0[kc].y}, zf{q4.x, q4.y});
      mac(t0, zf{a0[kc].z, a0[kc].w}, zf{q4.z, q4.w});
      mac(t1, zf{a1[kc].x, a1[kc].y}, zf{q4.x, q4.y});
      mac(t1, zf{a1[kc].z, a1[kc].w}, zf{q4.z, q4.w});
    }
  };
  if (nsp > 0) {
    take(0, p0, p1);
    send(0);
    cluster_arrive();
    for (int e = 1; e < nsp; ++e) {
      float4 a0[4], a1[4];
      take(e, a0, a1);
      cluster_wait();       // the partials of e - 1 are in place everywhere
      send(e);
      finish(e - 1, p0, p1);
      cluster_arrive();
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        p0[kc] = a0[kc];
        p1[kc] = a1[kc];
      }
    }
    cluster_wait();
    finish(nsp - 1, p0, p1);
  }
  // the two column halves of a row meet in shared memory
  if (h == 1) {
    th[ra] = t0;
    th[rb] = t1;
  }
  __syncthreads();
  if (h == 0 && ok) {
    if (ga < P.m) P.tpart[(int64_t)c * P.m + ga] = t0 + th[ra];
    if (gb < P.m) P.tpart[(int64_t)c * P.m + gb] = t1 + th[rb];
  }
  if (rank == 0 && wid == 0) {  // only rank 0 accumulated |q|^2
    qq_loc = warp_sum(qq_loc);
    if (lane == 0) P.qq_part[c] = (double)qq_loc;
  }
  if (!ok && tid == 0) {
    atomicExch(P.err, 1);
    for (int q = 0; q < kStages; ++q)   // copies still in flight (bounded waits)
      if ((pending >> q) & 1u) mbar_wait(&mbar[q], (parity >> q) & 1u, P.limit_ns);
  }
  cl.sync();   // no CTA leaves while a peer may still write into its shared memory
}

// t[i] = sum over the clusters of tpart[c][i], in FP64 and in cluster order
__global__ void __launch_bounds__(256)
cg_pair_finish_kernel(const zf *__restrict__ tpart, int nc, int m, zd *__restrict__ t, const int *__restrict__ skip) {
  if (skip && *skip) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double re = 0.0, im = 0.0;
  for (int c = 0; c < nc; ++c) {
    const zf v = tpart[(int64_t)c * m + i];
    re += (double)v.re;
    im += (double)v.im;
  }
  t[i] = {re, im};
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
  return 1024 + kStages * rows_pad * 128 + 3 * (size_t)m * sizeof(zd) + 2 * kPanel * sizeof(float) +
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
  P.skip = a.skip;
  P.withhold = a.withhold;
  const size_t smem = cg_fused_smem(a.m);
  cudaError_t e = cudaFuncSetAttribute(cg_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int NP = (int)((a.n + kPanel - 1) / kPanel);
  const int G = a.grid < NP ? a.grid : NP;
  // sub-panels per CTA kept in L2 between sweeps: a share of L2 (80 % unless tuned)
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
    l2 = 0;
  const double stage_bytes = (double)P.nbox * kBoxRows * 128;
  const double frac = a.keep_frac >= 0.0 ? a.keep_frac : 0.8;
  P.keep = (int)(frac * (double)l2 / ((double)G * stage_bytes));
  // a cooperative launch (every CTA resident: the grid barriers need it), made through
  // cudaLaunchKernelEx so that it can also be captured into a CUDA graph
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kCgThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  return cudaLaunchKernelEx(&cfg, cg_fused_kernel, map, P);
}

// ---- the one-pass product's launch ---------------------------------------------------
bool cg_pair_supported(int64_t m, int64_t n, int64_t lda, const void *A) {
  return m > kMaxFusedRows && m <= (int64_t)kPairRows * kPairMaxCluster && n >= kPanel && (lda % 2) == 0 &&
         (((uintptr_t)A) & 15) == 0 && get_encode() != nullptr;
}

static size_t cg_pair_smem() { return 1024 + (size_t)kStages * kPairStageBytes; }
static int cg_pair_cluster_size(int64_t m) { return (int)((m + kPairRows - 1) / kPairRows); }

static cudaLaunchConfig_t cg_pair_config(int cl, int nc, cudaLaunchAttribute *attr, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(cl * nc));
  cfg.blockDim = dim3(kCgThreads);
  cfg.dynamicSmemBytes = cg_pair_smem();
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// clusters of the one-pass product: as many as are resident at once (one CTA per SM), at most
// one per sub-panel; 0 when the cluster shape cannot be launched
int cg_pair_clusters(int64_t m, int64_t n) {
  if (m <= kMaxFusedRows || m > (int64_t)kPairRows * kPairMaxCluster) return 0;
  if (cudaFuncSetAttribute(cg_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cg_pair_smem()) !=
      cudaSuccess)
    return 0;
  const int cl = cg_pair_cluster_size(m);
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cg_pair_config(cl, 1, attr, nullptr);
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, cg_pair_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int64_t nsub = (n + kPanel - 1) / kPanel;
  return (int)std::min<int64_t>(nc, nsub);
}

cudaError_t launch_cg_pair(const CgPairArgs &a, cudaStream_t st) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc || a.nc < 1) return cudaErrorNotSupported;
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
  CgPairParams P;
  P.m = (int)a.m;
  P.n = (int)a.n;
  P.nsub = (int)((a.n + kPanel - 1) / kPanel);
  P.w = (const zf *)a.w32;
  P.tpart = (zf *)a.tpart;
  P.qq_part = a.qq_part;
  P.err = a.err;
  P.limit_ns = a.limit_ns;
  P.skip = a.skip;
  cudaError_t e = cudaFuncSetAttribute(cg_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)cg_pair_smem());
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = cg_pair_config(cg_pair_cluster_size(a.m), a.nc, attr, st);
  note_launch();
  if ((e = cudaLaunchKernelEx(&cfg, cg_pair_kernel, map, P)) != cudaSuccess) return e;
  note_launch();
  cg_pair_finish_kernel<<<(unsigned)((a.m + 255) / 256), 256, 0, st>>>((const zf *)a.tpart, a.nc, (int)a.m,
                                                                       (zd *)a.t, a.skip);
  return cudaGetLastError();
}

}  // namespace mn
