// qr.cu -- Step 2 of the algorithm (Eq. lineq): Householder QR with column
// pivoting of the sketch, Y P = Q R (the "classical pivoted QR based on
// Householder reflections" of Section 7, Golub & Van Loan ch. 5), then the
// preconditioner P R^{-1} used by Step 4.
//
// qrp_mail_kernel is one cooperative grid (up to two CTAs per SM). Per step k
// every CTA
//   1. takes the pivot p = the first column of largest partial norm among the
//      remaining ones, in the logical column order LAPACK's swaps produce
//      (agreed on at the end of the previous step),
//   2. in one block reduction forms ||Y[k+1:, p]||^2 and, for its share of the
//      trailing columns j, sum_r conj(Y[r,p]) Y[r,j] (the reflector's scale is
//      not needed for these sums, so all CTAs build the same reflector
//      H = I - tau v v^*, v = (1, Y[k+1:, p] / (Y[k,p] - beta)), beta real,
//      without waiting for each other),
//   3. applies H^* to its columns and downdates their partial norms (with
//      LAPACK's recomputation when the downdate loses half the digits),
//   4. posts its candidate for the next pivot and meets the others at a
//      mailbox exchange whose waits are bounded in time.
// The pivot column itself is left unscaled: only R and P are kept (Q is never
// needed: Steps 2-3 enter the solve through R alone, see solver.cu).
#include "common.cuh"
#include "kernels.h"

namespace mn {

constexpr int kQrThreads = 256;

__global__ void __launch_bounds__(kQrThreads)
qr_norms_kernel(const zd *__restrict__ Y, int l, double *__restrict__ vn1, double *__restrict__ vn2) {
  __shared__ double sc[kQrThreads / 32];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int r = threadIdx.x; r < l; r += blockDim.x) acc += abs2(Y[r + (int64_t)j * l]);
  const double t = block_sum(acc, sc);
  if (threadIdx.x == 0) { vn1[j] = sqrt(t); vn2[j] = sqrt(t); }
}

// Columns are assigned to CTAs afresh at every step: all CTAs keep the same
// logical order of the columns (a permutation updated by the same swaps
// LAPACK's zlaqp2 makes, so ties go to the same pivot as there), and CTA b
// takes the b-th equal share of the trailing positions k+1..m-1. Y stays in
// place in global memory (it is L2-resident for the sizes where the QR is
// latency-bound) and is read through L2 only (ld.global.cg), since other CTAs
// rewrite it between steps; the pivot column is staged in shared memory when
// it fits. Partial norms are indexed by physical column and double-buffered
// across steps.
//
// The steps are separated by a mailbox exchange instead of a counting
// barrier: after its update every CTA posts its own best candidate for the
// next pivot (largest partial norm, lowest logical position) and then raises
// its flag to k+1 with release semantics; every CTA polls all flags with
// acquire loads and reduces the posted candidates itself. The exchange is the
// step's only grid-wide synchronisation and also replaces a separate pivot
// search over all partial norms. Posts are double-buffered by the parity of k:
// a CTA can be at most one step ahead of any reader.
constexpr int kQrbThreads = 128;
constexpr int kQrMaxGrid = 320;

struct QrMail {
  unsigned long long key;  // bit pattern of the candidate's partial norm (non-negative), or 0
  int pos;                 // its logical position, or INT_MAX when the CTA had no columns
  int pad;
};

size_t qr_mail_bytes() { return 4 * (size_t)kQrMaxGrid + 2 * (size_t)kQrMaxGrid * 24 + 8 * (size_t)kQrMaxGrid; }

__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// On GB300 every FP64 warp instruction occupies the SM's FP64 pipe for tens of
// cycles, so the per-step scalar work is arranged to issue few of them: the
// pivot candidates are compared as integers (bit patterns of non-negative
// doubles), the block uses 4 warps so the reduction tree is short, and the
// factors of the own columns are computed by one lane each.
// The per-column loops are instantiated for the exact number of own columns
// (a predicated-off FP64 instruction still occupies the FP64 pipe).
template <int NC, int K>
__device__ __forceinline__ void qr_dots(const zd *yp, const zd *Y, const int *cols, int k, int l,
                                        zd *spiv, double (&part)[K]) {
  const zd *cp[NC > 0 ? NC : 1];
#pragma unroll
  for (int c = 0; c < NC; ++c) cp[c] = Y + (int64_t)cols[c] * l;
  int r = k + 1 + threadIdx.x;
  const int stride = blockDim.x;
  // several rows per thread in flight (the columns live in L2), fewer for many columns
  constexpr int U = NC <= 2 ? 4 : (NC <= 4 ? 2 : 1);
  for (; r + (U - 1) * stride < l; r += U * stride) {
    zd a[U], y[U][NC > 0 ? NC : 1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a[u] = ldcg(yp + r + u * stride);
#pragma unroll
      for (int c = 0; c < NC; ++c) y[u][c] = ldcg(cp[c] + r + u * stride);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (spiv) spiv[r + u * stride] = a[u];
      part[0] = fma(a[u].re, a[u].re, fma(a[u].im, a[u].im, part[0]));
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        part[1 + 2 * c] = fma(a[u].re, y[u][c].re, fma(a[u].im, y[u][c].im, part[1 + 2 * c]));
        part[2 + 2 * c] = fma(a[u].re, y[u][c].im, fma(-a[u].im, y[u][c].re, part[2 + 2 * c]));
      }
    }
  }
  for (; r < l; r += stride) {
    const zd a = ldcg(yp + r);
    if (spiv) spiv[r] = a;
    part[0] = fma(a.re, a.re, fma(a.im, a.im, part[0]));
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const zd y = ldcg(cp[c] + r);
      part[1 + 2 * c] = fma(a.re, y.re, fma(a.im, y.im, part[1 + 2 * c]));
      part[2 + 2 * c] = fma(a.re, y.im, fma(-a.im, y.re, part[2 + 2 * c]));
    }
  }
}

// rows k+1..l-1 of the own columns: y_j -= g_j v. The pivot column comes from
// shared memory (written by this same thread in qr_dots: the row mapping is
// the same) or from L2.
template <int NC>
__device__ __forceinline__ void qr_update(const zd *yp, zd *Y, const int *cols, const zd *g, int k, int l,
                                          const zd *spiv) {
  zd gg[NC > 0 ? NC : 1];
  zd *cp[NC > 0 ? NC : 1];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    gg[c] = g[c];
    cp[c] = Y + (int64_t)cols[c] * l;
  }
  int r = k + 1 + threadIdx.x;
  const int stride = blockDim.x;
  constexpr int U = NC <= 2 ? 4 : (NC <= 4 ? 2 : 1);
  for (; r + (U - 1) * stride < l; r += U * stride) {
    zd a[U], v[U][NC > 0 ? NC : 1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a[u] = spiv ? spiv[r + u * stride] : ldcg(yp + r + u * stride);
#pragma unroll
      for (int c = 0; c < NC; ++c) v[u][c] = ldcg(cp[c] + r + u * stride);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        zd t = v[u][c];
        t.re = fma(-gg[c].re, a[u].re, fma(gg[c].im, a[u].im, t.re));
        t.im = fma(-gg[c].re, a[u].im, fma(-gg[c].im, a[u].re, t.im));
        stcg(cp[c] + r + u * stride, t);
      }
    }
  }
  for (; r < l; r += stride) {
    const zd a = spiv ? spiv[r] : ldcg(yp + r);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      zd v = ldcg(cp[c] + r);
      v.re = fma(-gg[c].re, a.re, fma(gg[c].im, a.im, v.re));
      v.im = fma(-gg[c].re, a.im, fma(-gg[c].im, a.re, v.im));
      stcg(cp[c] + r, v);
    }
  }
}

#define MN_QR_SWITCH(NACT, CALL0, CALLN)                      \
  switch (NACT) {                                             \
    case 0: CALL0; break;                                     \
    case 1: CALLN((MAXC >= 1 ? 1 : 0)); break;                \
    case 2: CALLN((MAXC >= 2 ? 2 : 0)); break;                \
    case 3: CALLN((MAXC >= 3 ? 3 : 0)); break;                \
    case 4: CALLN((MAXC >= 4 ? 4 : 0)); break;                \
    case 5: CALLN((MAXC >= 5 ? 5 : 0)); break;                \
    case 6: CALLN((MAXC >= 6 ? 6 : 0)); break;                \
    case 7: CALLN((MAXC >= 7 ? 7 : 0)); break;                \
    case 8: CALLN((MAXC >= 8 ? 8 : 0)); break;                \
    case 9: CALLN((MAXC >= 9 ? 9 : 0)); break;                \
    case 10: CALLN((MAXC >= 10 ? 10 : 0)); break;             \
    case 11: CALLN((MAXC >= 11 ? 11 : 0)); break;             \
    case 12: CALLN((MAXC >= 12 ? 12 : 0)); break;             \
    case 13: CALLN((MAXC >= 13 ? 13 : 0)); break;             \
    case 14: CALLN((MAXC >= 14 ? 14 : 0)); break;             \
    case 15: CALLN((MAXC >= 15 ? 15 : 0)); break;             \
    default: CALLN((MAXC >= 16 ? 16 : 0)); break;             \
  }

// best (key, pos) of the pair: larger key, then lower position
__device__ __forceinline__ void qr_better(long long &bv, int &bq, long long ov, int oq) {
  if (ov > bv || (ov == bv && oq < bq)) { bv = ov; bq = oq; }
}

template <int MAXC>
__global__ void __launch_bounds__(kQrbThreads)
qrp_mail_kernel(zd *Y, int l, int m, double *vnA, double *vnB, double *vn2, double *__restrict__ beta,
                int32_t *__restrict__ piv, zd *__restrict__ Rout, unsigned int *flags, QrMail *mail, int *err,
                uint64_t limit_ns, int stage) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zd *spiv = stage ? reinterpret_cast<zd *>(smem_raw) : nullptr;                 // l: pivot column
  int *perm = reinterpret_cast<int *>(smem_raw + (stage ? sizeof(zd) * (size_t)l : 0));  // logical -> physical
  constexpr int K = 1 + 2 * MAXC;
  constexpr int NW = kQrbThreads / 32;
  __shared__ double red_scratch[NW * K];
  __shared__ double red_out[K];
  __shared__ long long s_val[NW];
  __shared__ int s_idx[NW];
  __shared__ int s_fail[NW];
  __shared__ int s_col[MAXC];
  __shared__ zd s_g[MAXC];
  __shared__ double s_nv[MAXC];
  __shared__ int s_rec[MAXC];
  __shared__ int s_nact, s_nrec, s_q0, s_abort;

  const int G = gridDim.x, b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const double tol3z = sqrt(0x1.0p-53);
  for (int j = tid; j < m; j += blockDim.x) perm[j] = j;

  // pivot of step 0: first maximum of the initial norms
  {
    long long best = -1;
    int bpos = 0x7fffffff;
    for (int q = tid; q < m; q += blockDim.x) qr_better(best, bpos, __double_as_longlong(ldcg(vnA + q)), q);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      qr_better(best, bpos, __shfl_xor_sync(0xffffffffu, best, o), __shfl_xor_sync(0xffffffffu, bpos, o));
    if (lane == 0) { s_val[wid] = best; s_idx[wid] = bpos; }
    __syncthreads();
    if (tid == 0) {
      long long bv = s_val[0];
      int bq = s_idx[0];
      for (int w = 1; w < NW; ++w) qr_better(bv, bq, s_val[w], s_idx[w]);
      perm[0] = bq;
      perm[bq] = 0;
      if (b == 0) piv[0] = bq;
    }
  }

  for (int k = 0; k < m; ++k) {
    const double *vn_cur = (k & 1) ? vnB : vnA;
    double *vn_nxt = (k & 1) ? vnA : vnB;
    if (tid == 0) {
      const int T = m - k - 1;
      const int q0 = k + 1 + (int)(((long long)T * b) / G), q1 = k + 1 + (int)(((long long)T * (b + 1)) / G);
      int na = 0;
      for (int q = q0; q < q1; ++q) s_col[na++] = perm[q];
      s_nact = na;
      s_q0 = q0;
      s_nrec = 0;
    }
    __syncthreads();
    const int p = perm[k];
    const int nact = s_nact;
    const zd *yp = Y + (int64_t)p * l;

    // scalars the reflector step needs, loaded before the reduction
    const bool scal_lane = tid < (nact > 0 ? nact : 1);
    zd alpha = {0.0, 0.0}, yk = {0.0, 0.0};
    double v1 = 0.0, v2 = 1.0;
    if (scal_lane) {
      alpha = ldcg(yp + k);
      if (tid < nact) {
        const int j = s_col[tid];
        yk = ldcg(Y + (int64_t)j * l + k);
        v1 = ldcg(vn_cur + j);
        v2 = ldcg(vn2 + j);
      }
    }

    // 1. one reduction: ||Y[k+1:,p]||^2 and conj(Y[k+1:,p])^T Y[k+1:,j] for own columns
    double part[K];
#pragma unroll
    for (int c = 0; c < K; ++c) part[c] = 0.0;
#define MN_DOTS(NC) qr_dots<NC, K>(yp, Y, s_col, k, l, spiv, part)
    if (MAXC <= 16) {
      MN_QR_SWITCH(nact, MN_DOTS(0), MN_DOTS)
    } else {
      for (int r = k + 1 + tid; r < l; r += blockDim.x) {
        const zd a = ldcg(yp + r);
        if (spiv) spiv[r] = a;
        part[0] = fma(a.re, a.re, fma(a.im, a.im, part[0]));
#pragma unroll
        for (int c = 0; c < MAXC; ++c) {
          if (c < nact) {
            const zd y = ldcg(Y + r + (int64_t)s_col[c] * l);
            part[1 + 2 * c] = fma(a.re, y.re, fma(a.im, y.im, part[1 + 2 * c]));
            part[2 + 2 * c] = fma(a.re, y.im, fma(-a.im, y.re, part[2 + 2 * c]));
          }
        }
      }
    }
#undef MN_DOTS
    block_sum_k<double, K>(part, red_scratch, red_out);

    // 2. reflector H = I - tau v v^*, identical in every CTA (LAPACK zlarfg convention),
    //    computed by each lane that owns a column (one lane when the CTA has none), then
    //    that column's factor, its row k, and its partial-norm downdate
    if (scal_lane) {
      const double xn2 = red_out[0];
      zd tau = {0.0, 0.0}, scale = {0.0, 0.0};
      double bt;
      if (xn2 == 0.0 && alpha.im == 0.0) {
        bt = alpha.re;
      } else {
        const double mag = sqrt(alpha.re * alpha.re + alpha.im * alpha.im + xn2);
        bt = alpha.re >= 0.0 ? -mag : mag;
        const double ib = 1.0 / bt;
        tau = {(bt - alpha.re) * ib, -alpha.im * ib};
        const double dr = alpha.re - bt, di = alpha.im;
        const double iden = 1.0 / (dr * dr + di * di);
        scale = {dr * iden, -di * iden};
      }
      if (tid == 0 && (k % G) == b) beta[k] = bt;  // read back by this CTA when it writes R
      if (tid < nact) {
        const int c = tid;
        const int j = s_col[c];
        const zd d = {red_out[1 + 2 * c], red_out[2 + 2 * c]};
        zd w = yk;
        macc(w, scale, d);                      // w = y_k + conj(scale) d
        const zd f = conjg(tau) * w;            // H^* = I - conj(tau) v v^*
        s_g[c] = f * scale;
        const zd rk = yk - f;
        stcg(Y + (int64_t)j * l + k, rk);
        // LAPACK zlaqp2 downdate: vn1 *= sqrt(1 - (|r_k|/vn1)^2) unless that loses half the digits
        double nv = v1;
        if (v1 != 0.0) {
          const double t = sqrt(abs2(rk)) / v1;
          double temp = 1.0 - t * t;
          temp = temp < 0.0 ? 0.0 : temp;
          const double ratio = v1 / v2;
          if (temp * ratio * ratio <= tol3z) s_rec[atomicAdd(&s_nrec, 1)] = c;
          else nv = v1 * sqrt(temp);
        }
        s_nv[c] = nv;
      }
    }
    __syncthreads();

    // 3. apply H^* to the own columns, rows k+1..l-1
#define MN_UPD(NC) qr_update<NC>(yp, Y, s_col, s_g, k, l, spiv)
    if (MAXC <= 16) {
      MN_QR_SWITCH(nact, (void)0, MN_UPD)
    } else {
      for (int r = k + 1 + tid; r < l; r += blockDim.x) {
        const zd a = spiv ? spiv[r] : ldcg(yp + r);
#pragma unroll
        for (int c = 0; c < MAXC; ++c) {
          if (c < nact) {
            zd *y = Y + r + (int64_t)s_col[c] * l;
            zd v = ldcg(y);
            const zd g = s_g[c];
            v.re = fma(-g.re, a.re, fma(g.im, a.im, v.re));
            v.im = fma(-g.re, a.im, fma(-g.im, a.re, v.im));
            stcg(y, v);
          }
        }
      }
    }
#undef MN_UPD
    if (k == m - 1) break;
    const int nrec = s_nrec;
    for (int q = 0; q < nrec; ++q) {  // rare: recompute a partial norm from scratch
      __syncthreads();
      const int c = s_rec[q];
      const int j = s_col[c];
      double acc = 0.0;
      for (int r = k + 1 + tid; r < l; r += blockDim.x) acc += abs2(ldcg(Y + r + (int64_t)j * l));
      const double t = sqrt(block_sum(acc, red_scratch));
      if (tid == 0) {
        const double v = (k < l - 1) ? t : 0.0;
        s_nv[c] = v;
        stcg(vn2 + j, v);
      }
    }
    __syncthreads();

    // 4. post: new partial norms, the CTA's best candidate, then the flag (release)
    if (tid == 0) {
      long long bv = 0;
      int bq = 0x7fffffff;
      const int q0 = s_q0;
      for (int c = 0; c < nact; ++c) {
        const double v = s_nv[c];
        stcg(vn_nxt + s_col[c], v);
        qr_better(bv, bq, __double_as_longlong(v), q0 + c);
      }
      QrMail *slot = mail + (k & 1) * kQrMaxGrid + b;
      stcg(&slot->key, (unsigned long long)bv);
      stcg(&slot->pos, bq);
      __threadfence();
      st_release_u32(flags + b, (unsigned int)(k + 1));
    }

    // 5. exchange: wait for every CTA's post of step k, reduce the candidates
    long long best = -1;
    int bpos = 0x7fffffff, fail = 0;
    for (int c = tid; c < G && !fail; c += blockDim.x) {
      const unsigned int want = (unsigned int)(k + 1);
      if (ld_acquire_u32(flags + c) < want) {
        const uint64_t t0 = global_ns();
        while (ld_acquire_u32(flags + c) < want) {
          if (ld_volatile_i32(err)) { fail = 1; break; }
          if (global_ns() - t0 > limit_ns) { atomicExch(err, 1); fail = 1; break; }
        }
      }
      if (!fail) {
        const QrMail *slot = mail + (k & 1) * kQrMaxGrid + c;
        qr_better(best, bpos, (long long)ldcg(&slot->key), ldcg(&slot->pos));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      qr_better(best, bpos, __shfl_xor_sync(0xffffffffu, best, o), __shfl_xor_sync(0xffffffffu, bpos, o));
      fail |= __shfl_xor_sync(0xffffffffu, fail, o);
    }
    if (lane == 0) { s_val[wid] = best; s_idx[wid] = bpos; s_fail[wid] = fail; }
    __syncthreads();
    if (tid == 0) {
      long long bv = s_val[0];
      int bq = s_idx[0], fl = s_fail[0];
      for (int w = 1; w < NW; ++w) { qr_better(bv, bq, s_val[w], s_idx[w]); fl |= s_fail[w]; }
      s_abort = fl;
      if (!fl) {
        const int tmp = perm[k + 1];
        perm[k + 1] = perm[bq];
        perm[bq] = tmp;
        if (b == 0) piv[k + 1] = perm[k + 1];
      }
    }
    __syncthreads();
    if (s_abort) return;
  }

  // R in pivot order: R[i, k] = Y[i, perm[k]] above the diagonal, beta_k on it
  __syncthreads();
  for (int k = b; k < m; k += G) {
    const int pk = perm[k];
    for (int i = tid; i < m; i += blockDim.x) {
      zd v = {0.0, 0.0};
      if (i < k) v = ldcg(Y + i + (int64_t)pk * l);
      else if (i == k) v = {beta[k], 0.0};
      Rout[i + (int64_t)k * m] = v;
    }
  }
}

// ---- register-tiled form for sketches of up to 2048 rows ----------------------
// Same steps and the same arithmetic as qrp_mail_kernel, arranged for the case
// where every CTA owns at most two trailing columns and a column's trailing
// rows fit 16 per thread. Four row warps copy the pivot rows and the own
// columns' rows into shared memory with cp.async (all of a step's loads in
// flight at once, one L2 read per step; every thread reads back only the rows
// it copied, so no barrier guards the tiles). A fifth warp computes
// the reflector, the factors and the norm downdates. The owner of the best
// column posts that column's exact ||Y[k+2:, j]||^2 with its candidate, so the
// next step's reflector needs no pass over the pivot column, and CTAs without
// columns do no FP64 work at all.
//
// A post is two 64-bit words, each tagged with the step (18 bits) so that a
// reader polling with relaxed loads knows when both halves are current:
//   wa = tag | position (14 bits) | high 32 bits of the norm's bit pattern
//   wb = tag | low 31 bits of the norm's bit pattern
// (a non-negative double has a zero sign bit). The writer fences before the
// tagged stores (release); a reader fences after seeing all tags (acquire).
constexpr int kQrNoPos = 0x3FFF;
constexpr bool kQrWide = false;  // the one-CTA-per-SM tile (256 row threads): measured no faster

// posts, one entry per CTA and step parity, in three dense arrays (a poll of
// all CTAs reads few cache lines)
struct QrPosts {
  unsigned long long *wa, *wb;  // [2][kQrMaxGrid] tagged words
  double *xn2;                  // [2][kQrMaxGrid] the candidate's ||Y[k+2:, j]||^2
  unsigned long long *smw;      // [kQrMaxGrid] 2^40 | SM id of each CTA, posted once at launch
};

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Warp sums of K = 2, 4 or 8 values with a transposed butterfly: each level
// sends half of the values still held and adds the other half, so a lane
// issues K - 1 + 5 - log2(K) additions instead of 5 K. Afterwards lane
// L holds the sum of v[L / (32 / K)] when L is a multiple of 32 / K.
template <int K>
__device__ __forceinline__ double warp_sum_t(const double (&v)[K], int lane) {
  static_assert(K == 2 || K == 4 || K == 8, "K");
  double z;
  if (K == 8) {
    // level 16: keep v[0..3] (lanes 0-15) or v[4..7]; level 8: keep two of them; level 4: one
    const bool lo = !(lane & 16);
    double w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double keep = lo ? v[q % K] : v[(q + 4) % K], send = lo ? v[(q + 4) % K] : v[q % K];
      w[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    const bool lo2 = !(lane & 8);
    const double u0 = (lo2 ? w[0] : w[2]) + __shfl_xor_sync(0xffffffffu, lo2 ? w[2] : w[0], 8);
    const double u1 = (lo2 ? w[1] : w[3]) + __shfl_xor_sync(0xffffffffu, lo2 ? w[3] : w[1], 8);
    const bool lo3 = !(lane & 4);
    z = (lo3 ? u0 : u1) + __shfl_xor_sync(0xffffffffu, lo3 ? u1 : u0, 4);
  } else if (K == 4) {
    const bool lo = !(lane & 16);
    const double s0 = lo ? v[2 % K] : v[0], s1 = lo ? v[3 % K] : v[1 % K];
    const double w0 = (lo ? v[0] : v[2 % K]) + __shfl_xor_sync(0xffffffffu, s0, 16);
    const double w1 = (lo ? v[1 % K] : v[3 % K]) + __shfl_xor_sync(0xffffffffu, s1, 16);
    const bool lo2 = !(lane & 8);
    z = (lo2 ? w0 : w1) + __shfl_xor_sync(0xffffffffu, lo2 ? w1 : w0, 8);
    z += __shfl_xor_sync(0xffffffffu, z, 4);
  } else {
    const bool lo = !(lane & 16);
    z = (lo ? v[0] : v[1 % K]) + __shfl_xor_sync(0xffffffffu, lo ? v[1 % K] : v[0], 16);
    z += __shfl_xor_sync(0xffffffffu, z, 8);
    z += __shfl_xor_sync(0xffffffffu, z, 4);
  }
  z += __shfl_xor_sync(0xffffffffu, z, 2);
  z += __shfl_xor_sync(0xffffffffu, z, 1);
  return z;
}

struct QrRegShared {
  double red[8 * 8];     // row-warp partial sums (up to 8 row warps x 8 values)
  double nv[4];          // new partial norms of the own columns
  double from[4];        // slow path: ||Y[k+2:, j]||^2 of the own columns
  double scratch[16];
  zd g[4];               // factors of the own columns
  int fl[4];             // own column needs its norm recomputed
  int cand;              // own column posted (-1: decided after the update)
  long long key[9];
  int pos[9], cta[9], fail[9];
  int win, abort_;
  double xn2_0;
};

// one step for a CTA that owns NC trailing columns (positions q0..q0+NC-1)
template <int NC, int RPT, int ROWT>
__device__ __forceinline__ void qr_reg_step(zd *Y, const int l, const int k, const int G, const int b,
                                            const int *perm, const int q0, const double *vn_cur, double *vn_nxt,
                                            double *vn2, double *beta, zd *spiv, QrRegShared &S, QrPosts P,
                                            const int slot, const double xn2, const double tol3z) {
  constexpr int NCV = NC > 0 ? NC : 1;
  constexpr int K = 2 * NCV <= 2 ? 2 : (2 * NCV <= 4 ? 4 : 8);  // partial sums, padded to a power of two
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool rowt = tid < ROWT;
  const int p = perm[k];
  const zd *yp = Y + (int64_t)p * l;
  zd *cp[NCV];
#pragma unroll
  for (int c = 0; c < NC; ++c) cp[c] = Y + (int64_t)perm[q0 + c] * l;
  zd *sy = spiv + RPT * ROWT;  // own columns: sy[c * RPT * 128 + i * 128 + tid]
  constexpr int CS = RPT * ROWT;
  zd tau = {0.0, 0.0}, scale = {0.0, 0.0}, yk = {0.0, 0.0};
  double v1 = 0.0, v2 = 1.0;

  // rows of this thread: k + 1 + tid + i * 128 for i < ni (loops stop there: on
  // GB300 an FP64 instruction costs its pipe time even when predicated off)
  const int rem = l - (k + 1) - tid;
  const int ni = rem > 0 ? (rem + ROWT - 1) / ROWT : 0;

  // 1. dot products (row warps) while the scalar warp forms the reflector
  if (rowt) {
    if (NC > 0) {
#pragma unroll 4
      for (int i = 0; i < ni; ++i) {
        const int r = k + 1 + tid + i * ROWT;
        cp_async16(spiv + i * ROWT + tid, yp + r, 16);
#pragma unroll
        for (int c = 0; c < NC; ++c) cp_async16(sy + c * CS + i * ROWT + tid, cp[c] + r, 16);
      }
      cp_async_wait_all();
      double part[K];
#pragma unroll
      for (int c = 0; c < K; ++c) part[c] = 0.0;
#pragma unroll 4
      for (int i = 0; i < ni; ++i) {
        const zd a = spiv[i * ROWT + tid];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const zd yv = sy[c * CS + i * ROWT + tid];
          part[2 * c] = fma(a.re, yv.re, fma(a.im, yv.im, part[2 * c]));
          part[2 * c + 1] = fma(a.re, yv.im, fma(-a.im, yv.re, part[2 * c + 1]));
        }
      }
      const double z = warp_sum_t<K>(part, lane);
      if ((lane & (32 / K - 1)) == 0) S.red[wid * K + lane / (32 / K)] = z;
    }
  } else {
    const zd alpha = ldcg(yp + k);
    if (lane < NC) {
      const int j = perm[q0 + lane];
      yk = ldcg(Y + (int64_t)j * l + k);
      v1 = ldcg(vn_cur + j);
      v2 = ldcg(vn2 + j);
    }
    // H = I - tau v v^*, LAPACK zlarfg convention (beta real)
    double bt;
    if (xn2 == 0.0 && alpha.im == 0.0) {
      bt = alpha.re;
    } else {
      const double mag = sqrt(alpha.re * alpha.re + alpha.im * alpha.im + xn2);
      bt = alpha.re >= 0.0 ? -mag : mag;
      const double ib = 1.0 / bt;
      tau = {(bt - alpha.re) * ib, -alpha.im * ib};
      const double dr = alpha.re - bt, di = alpha.im;
      const double iden = 1.0 / (dr * dr + di * di);
      scale = {dr * iden, -di * iden};
    }
    if (lane == 0 && (k % G) == b) beta[k] = bt;  // read back by this CTA when it writes R
  }
  if (NC == 0) return;  // uniform over the CTA
  __syncthreads();

  // 2. factors, row k and partial-norm downdates (one lane per own column)
  if (!rowt) {
    int flag = 0;
    if (lane < NC) {
      const int c = lane;
      zd d = {0.0, 0.0};
#pragma unroll
      for (int w = 0; w < ROWT / 32; ++w) {
        d.re += S.red[w * K + 2 * c];
        d.im += S.red[w * K + 2 * c + 1];
      }
      zd w = yk;
      macc(w, scale, d);                      // w = y_k + conj(scale) d
      const zd f = conjg(tau) * w;            // H^* = I - conj(tau) v v^*
      S.g[c] = f * scale;
      const zd rk = yk - f;
      stcg(Y + (int64_t)perm[q0 + c] * l + k, rk);
      // LAPACK zlaqp2 downdate: vn1 *= sqrt(1 - (|r_k|/vn1)^2) unless that loses half the digits
      double nv = v1;
      if (v1 != 0.0) {
        const double t = sqrt(abs2(rk)) / v1;
        double temp = 1.0 - t * t;
        temp = temp < 0.0 ? 0.0 : temp;
        const double ratio = v1 / v2;
        if (temp * ratio * ratio <= tol3z) flag = 1;
        else nv = v1 * sqrt(temp);
      }
      S.nv[c] = nv;
      S.fl[c] = flag;
    }
    // candidate among the own columns, unless a norm must first be recomputed
    const unsigned fl = __ballot_sync(0xffffffffu, flag);
    long long key = lane < NC ? __double_as_longlong(S.nv[lane < NC ? lane : 0]) : -1;
    int pos = lane < NC ? lane : 0x7fffffff;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) qr_better(key, pos, __shfl_xor_sync(0xffffffffu, key, o), __shfl_xor_sync(0xffffffffu, pos, o));
    if (lane == 0) S.cand = fl ? -1 : pos;
  }
  __syncthreads();

  // 3. update the own columns' rows k+1.. and the candidate's ||Y[k+2:, j]||^2
  const int cand = S.cand;
  if (rowt) {
    zd g[NCV];
#pragma unroll
    for (int c = 0; c < NC; ++c) g[c] = S.g[c];
    double xs = 0.0;
    // the candidate's norm skips row k+1 (thread 0's first row)
    const int i0 = (tid == 0) ? 1 : 0;
    if (tid == 0 && ni > 0) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        zd t = sy[c * CS + tid];
        const zd a = spiv[tid];
        t.re = fma(-g[c].re, a.re, fma(g[c].im, a.im, t.re));
        t.im = fma(-g[c].re, a.im, fma(-g[c].im, a.re, t.im));
        if (cand < 0) sy[c * CS + tid] = t;
        stcg(cp[c] + k + 1, t);
      }
    }
#pragma unroll 4
    for (int i = i0; i < ni; ++i) {
      const int r = k + 1 + tid + i * ROWT;
      const zd a = spiv[i * ROWT + tid];
      zd v = {0.0, 0.0};
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        zd t = sy[c * CS + i * ROWT + tid];
        t.re = fma(-g[c].re, a.re, fma(g[c].im, a.im, t.re));
        t.im = fma(-g[c].re, a.im, fma(-g[c].im, a.re, t.im));
        if (cand < 0) sy[c * CS + i * ROWT + tid] = t;
        stcg(cp[c] + r, t);
        v = (c == 0 || cand == c) ? t : v;
      }
      if (cand >= 0) xs = fma(v.re, v.re, fma(v.im, v.im, xs));
    }
    if (cand >= 0) {
      xs = warp_sum(xs);
      if (lane == 0) S.red[wid] = xs;
    }
  }
  if (cand < 0) {
    // slow path (rare): exact norms of the flagged columns, then the candidate's norm
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double fs = 0.0, fr = 0.0;
      if (rowt) {
#pragma unroll
        for (int i = 0; i < ni; ++i) {
          const double q = abs2(sy[c * CS + i * ROWT + tid]);
          fs += q;
          if (tid + i > 0) fr += q;  // rows k+2..
        }
      }
      const double full = block_sum(fs, S.scratch);
      const double from = block_sum(fr, S.scratch);
      if (tid == ROWT) {
        if (S.fl[c]) {
          const double v = (k < l - 1) ? sqrt(full) : 0.0;
          S.nv[c] = v;
          stcg(vn2 + perm[q0 + c], v);
        }
        S.from[c] = from;
      }
    }
  }
  __syncthreads();

  // 4. post the candidate (release: fence, then the tagged words)
  if (!rowt) {
    if (lane < NC) stcg(vn_nxt + perm[q0 + lane], S.nv[lane]);
    __syncwarp();
    if (lane == 0) {
      int c0 = cand;
      double xsum;
      if (c0 >= 0) {
        xsum = 0.0;
        for (int w = 0; w < ROWT / 32; ++w) xsum += S.red[w];
      } else {
        long long bk = -1;
        int bq = 0x7fffffff;
        for (int c = 0; c < NC; ++c) qr_better(bk, bq, __double_as_longlong(S.nv[c]), c);
        c0 = bq;
        xsum = S.from[c0];
      }
      const unsigned long long key = (unsigned long long)__double_as_longlong(S.nv[c0]);
      const unsigned long long tag = (unsigned long long)((k + 1) & 0x3FFFF) << 46;
      stcg(P.xn2 + slot, xsum);
      __threadfence();
      st_relaxed_u64(P.wa + slot, tag | ((unsigned long long)(q0 + c0) << 32) | (key >> 31));
      st_relaxed_u64(P.wb + slot, tag | (key & 0x7FFFFFFFull));
    }
  }
}

template <int RPT, int ROWT, int NCMAX>
__global__ void __launch_bounds__((ROWT + 32), (ROWT <= 128 ? 2 : 1))
qrp_reg_kernel(zd *Y, int l, int m, double *vnA, double *vnB, double *vn2, double *__restrict__ beta,
               int32_t *__restrict__ piv, zd *__restrict__ Rout, QrPosts P, int *err, uint64_t limit_ns,
               int npair) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zd *spiv = reinterpret_cast<zd *>(smem_raw);                         // RPT x 128 pivot rows, then 2 own columns
  int *perm = reinterpret_cast<int *>(spiv + (1 + NCMAX) * RPT * ROWT);  // logical -> physical
  __shared__ QrRegShared S;
  const int G = gridDim.x, b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int NW = (ROWT + 32) / 32;
  const double tol3z = sqrt(0x1.0p-53);
  for (int j = tid; j < m; j += blockDim.x) perm[j] = j;

  // with two CTAs on every SM (npair > 0), find this CTA's SM rank among the SMs and whether it
  // is the SM's second CTA: every CTA posts its SM id, waits for all, and ranks its own
  int sm_rank = 0, sm_half = 0;
  if (npair > 0) {
    unsigned int mysm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(mysm));
    if (tid == 0) st_relaxed_u64(P.smw + b, (1ull << 40) | mysm);
    int less = 0, before = 0, fail = 0;
    for (int c = tid; c < G; c += blockDim.x) {
      unsigned long long wv = ld_relaxed_u64(P.smw + c);
      if ((wv >> 40) != 1ull) {
        const uint64_t t0 = global_ns();
        while (((wv = ld_relaxed_u64(P.smw + c)) >> 40) != 1ull) {
          if (ld_volatile_i32(err)) { fail = 1; break; }
          if (global_ns() - t0 > limit_ns) { atomicExch(err, 1); fail = 1; break; }
        }
      }
      if (fail) break;
      const unsigned int sm = (unsigned int)(wv & 0xFFFFFFFFull);
      less += sm < mysm;
      before += (sm == mysm && c < b);
    }
    less = __reduce_add_sync(0xffffffffu, less);
    before = __reduce_add_sync(0xffffffffu, before);
    fail = __reduce_or_sync(0xffffffffu, fail);
    if (lane == 0) { S.pos[wid] = less; S.cta[wid] = before; S.fail[wid] = fail; }
    __syncthreads();
    int l_all = 0, b_all = 0, f_all = 0;
    for (int w = 0; w < NW; ++w) { l_all += S.pos[w]; b_all += S.cta[w]; f_all |= S.fail[w]; }
    if (f_all) return;
    sm_rank = l_all / 2;
    sm_half = b_all;
    __syncthreads();
  }

  // pivot of step 0 and its ||Y[1:, p]||^2 (every CTA)
  {
    long long best = -1;
    int bpos = 0x7fffffff;
    for (int q = tid; q < m; q += blockDim.x) qr_better(best, bpos, __double_as_longlong(ldcg(vnA + q)), q);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      qr_better(best, bpos, __shfl_xor_sync(0xffffffffu, best, o), __shfl_xor_sync(0xffffffffu, bpos, o));
    if (lane == 0) { S.key[wid] = best; S.pos[wid] = bpos; }
    __syncthreads();
    if (tid == 0) {
      long long bv = S.key[0];
      int bq = S.pos[0];
      for (int w = 1; w < NW; ++w) qr_better(bv, bq, S.key[w], S.pos[w]);
      perm[0] = bq;
      perm[bq] = 0;
      if (b == 0) piv[0] = bq;
      S.win = bq;
    }
    __syncthreads();
    const zd *y0 = Y + (int64_t)S.win * l;
    double acc = 0.0;
    for (int r = 1 + tid; r < l; r += blockDim.x) acc += abs2(ldcg(y0 + r));
    const double t = block_sum(acc, S.scratch);
    if (tid == 0) S.xn2_0 = t;
    __syncthreads();
  }

  int win = -1;
  for (int k = 0; k < m; ++k) {
    const double *vn_cur = (k & 1) ? vnB : vnA;
    double *vn_nxt = (k & 1) ? vnA : vnB;
    const double xn2 = (k == 0) ? S.xn2_0 : ldcg(P.xn2 + ((k - 1) & 1) * kQrMaxGrid + win);
    const int T = m - k - 1;
    int q0, nact;
    if (npair > 0) {
      // shares per SM first, then halved between the SM's two CTAs: no SM holds more than
      // ceil(T / npair) columns
      const int sm = sm_rank, half = sm_half;
      const int a0 = (int)(((long long)T * sm) / npair), a1 = (int)(((long long)T * (sm + 1)) / npair);
      const int c0 = (a1 - a0 + 1) / 2;
      q0 = k + 1 + a0 + (half ? c0 : 0);
      nact = half ? (a1 - a0 - c0) : c0;
    } else {
      q0 = k + 1 + (int)(((long long)T * b) / G);
      nact = k + 1 + (int)(((long long)T * (b + 1)) / G) - q0;
    }
    const int slot = (k & 1) * kQrMaxGrid + b;
    if (nact == 0) {
      qr_reg_step<0, RPT, ROWT>(Y, l, k, G, b, perm, q0, vn_cur, vn_nxt, vn2, beta, spiv, S, P, slot, xn2, tol3z);
      if (k == m - 1) break;
      if (tid == ROWT) {
        const unsigned long long tag = (unsigned long long)((k + 1) & 0x3FFFF) << 46;
        st_relaxed_u64(P.wa + slot, tag | ((unsigned long long)kQrNoPos << 32));
        st_relaxed_u64(P.wb + slot, tag);
      }
    } else if (nact == 1) {
      qr_reg_step<1, RPT, ROWT>(Y, l, k, G, b, perm, q0, vn_cur, vn_nxt, vn2, beta, spiv, S, P, slot, xn2, tol3z);
    } else if (NCMAX <= 2 || nact == 2) {
      qr_reg_step<2, RPT, ROWT>(Y, l, k, G, b, perm, q0, vn_cur, vn_nxt, vn2, beta, spiv, S, P, slot, xn2, tol3z);
    } else if (nact == 3) {
      qr_reg_step<(NCMAX >= 3 ? 3 : 2), RPT, ROWT>(Y, l, k, G, b, perm, q0, vn_cur, vn_nxt, vn2, beta, spiv, S, P,
                                                   slot, xn2, tol3z);
    } else {
      qr_reg_step<(NCMAX >= 4 ? 4 : 2), RPT, ROWT>(Y, l, k, G, b, perm, q0, vn_cur, vn_nxt, vn2, beta, spiv, S, P,
                                                   slot, xn2, tol3z);
    }

    // exchange: the scalar warp waits for every CTA's post of step k (relaxed polls of
    // the posts not yet seen, then an acquire fence) and reduces the candidates; the
    // row warps wait at the barrier
    if (tid >= ROWT) {
      constexpr int NT = (kQrMaxGrid + 31) / 32;
      const unsigned long long tagk = (unsigned long long)((k + 1) & 0x3FFFF);
      const unsigned long long *WA = P.wa + (k & 1) * kQrMaxGrid, *WB = P.wb + (k & 1) * kQrMaxGrid;
      unsigned long long wa[NT], wb[NT];
      unsigned pending = 0;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        wa[t] = 0;
        wb[t] = 0;
        if (lane + 32 * t < G) pending |= 1u << t;
      }
      int fail = 0;
      uint64_t t0 = 0;
      bool started = false;
      while (true) {
#pragma unroll
        for (int t = 0; t < NT; ++t)
          if (pending & (1u << t)) {
            wa[t] = ld_relaxed_u64(WA + lane + 32 * t);
            wb[t] = ld_relaxed_u64(WB + lane + 32 * t);
          }
        const int e = ld_volatile_i32(err);
#pragma unroll
        for (int t = 0; t < NT; ++t)
          if ((pending & (1u << t)) && (wa[t] >> 46) == tagk && (wb[t] >> 46) == tagk) pending &= ~(1u << t);
        if (__all_sync(0xffffffffu, pending == 0)) break;
        if (__any_sync(0xffffffffu, e != 0)) { fail = 1; break; }
        if (!started) { t0 = global_ns(); started = true; }
        else if (global_ns() - t0 > limit_ns) { atomicExch(err, 1); fail = 1; break; }
        __nanosleep(32);
      }
      fail = __any_sync(0xffffffffu, fail);
      __threadfence();
      long long best = -1;
      int bpos = 0x7fffffff, bcta = -1;
      if (!fail) {
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const int c = lane + 32 * t;
          if (c < G) {
            const long long kk = (long long)(((wa[t] & 0xFFFFFFFFull) << 31) | (wb[t] & 0x7FFFFFFFull));
            const int pp = (int)((wa[t] >> 32) & 0x3FFF);
            if (kk > best || (kk == best && pp < bpos)) { best = kk; bpos = pp; bcta = c; }
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ok = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, bpos, o);
        const int oc = __shfl_xor_sync(0xffffffffu, bcta, o);
        if (ok > best || (ok == best && op < bpos)) { best = ok; bpos = op; bcta = oc; }
      }
      if (lane == 0) {
        int fl = fail;
        if (!fl && (bpos < k + 1 || bpos >= m || bcta < 0)) { atomicExch(err, 1); fl = 1; }  // malformed post
        S.abort_ = fl;
        if (!fl) {
          const int tmp = perm[k + 1];
          perm[k + 1] = perm[bpos];
          perm[bpos] = tmp;
          if (b == 0) piv[k + 1] = perm[k + 1];
          S.win = bcta;
        }
      }
    }
    __syncthreads();
    if (S.abort_) return;
    win = S.win;
  }

  // R in pivot order: R[i, k] = Y[i, perm[k]] above the diagonal, beta_k on it
  __syncthreads();
  for (int k = b; k < m; k += G) {
    const int pk = perm[k];
    for (int i = tid; i < m; i += blockDim.x) {
      zd v = {0.0, 0.0};
      if (i < k) v = ldcg(Y + i + (int64_t)pk * l);
      else if (i == k) v = {beta[k], 0.0};
      Rout[i + (int64_t)k * m] = v;
    }
  }
}

template <int RPT, int ROWT, int NCMAX>
static cudaError_t try_qrp_reg(const QrArgs &a, int sms, cudaStream_t st, bool &launched) {
  launched = false;
  auto kern = qrp_reg_kernel<RPT, ROWT, NCMAX>;
  constexpr int per_sm = ROWT <= 128 ? 2 : 1;
  const size_t smem = sizeof(zd) * (1 + NCMAX) * RPT * ROWT + sizeof(int) * (size_t)a.m;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, (ROWT + 32), smem);
  if (e != cudaSuccess) return e;
  if (occ < per_sm) return cudaSuccess;  // the tile's column limit assumes per_sm CTAs on every SM
  int G = per_sm * sms;
  if (G > kQrMaxGrid) G = kQrMaxGrid;
  if (G > a.m) G = a.m;
  // widest share: ceil(T / G) columns, or with SM pairing half of ceil(T / sms), rounded up
  const int widest = (per_sm == 2 && G == 2 * sms) ? ((a.m - 1 + sms - 1) / sms + 1) / 2 : (a.m - 1 + G - 1) / G;
  if (widest > NCMAX) return cudaSuccess;
  zd *Y = (zd *)a.Y;
  double *vnB = a.vn1 + a.m;
  int l = a.l, m = a.m;
  zd *R = (zd *)a.R;
  unsigned char *pbase = (unsigned char *)a.mail + 4 * (size_t)kQrMaxGrid;
  QrPosts posts;
  posts.wa = (unsigned long long *)pbase;
  posts.wb = posts.wa + 2 * kQrMaxGrid;
  posts.xn2 = (double *)(posts.wb + 2 * kQrMaxGrid);
  posts.smw = (unsigned long long *)(posts.xn2 + 2 * kQrMaxGrid);
  uint64_t lim = a.limit_ns;
  // two CTAs on every SM (G co-resident CTAs, at most two per SM): shares are balanced per SM
  int npair = (per_sm == 2 && G == 2 * sms) ? sms : 0;
  void *args[] = {&Y, &l, &m, (void *)&a.vn1, &vnB, (void *)&a.vn2, (void *)&a.beta, (void *)&a.piv,
                  &R, &posts, (void *)&a.err, &lim, &npair};
  note_launch();
  launched = true;
  return cudaLaunchCooperativeKernel((const void *)kern, dim3(G), dim3((ROWT + 32)), args, smem, st);
}

template <int MAXC>
static cudaError_t launch_qrp_mail_t(const QrArgs &a, int G, size_t smem, int stage, cudaStream_t st) {
  zd *Y = (zd *)a.Y;
  double *vnB = a.vn1 + a.m;  // the vn1 buffer holds 2m doubles
  int l = a.l, m = a.m;
  zd *R = (zd *)a.R;
  unsigned int *flags = (unsigned int *)a.mail;
  QrMail *mail = (QrMail *)((unsigned char *)a.mail + 4 * (size_t)kQrMaxGrid);
  uint64_t lim = a.limit_ns;
  void *args[] = {&Y, &l, &m, (void *)&a.vn1, &vnB, (void *)&a.vn2, (void *)&a.beta, (void *)&a.piv,
                  &R, &flags, &mail, (void *)&a.err, &lim, &stage};
  note_launch();
  return cudaLaunchCooperativeKernel((const void *)qrp_mail_kernel<MAXC>, dim3(G), dim3(kQrbThreads), args, smem,
                                     st);
}

template <int MAXC>
static cudaError_t qrp_plan(const QrArgs &a, int sms, int &G, size_t &smem, int &stage) {
  auto kern = qrp_mail_kernel<MAXC>;
  // stage the pivot column in shared memory when two CTAs per SM still fit
  const size_t perm_bytes = sizeof(int) * (size_t)a.m;
  const size_t piv_bytes = sizeof(zd) * (size_t)a.l;
  stage = (perm_bytes + piv_bytes) <= 96 * 1024 ? 1 : 0;
  smem = perm_bytes + (stage ? piv_bytes : 0);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kQrbThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  // two CTAs per SM: one CTA's latency-bound scalar phases overlap the other's FP64 loops
  const int per_sm = occ < 2 ? occ : 2;
  G = per_sm * sms;
  if (G > kQrMaxGrid) G = kQrMaxGrid;
  if (G > a.m) G = a.m;
  return cudaSuccess;
}

cudaError_t launch_qrp(const QrArgs &a, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (!a.mail) return cudaErrorInvalidValue;
  // flags and posts must start at zero (posts carry the step number)
  cudaError_t e = cudaMemsetAsync(a.mail, 0, qr_mail_bytes(), st);
  if (e != cudaSuccess) return e;
  note_launch();
  qr_norms_kernel<<<a.m, kQrThreads, 0, st>>>((const zd *)a.Y, a.l, a.vn1, a.vn2);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // register/shared-tiled form when a column's trailing rows fit the tile
  if (a.m <= 16383) {
    bool launched = false;
    if (kQrWide && a.l - 1 <= 8 * 256) {
      // one CTA per SM, 256 row threads, up to 4 own columns
      e = try_qrp_reg<8, 256, 4>(a, sms, st, launched);
      if (e != cudaSuccess || launched) return e;
    }
    if (a.l - 1 <= 4 * 128) e = try_qrp_reg<4, 128, 2>(a, sms, st, launched);
    else if (a.l - 1 <= 8 * 128) e = try_qrp_reg<8, 128, 2>(a, sms, st, launched);
    else if (a.l - 1 <= 16 * 128) e = try_qrp_reg<16, 128, 2>(a, sms, st, launched);
    if (e != cudaSuccess || launched) return e;
  }
  // the widest own-column share is the one at step 0; choose the instantiation for it
  int G = 0, stage = 0;
  size_t smem = 0;
#define MN_QR_TRY(MC)                                           \
  {                                                             \
    e = qrp_plan<MC>(a, sms, G, smem, stage);                   \
    if (e != cudaSuccess) return e;                             \
    if ((a.m - 1 + G - 1) / G <= MC) return launch_qrp_mail_t<MC>(a, G, smem, stage, st); \
  }
  MN_QR_TRY(2)
  MN_QR_TRY(4)
  MN_QR_TRY(8)
  MN_QR_TRY(16)
  MN_QR_TRY(32)
#undef MN_QR_TRY
  return cudaErrorInvalidValue;
}

// ---- P R^{-1} ---------------------------------------------------------------
// One CTA per column k of R^{-1}: back substitution R w = e_k, column-oriented
// (after w_j is final, subtract w_j R[0:j, j] from the entries above). Writes
// Wp = P R^{-1} (row piv[i] of Wp is row i of R^{-1}) and WpH = Wp^*, both
// row-major; the caller zeroes them first.
//
// The chain of k steps is latency-bound, so each step is kept short: the
// reciprocals of R's (real) diagonal are formed once per CTA, the thread that
// finishes w_{j-1} scales it at once (no FP64 division inside the chain, one
// FP64 instruction per step instead of one per thread), w_j goes to Wp and WpH
// as soon as it is final (its pivot index read a step ahead), and with STAGE
// the next column of R is copied into shared memory by cp.async while the
// current one is applied (each thread copies and reads only its own rows).
template <bool STAGE>
__global__ void __launch_bounds__(128)
prinv_kernel(const zd *__restrict__ R, const int32_t *__restrict__ piv, int m, zd *__restrict__ Wp,
             zd *__restrict__ WpH) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  zd *w = reinterpret_cast<zd *>(smem_raw);
  zd *rcol = w + m;                                         // STAGE: 2 x m
  double *rinv = reinterpret_cast<double *>(rcol + (STAGE ? 2 * m : 0));
  __shared__ zd s_wj[2];
  const int tid = threadIdx.x;
  const int k = m - 1 - blockIdx.x;  // longest columns first: they bound the kernel's duration
  for (int i = tid; i <= k; i += blockDim.x) {
    w[i] = {i == k ? 1.0 : 0.0, 0.0};
    rinv[i] = 1.0 / R[i + (int64_t)i * m].re;
  }
  if (STAGE) {
    for (int i = tid; i < k; i += blockDim.x)
      cp_async16(rcol + (k & 1) * m + i, R + i + (int64_t)k * m, 16);
    cp_async_wait_all();
  }
  __syncthreads();
  if (tid == 0) s_wj[k & 1] = {rinv[k], 0.0};
  int pj = tid == 0 ? piv[k] : 0;
  for (int j = k; j >= 0; --j) {
    __syncthreads();  // s_wj[j & 1] = w_j / r_jj
    const zd wj = s_wj[j & 1];
    if (tid == 0) {
      Wp[(int64_t)pj * m + k] = wj;
      WpH[(int64_t)k * m + pj] = conjg(wj);
      if (j > 0) pj = piv[j - 1];
    }
    if (STAGE && j > 0)  // column j-1 for the next step
      for (int i = tid; i < j - 1; i += blockDim.x)
        cp_async16(rcol + ((j - 1) & 1) * m + i, R + i + (int64_t)(j - 1) * m, 16);
    const zd *rj = STAGE ? rcol + (j & 1) * m : R + (int64_t)j * m;
    for (int i = tid; i < j; i += blockDim.x) {
      zd v = w[i];
      const zd a = rj[i];
      v.re = fma(-a.re, wj.re, fma(a.im, wj.im, v.re));
      v.im = fma(-a.re, wj.im, fma(-a.im, wj.re, v.im));
      w[i] = v;
      if (i == j - 1) s_wj[i & 1] = {v.re * rinv[i], v.im * rinv[i]};
    }
    if (STAGE) cp_async_wait_all();
  }
}

cudaError_t launch_prinv(const void *R, const int32_t *piv, int m, void *Wp, void *WpH, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(Wp, 0, sizeof(zd) * (size_t)m * m, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(WpH, 0, sizeof(zd) * (size_t)m * m, st);
  if (e != cudaSuccess) return e;
  // staged while two CTAs per SM still fit (m <= 2048)
  const size_t staged = (sizeof(zd) * 3 + sizeof(double)) * (size_t)m;
  const bool stage = staged <= 112 * 1024;
  const size_t smem = stage ? staged : (sizeof(zd) + sizeof(double)) * (size_t)m;
  auto kern = stage ? prinv_kernel<true> : prinv_kernel<false>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  note_launch();
  kern<<<m, 128, smem, st>>>((const zd *)R, piv, m, (zd *)Wp, (zd *)WpH);
  return cudaGetLastError();
}

}  // namespace mn
