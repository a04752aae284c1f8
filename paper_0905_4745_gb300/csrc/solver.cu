// solver.cu -- the plan object and the C ABI of include/minnorm.h: Steps 1-5
// of the randomized minimal-norm algorithm (Section 4) on one GPU.
//
// Steps 2-3 (z = Q R^{-*} P^T b, c = T^* z) enter Step 4 only through R and
// P: with M = A^* P R^{-1}, the normal equations of min_u ||M u - c|| are
// (R^{-*} P^T A A^* P R^{-1}) u = R^{-*} P^T A c = R^{-*} P^T b (Lemma 5.1,
// Eq. easy: A c = b). So after the sketch and its QR, the solve runs CG on
// that system (two passes over A per iteration: q = A^* (P R^{-1} p), then
// A q), and Step 5 is x = A^* y with y = P R^{-1} u.
//
// Because the error of FP64 arithmetic in x = A^* y and in b - A x grows like
// kappa(A) * 2^-53 (about 1e-10 at kappa = 1e6; the paper's Tables 2 and 4
// show raw errors near 1e-9), the CG runs as the inner solver of an outer
// refinement loop on A A^* y = b (a generalisation of Remark 4.2's extra CG
// iterations): y is kept as a double-double pair, and after every inner solve
// x = A^* y and r = b - A x are formed exactly in fixed point on the integer
// pipe (xprod.cu). The loop stops on the a-posteriori bound
// ||x - p|| <= ||R^{-*} P^T r||, which holds because T has orthonormal rows
// (sigma_min(M) >= 1, so ||x - p|| = ||M (u - u*)|| <= ||M^* M (u - u*)||).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/minnorm.h"
#include "common.cuh"
#include "dw.cuh"
#include "kernels.h"
#include "params.h"
#include "vec.h"

using namespace mn;

namespace mn {
static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace mn

namespace {

constexpr int kSeg = 2048;                 // chain segment (outputs per CTA)
constexpr int kChainScanThreads = 256;     // threads of a chain CTA (sketch.cu)
constexpr int kChainCap = 4096;            // loaded elements per chain CTA
constexpr int kMaxOuter = 12;

struct KernelTimer {
  int cls;
  cudaEvent_t a, b;
};

}  // namespace

// m x n-sized scratch a batch shares among its plans (solved in turn)
struct ScratchPool {
  void *S1 = nullptr, *S2 = nullptr, *afix = nullptr, *A32 = nullptr;
  size_t s_bytes = 0, afix_bytes = 0, a32_bytes = 0;
};

// kernel classes of minnorm_kernel_stats (see minnorm.h)
constexpr int kNumClasses = 8;
// Step 2 by the blocked QR (qrblk.cu) for sketches of more than this many rows
constexpr int64_t kQrBlockedMinRows = 2048;
// relative residual reduction of an inner CG solve in mixed precision (each refinement step
// then reduces the error by about this much, or by the floor the complex64 A sets)
constexpr double kInnerTolMixed = 2e-3;

struct minnorm_plan_s {
  const ScratchPool *pool = nullptr;  // if set, S1, S2, afix and A32 point into it
  int64_t m = 0, n = 0, l = 0;
  minnorm_dtype dtype = MINNORM_C128;
  minnorm_precision prec = MINNORM_FP64;
  uint32_t flags = 0;
  cudaStream_t st = nullptr;
  int device = 0, sms = 152;
  bool fp32 = false;        // CG products in FP32
  int sk_arith = kArithF64;  // sketch arithmetic: FP64, or double-word (mixed precision)
  bool sketched = false;
  bool failed = false;
  SrftParams P;

  // sketch tables
  int logn = 0, logN1 = 0, tj = 0, tk = 0;  // FFT geometry of length L = 2^logn
  bool bluestein = false;                    // n not a power of two: L >= 2n - 1
  void *d_chirp = nullptr, *d_bhat = nullptr;  // Bluestein tables (compute precision)
  double *d_fac = nullptr;                   // l complex128: c_{s_t} / sqrt(n)
  cudaEvent_t ev_sk0 = nullptr, ev_sk1 = nullptr, ev_sk2 = nullptr;  // sketch / QR timing events
  double *h_qr = nullptr;                    // pinned: QR error word, |R_11|, |R_mm| of the last sketch,
                                             // ||R||_F^2, ||P R^{-1}||_F^2, ||A||_F^2 (upper bound)
  // the certificate sigma_min(A^* P R^{-1}) >= 1 - delta (see cert_delta)
  double eps_sk = 0.0;   // a priori bound of the sketch's rounding, relative to each row's norm
  double eps_qr = 0.0;   // a priori bound of the QR's backward error, relative to ||Y||_F
  double cert_delta = 1.0, inv_eta = 0.0, r_fro = 0.0, rinv_fro = 0.0, a_fro = 0.0;
  double *d_rown2 = nullptr;  // per row of A: an upper bound of ||A[i, :]||^2
  double *d_cert = nullptr;   // ||R||_F^2, ||P R^{-1}||_F^2, sum of d_rown2
  // block right-hand sides (allocated by the first multi-column mixed solve)
  bool blk_ready = false;
  void *d_bG = nullptr, *d_bR = nullptr, *d_bU = nullptr, *d_bS = nullptr, *d_bP = nullptr, *d_bT = nullptr,
       *d_bNp = nullptr, *d_bdY = nullptr, *d_bYh = nullptr, *d_bYl = nullptr, *d_bW32 = nullptr, *d_bQ = nullptr,
       *d_btpart = nullptr;
  float *d_bqqp = nullptr;
  void *d_bsplit = nullptr;   // BF16 pieces of W for the tensor-core adjoint product
  void *d_bsplit2 = nullptr;  // BF16 pieces of Q for the tensor-core forward product
  int blk_nsplit_tc = 0;
  double *d_bpart = nullptr, *d_bscal = nullptr;  // scal: gam, gam0, alpha, beta (KB each)
  int *d_bint = nullptr;                           // use, active, iters (KB each), alldone
  int blk_nsplit = 1;
  double *h_bpart = nullptr;                       // pinned: column-norm partials
  int *h_bint = nullptr;                           // pinned: a copy of d_bint
  double *h_bx = nullptr;                          // pinned: ||x_c||^2 per column
  int cap1 = 0, cap2 = 0;
  int32_t *d_idx1 = nullptr, *d_idx2 = nullptr, *d_halo1 = nullptr, *d_halo2 = nullptr;
  void *d_ph1 = nullptr, *d_ph2 = nullptr, *d_cs1 = nullptr, *d_cs2 = nullptr, *d_post = nullptr, *d_tw = nullptr;
  int32_t *d_samp_off = nullptr, *d_samp_t = nullptr, *d_samp_loc = nullptr;
  void *d_S1 = nullptr, *d_S2 = nullptr;
  zd *d_Y = nullptr, *d_Ykeep = nullptr;
  // factor
  double *d_vn1 = nullptr, *d_vn2 = nullptr, *d_beta = nullptr;
  int32_t *d_piv = nullptr;
  zd *d_R = nullptr, *d_Wp = nullptr, *d_WpH = nullptr;
  GridBarrier *d_bar = nullptr;
  void *d_qrmail = nullptr;
  int *d_err = nullptr;
  double rdiag_max = 0, rdiag_min = 0;
  // products
  zf *d_A32 = nullptr;
  GemvPlan g_cg{}, g_hp{};
  void *d_part = nullptr;
  size_t part_bytes = 0;
  double *d_qq = nullptr;
  int nqq = 0;
  double *d_red = nullptr;     // reduction partials
  double *d_norms = nullptr;   // [0] = ||g||^2, [1] = ||x||^2
  CgScalars *d_cg = nullptr;
  // vectors
  zd *d_r = nullptr, *d_g = nullptr, *d_u = nullptr, *d_s = nullptr, *d_p = nullptr, *d_w = nullptr,
     *d_t = nullptr, *d_np = nullptr, *d_dy = nullptr, *d_yh = nullptr, *d_yl = nullptr, *d_vh = nullptr,
     *d_vl = nullptr;
  zf *d_w32 = nullptr;
  void *d_q = nullptr;
  zd *d_xh = nullptr, *d_xl = nullptr, *d_d = nullptr;
  // fixed-point A for the exact residual
  void *d_afix = nullptr;
  int32_t *d_E = nullptr;
  void *d_yfix = nullptr, *d_xpart = nullptr, *d_xapart = nullptr, *d_xfix = nullptr;
  int *d_F = nullptr;   // [0] = Fy, [1] = Fx
  int x_nchunk = 1;
  int64_t x_chunk = 1;
  int x_nchunk_max = 1;   // the forward partial buffer holds this many column chunks
  int x_split = 0;        // row splits of x = A^* y (0: the default)
  bool x_tuned = false;
  double cg_keep = -1.0;  // fused CG: share of L2 kept between sweeps (negative: the default)
  bool cg_tuned = false;
  // fused CG (mixed precision, m <= 512)
  bool fused_ok = false;
  int pair_nc = 0;           // clusters of the one-pass CG product (mixed, 512 < m <= 4096), 0: two passes
  zf *d_tpart = nullptr;
  double *d_qqp = nullptr, *d_ggp = nullptr;
  // host staging (minnorm_solve_host): A arrives in row blocks on a copy stream
  void *d_Ah = nullptr;
  zd *d_bh = nullptr, *d_xo = nullptr;
  cudaStream_t st_copy = nullptr;
  cudaEvent_t ev_host[9] = {};
  // host pinned scalars
  double *h_norms = nullptr;
  CgScalars *h_cg = nullptr;
  // asynchronous solve (minnorm_solve with info == NULL): device state, pinned copy, pending flag
  SolveState *d_ss = nullptr, *h_ss = nullptr;
  bool async_pending = false;
  // bounded device-side waits: their limit, and (tests) a CTA of the next fused CG launch that
  // withholds its arrival at the grid barrier
  uint64_t wait_limit_ns = kBarrierLimitNs;
  int withhold = 0;
  // the asynchronous solve's CUDA graph (captured on st_cap for one (A, b, x, lda); the
  // certificate's constants are read from d_cc, written before each launch)
  cudaGraphExec_t ga_exec = nullptr;
  const void *ga_A = nullptr, *ga_b = nullptr;
  void *ga_x = nullptr;
  int64_t ga_lda = 0;
  int ga_withhold = 0;
  cudaStream_t st_cap = nullptr, st_cap2 = nullptr;
  CertConsts *d_cc = nullptr;
  bool capturing = false;
  // blocked QR of the sketch (allocated on first use)
  QrBlkWork qb;
  bool qb_ready = false;
  bool qr_blocked = false;   // Step 2 by the blocked QR (qrblk.cu) rather than the column-by-column kernel
  cudaEvent_t ev_as0 = nullptr, ev_as1 = nullptr;
  // timing
  std::vector<KernelTimer> timers;
  std::vector<cudaEvent_t> event_pool;
  size_t event_next = 0;
  int stat_launches[kNumClasses] = {};
  double stat_ms[kNumClasses] = {};
  float ms_sketch = 0, ms_qr = 0, ms_solve = 0;
  int fused_iters = 0;
  std::vector<void *> allocs;
};

namespace {

#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) {                       \
      plan->failed = true;                         \
      return MINNORM_ECUDA;                        \
    }                                              \
  } while (0)

template <typename T>
minnorm_status dalloc(minnorm_plan_t plan, T **ptr, size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return MINNORM_ENOMEM;
  }
  plan->allocs.push_back(p);
  *ptr = reinterpret_cast<T *>(p);
  return MINNORM_OK;
}

#define ALLOC(ptr, bytes)                               \
  do {                                                  \
    minnorm_status s_ = dalloc(plan, &(ptr), (bytes));  \
    if (s_ != MINNORM_OK) return s_;                    \
  } while (0)

// transform length of the sketch: n, or Bluestein's power of two >= 2n - 1
int64_t fft_length(int64_t n) {
  if ((n & (n - 1)) == 0) return n;
  int64_t L = 1;
  while (L < 2 * n - 1) L <<= 1;
  return L;
}

// bytes of the pooled scratch of one plan
void scratch_sizes(int64_t m, int64_t n, minnorm_precision prec, minnorm_dtype dtype, size_t &s_bytes,
                   size_t &afix_bytes, size_t &a32_bytes) {
  const bool fp32 = prec == MINNORM_MIXED;
  // the sketch's transform buffers: complex FP64 or complex double-word, 16 bytes either way
  s_bytes = sizeof(zd) * (size_t)m * (size_t)fft_length(n);
  afix_bytes = sizeof(int64_t) * 2 * (size_t)m * (size_t)n;
  a32_bytes = (fp32 && dtype == MINNORM_C128) ? sizeof(zf) * (size_t)m * (size_t)n : 0;
}

int ilog2(int64_t v) {
  int k = 0;
  while ((int64_t(1) << k) < v) ++k;
  return k;
}

cudaEvent_t next_event(minnorm_plan_t plan) {
  if (plan->event_next >= plan->event_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    plan->event_pool.push_back(e);
  }
  return plan->event_pool[plan->event_next++];
}

// Record a timed region around a kernel class when timing is on.
struct Timed {
  minnorm_plan_t plan;
  int cls;
  cudaEvent_t b{};
  bool on;
  Timed(minnorm_plan_t p, int c) : plan(p), cls(c), on((p->flags & MINNORM_FLAG_TIMING) != 0 && !p->capturing) {
    if (on) {
      cudaEvent_t a = next_event(plan);
      b = next_event(plan);
      cudaEventRecord(a, plan->st);
      plan->timers.push_back({cls, a, b});
    }
  }
  ~Timed() {
    if (on) cudaEventRecord(b, plan->st);
  }
};

void reset_stats(minnorm_plan_t plan) {
  for (int k = 0; k < kNumClasses; ++k) { plan->stat_launches[k] = 0; plan->stat_ms[k] = 0; }
  plan->fused_iters = 0;
}

void collect_timers(minnorm_plan_t plan) {
  for (auto &t : plan->timers) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      plan->stat_launches[t.cls] += 1;
      plan->stat_ms[t.cls] += ms;
    }
  }
  plan->timers.clear();
  plan->event_next = 0;
}

// ---- the certificate --------------------------------------------------------
// The refinement stops on ||x - p|| <= ||R^{-*} P^T (b - A x)|| / sigma_min(M), M = A^* P R^{-1}.
// For the exact sketch Y = T A^* and an exact QR, T M = Q has orthonormal columns and T has
// orthonormal rows (Section 3), so sigma_min(M) >= 1. With the computed sketch Y' = T A^* + E and
// the computed R (Y' P + dY = Q R, Q orthonormal), T M = Q - (dY + E P) R^{-1}, hence
//   sigma_min(M) >= 1 - delta,  delta = (||E||_F + ||dY||_F) ||R^{-1}||_F
//                               <= (eps_sk + eps_qr (1 + eps_sk)) ||A||_F ||R^{-1}||_F,
// with a priori bounds of the rounding of both (relative to each row of A, and to ||Y||_F). The
// bound also pays for the rounding of P R^{-1} itself (back substitution: relative error within
// 4 m 2^-53 ||R||_F ||R^{-1}||_F) and for the final rounding of x to complex128.

// Weight of a Givens chain's recurrence C_k = cos_k v_k + sin_k C_{k+1}: C_k is a sum over j >= k
// of v_j times products of |sin| over k..j-1; the largest row sum T_k = 1 + |sin_k| T_{k+1} and
// column sum U_j = 1 + |sin_{j-1}| U_{j-1} bound the 2-norm of the weight matrix by
// sqrt(max T max U) (Schur's test), so a rounding of relative size u in every term of every sum
// moves the chain's outputs by at most u sqrt(max T max U) ||v|| per rounding level.
static double chain_weight(const std::vector<double> &theta, int64_t n) {
  double t = 1.0, tmax = 1.0, u = 1.0, umax = 1.0;
  for (int64_t k = n - 2; k >= 0; --k) {
    t = 1.0 + std::fabs(std::sin(theta[k])) * t;
    tmax = std::max(tmax, t);
  }
  for (int64_t j = 1; j < n; ++j) {
    u = 1.0 + std::fabs(std::sin(theta[j - 1])) * u;
    umax = std::max(umax, u);
  }
  return std::sqrt(tmax * umax);
}

// A priori bound of ||y'_i - T conj(a_i)|| / ||a_i|| for the sketch's arithmetic (unit ua per
// operation: 2^-46 for double-word products and sums, 2^-53 for FP64). T is a product of unitary
// stages (phases, Givens chains, the DFT) and a row selection, so the stages' errors add:
//   input rounding (complex128 to double-word): 2^-48
//   each of the three phase products (the table entry rounded, four products, two sums): 8 ua
//   each chain: (depth + 2) ua sqrt(max T max U) + the halo truncation (2^-60 or 2^-72)
//     with depth 6 per + 40 roundings along a term's path through the block scan (per: elements
//     per thread, both serial passes) plus the warp and block levels
//   the FFT: 6 ua per radix-2 stage (twiddle product and the butterfly's sum) + 8 ua for the
//     four-step twiddle pass; Bluestein: two FFTs of length L and two chirp products, amplified
//     by amp = L max|bh| / sqrt(n) (the intermediate vectors' norm relative to ||a_i||)
//   the output rounding to complex128: 2^-53.
double sketch_error_bound(minnorm_plan_t plan, double chain_w, int per, double halo_tol, double amp) {
  const bool dw = plan->sk_arith == kArithDW;
  const double ua = dw ? 0x1.0p-46 : 0x1.0p-53;
  const double e_in = (dw && plan->dtype == MINNORM_C128) ? 0x1.0p-48 : 0.0;
  const double e_ph = 8.0 * ua;
  const double e_ch = (6.0 * per + 42.0) * ua * chain_w + halo_tol * std::sqrt((double)plan->n);
  const double e_fft1 = (6.0 * plan->logn + (plan->logN1 ? 8.0 : 0.0)) * ua;
  const double e_fft = plan->bluestein ? (2.0 * e_fft1 + 16.0 * ua) * std::max(1.0, amp) : e_fft1;
  return e_in + 3.0 * e_ph + 2.0 * e_ch + e_fft + 0x1.0p-53;
}

// delta from the norms of the last sketch (see above); a delta >= 1/2 certifies nothing
void certificate_delta(minnorm_plan_t plan, double r2, double rinv2, double a2) {
  const double slack = 1.0 + 1e-12;  // the FP64 sums of the squares
  plan->r_fro = std::sqrt(r2 * slack);
  plan->rinv_fro = std::sqrt(rinv2 * slack);
  plan->a_fro = std::sqrt(a2 * slack);
  const double e = plan->eps_sk + plan->eps_qr * (1.0 + plan->eps_sk);
  plan->cert_delta = e * plan->a_fro * plan->rinv_fro;
  plan->inv_eta = 4.0 * (double)plan->m * 0x1.0p-53 * plan->r_fro * plan->rinv_fro;
  if (!(plan->cert_delta < 0.5)) plan->cert_delta = 1.0;
}

// the factor-related fields of minnorm_info (the rest is zeroed)
void fill_factor_info(minnorm_plan_t plan, minnorm_info *info) {
  info->rdiag_max = plan->rdiag_max;
  info->rdiag_min = plan->rdiag_min;
  info->sigma_min_R = plan->rinv_fro > 0.0 ? 1.0 / plan->rinv_fro : 0.0;
  info->sigma_max_R = plan->r_fro;
  info->cert_delta = plan->cert_delta;
  info->ms_sketch = plan->ms_sketch;
  info->ms_qr = plan->ms_qr;
  info->ms_solve = info->ms_cg = info->ms_refine = info->reserved = 0.0f;
}

// ||x - p|| / ||x|| <= certified(||R^{-*} P^T r||, ||x||)
double certified(minnorm_plan_t plan, double gnorm, double xnorm) {
  if (!(xnorm > 0.0) || !(plan->cert_delta < 0.5)) return INFINITY;
  return gnorm * (1.0 + plan->inv_eta + 4.0 * (double)plan->m * 0x1.0p-53) / ((1.0 - plan->cert_delta) * xnorm) +
         0x1.0p-52;
}

// Upload the derived tables of the current parameters.
minnorm_status upload_params(minnorm_plan_t plan) {
  const int64_t n = plan->n, l = plan->l;
  const SrftParams &P = plan->P;
  const bool dw = plan->sk_arith == kArithDW;
  const size_t csz = sizeof(zd);  // complex FP64 or complex double-word: 16 bytes
  auto put_complex = [&](void *dst, const std::vector<std::complex<double>> &v) -> cudaError_t {
    std::vector<unsigned char> buf(v.size() * csz);
    for (size_t i = 0; i < v.size(); ++i) {
      if (dw) {
        zw z{df(v[i].real()), df(v[i].imag())};  // nearest double-words (2^-48 relative)
        memcpy(&buf[i * csz], &z, csz);
      } else {
        zd z{v[i].real(), v[i].imag()};
        memcpy(&buf[i * csz], &z, csz);
      }
    }
    return cudaMemcpy(dst, buf.data(), buf.size(), cudaMemcpyHostToDevice);
  };
  std::vector<std::complex<double>> tmp(n);
  std::vector<int32_t> idx(n);
  // chain 1: gather Pi~ after Z~  => v[j] = zeta~[pi~[j]] * conj(a[pi~[j]])
  for (int64_t j = 0; j < n; ++j) { idx[j] = (int32_t)P.pi_t[j]; tmp[j] = P.zeta_t[P.pi_t[j]]; }
  CK(cudaMemcpy(plan->d_idx1, idx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  CK(put_complex(plan->d_ph1, tmp));
  for (int64_t j = 0; j < n; ++j) tmp[j] = j < n - 1 ? std::complex<double>(cos(P.theta_t[j]), sin(P.theta_t[j]))
                                                     : std::complex<double>(1.0, 0.0);
  CK(put_complex(plan->d_cs1, tmp));
  // chain 2: Z then Pi  => v[j] = zeta[pi[j]] * w[pi[j]]
  for (int64_t j = 0; j < n; ++j) { idx[j] = (int32_t)P.pi[j]; tmp[j] = P.zeta[P.pi[j]]; }
  CK(cudaMemcpy(plan->d_idx2, idx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  CK(put_complex(plan->d_ph2, tmp));
  for (int64_t j = 0; j < n; ++j) tmp[j] = j < n - 1 ? std::complex<double>(cos(P.theta[j]), sin(P.theta[j]))
                                                     : std::complex<double>(1.0, 0.0);
  CK(put_complex(plan->d_cs2, tmp));
  CK(put_complex(plan->d_post, P.d));
  // halos
  const double tol = (dw ? 0x1.0p-60 : 0x1.0p-72) / std::sqrt((double)n);
  int h1 = 0, h2 = 0;
  std::vector<int32_t> halo1 = chain_halos(P.theta_t, n, kSeg, tol, &h1);
  std::vector<int32_t> halo2 = chain_halos(P.theta, n, kSeg, tol, &h2);
  if (std::min<int64_t>(kSeg, n) + std::max(h1, h2) + 1 > kChainCap) return MINNORM_ENOTSUP;
  plan->cap1 = (int)std::min<int64_t>(kSeg, n) + h1 + 1;
  plan->cap2 = (int)std::min<int64_t>(kSeg, n) + h2 + 1;
  CK(cudaMemcpy(plan->d_halo1, halo1.data(), sizeof(int32_t) * halo1.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(plan->d_halo2, halo2.data(), sizeof(int32_t) * halo2.size(), cudaMemcpyHostToDevice));
  const double chain_w = std::max(chain_weight(P.theta_t, n), chain_weight(P.theta, n));
  const int per = (std::max(plan->cap1, plan->cap2) + kChainScanThreads - 1) / kChainScanThreads;
  // samples: for each output t, where X[s_t] sits in the pass that produces it
  const int logn = plan->logn, logN1 = plan->logN1;
  std::vector<int32_t> off, st_t(l), st_loc(l);
  if (logN1 == 0) {
    off = {0, (int32_t)l};
    for (int64_t t = 0; t < l; ++t) { st_t[t] = (int32_t)t; st_loc[t] = (int32_t)P.s[t]; }
  } else {
    const int64_t N1 = int64_t(1) << logN1, N2 = int64_t(1) << (logn - logN1);
    const int64_t nb = N2 / plan->tk;
    std::vector<int32_t> cnt(nb + 1, 0);
    for (int64_t t = 0; t < l; ++t) cnt[(P.s[t] % N2) / plan->tk + 1] += 1;
    for (int64_t b = 0; b < nb; ++b) cnt[b + 1] += cnt[b];
    off = cnt;
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t t = 0; t < l; ++t) {
      const int64_t k = P.s[t], k2 = k % N2, k1 = k / N2, b = k2 / plan->tk, kk = k2 - b * plan->tk;
      const int32_t pos = fill[b]++;
      st_t[pos] = (int32_t)t;
      st_loc[pos] = (int32_t)(kk * (N1 + 1) + k1);  // pass B's sequences are padded by one element
    }
  }
  CK(cudaMemcpy(plan->d_samp_off, off.data(), sizeof(int32_t) * off.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(plan->d_samp_t, st_t.data(), sizeof(int32_t) * l, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(plan->d_samp_loc, st_loc.data(), sizeof(int32_t) * l, cudaMemcpyHostToDevice));
  // twiddles e^{-2 pi i k / L}
  const int64_t L = int64_t(1) << logn;
  const double two_pi = 6.283185307179586476925286766559;
  tmp.resize(L);
  for (int64_t k = 0; k < L; ++k) {
    const double a = two_pi * (double)k / (double)L;
    tmp[k] = std::complex<double>(cos(a), -sin(a));
  }
  CK(put_complex(plan->d_tw, tmp));
  if (plan->bluestein) {
    std::vector<std::complex<double>> chirp, bh;
    bluestein_tables(n, L, chirp, bh);
    CK(put_complex(plan->d_chirp, chirp));
    CK(put_complex(plan->d_bhat, bh));
    std::vector<double> fac(2 * l);
    const double sc = 1.0 / std::sqrt((double)n);
    for (int64_t t = 0; t < l; ++t) {
      fac[2 * t] = chirp[P.s[t]].real() * sc;
      fac[2 * t + 1] = chirp[P.s[t]].imag() * sc;
    }
    CK(cudaMemcpy(plan->d_fac, fac.data(), sizeof(double) * 2 * l, cudaMemcpyHostToDevice));
    double bmax = 0.0;
    for (const auto &z : bh) bmax = std::max(bmax, std::abs(z));
    plan->eps_sk = sketch_error_bound(plan, chain_w, per, tol, (double)L * bmax / std::sqrt((double)n));
  } else {
    plan->eps_sk = sketch_error_bound(plan, chain_w, per, tol, 0.0);
  }
  // Householder QR (FP64): backward error within 8 m (d + 4) 2^-53 ||Y||_F, d the depth of its
  // dot products' sums (a thread's run of rows plus the warp, block and grid trees). The blocked
  // form adds its two QRs' bounds: the l x m one, then the m x m pivoted one. In the l x m one a
  // panel's sums have depth at most max(l / (8 G), 2) + 1 (a thread's rows) + 8 (the block's
  // warps) + G / 8 + 8 (the grid's partials) + 2 (the reflector's scalars), G <= sms; the adjoint
  // trailing product of complex length K <= l errs by at most 2^-53 (2 sqrt(K) / 256 + K / 4096 +
  // 4) ||v|| ||c|| (63-bit operand truncation; the dropped slice levels, K 2^-65.9 max|v| max|c|;
  // the roundings of the K splits and of their compensated sum, 2^-51.5 |v|^T |c|), and the
  // K = 32 update by at most 24 more units.
  if (plan->qr_blocked) {
    const double G = plan->sms, L = (double)l;
    const double d_panel = std::max(L / (8.0 * G), 2.0) + 1.0 + 8.0 + G / 8.0 + 8.0 + 2.0;
    const double d_prod = 2.0 * std::sqrt(L) / 256.0 + L / 4096.0 + 4.0 + 24.0;
    const double d2 = (double)((plan->m + 127) / 128 + 20);
    plan->eps_qr = 8.0 * (double)plan->m * (d_panel + d_prod + d2 + 8.0) * 0x1.0p-53;
  } else {
    plan->eps_qr = 8.0 * (double)plan->m * (double)((l + 127) / 128 + 20) * 0x1.0p-53;
  }
  plan->sketched = false;
  return MINNORM_OK;
}

minnorm_status qrblk_alloc(minnorm_plan_t plan);

minnorm_status create_impl(minnorm_plan_t plan, int64_t m, int64_t n, int64_t l, minnorm_dtype dtype,
                           minnorm_precision prec, uint64_t seed, uint32_t flags, void *stream) {
  plan->m = m;
  plan->n = n;
  plan->l = l;
  plan->dtype = dtype;
  plan->prec = prec;
  plan->flags = flags;
  plan->st = (cudaStream_t)stream;
  plan->fp32 = (prec == MINNORM_MIXED);
  plan->sk_arith = (prec == MINNORM_MIXED) ? kArithDW : kArithF64;
  CK(cudaGetDevice(&plan->device));
  CK(cudaDeviceGetAttribute(&plan->sms, cudaDevAttrMultiProcessorCount, plan->device));
  // FFT geometry: length L = n for a power of two, else the Bluestein length 2^ceil(log2(2n - 1))
  plan->bluestein = (n & (n - 1)) != 0;
  const int64_t L = fft_length(n);
  plan->logn = ilog2(L);
  const int cap = 4096;  // complex elements of 16 bytes per FFT tile in shared memory
  if (L <= cap) {
    plan->logN1 = 0;
  } else {
    plan->logN1 = plan->logn / 2;
    const int64_t N1 = int64_t(1) << plan->logN1, N2 = L / N1;
    if (N2 > cap) return MINNORM_ENOTSUP;
    plan->tj = (int)std::min<int64_t>(N1, cap / N2);
    plan->tk = (int)std::min<int64_t>(N2, cap / N1);
  }
  const size_t rc = plan->fp32 ? sizeof(zf) : sizeof(zd);  // complex size of the CG products
  const size_t rs = sizeof(zd);  // complex size of the sketch (FP64 or double-word)
  const int64_t nseg = (n + kSeg - 1) / kSeg;
  ALLOC(plan->d_idx1, sizeof(int32_t) * n);
  ALLOC(plan->d_idx2, sizeof(int32_t) * n);
  ALLOC(plan->d_halo1, sizeof(int32_t) * nseg);
  ALLOC(plan->d_halo2, sizeof(int32_t) * nseg);
  ALLOC(plan->d_ph1, rs * n);
  ALLOC(plan->d_ph2, rs * n);
  ALLOC(plan->d_cs1, rs * n);
  ALLOC(plan->d_cs2, rs * n);
  ALLOC(plan->d_post, rs * n);
  ALLOC(plan->d_tw, rs * L);
  if (plan->bluestein) {
    ALLOC(plan->d_chirp, rs * n);
    ALLOC(plan->d_bhat, rs * L);
    ALLOC(plan->d_fac, 2 * sizeof(double) * l);
  }
  const int64_t nbB = plan->logN1 ? ((L >> plan->logN1) / plan->tk) : 1;
  ALLOC(plan->d_samp_off, sizeof(int32_t) * (nbB + 1));
  ALLOC(plan->d_samp_t, sizeof(int32_t) * l);
  ALLOC(plan->d_samp_loc, sizeof(int32_t) * l);
  if (plan->pool) {
    size_t sb = 0, ab = 0, a32 = 0;
    scratch_sizes(m, n, prec, dtype, sb, ab, a32);
    if (sb > plan->pool->s_bytes || ab > plan->pool->afix_bytes || a32 > plan->pool->a32_bytes)
      return MINNORM_EINVAL;
    plan->d_S1 = plan->pool->S1;
    plan->d_S2 = plan->pool->S2;
  } else {
    ALLOC(plan->d_S1, rs * (size_t)m * L);
    ALLOC(plan->d_S2, rs * (size_t)m * L);
  }
  ALLOC(plan->d_Y, sizeof(zd) * (size_t)l * m);
  if (flags & MINNORM_FLAG_KEEP_SKETCH) ALLOC(plan->d_Ykeep, sizeof(zd) * (size_t)l * m);
  ALLOC(plan->d_vn1, sizeof(double) * 2 * m);
  ALLOC(plan->d_vn2, sizeof(double) * m);
  ALLOC(plan->d_beta, sizeof(double) * m);
  ALLOC(plan->d_piv, sizeof(int32_t) * m);
  ALLOC(plan->d_R, sizeof(zd) * (size_t)m * m);
  ALLOC(plan->d_Wp, sizeof(zd) * (size_t)m * m);
  ALLOC(plan->d_WpH, sizeof(zd) * (size_t)m * m);
  ALLOC(plan->d_bar, sizeof(GridBarrier));
  ALLOC(plan->d_qrmail, qr_mail_bytes());
  ALLOC(plan->d_err, sizeof(int));
  if (plan->fp32 && dtype == MINNORM_C128) {
    if (plan->pool) plan->d_A32 = static_cast<zf *>(plan->pool->A32);
    else ALLOC(plan->d_A32, sizeof(zf) * (size_t)m * n);
  }
  // products: g_cg for the CG passes, g_hp for FP64 / double-double passes on the stored A
  const int hp_mode = dtype == MINNORM_C128 ? 0 : 2;
  gemv_configure(plan->g_hp, m, n, n, hp_mode, plan->sms);
  gemv_configure(plan->g_cg, m, n, n, plan->fp32 ? 1 : hp_mode, plan->sms);
  size_t pb = 0;
  pb = std::max(pb, gemv_adj_partial_elems(plan->g_cg) * rc);
  pb = std::max(pb, gemv_fwd_partial_elems(plan->g_cg) * rc);
  pb = std::max(pb, gemv_adj_partial_elems(plan->g_hp) * sizeof(zd));
  pb = std::max(pb, gemv_fwd_partial_elems(plan->g_hp) * sizeof(zd));
  plan->part_bytes = pb;
  ALLOC(plan->d_part, pb);
  plan->nqq = (int)std::min<int64_t>(1024, (n + 255) / 256);
  ALLOC(plan->d_qq, sizeof(double) * 1024);
  ALLOC(plan->d_red, sizeof(double) * 2048);
  ALLOC(plan->d_norms, sizeof(double) * 4);
  ALLOC(plan->d_rown2, sizeof(double) * m);
  ALLOC(plan->d_cert, sizeof(double) * 4);
  ALLOC(plan->d_cg, sizeof(CgScalars));
  zd **mvecs[] = {&plan->d_r, &plan->d_g, &plan->d_u, &plan->d_s, &plan->d_p, &plan->d_w, &plan->d_t,
                  &plan->d_np, &plan->d_dy, &plan->d_yh, &plan->d_yl, &plan->d_vh, &plan->d_vl};
  for (zd **v : mvecs) ALLOC(*v, sizeof(zd) * m);
  ALLOC(plan->d_w32, sizeof(zf) * m);
  ALLOC(plan->d_q, rc * n);
  ALLOC(plan->d_xh, sizeof(zd) * n);
  ALLOC(plan->d_xl, sizeof(zd) * n);
  ALLOC(plan->d_d, sizeof(zd) * n);
  if (plan->pool) plan->d_afix = plan->pool->afix;
  else ALLOC(plan->d_afix, sizeof(int64_t) * 2 * (size_t)m * n);
  ALLOC(plan->d_E, sizeof(int32_t) * m);
  ALLOC(plan->d_yfix, 32 * (size_t)m);
  ALLOC(plan->d_F, sizeof(int) * 2);
  {
    const int64_t row_blocks = (m + 7) / 8;
    int64_t nchunk = 1;
    while (row_blocks * nchunk < 8 * plan->sms && n / (nchunk * 2) >= 1024) nchunk *= 2;
    plan->x_nchunk = (int)nchunk;
    plan->x_chunk = (n + nchunk - 1) / nchunk;
    plan->x_nchunk_max = n / (nchunk * 2) >= 256 ? (int)nchunk * 2 : (int)nchunk;
    ALLOC(plan->d_xpart, xprod_partial_bytes(m, plan->x_nchunk_max));
    ALLOC(plan->d_xapart, xadj_partial_bytes(m, n));
    ALLOC(plan->d_xfix, xfix_bytes(n));
  }
  if (plan->fp32 && m <= 512) {
    plan->fused_ok = true;
    ALLOC(plan->d_tpart, sizeof(zf) * (size_t)plan->sms * m);
    ALLOC(plan->d_qqp, sizeof(double) * plan->sms);
    ALLOC(plan->d_ggp, sizeof(double) * plan->sms);
  } else if (plan->fp32 && (plan->pair_nc = cg_pair_clusters(m, n)) > 0) {
    ALLOC(plan->d_tpart, sizeof(zf) * (size_t)plan->pair_nc * m);
    ALLOC(plan->d_qqp, sizeof(double) * plan->pair_nc);
  }
  // Step 2 for tall sketches: the blocked QR with tensor-core trailing updates (its workspace now)
  plan->qr_blocked = l > kQrBlockedMinRows && !plan->pool && qrblk_panel_grid(l, plan->sms) > 0;
  if (plan->qr_blocked) {
    minnorm_status qs = qrblk_alloc(plan);
    if (qs != MINNORM_OK) return qs;
  }
  if (cudaMallocHost(&plan->h_norms, sizeof(double) * 4) != cudaSuccess) return MINNORM_ENOMEM;
  if (cudaMallocHost(&plan->h_cg, sizeof(CgScalars)) != cudaSuccess) return MINNORM_ENOMEM;
  if (cudaMallocHost(&plan->h_ss, sizeof(SolveState)) != cudaSuccess) return MINNORM_ENOMEM;
  ALLOC(plan->d_ss, sizeof(SolveState));
  ALLOC(plan->d_cc, sizeof(CertConsts));
  if (cudaMallocHost(&plan->h_qr, sizeof(double) * 6) != cudaSuccess) return MINNORM_ENOMEM;
  draw_srft_params(seed, n, l, plan->P);
  return upload_params(plan);
}

// Step 1 on the plan's stream: the fixed-point (and complex64) copies of A, then Y = T A^*.
minnorm_status sketch_transform(minnorm_plan_t plan, const void *A, int64_t lda) {
  cudaStream_t st = plan->st;
  const int64_t m = plan->m, n = plan->n, l = plan->l;
  const bool timing = plan->flags & MINNORM_FLAG_TIMING;
  reset_stats(plan);
  plan->sketched = false;
  if (timing) {
    plan->ev_sk0 = next_event(plan);
    plan->ev_sk1 = next_event(plan);
    CK(cudaEventRecord(plan->ev_sk0, st));
  }
  const bool src_c64 = plan->dtype == MINNORM_C64;
  // fixed-point copy of A for the exact residuals (and the complex64 copy in mixed mode)
  CK(launch_fix_prep(A, lda, src_c64, m, n, plan->d_afix, plan->d_E, plan->d_A32, st, plan->d_rown2));
  {
    // the sketch reads A as stored (FP64 or double-word arithmetic: the R the error bound uses
    // is that of an FP64-class sketch of A itself)
    Timed tm(plan, 4);
    const int ar = plan->sk_arith;
    ChainArgs c1{A, lda, plan->d_S1, n, plan->d_idx1, plan->d_ph1, plan->d_cs1, nullptr, plan->d_halo1,
                 (int)n, kSeg, plan->cap1, (int)m, src_c64 ? kSrcC64 : kSrcC128, true, ar};
    CK(launch_chain(c1, st));
    ChainArgs c2{plan->d_S1, n, plan->d_S2, n, plan->d_idx2, plan->d_ph2, plan->d_cs2, plan->d_post,
                 plan->d_halo2, (int)n, kSeg, plan->cap2, (int)m, ar == kArithDW ? kSrcDW : kSrcC128, false, ar};
    CK(launch_chain(c2, st));
    const int64_t L = int64_t(1) << plan->logn;
    FftArgs f{};
    f.tw = plan->d_tw;
    f.logn = plan->logn;
    f.logN1 = plan->logN1;
    f.tj = plan->tj;
    f.tk = plan->tk;
    f.samp_off = plan->d_samp_off;
    f.samp_t = plan->d_samp_t;
    f.samp_loc = plan->d_samp_loc;
    f.l = (int)l;
    f.rows = (int)m;
    f.Y = plan->d_Y;
    f.ldy = l;
    f.arith = ar;
    if (!plan->bluestein) {
      f.src = plan->d_S2;
      f.ld = n;
      f.work = plan->d_S1;
      f.ldw = n;
      CK(launch_fft(f, st));
    } else {
      // stage 1: conj(FFT_L(x c) bh) in full; stage 2: FFT_L of that, sampled with c_k / sqrt(n)
      // (single pass: S2 -> S1 -> Y; four-step: S2 -> S1 -> S2, then S2 -> S1 -> Y)
      FftArgs f1 = f;
      f1.src = plan->d_S2;
      f1.ld = n;
      f1.work = plan->d_S1;
      f1.ldw = L;
      f1.chirp = plan->d_chirp;
      f1.nin = (int)n;
      f1.full = plan->logN1 ? plan->d_S2 : plan->d_S1;
      f1.bh = plan->d_bhat;
      f1.ldf = L;
      CK(launch_fft(f1, st));
      FftArgs f2 = f;
      f2.src = f1.full;
      f2.ld = L;
      f2.work = plan->d_S1;
      f2.ldw = L;
      f2.fac = plan->d_fac;
      CK(launch_fft(f2, st));
    }
  }
  if (plan->d_Ykeep) CK(cudaMemcpyAsync(plan->d_Ykeep, plan->d_Y, sizeof(zd) * l * m, cudaMemcpyDeviceToDevice, st));
  if (timing) CK(cudaEventRecord(plan->ev_sk1, st));
  return MINNORM_OK;
}

// Step 2 on the plan's stream: pivoted QR of Y, then P R^{-1}; the status words are copied
// to pinned host memory (read by sketch_finish after the stream has reached them).
minnorm_status sketch_factor(minnorm_plan_t plan) {
  cudaStream_t st = plan->st;
  const int64_t m = plan->m, l = plan->l;
  QrArgs q{plan->d_Y, (int)l, (int)m, plan->d_vn1, plan->d_vn2, plan->d_beta, plan->d_piv, plan->d_R,
           plan->d_qrmail, plan->d_err, plan->wait_limit_ns};
  {
    Timed tm(plan, 3);
    CK(cudaMemsetAsync(plan->d_err, 0, sizeof(int), st));
    if (plan->qr_blocked) CK(launch_qr_tall(plan->qb, q, plan->sms, st));
    else CK(launch_qrp(q, st));
  }
  if (plan->qr_blocked) {
    Timed tm(plan, 6);
    CK(launch_qr_triangle(plan->qb, q, st));
  }
  {
    Timed tm(plan, 7);
    if (plan->qr_blocked && m >= kPinvBlockedMinM)
      CK(launch_prinv_blocked(plan->qb, plan->d_R, plan->d_piv, (int)m, plan->d_Wp, plan->d_WpH, plan->d_err,
                              plan->wait_limit_ns, st));
    else
      CK(launch_prinv(plan->d_R, plan->d_piv, (int)m, plan->d_Wp, plan->d_WpH, st));
    // ||R||_F, ||P R^{-1}||_F and ||A||_F for the certificate's delta
    CK(launch_sumsq(m * m, plan->d_R, plan->d_red, plan->d_cert, st));
    CK(launch_sumsq(m * m, plan->d_Wp, plan->d_red + 1024, plan->d_cert + 1, st));
    CK(launch_sum((int)m, plan->d_rown2, plan->d_cert + 2, st));
  }
  if (plan->flags & MINNORM_FLAG_TIMING) {
    plan->ev_sk2 = next_event(plan);
    CK(cudaEventRecord(plan->ev_sk2, st));
  }
  CK(cudaMemcpyAsync(&plan->h_qr[0], plan->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&plan->h_qr[1], plan->d_beta, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&plan->h_qr[2], plan->d_beta + (m - 1), sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&plan->h_qr[3], plan->d_cert, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  return MINNORM_OK;
}

// After the stream has passed sketch_factor: timings, the QR's status and the rank test.
minnorm_status sketch_finish(minnorm_plan_t plan) {
  CK(cudaStreamSynchronize(plan->st));
  if (plan->flags & MINNORM_FLAG_TIMING) {
    cudaEventElapsedTime(&plan->ms_sketch, plan->ev_sk0, plan->ev_sk1);
    cudaEventElapsedTime(&plan->ms_qr, plan->ev_sk1, plan->ev_sk2);
    collect_timers(plan);
  }
  int err = 0;
  double b0 = 0, bm = 0;
  memcpy(&err, &plan->h_qr[0], sizeof(int));
  memcpy(&b0, &plan->h_qr[1], sizeof(double));
  memcpy(&bm, &plan->h_qr[2], sizeof(double));
  if (err) {
    plan->failed = true;
    return MINNORM_ETIMEOUT;
  }
  plan->rdiag_max = std::fabs(b0);
  plan->rdiag_min = std::fabs(bm);
  certificate_delta(plan, plan->h_qr[3], plan->h_qr[4], plan->h_qr[5]);
  plan->sketched = true;
  if (!(plan->rdiag_min > 64.0 * (double)plan->m * 0x1.0p-53 * plan->rdiag_max)) return MINNORM_ERANK;
  return MINNORM_OK;
}

// ---- Step 1 + Step 2 --------------------------------------------------------
minnorm_status sketch_impl(minnorm_plan_t plan, const void *A, int64_t lda) {
  minnorm_status s = sketch_transform(plan, A, lda);
  if (s != MINNORM_OK) return s;
  s = sketch_factor(plan);
  if (s != MINNORM_OK) return s;
  return sketch_finish(plan);
}

// ---- Steps 1-2 with A in host memory ------------------------------------------
// A is copied to the plan's staging buffer in kHostBlocks row blocks on a copy stream, and
// each block's part of Step 1 (fixed-point copy, chains, FFT) runs on the plan's stream as
// soon as its rows have arrived: every kernel of the sketch is row-local, so the result is
// the one sketch_transform gives over all rows, and the copy of block k + 1 overlaps the
// sketch of block k. Power-of-two n (the Bluestein path keeps the single copy).
static constexpr int kHostBlocks = 8;

minnorm_status sketch_from_host(minnorm_plan_t plan, const void *A_host, int64_t lda) {
  cudaStream_t st = plan->st;
  const int64_t m = plan->m, n = plan->n;
  const size_t es = plan->dtype == MINNORM_C128 ? sizeof(zd) : sizeof(zf);
  const size_t rs = sizeof(zd);  // sketch buffers: complex FP64 or complex double-word
  const bool timing = plan->flags & MINNORM_FLAG_TIMING;
  if (!plan->st_copy) {
    CK(cudaStreamCreateWithFlags(&plan->st_copy, cudaStreamNonBlocking));
    for (cudaEvent_t &e : plan->ev_host) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  reset_stats(plan);
  plan->sketched = false;
  plan->g_hp.ld = n;
  plan->g_cg.ld = n;
  if (timing) {
    plan->ev_sk0 = next_event(plan);
    plan->ev_sk1 = next_event(plan);
    CK(cudaEventRecord(plan->ev_sk0, st));
  }
  // the staging buffer is free once the plan's stream has finished its earlier work
  CK(cudaEventRecord(plan->ev_host[kHostBlocks], st));
  CK(cudaStreamWaitEvent(plan->st_copy, plan->ev_host[kHostBlocks], 0));
  const int K = (int)std::min<int64_t>(kHostBlocks, m);
  const int ar = plan->sk_arith;
  for (int k = 0; k < K; ++k) {
    const int64_t r0 = m * k / K, r1 = m * (k + 1) / K, rows = r1 - r0;
    char *Ab = static_cast<char *>(plan->d_Ah) + (size_t)r0 * n * es;
    CK(cudaMemcpy2DAsync(Ab, es * n, static_cast<const char *>(A_host) + (size_t)r0 * lda * es, es * lda, es * n,
                         rows, cudaMemcpyHostToDevice, plan->st_copy));
    CK(cudaEventRecord(plan->ev_host[k], plan->st_copy));
    CK(cudaStreamWaitEvent(st, plan->ev_host[k], 0));
    zf *A32 = plan->d_A32 ? plan->d_A32 + r0 * n : nullptr;
    CK(launch_fix_prep(Ab, n, plan->dtype == MINNORM_C64, rows, n,
                       reinterpret_cast<char *>(plan->d_afix) + (size_t)r0 * n * 2 * sizeof(int64_t), plan->d_E + r0,
                       A32, st, plan->d_rown2 + r0));
    const bool src_c64 = plan->dtype == MINNORM_C64;
    char *S1 = reinterpret_cast<char *>(plan->d_S1) + (size_t)r0 * n * rs;
    char *S2 = reinterpret_cast<char *>(plan->d_S2) + (size_t)r0 * n * rs;
    Timed tm(plan, 4);
    ChainArgs c1{Ab, n, S1, n, plan->d_idx1, plan->d_ph1, plan->d_cs1, nullptr, plan->d_halo1,
                 (int)n, kSeg, plan->cap1, (int)rows, src_c64 ? kSrcC64 : kSrcC128, true, ar};
    CK(launch_chain(c1, st));
    ChainArgs c2{S1, n, S2, n, plan->d_idx2, plan->d_ph2, plan->d_cs2, plan->d_post,
                 plan->d_halo2, (int)n, kSeg, plan->cap2, (int)rows, ar == kArithDW ? kSrcDW : kSrcC128, false, ar};
    CK(launch_chain(c2, st));
    FftArgs f{};
    f.tw = plan->d_tw;
    f.logn = plan->logn;
    f.logN1 = plan->logN1;
    f.tj = plan->tj;
    f.tk = plan->tk;
    f.samp_off = plan->d_samp_off;
    f.samp_t = plan->d_samp_t;
    f.samp_loc = plan->d_samp_loc;
    f.l = (int)plan->l;
    f.rows = (int)rows;
    f.Y = plan->d_Y;
    f.ldy = plan->l;
    f.row_offset = (int)r0;
    f.arith = ar;
    f.src = S2;
    f.ld = n;
    f.work = S1;
    f.ldw = n;
    CK(launch_fft(f, st));
  }
  if (plan->d_Ykeep)
    CK(cudaMemcpyAsync(plan->d_Ykeep, plan->d_Y, sizeof(zd) * plan->l * m, cudaMemcpyDeviceToDevice, st));
  if (timing) CK(cudaEventRecord(plan->ev_sk1, st));
  minnorm_status s = sketch_factor(plan);
  if (s != MINNORM_OK) return s;
  return sketch_finish(plan);
}

// autotuning caches, keyed by the system's shape and the SM count (process-wide)
struct TuneKey {
  int64_t m, n;
  int sms;
  bool operator<(const TuneKey &o) const {
    return m != o.m ? m < o.m : (n != o.n ? n < o.n : sms < o.sms);
  }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, int>> g_tune_cache;  // -> (column chunks, row splits)
static std::map<TuneKey, double> g_cg_keep_cache;             // -> fused CG L2 share

// The fused CG's L2 share (how much of each sweep's tail is loaded with an evict-last hint
// for the next, reversed sweep) is a cache hint: every choice gives the same bits. On a plan's
// first inner solve the candidates run that solve (from the same g, so the run afterwards is
// unchanged) and the fastest is kept, for later plans of the same shape too. Small systems,
// whose A fits in L2, keep the default.
minnorm_status tune_cg_keep(minnorm_plan_t plan, CgFusedArgs a) {
  plan->cg_tuned = true;
  const int64_t m = plan->m, n = plan->n;
  if (m * n * (int64_t)sizeof(zf) < ((int64_t)64 << 20)) return MINNORM_OK;
  const TuneKey key{m, n, plan->sms};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_cg_keep_cache.find(key);
    if (it != g_cg_keep_cache.end()) {
      plan->cg_keep = it->second;
      return MINNORM_OK;
    }
  }
  cudaStream_t st = plan->st;
  const double cand[] = {0.0, 0.4, 0.6, 0.8, 1.0};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = INFINITY;
  double best_f = -1.0;
  for (double f : cand) {
    a.keep_frac = f;
    for (int rep = 0; rep < 2; ++rep) {  // warm, then timed
      CK(cudaMemsetAsync(plan->d_bar, 0, sizeof(GridBarrier), st));
      CK(cudaMemsetAsync(plan->d_err, 0, sizeof(int), st));
      if (rep == 1) CK(cudaEventRecord(e0, st));
      CK(launch_cg_fused(a, st));
      if (rep == 1) CK(cudaEventRecord(e1, st));
    }
    int err = 0;
    CK(cudaMemcpyAsync(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      plan->failed = true;
      return MINNORM_ETIMEOUT;
    }
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      best_f = f;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaMemsetAsync(plan->d_bar, 0, sizeof(GridBarrier), st));
  CK(cudaMemsetAsync(plan->d_err, 0, sizeof(int), st));
  plan->cg_keep = best_f;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_cg_keep_cache[key] = best_f;
  return MINNORM_OK;
}

// ---- Steps 3-5 --------------------------------------------------------------
// Inner solve: CG on (Wp^* A A^* Wp) du = g, Wp = P R^{-1}; dy = Wp du.
minnorm_status enqueue_cg_iters(minnorm_plan_t plan, const void *Acg, double tol, int k);
static bool cg_pair_on(minnorm_plan_t plan, const void *Acg);

minnorm_status inner_cg(minnorm_plan_t plan, const void *Acg, double tol, int maxit, int *iters) {
  cudaStream_t st = plan->st;
  const int m = (int)plan->m;
  const int64_t lda_cg = plan->g_cg.ld;
  if (plan->fused_ok && cg_fused_supported(plan->m, plan->n, lda_cg, Acg)) {
    CK(cudaMemsetAsync(plan->d_bar, 0, sizeof(GridBarrier), st));
    CK(cudaMemsetAsync(plan->d_err, 0, sizeof(int), st));
    CgFusedArgs a{};
    a.A = Acg;
    a.m = plan->m;
    a.n = plan->n;
    a.lda = lda_cg;
    a.Wp = plan->d_Wp;
    a.WpH = plan->d_WpH;
    a.g = plan->d_g;
    a.u = plan->d_u;
    a.s = plan->d_s;
    a.w = plan->d_w;
    a.t = plan->d_t;
    a.dy = plan->d_dy;
    a.tpart = plan->d_tpart;
    a.qq_part = plan->d_qqp;
    a.gg_part = plan->d_ggp;
    a.sc = plan->d_cg;
    a.tol2 = tol * tol;
    a.maxit = maxit;
    a.bar = plan->d_bar;
    a.err = plan->d_err;
    a.limit_ns = plan->wait_limit_ns;
    a.grid = plan->sms;
    if (!plan->cg_tuned) {
      minnorm_status ts = tune_cg_keep(plan, a);
      if (ts != MINNORM_OK) return ts;
    }
    a.keep_frac = plan->cg_keep;
    a.withhold = plan->withhold;
    plan->withhold = 0;
    {
      Timed tm(plan, 5);
      CK(launch_cg_fused(a, st));
    }
    int err = 0;
    CK(cudaMemcpyAsync(plan->h_cg, plan->d_cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err) {
      plan->failed = true;
      return MINNORM_ETIMEOUT;
    }
    *iters = plan->h_cg->iters;
    plan->fused_iters += *iters;
    return MINNORM_OK;
  }
  CK(launch_cg_init(m, plan->d_g, plan->d_u, plan->d_s, plan->d_p, plan->d_cg, st));
  const int chunk = plan->fp32 ? 4 : 8;
  const bool pair = cg_pair_on(plan, Acg);   // its loads' waits are bounded: their error word
  if (pair) CK(cudaMemsetAsync(plan->d_err, 0, sizeof(int), st));
  int it = 0, err = 0;
  while (it < maxit) {
    const int todo = std::min(chunk, maxit - it);
    minnorm_status cs = enqueue_cg_iters(plan, Acg, tol, todo);
    if (cs != MINNORM_OK) return cs;
    it += todo;
    CK(cudaMemcpyAsync(plan->h_cg, plan->d_cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
    if (pair) CK(cudaMemcpyAsync(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err) {
      plan->failed = true;
      return MINNORM_ETIMEOUT;
    }
    if (plan->h_cg->done) break;
  }
  *iters = plan->h_cg->iters;
  // dy = Wp u
  CK(launch_small_gemv(plan->d_Wp, m, plan->d_u, plan->d_dy, nullptr, nullptr, st));
  return MINNORM_OK;
}

minnorm_status norms(minnorm_plan_t plan, bool with_x, double *gnorm, double *xnorm) {
  cudaStream_t st = plan->st;
  CK(launch_sumsq(plan->m, plan->d_g, plan->d_red, plan->d_norms, st));
  if (with_x) CK(launch_sumsq(plan->n, plan->d_xh, plan->d_red + 1024, plan->d_norms + 1, st));
  CK(cudaMemcpyAsync(plan->h_norms, plan->d_norms, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *gnorm = std::sqrt(plan->h_norms[0]);
  *xnorm = with_x ? std::sqrt(plan->h_norms[1]) : 0.0;
  return MINNORM_OK;
}

XprodArgs xargs(minnorm_plan_t plan, const void *b) {
  XprodArgs a{};
  a.afix = plan->d_afix;
  a.E = plan->d_E;
  a.rows = plan->m;
  a.cols = plan->n;
  a.yh = plan->d_yh;
  a.yl = plan->d_yl;
  a.yfix = plan->d_yfix;
  a.Fy = plan->d_F;
  a.Fx = plan->d_F + 1;
  a.xh = plan->d_xh;
  a.xl = plan->d_xl;
  a.b = b;
  a.r = plan->d_r;
  a.partial = plan->d_xpart;
  a.nchunk = plan->x_nchunk;
  a.chunk = plan->x_chunk;
  a.xpart = plan->d_xapart;
  a.xfix = plan->d_xfix;
  a.xsplit = plan->x_split;
  return a;
}

// ---- autotuning of the exact residual's work split ------------------------------
// The exact residual (x = A^* y and b - A x in 128-bit fixed point) gives bit-identical
// results for any split of its work, so on a plan's first residual the candidates
// (column chunks of the forward pass: the default, half, twice; row splits of the
// adjoint pass: 1, 2, 4, 8) are run on the actual data, timed with CUDA events on the
// plan's stream, and the fastest kept, also for later plans of the same shape (process-
// wide cache). Small systems keep the default split (a residual there takes microseconds).

minnorm_status tune_xresidual(minnorm_plan_t plan, const void *b) {
  plan->x_tuned = true;
  const int64_t m = plan->m, n = plan->n;
  if (m * n < ((int64_t)1 << 22)) return MINNORM_OK;
  const TuneKey key{m, n, plan->sms};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      plan->x_nchunk = it->second.first;
      plan->x_chunk = (n + plan->x_nchunk - 1) / plan->x_nchunk;
      plan->x_split = it->second.second;
      return MINNORM_OK;
    }
  }
  cudaStream_t st = plan->st;
  std::vector<int> chunks = {plan->x_nchunk};
  if (plan->x_nchunk > 1) chunks.push_back(plan->x_nchunk / 2);
  if (plan->x_nchunk_max > plan->x_nchunk) chunks.push_back(plan->x_nchunk_max);
  std::vector<int> splits;
  for (int sp = 1; sp <= xadj_max_splits(m); sp *= 2) splits.push_back(sp);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = INFINITY;
  int best_c = plan->x_nchunk, best_s = 0;
  for (int nc : chunks) {
    for (int sp : splits) {
      XprodArgs a = xargs(plan, b);
      a.nchunk = nc;
      a.chunk = (n + nc - 1) / nc;
      a.xsplit = sp;
      CK(launch_xresidual(a, st));  // warm
      CK(cudaEventRecord(e0, st));
      CK(launch_xresidual(a, st));
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_c = nc;
        best_s = sp;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan->x_nchunk = best_c;
  plan->x_chunk = (n + best_c - 1) / best_c;
  plan->x_split = best_s;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = {best_c, best_s};
  return MINNORM_OK;
}

// one exact residual with the plan's (tuned) split
minnorm_status xresidual(minnorm_plan_t plan, const void *b, const int *skip = nullptr) {
  if (!plan->x_tuned && !skip) {  // an asynchronous solve keeps the current split (no host round trip)
    minnorm_status s = tune_xresidual(plan, b);
    if (s != MINNORM_OK) return s;
  }
  XprodArgs a = xargs(plan, b);
  a.skip = skip;
  CK(launch_xresidual(a, plan->st));
  return MINNORM_OK;
}

minnorm_status solve_impl(minnorm_plan_t plan, const void *A, int64_t lda, const void *b, double eps, void *x,
                          minnorm_info *info) {
  cudaStream_t st = plan->st;
  const int64_t m = plan->m, n = plan->n;
  (void)lda;
  const bool timing = plan->flags & MINNORM_FLAG_TIMING;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double ms0[6];
  memcpy(ms0, plan->stat_ms, sizeof(ms0));
  if (timing) { e0 = next_event(plan); e1 = next_event(plan); CK(cudaEventRecord(e0, st)); }
  const void *Acg = plan->d_A32 ? (const void *)plan->d_A32 : A;
  // y = 0, x = 0, r = b
  CK(cudaMemsetAsync(plan->d_yh, 0, sizeof(zd) * m, st));
  CK(cudaMemsetAsync(plan->d_yl, 0, sizeof(zd) * m, st));
  CK(cudaMemsetAsync(plan->d_xh, 0, sizeof(zd) * n, st));
  CK(cudaMemsetAsync(plan->d_xl, 0, sizeof(zd) * n, st));
  CK(cudaMemcpyAsync(plan->d_r, b, sizeof(zd) * m, cudaMemcpyDeviceToDevice, st));
  const double tol_inner = plan->fp32 ? kInnerTolMixed : 1e-11;
  const int maxit = plan->fp32 ? 40 : 300;
  double err = INFINITY, best = INFINITY, prev = INFINITY;
  int cg_total = 0, dd_passes = 0, outer = 0, stagnant = 0;
  (void)A;
  minnorm_status status = MINNORM_ENOCONV;
  for (outer = 0; outer < kMaxOuter; ++outer) {
    // g = Wp^* r (the preconditioned residual), and the bound ||x - p|| <= ||g||
    CK(launch_small_gemv(plan->d_WpH, (int)m, plan->d_r, plan->d_g, nullptr, nullptr, st));
    double gnorm = 0, xnorm = 0;
    minnorm_status s = norms(plan, outer > 0, &gnorm, &xnorm);
    if (s != MINNORM_OK) return s;
    if (outer > 0) {
      err = certified(plan, gnorm, xnorm);
      if (err <= eps) { status = MINNORM_OK; break; }
      if (err < best) best = err;
      stagnant = (err > 0.5 * prev) ? stagnant + 1 : 0;
      if (stagnant >= 2) { status = MINNORM_EFLOOR; break; }
      prev = err;
    } else if (gnorm == 0.0) {
      err = 0.0;
      status = MINNORM_OK;
      break;
    }
    int it = 0;
    s = inner_cg(plan, Acg, tol_inner, maxit, &it);
    if (s != MINNORM_OK) return s;
    cg_total += it;
    CK(launch_dd_accumulate(m, plan->d_yh, plan->d_yl, plan->d_dy, st));
    {
      Timed tm(plan, 2);
      { minnorm_status xs = xresidual(plan, b); if (xs != MINNORM_OK) return xs; }
      dd_passes += 2;
    }
  }
  if (status == MINNORM_ENOCONV && outer == kMaxOuter) {
    // final bound for the last iterate
    CK(launch_small_gemv(plan->d_WpH, (int)m, plan->d_r, plan->d_g, nullptr, nullptr, st));
    double gnorm = 0, xnorm = 0;
    minnorm_status s = norms(plan, true, &gnorm, &xnorm);
    if (s != MINNORM_OK) return s;
    err = certified(plan, gnorm, xnorm);
    if (err <= eps) status = MINNORM_OK;
  }
  CK(cudaMemcpyAsync(x, plan->d_xh, sizeof(zd) * n, cudaMemcpyDeviceToDevice, st));
  if (timing) CK(cudaEventRecord(e1, st));
  if (info || timing) {
    CK(launch_sumsq(m, plan->d_r, plan->d_red, plan->d_norms + 2, st));
    CK(launch_sumsq(m, (const zd *)b, plan->d_red + 1024, plan->d_norms + 3, st));
    CK(cudaMemcpyAsync(plan->h_norms, plan->d_norms, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  if (timing) {
    cudaEventElapsedTime(&plan->ms_solve, e0, e1);
    collect_timers(plan);
  }
  if (info) {
    info->outer_steps = outer;
    info->cg_iters = cg_total;
    info->exact_passes = dd_passes;
    info->status = status;
    info->err_bound = err;
    const double bn = std::sqrt(plan->h_norms[3]);
    info->resid_rel = bn > 0 ? std::sqrt(plan->h_norms[2]) / bn : 0.0;
    fill_factor_info(plan, info);
    info->ms_solve = plan->ms_solve;
    info->ms_cg = (float)(plan->stat_ms[0] + plan->stat_ms[1] + plan->stat_ms[5] - ms0[0] - ms0[1] - ms0[5]);
    info->ms_refine = (float)(plan->stat_ms[2] - ms0[2]);
  }
  return status;
}

// ---- Steps 3-5 without host round trips (minnorm_solve with info == NULL) -----------
// The refinement loop of solve_impl, enqueued whole: kMaxOuter steps, each opened by the
// stopping test on the device (solve_stop_kernel, the same rule and certificate as the host
// loop). Once the test fires it sets SolveState::done, and every kernel of the later steps
// (the small products, the CG kernels through their `done` word, the accumulation of y and the
// exact residual) returns at once. The inner CG of the two-pass form enqueues its maxit
// iterations (each kernel returns once the CG's own test has fired). Nothing is tuned here: a
// plan that has not yet run a synchronous solve uses the default work splits. The status, the
// step counts and the bound stay on the device until minnorm_solve_wait.
// k iterations of the two-pass CG (each kernel returns once the CG's test has fired)
// the one-pass product serves this plan's mixed CG (A's layout permitting)
static bool cg_pair_on(minnorm_plan_t plan, const void *Acg) {
  return plan->fp32 && plan->pair_nc > 0 && cg_pair_supported(plan->m, plan->n, plan->g_cg.ld, Acg);
}

minnorm_status enqueue_cg_iters(minnorm_plan_t plan, const void *Acg, double tol, int k) {
  cudaStream_t st = plan->st;
  const int *done = &plan->d_cg->done;
  const int mi = (int)plan->m;
  const bool pair = cg_pair_on(plan, Acg);
  for (int i = 0; i < k; ++i) {
    if (pair) {
      CK(launch_small_gemv(plan->d_Wp, mi, plan->d_p, plan->d_w, plan->d_w32, done, st));
      CgPairArgs pa{Acg, plan->g_cg.ld, plan->m, plan->n, plan->d_w32, plan->d_t, plan->d_tpart, plan->d_qqp,
                    plan->pair_nc, plan->d_err, plan->wait_limit_ns, done};
      Timed tm(plan, 0);
      CK(launch_cg_pair(pa, st));
    } else if (plan->fp32) {
      CK(launch_small_gemv(plan->d_Wp, mi, plan->d_p, plan->d_w, plan->d_w32, done, st));
      { Timed tm(plan, 0); CK(launch_gemv_adj_f32(plan->g_cg, Acg, plan->d_w32, plan->d_q, plan->d_part, plan->d_qq, done, st)); }
      { Timed tm(plan, 1); CK(launch_gemv_fwd_f32(plan->g_cg, Acg, plan->d_q, plan->d_t, plan->d_part, done, st)); }
    } else {
      CK(launch_small_gemv(plan->d_Wp, mi, plan->d_p, plan->d_w, nullptr, done, st));
      { Timed tm(plan, 0); CK(launch_gemv_adj(plan->g_cg, Acg, plan->d_w, plan->d_q, plan->d_part, plan->d_qq, done, st)); }
      { Timed tm(plan, 1); CK(launch_gemv_fwd(plan->g_cg, Acg, plan->d_q, plan->d_t, plan->d_part, done, st)); }
    }
    CK(launch_small_gemv(plan->d_WpH, mi, plan->d_t, plan->d_np, nullptr, done, st));
    CK(launch_cg_update(mi, pair ? plan->d_qqp : plan->d_qq, pair ? plan->pair_nc : plan->nqq, plan->d_np, plan->d_u,
                        plan->d_s, plan->d_p, plan->d_cg, tol * tol, st));
  }
  return MINNORM_OK;
}

// Inside the capture of the asynchronous solve: the two-pass CG's iterations as a WHILE node of
// the graph whose body is a chunk of kAsyncChunk iterations followed by a kernel that sets the
// node's condition (cleared once the CG's test has fired or maxit iterations have run; maxit is
// a multiple of the chunk, so the cap is the synchronous form's). The graph holds one copy of the
// chunk however many iterations run.
constexpr int kAsyncChunk = 4;
minnorm_status capture_cg_while(minnorm_plan_t plan, const void *Acg, double tol, int maxit) {
  cudaStream_t st = plan->st;
  if (!plan->st_cap2) CK(cudaStreamCreateWithFlags(&plan->st_cap2, cudaStreamNonBlocking));
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *edges = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edges, &nd));
  if (cs != cudaStreamCaptureStatusActive) return MINNORM_ECUDA;
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, edges, nd, &cp));
  CK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(plan->st_cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  plan->st = plan->st_cap2;
  minnorm_status s = enqueue_cg_iters(plan, Acg, tol, kAsyncChunk);
  if (s == MINNORM_OK && launch_cg_continue(h, plan->d_cg, maxit, plan->st_cap2) != cudaSuccess) s = MINNORM_ECUDA;
  plan->st = st;
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(plan->st_cap2, &out);
  if (s != MINNORM_OK) return s;
  CK(e);
  return MINNORM_OK;
}

minnorm_status solve_async_body(minnorm_plan_t plan, const void *A, const void *b, void *x) {
  cudaStream_t st = plan->st;
  const int64_t m = plan->m, n = plan->n;
  const void *Acg = plan->d_A32 ? (const void *)plan->d_A32 : A;
  const int *skip = &plan->d_ss->done;
  CK(cudaMemsetAsync(plan->d_yh, 0, sizeof(zd) * m, st));
  CK(cudaMemsetAsync(plan->d_yl, 0, sizeof(zd) * m, st));
  CK(cudaMemsetAsync(plan->d_xh, 0, sizeof(zd) * n, st));
  CK(cudaMemsetAsync(plan->d_xl, 0, sizeof(zd) * n, st));
  CK(cudaMemcpyAsync(plan->d_r, b, sizeof(zd) * m, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(plan->d_err, 0, sizeof(int), st));
  CK(launch_solve_state_init(plan->d_ss, st));
  const CertConsts *cc = plan->d_cc;
  const double tol_inner = plan->fp32 ? kInnerTolMixed : 1e-11;
  const int maxit = plan->fp32 ? 40 : 300;
  const bool fused = plan->fused_ok && cg_fused_supported(plan->m, plan->n, plan->g_cg.ld, Acg);
  for (int outer = 0; outer <= kMaxOuter; ++outer) {
    const bool final = outer == kMaxOuter;
    CK(launch_small_gemv(plan->d_WpH, (int)m, plan->d_r, plan->d_g, nullptr, skip, st));
    CK(launch_sumsq(m, plan->d_g, plan->d_red, plan->d_norms, st));
    if (outer > 0) CK(launch_sumsq(n, plan->d_xh, plan->d_red + 1024, plan->d_norms + 1, st));
    CK(launch_solve_stop(plan->d_ss, plan->d_norms, outer, final, cc, outer > 0 ? plan->d_cg : nullptr, st));
    if (final) break;
    if (fused) {
      CK(cudaMemsetAsync(plan->d_bar, 0, sizeof(GridBarrier), st));
      CgFusedArgs a{};
      a.A = Acg;
      a.m = plan->m;
      a.n = plan->n;
      a.lda = plan->g_cg.ld;
      a.Wp = plan->d_Wp;
      a.WpH = plan->d_WpH;
      a.g = plan->d_g;
      a.u = plan->d_u;
      a.s = plan->d_s;
      a.w = plan->d_w;
      a.t = plan->d_t;
      a.dy = plan->d_dy;
        a.tpart = plan->d_tpart;
      a.qq_part = plan->d_qqp;
      a.gg_part = plan->d_ggp;
      a.sc = plan->d_cg;
      a.tol2 = tol_inner * tol_inner;
      a.maxit = maxit;
      a.bar = plan->d_bar;
      a.err = plan->d_err;
      a.limit_ns = plan->wait_limit_ns;
      a.grid = plan->sms;
      a.keep_frac = plan->cg_keep;
      a.skip = skip;
      a.withhold = plan->withhold;
      plan->withhold = 0;
      Timed tm(plan, 5);
      CK(launch_cg_fused(a, st));
    } else {
      const int mi = (int)m;
      CK(launch_cg_init(mi, plan->d_g, plan->d_u, plan->d_s, plan->d_p, plan->d_cg, st, skip));
      minnorm_status ws = capture_cg_while(plan, Acg, tol_inner, maxit);
      if (ws != MINNORM_OK) return ws;
      CK(launch_small_gemv(plan->d_Wp, mi, plan->d_u, plan->d_dy, nullptr, skip, st));
    }
    CK(launch_dd_accumulate(m, plan->d_yh, plan->d_yl, plan->d_dy, st, skip));
    {
      Timed tm(plan, 2);
      minnorm_status xs = xresidual(plan, b, skip);
      if (xs != MINNORM_OK) return xs;
    }
  }
  CK(cudaMemcpyAsync(x, plan->d_xh, sizeof(zd) * n, cudaMemcpyDeviceToDevice, st));
  // ||r||^2 and ||b||^2 for the report, kept on the device
  CK(launch_sumsq(m, plan->d_r, plan->d_red, plan->d_norms + 2, st));
  CK(launch_sumsq(m, (const zd *)b, plan->d_red + 1024, plan->d_norms + 3, st));
  return MINNORM_OK;
}

// The loop above holds up to a few thousand kernels (the two-pass CG enqueues its iterations),
// more than a stream's launch queue takes without blocking the host, so it is captured once into
// a CUDA graph (on a private stream: the plan's may be the legacy default stream) and each
// asynchronous solve is one graph launch. The graph is kept for the plan's (A, b, x, lda) and
// captured again when they change; everything else it reads (the factors, the certificate's
// constants in d_cc, eps) is read from device memory at run time.
minnorm_status solve_async(minnorm_plan_t plan, const void *A, int64_t lda, const void *b, double eps, void *x) {
  const bool timing = plan->flags & MINNORM_FLAG_TIMING;
  if (!plan->ev_as0) {
    CK(cudaEventCreate(&plan->ev_as0));
    CK(cudaEventCreate(&plan->ev_as1));
  }
  if (!plan->st_cap) CK(cudaStreamCreateWithFlags(&plan->st_cap, cudaStreamNonBlocking));
  const bool same = plan->ga_exec && plan->ga_A == A && plan->ga_b == b && plan->ga_x == x && plan->ga_lda == lda &&
                    plan->withhold == 0 && plan->ga_withhold == 0;
  if (!same) {
    if (plan->ga_exec) {
      cudaGraphExecDestroy(plan->ga_exec);
      plan->ga_exec = nullptr;
    }
    cudaStream_t keep = plan->st;
    plan->st = plan->st_cap;
    plan->capturing = true;
    plan->ga_withhold = plan->withhold;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(plan->st_cap, cudaStreamCaptureModeThreadLocal);
    minnorm_status bs = MINNORM_OK;
    if (e == cudaSuccess) {
      bs = solve_async_body(plan, A, b, x);
      e = cudaStreamEndCapture(plan->st_cap, &g);
    }
    plan->st = keep;
    plan->capturing = false;
    if (bs != MINNORM_OK) {
      if (g) cudaGraphDestroy(g);
      return bs;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->ga_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      plan->ga_exec = nullptr;
      plan->failed = true;
      return MINNORM_ECUDA;
    }
    plan->ga_A = A;
    plan->ga_b = b;
    plan->ga_x = x;
    plan->ga_lda = lda;
  }
  cudaStream_t st = plan->st;
  // the certificate's constants for this sketch and eps (as kernel arguments: nothing on the
  // host has to outlive the call, and no pageable copy waits for the stream)
  const CertConsts cc{plan->cert_delta, 1.0 + plan->inv_eta + 4.0 * (double)plan->m * 0x1.0p-53, eps};
  CK(launch_set_cert(plan->d_cc, cc, st));
  if (timing) CK(cudaEventRecord(plan->ev_as0, st));
  note_launch();
  CK(cudaGraphLaunch(plan->ga_exec, st));
  if (timing) CK(cudaEventRecord(plan->ev_as1, st));
  plan->async_pending = true;
  return MINNORM_OK;
}

// workspace of the blocked QR (qrblk.cu), allocated on first use
minnorm_status qrblk_alloc(minnorm_plan_t plan) {
  if (plan->qb_ready) return MINNORM_OK;
  size_t b[18];
  qrblk_sizes(plan->l, plan->m, plan->sms, b);
  QrBlkWork &w = plan->qb;
  w.l = plan->l;
  w.m = plan->m;
  ALLOC(w.sA, b[0]);
  ALLOC(w.sB, b[1]);
  ALLOC(w.sV, b[2]);
  ALLOC(w.sZ, b[3]);
  ALLOC(w.eA, b[4]);
  ALLOC(w.eB, b[5]);
  ALLOC(w.eV, b[6]);
  ALLOC(w.eZ, b[7]);
  ALLOC(w.part, b[8]);
  w.part_bytes = b[8];
  ALLOC(w.W, b[9]);
  ALLOC(w.Z, b[10]);
  ALLOC(w.T, b[11]);
  ALLOC(w.tau, b[12]);
  ALLOC(w.Vb, b[13]);
  ALLOC(w.R1, b[14]);
  ALLOC(w.ppart, b[15]);
  ALLOC(w.rowb, b[16]);
  ALLOC(w.bar, b[17]);
  if (cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking) != cudaSuccess) return MINNORM_ENOMEM;
  if (cudaEventCreateWithFlags(&w.ev_panel, cudaEventDisableTiming) != cudaSuccess) return MINNORM_ENOMEM;
  if (cudaEventCreateWithFlags(&w.ev_t, cudaEventDisableTiming) != cudaSuccess) return MINNORM_ENOMEM;
  plan->qb_ready = true;
  return MINNORM_OK;
}

// argument checks of minnorm_plan_create (no device access)
minnorm_status check_plan_args(int64_t m, int64_t n, int64_t &l, minnorm_dtype dtype, minnorm_precision prec,
                               uint32_t flags) {
  if (m < 1 || n < 2 || m >= n) return MINNORM_EINVAL;
  if (l == 0) l = std::min<int64_t>(4 * m, n);
  if (l <= m || l > n) return MINNORM_EINVAL;
  if (dtype != MINNORM_C128 && dtype != MINNORM_C64) return MINNORM_EINVAL;
  if (prec != MINNORM_FP64 && prec != MINNORM_MIXED) return MINNORM_EINVAL;
  if ((flags & ~(MINNORM_FLAG_TIMING | MINNORM_FLAG_KEEP_SKETCH)) != 0) return MINNORM_EINVAL;
  if (n > (int64_t(1) << 30) || m > 4864) return MINNORM_ENOTSUP;
  return MINNORM_OK;
}

minnorm_status plan_create_pooled(minnorm_plan_t *out, int64_t m, int64_t n, int64_t l, minnorm_dtype dtype,
                                  minnorm_precision prec, uint64_t seed, uint32_t flags, void *stream,
                                  const ScratchPool *pool) {
  if (!out) return MINNORM_EINVAL;
  *out = nullptr;
  minnorm_status c = check_plan_args(m, n, l, dtype, prec, flags);
  if (c != MINNORM_OK) return c;
  minnorm_plan_t plan = new (std::nothrow) minnorm_plan_s();
  if (!plan) return MINNORM_ENOMEM;
  plan->pool = pool;
  minnorm_status s = create_impl(plan, m, n, l, dtype, prec, seed, flags, stream);
  if (s != MINNORM_OK) {
    minnorm_plan_destroy(plan);
    return s;
  }
  *out = plan;
  return MINNORM_OK;
}

// ---- Steps 3-5 for blocks of right-hand sides (mixed precision) -------------------
minnorm_status block_alloc(minnorm_plan_t plan) {
  if (plan->blk_ready) return MINNORM_OK;
  const int64_t m = plan->m, n = plan->n;
  const size_t bz = sizeof(zd) * (size_t)m * kBlockRhs;
  void **bufs[] = {&plan->d_bG, &plan->d_bR, &plan->d_bU, &plan->d_bS, &plan->d_bP, &plan->d_bT, &plan->d_bNp,
                   &plan->d_bdY, &plan->d_bYh, &plan->d_bYl};
  for (void **b : bufs) ALLOC(*b, bz);
  ALLOC(plan->d_bW32, sizeof(zf) * (size_t)m * kBlockRhs);
  ALLOC(plan->d_bQ, sizeof(zf) * (size_t)n * kBlockRhs);
  ALLOC(plan->d_bqqp, sizeof(float) * (size_t)block_adj_parts(n) * kBlockRhs);
  ALLOC(plan->d_bsplit, tc_split_bytes(m));
  ALLOC(plan->d_bsplit2, tc_split2_bytes(n));
  plan->blk_nsplit = block_fwd_splits(m, n, plan->sms);
  plan->blk_nsplit_tc = tc_fwd_splits(m, n, plan->sms);
  ALLOC(plan->d_btpart,
        sizeof(zf) * (size_t)std::max(plan->blk_nsplit, plan->blk_nsplit_tc) * m * kBlockRhs);
  ALLOC(plan->d_bpart, sizeof(double) * (size_t)block_col_parts(m) * kBlockRhs);
  ALLOC(plan->d_bscal, sizeof(double) * 4 * kBlockRhs);
  ALLOC(plan->d_bint, sizeof(int) * (3 * kBlockRhs + 1));
  if (cudaMallocHost(&plan->h_bpart, sizeof(double) * (size_t)block_col_parts(m) * kBlockRhs) != cudaSuccess)
    return MINNORM_ENOMEM;
  if (cudaMallocHost(&plan->h_bint, sizeof(int) * (3 * kBlockRhs + 1)) != cudaSuccess) return MINNORM_ENOMEM;
  if (cudaMallocHost(&plan->h_bx, sizeof(double) * kBlockRhs) != cudaSuccess) return MINNORM_ENOMEM;
  plan->blk_ready = true;
  return MINNORM_OK;
}

// per-column ||G_c|| (host, after a sync)
minnorm_status block_gnorms(minnorm_plan_t plan, double *gn) {
  cudaStream_t st = plan->st;
  const int m = (int)plan->m, np = block_col_parts(m);
  CK(launch_block_colnorms(m, plan->d_bG, plan->d_bpart, st));
  CK(cudaMemcpyAsync(plan->h_bpart, plan->d_bpart, sizeof(double) * np * kBlockRhs, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int c = 0; c < kBlockRhs; ++c) {
    double t = 0.0;
    for (int q = 0; q < np; ++q) t += plan->h_bpart[q * kBlockRhs + c];
    gn[c] = std::sqrt(t);
  }
  return MINNORM_OK;
}

// the block inner CG on G (columns with use[c]); returns the iterations taken (max over columns)
minnorm_status block_inner_cg(minnorm_plan_t plan, const void *Acg, int64_t lda_cg, double tol, int maxit,
                              int *iters_out) {
  cudaStream_t st = plan->st;
  const int m = (int)plan->m;
  double *gam = plan->d_bscal, *gam0 = gam + kBlockRhs, *alpha = gam0 + kBlockRhs, *beta = alpha + kBlockRhs;
  int *use = plan->d_bint, *active = use + kBlockRhs, *iters = active + kBlockRhs, *alldone = iters + kBlockRhs;
  CK(cudaMemsetAsync(iters, 0, sizeof(int) * kBlockRhs, st));
  CK(launch_block_cg_init(m, plan->d_bG, plan->d_bU, plan->d_bS, plan->d_bP, plan->d_bpart, use, gam, gam0, active,
                          alldone, st));
  BlockProductArgs pa{};
  pa.A = Acg;
  pa.m = plan->m;
  pa.n = plan->n;
  pa.lda = lda_cg;
  pa.W32 = plan->d_bW32;
  pa.Q = plan->d_bQ;
  pa.qqp = plan->d_bqqp;
  pa.gam = gam;
  pa.active = active;
  pa.alpha = alpha;
  pa.tpart = plan->d_btpart;
  pa.nsplit = plan->blk_nsplit;
  pa.T = plan->d_bT;
  pa.alldone = alldone;
  pa.Bsplit = plan->d_bsplit;
  pa.Bsplit2 = plan->d_bsplit2;
  pa.nsplit_tc = plan->blk_nsplit_tc;
  pa.err = plan->d_err;
  pa.limit_ns = plan->wait_limit_ns;
  pa.sms = plan->sms;
  CK(cudaMemsetAsync(plan->d_err, 0, sizeof(int), st));
  int it = 0;
  while (it < maxit) {
    const int todo = std::min(4, maxit - it);
    for (int k = 0; k < todo; ++k) {
      CK(launch_block_mm(plan->d_Wp, m, plan->d_bP, nullptr, plan->d_bW32, alldone, st));
      { Timed tm(plan, 0); CK(launch_block_adj(pa, st)); }
      { Timed tm(plan, 1); CK(launch_block_fwd(pa, st)); }
      CK(launch_block_mm(plan->d_WpH, m, plan->d_bT, plan->d_bNp, nullptr, alldone, st));
      CK(launch_block_cg_update(m, alpha, plan->d_bP, plan->d_bNp, plan->d_bU, plan->d_bS, plan->d_bpart, tol * tol,
                                gam, gam0, active, beta, iters, alldone, st));
    }
    it += todo;
    CK(cudaMemcpyAsync(plan->h_bint, plan->d_bint, sizeof(int) * (3 * kBlockRhs + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (plan->h_bint[3 * kBlockRhs]) break;
  }
  int err = 0;
  CK(cudaMemcpyAsync(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (err) {
    plan->failed = true;
    return MINNORM_ETIMEOUT;
  }
  int mx = 0;
  for (int c = 0; c < kBlockRhs; ++c) mx = std::max(mx, plan->h_bint[2 * kBlockRhs + c]);
  *iters_out = mx;
  return MINNORM_OK;
}

// Steps 3-5 for columns j0 .. j0 + kc - 1 of B (kc <= kBlockRhs), mixed precision: the block
// CG replaces the per-column CG; the refinement's exact residuals and stopping tests stay per
// column, exactly as in solve_impl.
minnorm_status solve_block_chunk(minnorm_plan_t plan, const void *A, int64_t lda, const zd *B, int64_t ldb, int kc,
                                 double eps, zd *X, int64_t ldx, minnorm_info *infos) {
  cudaStream_t st = plan->st;
  const int64_t m = plan->m, n = plan->n;
  const void *Acg = plan->d_A32 ? (const void *)plan->d_A32 : A;
  const int64_t lda_cg = plan->d_A32 ? n : lda;
  const double tol_inner = kInnerTolMixed;
  const int maxit = 40;
  int *use = plan->d_bint;
  struct Col {
    int outer = 0, stagnant = 0, cg = 0, passes = 0;
    double err = INFINITY, best = INFINITY, prev = INFINITY;
    minnorm_status status = MINNORM_ENOCONV;
    bool done = false;
  };
  std::vector<Col> col(kc);
  CK(cudaMemsetAsync(plan->d_bYh, 0, sizeof(zd) * m * kBlockRhs, st));
  CK(cudaMemsetAsync(plan->d_bYl, 0, sizeof(zd) * m * kBlockRhs, st));
  CK(launch_block_load_rhs((int)m, kc, B, ldb, plan->d_bR, st));
  for (int c = 0; c < kc; ++c) CK(cudaMemsetAsync(X + c * ldx, 0, sizeof(zd) * n, st));
  std::vector<double> gn(kBlockRhs);
  std::vector<int> huse(kBlockRhs);
  for (int outer = 0; outer <= kMaxOuter; ++outer) {
    // G = Wp^* R; per-column bound ||x - p|| <= ||g|| (x as of the last exact residual)
    CK(launch_block_mm(plan->d_WpH, (int)m, plan->d_bR, plan->d_bG, nullptr, nullptr, st));
    minnorm_status s = block_gnorms(plan, gn.data());
    if (s != MINNORM_OK) return s;
    bool any = false;
    for (int c = 0; c < kBlockRhs; ++c) {
      huse[c] = 0;
      if (c >= kc || col[c].done) continue;
      Col &q = col[c];
      if (outer > 0) {
        const double xn = std::sqrt(plan->h_bx[c]);
        q.err = certified(plan, gn[c], xn);
        if (q.err <= eps) { q.status = MINNORM_OK; q.done = true; continue; }
        if (q.err < q.best) q.best = q.err;
        q.stagnant = (q.err > 0.5 * q.prev) ? q.stagnant + 1 : 0;
        if (q.stagnant >= 2) { q.status = MINNORM_EFLOOR; q.done = true; continue; }
        q.prev = q.err;
      } else if (gn[c] == 0.0) {
        q.err = 0.0;
        q.status = MINNORM_OK;
        q.done = true;
        continue;
      }
      if (outer == kMaxOuter) { q.done = true; continue; }  // ENOCONV with the bound just taken
      huse[c] = 1;
      any = true;
      q.outer = outer + 1;
    }
    if (!any) break;
    CK(cudaMemcpyAsync(use, huse.data(), sizeof(int) * kBlockRhs, cudaMemcpyHostToDevice, st));
    int it = 0;
    s = block_inner_cg(plan, Acg, lda_cg, tol_inner, maxit, &it);
    if (s != MINNORM_OK) return s;
    // dY = Wp U; y += dY (double-double) on the iterating columns
    CK(launch_block_mm(plan->d_Wp, (int)m, plan->d_bU, plan->d_bdY, nullptr, nullptr, st));
    CK(launch_block_dd_acc((int)m, use, plan->d_bYh, plan->d_bYl, plan->d_bdY, st));
    // exact x = A^* y and r = b - A x per iterating column
    for (int c = 0; c < kc; ++c) {
      if (!huse[c]) continue;
      col[c].cg += plan->h_bint[2 * kBlockRhs + c];
      CK(launch_block_get_col((int)m, plan->d_bYh, c, plan->d_yh, st));
      CK(launch_block_get_col((int)m, plan->d_bYl, c, plan->d_yl, st));
      {
        Timed tm(plan, 2);
        { minnorm_status xs = xresidual(plan, B + c * ldb); if (xs != MINNORM_OK) return xs; }
      }
      col[c].passes += 2;
      CK(launch_block_set_col((int)m, plan->d_r, c, plan->d_bR, st));
      CK(cudaMemcpyAsync(X + c * ldx, plan->d_xh, sizeof(zd) * n, cudaMemcpyDeviceToDevice, st));
      CK(launch_sumsq(n, plan->d_xh, plan->d_red + 1024, plan->d_norms + 1, st));
      CK(cudaMemcpyAsync(plan->h_bx + c, plan->d_norms + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
  }
  if (infos) {
    for (int c = 0; c < kc; ++c) {
      // residual norm for the report
      CK(launch_block_get_col((int)m, plan->d_bR, c, plan->d_r, st));
      CK(launch_sumsq(m, plan->d_r, plan->d_red, plan->d_norms + 2, st));
      CK(launch_sumsq(m, B + c * ldb, plan->d_red + 1024, plan->d_norms + 3, st));
      CK(cudaMemcpyAsync(plan->h_norms, plan->d_norms, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      minnorm_info &f = infos[c];
      fill_factor_info(plan, &f);
      f.outer_steps = col[c].outer;
      f.cg_iters = col[c].cg;
      f.exact_passes = col[c].passes;
      f.status = col[c].status;
      f.err_bound = col[c].err;
      const double bn = std::sqrt(plan->h_norms[3]);
      f.resid_rel = bn > 0 ? std::sqrt(plan->h_norms[2]) / bn : 0.0;
    }
  } else {
    CK(cudaStreamSynchronize(st));
  }
  minnorm_status first = MINNORM_OK;
  for (int c = 0; c < kc; ++c)
    if (col[c].status != MINNORM_OK && first == MINNORM_OK) first = col[c].status;
  return first;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

// =============================================================================
// C ABI
// =============================================================================
extern "C" {

const char *minnorm_status_string(minnorm_status s) {
  switch (s) {
    case MINNORM_OK: return "MINNORM_OK";
    case MINNORM_EINVAL: return "MINNORM_EINVAL: invalid argument";
    case MINNORM_ESTATE: return "MINNORM_ESTATE: call order or failed plan";
    case MINNORM_ENOMEM: return "MINNORM_ENOMEM: allocation failed";
    case MINNORM_ECUDA: return "MINNORM_ECUDA: a CUDA call failed";
    case MINNORM_ERANK: return "MINNORM_ERANK: sketch numerically rank deficient";
    case MINNORM_ENOCONV: return "MINNORM_ENOCONV: refinement step cap reached";
    case MINNORM_EFLOOR: return "MINNORM_EFLOOR: refinement stagnated above eps";
    case MINNORM_ETIMEOUT: return "MINNORM_ETIMEOUT: a bounded device wait expired";
    case MINNORM_ENOTSUP: return "MINNORM_ENOTSUP: unsupported size";
  }
  return "MINNORM_UNKNOWN";
}

minnorm_status minnorm_plan_create(minnorm_plan_t *out, int64_t m, int64_t n, int64_t l, minnorm_dtype dtype,
                                   minnorm_precision prec, uint64_t seed, uint32_t flags, void *stream) {
  return plan_create_pooled(out, m, n, l, dtype, prec, seed, flags, stream, nullptr);
}

minnorm_status minnorm_plan_set_params(minnorm_plan_t plan, const double *zeta_t, const int64_t *pi_t,
                                       const double *theta_t, const double *zeta, const int64_t *pi,
                                       const double *theta, const double *d, const int64_t *s) {
  if (!plan || !zeta_t || !pi_t || !theta_t || !zeta || !pi || !theta || !d || !s) return MINNORM_EINVAL;
  const int64_t n = plan->n, l = plan->l;
  SrftParams Q;
  Q.n = n;
  Q.l = l;
  auto cplx = [&](const double *src, std::vector<std::complex<double>> &dst) {
    dst.resize(n);
    for (int64_t j = 0; j < n; ++j) dst[j] = std::complex<double>(src[2 * j], src[2 * j + 1]);
  };
  cplx(zeta_t, Q.zeta_t);
  cplx(zeta, Q.zeta);
  cplx(d, Q.d);
  Q.pi_t.assign(pi_t, pi_t + n);
  Q.pi.assign(pi, pi + n);
  Q.theta_t.assign(theta_t, theta_t + (n - 1));
  Q.theta.assign(theta, theta + (n - 1));
  Q.s.assign(s, s + l);
  if (!validate_srft_params(Q)) return MINNORM_EINVAL;
  SrftParams old = plan->P;
  plan->P = Q;
  minnorm_status st = upload_params(plan);
  if (st == MINNORM_ENOTSUP) {
    plan->P = old;
    minnorm_status back = upload_params(plan);
    return back == MINNORM_OK ? MINNORM_ENOTSUP : back;
  }
  return st;
}

minnorm_status minnorm_plan_export_params(minnorm_plan_t plan, double *zeta_t, int64_t *pi_t, double *theta_t,
                                          double *zeta, int64_t *pi, double *theta, double *d, int64_t *s) {
  if (!plan) return MINNORM_EINVAL;
  const SrftParams &P = plan->P;
  const int64_t n = plan->n, l = plan->l;
  auto cplx = [&](const std::vector<std::complex<double>> &src, double *dst) {
    if (!dst) return;
    for (int64_t j = 0; j < n; ++j) { dst[2 * j] = src[j].real(); dst[2 * j + 1] = src[j].imag(); }
  };
  cplx(P.zeta_t, zeta_t);
  cplx(P.zeta, zeta);
  cplx(P.d, d);
  if (pi_t) std::copy(P.pi_t.begin(), P.pi_t.end(), pi_t);
  if (pi) std::copy(P.pi.begin(), P.pi.end(), pi);
  if (theta_t) std::copy(P.theta_t.begin(), P.theta_t.begin() + (n - 1), theta_t);
  if (theta) std::copy(P.theta.begin(), P.theta.begin() + (n - 1), theta);
  if (s) std::copy(P.s.begin(), P.s.begin() + l, s);
  return MINNORM_OK;
}

minnorm_status minnorm_sketch(minnorm_plan_t plan, const void *A, int64_t lda) {
  if (!plan || !A) return MINNORM_EINVAL;
  if (plan->failed) return MINNORM_ESTATE;
  if (lda < plan->n) return MINNORM_EINVAL;
  if (!aligned16(A) && plan->dtype == MINNORM_C128) return MINNORM_EINVAL;
  plan->sketched = false;
  plan->g_hp.ld = lda;
  plan->g_cg.ld = plan->d_A32 ? plan->n : lda;
  return sketch_impl(plan, A, lda);
}

minnorm_status minnorm_solve(minnorm_plan_t plan, const void *A, int64_t lda, const void *b, double eps, void *x,
                             minnorm_info *info) {
  if (!plan || !A || !b || !x) return MINNORM_EINVAL;
  if (plan->failed) return MINNORM_ESTATE;
  if (!plan->sketched) return MINNORM_ESTATE;
  if (lda < plan->n) return MINNORM_EINVAL;
  if (!(eps > 0.0 && eps < 1.0)) return MINNORM_EINVAL;
  plan->g_hp.ld = lda;
  plan->g_cg.ld = plan->d_A32 ? plan->n : lda;
  plan->async_pending = false;
  if (!info) return solve_async(plan, A, lda, b, eps, x);
  return solve_impl(plan, A, lda, b, eps, x, info);
}

minnorm_status minnorm_trailing_products(minnorm_plan_t plan, const void *V, int64_t ldv, void *C, int64_t ldc,
                                         int64_t rows, int64_t cols, const void *Z, int64_t ldz, void *W) {
  if (!plan || !V || !C) return MINNORM_EINVAL;
  if (plan->failed) return MINNORM_ESTATE;
  if (rows < 1 || cols < 1 || rows > plan->l || cols > plan->m || ldv < rows || ldc < rows || (Z && ldz < 32))
    return MINNORM_EINVAL;
  minnorm_status s = qrblk_alloc(plan);
  if (s != MINNORM_OK) return s;
  cudaStream_t st = plan->st;
  CK(cudaMemsetAsync(plan->d_err, 0, sizeof(int), st));
  CK(launch_trailing_products(plan->qb, V, ldv, C, ldc, rows, cols, Z, ldz, W, plan->d_err, plan->wait_limit_ns, st));
  int err = 0;
  CK(cudaMemcpyAsync(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (err) {
    plan->failed = true;
    return MINNORM_ETIMEOUT;
  }
  return MINNORM_OK;
}

minnorm_status minnorm_plan_set_wait_limit(minnorm_plan_t plan, uint64_t limit_ns, int32_t withhold) {
  if (!plan || limit_ns < 1000000ull || limit_ns > kBarrierLimitNs || withhold < 0 || withhold > 1)
    return MINNORM_EINVAL;
  plan->wait_limit_ns = limit_ns;
  plan->withhold = withhold;
  return MINNORM_OK;
}

minnorm_status minnorm_solve_wait(minnorm_plan_t plan, minnorm_info *info) {
  if (!plan) return MINNORM_EINVAL;
  if (!plan->async_pending) return MINNORM_ESTATE;
  plan->async_pending = false;
  cudaStream_t st = plan->st;
  int err = 0;
  CK(cudaMemcpyAsync(plan->h_ss, plan->d_ss, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(plan->h_norms + 2, plan->d_norms + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (err) {
    plan->failed = true;
    return MINNORM_ETIMEOUT;
  }
  const SolveState ss = *plan->h_ss;
  if (info) {
    fill_factor_info(plan, info);
    info->outer_steps = ss.outer;
    info->cg_iters = ss.cg_total;
    info->exact_passes = 2 * ss.outer;
    info->status = ss.status;
    info->err_bound = ss.err;
    const double bn = std::sqrt(plan->h_norms[3]);
    info->resid_rel = bn > 0 ? std::sqrt(plan->h_norms[2]) / bn : 0.0;
    if (plan->flags & MINNORM_FLAG_TIMING) {
      cudaEventElapsedTime(&info->ms_solve, plan->ev_as0, plan->ev_as1);
      double ms0[6];
      memcpy(ms0, plan->stat_ms, sizeof(ms0));
      collect_timers(plan);
      info->ms_cg = (float)(plan->stat_ms[0] + plan->stat_ms[1] + plan->stat_ms[5] - ms0[0] - ms0[1] - ms0[5]);
      info->ms_refine = (float)(plan->stat_ms[2] - ms0[2]);
    }
  } else if (plan->flags & MINNORM_FLAG_TIMING) {
    collect_timers(plan);
  }
  return (minnorm_status)ss.status;
}

minnorm_status minnorm_solve_many(minnorm_plan_t plan, const void *A, int64_t lda, const void *B, int64_t ldb,
                                  int64_t nrhs, double eps, void *X, int64_t ldx, minnorm_info *infos) {
  if (!plan || !A || !B || !X) return MINNORM_EINVAL;
  if (plan->failed || !plan->sketched) return MINNORM_ESTATE;
  if (lda < plan->n || ldb < plan->m || ldx < plan->n || nrhs < 1) return MINNORM_EINVAL;
  if (!(eps > 0.0 && eps < 1.0)) return MINNORM_EINVAL;
  plan->g_hp.ld = lda;
  plan->g_cg.ld = plan->d_A32 ? plan->n : lda;
  minnorm_status first = MINNORM_OK;
  if (plan->fp32 && nrhs > 1) {
    // mixed precision: block CG over chunks of up to kBlockRhs columns
    minnorm_status s = block_alloc(plan);
    if (s != MINNORM_OK) return s;
    for (int64_t j0 = 0; j0 < nrhs; j0 += kBlockRhs) {
      const int kc = (int)std::min<int64_t>(kBlockRhs, nrhs - j0);
      s = solve_block_chunk(plan, A, lda, static_cast<const zd *>(B) + j0 * ldb, ldb, kc, eps,
                            static_cast<zd *>(X) + j0 * ldx, ldx, infos ? infos + j0 : nullptr);
      if (s == MINNORM_EINVAL || s == MINNORM_ESTATE || s == MINNORM_ECUDA || s == MINNORM_ENOMEM ||
          s == MINNORM_ETIMEOUT)
        return s;
      if (s != MINNORM_OK && first == MINNORM_OK) first = s;
    }
    if (plan->flags & MINNORM_FLAG_TIMING) collect_timers(plan);
    return first;
  }
  for (int64_t j = 0; j < nrhs; ++j) {
    const minnorm_status s = solve_impl(plan, A, lda, static_cast<const zd *>(B) + j * ldb, eps,
                                        static_cast<zd *>(X) + j * ldx, infos ? infos + j : nullptr);
    // a failed plan (ETIMEOUT) or a missing allocation stops at once, as in the block path
    if (s == MINNORM_EINVAL || s == MINNORM_ESTATE || s == MINNORM_ECUDA || s == MINNORM_ENOMEM ||
        s == MINNORM_ETIMEOUT)
      return s;
    if (s != MINNORM_OK && first == MINNORM_OK) first = s;
  }
  return first;
}

minnorm_status minnorm_solve_host(minnorm_plan_t plan, const void *A_host, int64_t lda, const void *b_host,
                                  double eps, void *x_host, minnorm_info *info) {
  if (!plan || !A_host || !b_host || !x_host) return MINNORM_EINVAL;
  if (plan->failed) return MINNORM_ESTATE;
  if (lda < plan->n) return MINNORM_EINVAL;
  if (!(eps > 0.0 && eps < 1.0)) return MINNORM_EINVAL;
  const int64_t m = plan->m, n = plan->n;
  const size_t es = plan->dtype == MINNORM_C128 ? sizeof(zd) : sizeof(zf);
  if (!plan->d_Ah) {
    ALLOC(plan->d_Ah, es * (size_t)m * n);
    ALLOC(plan->d_bh, sizeof(zd) * m);
    ALLOC(plan->d_xo, sizeof(zd) * n);
  }
  cudaStream_t st = plan->st;
  minnorm_status s;
  if (!plan->bluestein) {  // copy in row blocks, each sketched as it arrives
    s = sketch_from_host(plan, A_host, lda);
    if (s != MINNORM_OK) return s;
    CK(cudaMemcpyAsync(plan->d_bh, b_host, sizeof(zd) * m, cudaMemcpyHostToDevice, st));
  } else {
    CK(cudaMemcpy2DAsync(plan->d_Ah, es * n, A_host, es * lda, es * n, m, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(plan->d_bh, b_host, sizeof(zd) * m, cudaMemcpyHostToDevice, st));
    s = minnorm_sketch(plan, plan->d_Ah, n);
    if (s != MINNORM_OK) return s;
  }
  minnorm_info local{};
  minnorm_status r = minnorm_solve(plan, plan->d_Ah, n, plan->d_bh, eps, plan->d_xo, info ? info : &local);
  if (r != MINNORM_OK && r != MINNORM_ENOCONV && r != MINNORM_EFLOOR) return r;
  CK(cudaMemcpyAsync(x_host, plan->d_xo, sizeof(zd) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return r;
}

minnorm_status minnorm_plan_destroy(minnorm_plan_t plan) {
  if (!plan) return MINNORM_OK;
  if (plan->st) cudaStreamSynchronize(plan->st);
  else cudaDeviceSynchronize();
  if (plan->st_copy) {
    cudaStreamSynchronize(plan->st_copy);
    cudaStreamDestroy(plan->st_copy);
    for (cudaEvent_t e : plan->ev_host) cudaEventDestroy(e);
  }
  if (plan->qb.side) {
    cudaStreamSynchronize(plan->qb.side);
    cudaStreamDestroy(plan->qb.side);
  }
  if (plan->qb.ev_panel) cudaEventDestroy(plan->qb.ev_panel);
  if (plan->qb.ev_t) cudaEventDestroy(plan->qb.ev_t);
  for (void *p : plan->allocs) cudaFree(p);
  for (cudaEvent_t e : plan->event_pool) cudaEventDestroy(e);
  if (plan->h_norms) cudaFreeHost(plan->h_norms);
  if (plan->h_cg) cudaFreeHost(plan->h_cg);
  if (plan->h_ss) cudaFreeHost(plan->h_ss);
  if (plan->ev_as0) cudaEventDestroy(plan->ev_as0);
  if (plan->ga_exec) cudaGraphExecDestroy(plan->ga_exec);
  if (plan->st_cap) cudaStreamDestroy(plan->st_cap);
  if (plan->st_cap2) cudaStreamDestroy(plan->st_cap2);
  if (plan->ev_as1) cudaEventDestroy(plan->ev_as1);
  if (plan->h_qr) cudaFreeHost(plan->h_qr);
  if (plan->h_bpart) cudaFreeHost(plan->h_bpart);
  if (plan->h_bint) cudaFreeHost(plan->h_bint);
  if (plan->h_bx) cudaFreeHost(plan->h_bx);
  delete plan;
  return MINNORM_OK;
}

minnorm_status minnorm_get_sketch(minnorm_plan_t plan, void *Y_out) {
  if (!plan || !Y_out) return MINNORM_EINVAL;
  if (!plan->d_Ykeep || !plan->sketched) return MINNORM_ESTATE;
  if (cudaMemcpyAsync(Y_out, plan->d_Ykeep, sizeof(zd) * plan->l * plan->m, cudaMemcpyDeviceToDevice, plan->st) !=
      cudaSuccess)
    return MINNORM_ECUDA;
  return MINNORM_OK;
}

namespace {
__global__ void piv_widen_kernel(const int32_t *a, int64_t *b, int m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) b[i] = a[i];
}
}  // namespace

minnorm_status minnorm_get_factor(minnorm_plan_t plan, void *R_out, void *piv_out) {
  if (!plan || !R_out || !piv_out) return MINNORM_EINVAL;
  if (!plan->sketched) return MINNORM_ESTATE;
  CK(cudaMemcpyAsync(R_out, plan->d_R, sizeof(zd) * plan->m * plan->m, cudaMemcpyDeviceToDevice, plan->st));
  note_launch();
  piv_widen_kernel<<<(int)((plan->m + 255) / 256), 256, 0, plan->st>>>(plan->d_piv, (int64_t *)piv_out, (int)plan->m);
  CK(cudaGetLastError());
  return MINNORM_OK;
}

// out = conj(in), n complex entries
__global__ void conj_copy_kernel(const zd *__restrict__ in, zd *__restrict__ out, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = conjg(in[e]);
}

minnorm_status minnorm_get_preconditioner(minnorm_plan_t plan, void *W_out) {
  if (!plan || !W_out) return MINNORM_EINVAL;
  if (!plan->sketched) return MINNORM_ESTATE;
  // column-major P R^{-1}: entry (i, k) at i + k m, the conjugate of WpH's row-major (k, i)
  note_launch();
  conj_copy_kernel<<<1024, 256, 0, plan->st>>>(plan->d_WpH, static_cast<zd *>(W_out), plan->m * plan->m);
  CK(cudaGetLastError());
  return MINNORM_OK;
}

minnorm_status minnorm_cg_products(minnorm_plan_t plan, const void *A, int64_t lda, const void *w, void *q,
                                   void *t) {
  if (!plan || !A || !w) return MINNORM_EINVAL;
  if (lda < plan->n) return MINNORM_EINVAL;
  if (!plan->sketched) return MINNORM_ESTATE;
  plan->g_hp.ld = lda;
  plan->g_cg.ld = plan->d_A32 ? plan->n : lda;
  cudaStream_t st = plan->st;
  const int64_t m = plan->m, n = plan->n;
  const void *Acg = plan->d_A32 ? (const void *)plan->d_A32 : A;
  if (!q && t && cg_pair_on(plan, Acg)) {   // t alone: the CG's one-pass form
    CK(launch_narrow(m, w, plan->d_w32, st));
    CK(cudaMemsetAsync(plan->d_err, 0, sizeof(int), st));
    CgPairArgs pa{Acg, plan->g_cg.ld, m, n, plan->d_w32, t, plan->d_tpart, plan->d_qqp, plan->pair_nc, plan->d_err,
                  plan->wait_limit_ns, nullptr};
    CK(launch_cg_pair(pa, st));
    int err = 0;
    CK(cudaMemcpyAsync(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err) {
      plan->failed = true;
      return MINNORM_ETIMEOUT;
    }
    return MINNORM_OK;
  }
  if (plan->fp32) {
    CK(launch_narrow(m, w, plan->d_w32, st));
    CK(launch_gemv_adj_f32(plan->g_cg, Acg, plan->d_w32, plan->d_q, plan->d_part, plan->d_qq, nullptr, st));
    if (q) CK(launch_widen(n, plan->d_q, q, st));
    if (t) CK(launch_gemv_fwd_f32(plan->g_cg, Acg, plan->d_q, t, plan->d_part, nullptr, st));
  } else {
    CK(launch_gemv_adj(plan->g_cg, Acg, w, plan->d_q, plan->d_part, plan->d_qq, nullptr, st));
    if (q) CK(cudaMemcpyAsync(q, plan->d_q, sizeof(zd) * n, cudaMemcpyDeviceToDevice, st));
    if (t) CK(launch_gemv_fwd(plan->g_cg, Acg, plan->d_q, t, plan->d_part, nullptr, st));
  }
  return MINNORM_OK;
}

minnorm_status minnorm_block_products(minnorm_plan_t plan, const void *A, int64_t lda, const void *W, void *Q,
                                      void *T) {
  if (!plan || !A || !W || !Q || !T) return MINNORM_EINVAL;
  if (lda < plan->n || !plan->fp32) return MINNORM_EINVAL;
  if (plan->dtype == MINNORM_C128 && !plan->sketched) return MINNORM_ESTATE;
  minnorm_status s = block_alloc(plan);
  if (s != MINNORM_OK) return s;
  cudaStream_t st = plan->st;
  const int64_t m = plan->m, n = plan->n;
  const void *Acg = plan->d_A32 ? (const void *)plan->d_A32 : A;
  const int64_t lda_cg = plan->d_A32 ? n : lda;
  double *gam = plan->d_bscal, *gam0 = gam + kBlockRhs, *alpha = gam0 + kBlockRhs;
  int *use = plan->d_bint, *active = use + kBlockRhs, *alldone = active + 2 * kBlockRhs;
  CK(cudaMemsetAsync(plan->d_bscal, 0, sizeof(double) * 4 * kBlockRhs, st));
  CK(cudaMemsetAsync(plan->d_bint, 0, sizeof(int) * (3 * kBlockRhs + 1), st));
  CK(cudaMemsetAsync(plan->d_err, 0, sizeof(int), st));
  CK(launch_narrow(m * kBlockRhs, W, plan->d_bW32, st));
  BlockProductArgs pa{};
  pa.A = Acg;
  pa.m = m;
  pa.n = n;
  pa.lda = lda_cg;
  pa.W32 = plan->d_bW32;
  pa.Q = plan->d_bQ;
  pa.qqp = plan->d_bqqp;
  pa.gam = gam;
  pa.active = active;
  pa.alpha = alpha;
  pa.tpart = plan->d_btpart;
  pa.nsplit = plan->blk_nsplit;
  pa.T = T;
  pa.alldone = alldone;
  pa.Bsplit = plan->d_bsplit;
  pa.Bsplit2 = plan->d_bsplit2;
  pa.nsplit_tc = plan->blk_nsplit_tc;
  pa.err = plan->d_err;
  pa.limit_ns = plan->wait_limit_ns;
  pa.sms = plan->sms;
  CK(launch_block_adj(pa, st));
  CK(launch_block_fwd(pa, st));
  CK(launch_widen(n * kBlockRhs, plan->d_bQ, Q, st));
  int err = 0;
  CK(cudaMemcpyAsync(&err, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return err ? MINNORM_ETIMEOUT : MINNORM_OK;
}

minnorm_status minnorm_residual_dd(minnorm_plan_t plan, const void *A, int64_t lda, const void *y_hi,
                                   const void *y_lo, const void *b, void *r, void *x_hi, void *x_lo) {
  if (!plan || !A || !y_hi || !b || !r || !x_hi || !x_lo) return MINNORM_EINVAL;
  if (lda < plan->n) return MINNORM_EINVAL;
  cudaStream_t st = plan->st;
  CK(launch_fix_prep(A, lda, plan->dtype == MINNORM_C64, plan->m, plan->n, plan->d_afix, plan->d_E, nullptr, st));
  XprodArgs a = xargs(plan, b);
  a.yh = y_hi;
  a.yl = y_lo;
  a.xh = x_hi;
  a.xl = x_lo;
  a.r = r;
  CK(launch_xresidual(a, st));
  return MINNORM_OK;
}

int64_t minnorm_launch_count(void) { return (int64_t)launches_so_far(); }

minnorm_status minnorm_plan_tuning(minnorm_plan_t plan, int32_t *x_chunks, int32_t *x_splits,
                                   int32_t *cg_l2_keep_pct) {
  if (!plan || !x_chunks || !x_splits || !cg_l2_keep_pct) return MINNORM_EINVAL;
  *x_chunks = plan->x_nchunk;
  *x_splits = plan->x_split > 0 ? plan->x_split : xadj_splits(plan->m, plan->n);
  *cg_l2_keep_pct = (int32_t)std::lround(100.0 * (plan->cg_keep >= 0.0 ? plan->cg_keep : 0.8));
  return plan->x_tuned ? MINNORM_OK : MINNORM_ESTATE;
}

minnorm_status minnorm_kernel_stats(minnorm_plan_t plan, int32_t k, int32_t *launches, double *ms) {
  if (!plan || k < 0 || k >= kNumClasses || !launches || !ms) return MINNORM_EINVAL;
  *launches = k == 5 ? plan->fused_iters : plan->stat_launches[k];
  *ms = plan->stat_ms[k];
  return MINNORM_OK;
}


// ---- batches ----------------------------------------------------------------
struct minnorm_batch_s {
  std::vector<minnorm_plan_t> plans;
  ScratchPool pool;
  std::vector<void *> allocs;
  cudaStream_t st = nullptr;                // the batch's stream
  std::vector<cudaStream_t> side;           // streams the systems' QRs are spread over
  std::vector<cudaEvent_t> ev;              // one per side stream, plus one for the batch stream
};

static constexpr int kBatchSideStreams = 8;

minnorm_status minnorm_batch_destroy(minnorm_batch_t batch) {
  if (!batch) return MINNORM_OK;
  for (minnorm_plan_t p : batch->plans) minnorm_plan_destroy(p);  // synchronizes the stream
  for (cudaStream_t s : batch->side) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (cudaEvent_t e : batch->ev) cudaEventDestroy(e);
  for (void *p : batch->allocs) cudaFree(p);
  delete batch;
  return MINNORM_OK;
}

minnorm_status minnorm_batch_create(minnorm_batch_t *out, int32_t count, const int64_t *m, const int64_t *n,
                                    minnorm_dtype dtype, minnorm_precision precision, uint64_t seed,
                                    uint32_t flags, void *stream) {
  if (!out) return MINNORM_EINVAL;
  *out = nullptr;
  if (count < 1 || !m || !n) return MINNORM_EINVAL;
  size_t sb = 0, ab = 0, a32 = 0;
  for (int32_t i = 0; i < count; ++i) {
    int64_t l = 0;
    const minnorm_status c = check_plan_args(m[i], n[i], l, dtype, precision, flags);
    if (c != MINNORM_OK) return c;
    size_t s1 = 0, s2 = 0, s3 = 0;
    scratch_sizes(m[i], n[i], precision, dtype, s1, s2, s3);
    sb = std::max(sb, s1);
    ab = std::max(ab, s2);
    a32 = std::max(a32, s3);
  }
  minnorm_batch_t b = new (std::nothrow) minnorm_batch_s();
  if (!b) return MINNORM_ENOMEM;
  auto grab = [&](void **p, size_t bytes) -> bool {
    if (bytes == 0) return true;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    b->allocs.push_back(*p);
    return true;
  };
  if (!grab(&b->pool.S1, sb) || !grab(&b->pool.S2, sb) || !grab(&b->pool.afix, ab) || !grab(&b->pool.A32, a32)) {
    minnorm_batch_destroy(b);
    return MINNORM_ENOMEM;
  }
  b->pool.s_bytes = sb;
  b->pool.afix_bytes = ab;
  b->pool.a32_bytes = a32;
  b->st = (cudaStream_t)stream;
  for (int i = 0; i < kBatchSideStreams + 1; ++i) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      minnorm_batch_destroy(b);
      return MINNORM_ECUDA;
    }
    b->ev.push_back(e);
    if (i == kBatchSideStreams) break;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      minnorm_batch_destroy(b);
      return MINNORM_ECUDA;
    }
    b->side.push_back(s);
  }
  b->plans.reserve(count);
  for (int32_t i = 0; i < count; ++i) {
    minnorm_plan_t p = nullptr;
    const minnorm_status s =
        plan_create_pooled(&p, m[i], n[i], 0, dtype, precision, seed + (uint64_t)i, flags, stream, &b->pool);
    if (s != MINNORM_OK) {
      minnorm_batch_destroy(b);
      return s;
    }
    b->plans.push_back(p);
  }
  *out = b;
  return MINNORM_OK;
}

minnorm_status minnorm_batch_solve(minnorm_batch_t batch, const void *const *A, const int64_t *lda,
                                   const void *const *b, double eps, void *const *x, minnorm_info *infos) {
  if (!batch || !A || !b || !x) return MINNORM_EINVAL;
  if (!(eps > 0.0 && eps < 1.0)) return MINNORM_EINVAL;
  const size_t N = batch->plans.size();
  for (size_t i = 0; i < N; ++i) {
    const minnorm_plan_t p = batch->plans[i];
    const int64_t ld = lda ? lda[i] : p->n;
    if (!A[i] || !b[i] || !x[i] || ld < p->n) return MINNORM_EINVAL;
    if (!aligned16(A[i]) && p->dtype == MINNORM_C128) return MINNORM_EINVAL;
    if (p->failed) return MINNORM_ESTATE;
  }
#define BCK(expr)                                                    \
  do {                                                               \
    if ((expr) != cudaSuccess) {                                     \
      for (minnorm_plan_t q_ : batch->plans) {                       \
        q_->st = batch->st;                                          \
        q_->failed = true;                                           \
      }                                                              \
      return MINNORM_ECUDA;                                          \
    }                                                                \
  } while (0)
  auto fatal = [](minnorm_status s) {
    return s == MINNORM_EINVAL || s == MINNORM_ECUDA || s == MINNORM_ETIMEOUT || s == MINNORM_ESTATE ||
           s == MINNORM_ENOMEM;
  };
  std::vector<minnorm_status> st(N, MINNORM_OK);
  // 1. Step 1 of every system, in turn on the batch stream (the shared pool holds a system's
  //    transform buffers only while its Step 1 runs; Y is the system's own)
  for (size_t i = 0; i < N; ++i) {
    minnorm_plan_t p = batch->plans[i];
    const int64_t ld = lda ? lda[i] : p->n;
    p->g_hp.ld = ld;
    p->g_cg.ld = p->d_A32 ? p->n : ld;
    const minnorm_status s = sketch_transform(p, A[i], ld);
    if (s != MINNORM_OK) return s;
  }
  // 2. Step 2 of every system, spread over the side streams: the QRs are latency-bound
  //    cooperative grids on per-system buffers, so those of different systems overlap
  BCK(cudaEventRecord(batch->ev.back(), batch->st));
  for (cudaStream_t s : batch->side) BCK(cudaStreamWaitEvent(s, batch->ev.back(), 0));
  for (size_t i = 0; i < N; ++i) {
    minnorm_plan_t p = batch->plans[i];
    p->st = batch->side[i % batch->side.size()];
    const minnorm_status s = sketch_factor(p);
    if (s != MINNORM_OK) {
      for (minnorm_plan_t q : batch->plans) q->st = batch->st;
      return s;
    }
  }
  for (size_t k = 0; k < batch->side.size(); ++k) {
    BCK(cudaEventRecord(batch->ev[k], batch->side[k]));
    BCK(cudaStreamWaitEvent(batch->st, batch->ev[k], 0));
  }
  for (minnorm_plan_t p : batch->plans) p->st = batch->st;
  for (size_t i = 0; i < N; ++i) {
    st[i] = sketch_finish(batch->plans[i]);
    if (fatal(st[i])) return st[i];
  }
  // 3. Steps 3-5 of every system, in turn; the pooled fixed-point (and complex64) copy of A is
  //    rebuilt first, since later systems' Step 1 overwrote it
  minnorm_status first = MINNORM_OK;
  for (size_t i = 0; i < N; ++i) {
    minnorm_plan_t p = batch->plans[i];
    const int64_t ld = lda ? lda[i] : p->n;
    minnorm_status s = st[i];
    if (s == MINNORM_OK) {
      BCK(launch_fix_prep(A[i], ld, p->dtype == MINNORM_C64, p->m, p->n, p->d_afix, p->d_E, p->d_A32, p->st));
      minnorm_info local{};
      s = minnorm_solve(p, A[i], ld, b[i], eps, x[i], infos ? infos + i : &local);
    } else if (infos) {
      memset(infos + i, 0, sizeof(minnorm_info));
      infos[i].status = s;
    }
    if (fatal(s)) return s;
    if (s != MINNORM_OK && first == MINNORM_OK) first = s;
  }
  return first;
}
#undef BCK

minnorm_status minnorm_batch_kernel_stats(minnorm_batch_t batch, int32_t system, int32_t k, int32_t *launches,
                                          double *ms) {
  if (!batch || !launches || !ms || k < 0 || k >= kNumClasses) return MINNORM_EINVAL;
  if (system < -1 || system >= (int32_t)batch->plans.size()) return MINNORM_EINVAL;
  int32_t nl = 0;
  double t = 0.0;
  for (int32_t i = 0; i < (int32_t)batch->plans.size(); ++i) {
    if (system >= 0 && i != system) continue;
    int32_t a = 0;
    double b = 0.0;
    minnorm_kernel_stats(batch->plans[i], k, &a, &b);
    nl += a;
    t += b;
  }
  *launches = nl;
  *ms = t;
  return MINNORM_OK;
}

}  // extern "C"
