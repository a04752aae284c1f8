// kernels.h -- host-side launchers of the sm_103a kernels (internal to the
// library; the public interface is include/minnorm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mn {

struct GridBarrier;

// Longest a bounded device-side wait (a grid barrier, a pivot exchange, an
// mbarrier phase) may spin before the kernel records MINNORM_ETIMEOUT and
// returns: 2 s. Every entry point passes this same limit.
constexpr uint64_t kBarrierLimitNs = 2000000000ULL;

// count of kernels launched by this library (every launch site calls it)
void note_launch();
long long launches_so_far();

// ---- sketch.cu ------------------------------------------------------------
// arithmetic of the sketch: complex FP64, or complex double-word (pairs of
// floats on the FP32 pipe, dw.cuh); element kinds of a chain's source rows
constexpr int kArithF64 = 0, kArithDW = 2;
constexpr int kSrcC128 = 0, kSrcC64 = 1, kSrcDW = 2;

struct ChainArgs {
  const void *src;       // rows x n, of kind src_kind (complex128, complex64 or complex double-word)
  int64_t ld_src;
  void *dst;             // rows x n complex of the compute precision
  int64_t ld_dst;
  const int32_t *idx;    // gather permutation (n)
  const void *phase;     // n unit phases (compute precision), applied after the gather
  const void *cs;        // n (cos, sin) pairs, entry n-1 = (1, 0)
  const void *post;      // n phases applied to the output, or nullptr
  const int32_t *halo;   // per-segment right halo
  int n, seg, cap, rows;
  int src_kind;          // kSrcC128, kSrcC64 or kSrcDW
  bool conj;
  int arith;             // kArithF64 or kArithDW (dst, phase, cs and post in that arithmetic)
};
cudaError_t launch_chain(const ChainArgs &a, cudaStream_t st);

struct FftArgs {
  const void *src;        // rows of the input (compute precision), row stride ld
  int64_t ld;
  void *work;             // rows x L scratch for the four-step path, row stride ldw
  int64_t ldw;
  const void *tw;         // L twiddles e^{-2 pi i k/L}
  int logn, logN1;        // L = 2^logn; logN1 = 0: single-pass row FFT
  int tj, tk;             // tile widths of pass A / B
  const int32_t *samp_off, *samp_t, *samp_loc;
  int l, rows;
  void *Y;                // l x m complex128, column-major
  int64_t ldy;
  int row_offset;
  int arith;              // kArithF64 or kArithDW (src, work, tw, chirp, full, bh in that arithmetic)
  // Bluestein stages (n not a power of two; see params.h):
  const void *chirp;      // if set: the input is x_j chirp_j for j < nin and 0 for nin <= j < L
  int nin;
  void *full;             // if set: store conj(X_k bh_k) for all k < L (row stride ldf), no sampling
  const void *bh;
  int64_t ldf;
  const double *fac;      // if set: sampled outputs are conj(X) * fac[t] (complex128) instead of X / sqrt(L)
};
cudaError_t launch_fft(const FftArgs &a, cudaStream_t st);
cudaError_t launch_to_c64(const void *A, int64_t lda, void *B, int64_t ldb, int64_t rows, int64_t cols,
                          cudaStream_t st);
// vectors: complex128 -> complex64 and back
cudaError_t launch_narrow(int64_t len, const void *src, void *dst, cudaStream_t st);
cudaError_t launch_widen(int64_t len, const void *src, void *dst, cudaStream_t st);

// ---- qr.cu ----------------------------------------------------------------
struct QrArgs {
  void *Y;                // l x m complex128 column-major, overwritten
  int l, m;
  double *vn1, *vn2;      // m
  double *beta;           // m: real diagonal of R
  int32_t *piv;           // m
  void *R;                // m x m complex128 column-major (out)
  void *mail;             // qr_mail_bytes() of exchange words (cleared by launch_qrp)
  int *err;
  uint64_t limit_ns;
};
cudaError_t launch_qrp(const QrArgs &a, cudaStream_t st);
size_t qr_mail_bytes();

// Wp = P R^{-1} (row-major m x m) and WpH = Wp^* (row-major)
cudaError_t launch_prinv(const void *R, const int32_t *piv, int m, void *Wp, void *WpH, cudaStream_t st);

// ---- gemv.cu --------------------------------------------------------------
// Element/compute types: 0 = complex128 matrix / FP64 compute, 1 = complex64
// matrix / FP32 compute, 2 = complex64 matrix / FP64 compute.
struct GemvPlan {
  int64_t rows, cols, ld;
  int mode;               // as above
  int adj_split;          // row splits of the adjoint product
  int fwd_rows;           // rows per CTA of the forward product
  int fwd_chunk;          // columns per CTA of the forward product
  int fwd_nchunk;
};
void gemv_configure(GemvPlan &g, int64_t rows, int64_t cols, int64_t ld, int mode, int num_sms);
size_t gemv_adj_partial_elems(const GemvPlan &g);   // complex elements of partial storage (compute type)
size_t gemv_fwd_partial_elems(const GemvPlan &g);

// out = A^* v: v (rows, complex128), out (cols, complex128); partials scratch
cudaError_t launch_gemv_adj(const GemvPlan &g, const void *A, const void *v, void *out, void *partial,
                            double *qq_partial, const int *skip, cudaStream_t st);
// out = A v: v (cols, complex128 or complex64 when compute is FP32), out (rows, complex128)
cudaError_t launch_gemv_fwd(const GemvPlan &g, const void *A, const void *v, void *out, void *partial,
                            const int *skip, cudaStream_t st);
// mixed-precision entry points working on FP32 vectors
cudaError_t launch_gemv_adj_f32(const GemvPlan &g, const void *A, const void *v32, void *out32,
                                void *partial, double *qq, const int *skip, cudaStream_t st);
cudaError_t launch_gemv_fwd_f32(const GemvPlan &g, const void *A, const void *v32, void *out64,
                                void *partial, const int *skip, cudaStream_t st);


// ---- xprod.cu --------------------------------------------------------------
// exact fixed-point products of the refinement (see xprod.cu)
struct XprodArgs {
  const void *afix;       // rows x cols fixed-point A (2 int64 per element)
  const int32_t *E;       // rows: per-row exponents
  int64_t rows, cols;
  const void *yh, *yl;    // rows complex128: y = yh + yl (yl may be nullptr)
  void *yfix;             // rows x 32 bytes scratch
  int *Fy, *Fx;           // device scalars
  void *xh, *xl;          // cols complex128 out: x = A^* y as double-double
  const void *b;          // rows complex128, or nullptr to stop after x
  void *r;                // rows complex128 out: b - A x (may be nullptr)
  void *th, *tl;          // rows complex128 out: A x as double-double (may be nullptr)
  void *partial;          // xprod_partial_bytes(rows, nchunk)
  int nchunk;
  int64_t chunk;
  void *xpart;            // xadj_partial_bytes(rows, cols): row-split partial sums of A^* y
  void *xfix;             // xfix_bytes(cols): x in 128-bit fixed point for the forward product
  int xsplit;             // row splits of x = A^* y (0: xadj_splits); at most xadj_max_splits(rows)
  const int *skip;        // if set and nonzero on the device, every kernel returns at once
};
// The fixed-point copy of A (and its complex64 copy when A32 is set); with rown2 set, also an
// upper bound of ||A[i, :]||^2 per row (rigorous: the rounding of the float sums is added).
cudaError_t launch_fix_prep(const void *A, int64_t lda, bool c64, int64_t rows, int64_t cols, void *afix,
                            int32_t *E, void *A32, cudaStream_t st, double *rown2 = nullptr);
cudaError_t launch_xresidual(const XprodArgs &a, cudaStream_t st);
size_t xprod_partial_bytes(int64_t rows, int nchunk);
int xadj_splits(int64_t rows, int64_t cols);
int xadj_max_splits(int64_t rows);
size_t xadj_partial_bytes(int64_t rows, int64_t cols);
size_t xfix_bytes(int64_t cols);

// ---- cgfused.cu ---------------------------------------------------------------
struct CgScalars;
struct CgFusedArgs {
  const void *A;           // complex64, row-major, lda even, 16-byte aligned
  int64_t m, n, lda;
  const void *Wp, *WpH, *g;
  void *u, *s, *w, *t, *dy;
  void *tpart;             // grid x m complex64
  double *qq_part, *gg_part;  // grid each
  CgScalars *sc;
  double tol2;
  int maxit;
  GridBarrier *bar;
  int *err;
  uint64_t limit_ns;
  int grid;                // CTAs (one per SM)
  double keep_frac;        // share of L2 the tail of each sweep is loaded into with an evict-last hint
                           // (negative: the default); a cache hint only, results do not depend on it
  const int *skip;         // if set and nonzero on the device, the kernel returns at once
  int withhold;            // 1: CTA 0 returns at once without arriving at the grid barrier (tests of
                           // the bounded wait: the others time out and report it)
};
bool cg_fused_supported(int64_t m, int64_t n, int64_t lda, const void *A);
cudaError_t launch_cg_fused(const CgFusedArgs &a, cudaStream_t st);
// One pass over A per mixed-precision CG iteration for 512 < m <= 4096: t = A (A^* w) (m complex128)
// and the partial sums of ||A^* w||^2 (one per cluster), by clusters of ceil(m / 512) CTAs
struct CgPairArgs {
  const void *A;          // complex64, row-major m x n, leading dimension lda (even, 16-byte aligned)
  int64_t lda, m, n;
  const void *w32;        // m complex64
  void *t;                // m complex128
  void *tpart;            // nc x m complex64
  double *qq_part;        // nc
  int nc;                 // clusters (cg_pair_clusters)
  int *err;
  uint64_t limit_ns;
  const int *skip;        // returns at once when *skip != 0
};
bool cg_pair_supported(int64_t m, int64_t n, int64_t lda, const void *A);
int cg_pair_clusters(int64_t m, int64_t n);
cudaError_t launch_cg_pair(const CgPairArgs &a, cudaStream_t st);

// ---- ozaki.cu ----------------------------------------------------------------------
// FP64-accurate complex products on the tensor cores (the trailing updates of the blocked
// Householder QR, qrblk.cu). Every FP64 operand entry is truncated to 8 S - 1 bits below its
// row's scale (one exponent per operand row) and split exactly into S BF16 slices of balanced
// base-256 digits; the pair products of every kept slice level are accumulated EXACTLY in FP32
// in tensor memory (one accumulator per level: their integer sums over kOzDrain K-blocks fit in
// 24 bits) and moved into int64 sums every kOzDrain K-blocks. The adjoint product (K = the
// trailing block's rows, up to l) keeps 63 bits and the levels s + t <= 8 (43 slice pairs): its
// error is within a few units of 2^-53 ||v|| ||c|| at any K. The update (K = 32 reflectors)
// keeps 55 bits and the levels s + t <= 7 (34 pairs) on wider tiles.
constexpr int kOzSlicesAdj = 8, kOzLevelsAdj = 9, kOzNAdj = 32;
constexpr int kOzSlicesFwd = 7, kOzLevelsFwd = 8, kOzNFwd = 64;
constexpr int kOzM = 128;         // output rows per tile
constexpr int kOzK = 64;          // K per block (one 128-byte row of BF16)
constexpr int kOzDrain = 2;       // K-blocks per exact accumulation: 8 x 128 x 2^14 <= 2^24
constexpr int kOzKbMax = 480;     // K-blocks per CTA: the int64 level sums stay below 2^53
// Operand slices: [ns][rows_pad][k_pad] BF16, K contiguous (rows_pad a multiple of 128 (64 for
// the update's B), k_pad of 64, zero padded), with one int32 exponent per row.
struct OzOperand {
  void *slices;
  int32_t *expo;
  int64_t rows, rows_pad, k, k_pad;
  int ns;                 // slices
};
size_t oz_slice_bytes(int64_t rows, int64_t k, int ns);
// A rows from C's columns: row c = (Re C[r, c], Im C[r, c]) for r = 0..rows-1 interleaved along K
cudaError_t launch_oz_slice_cols(const void *C, int64_t ldc, int64_t rows, int64_t cols, OzOperand &out,
                                 cudaStream_t st);
// B rows from the 32 reflectors V (rows x 32, column-major, ldv): row j < 32 = (Re V[:, j], Im V[:, j])
// interleaved; row 32 + j = (Im V[:, j], -Re V[:, j])
cudaError_t launch_oz_slice_v_adj(const void *V, int64_t ldv, int64_t rows, OzOperand &out, cudaStream_t st);
// A rows for C -= V Z: row 2i = (Re V[i, j], -Im V[i, j]), row 2i + 1 = (Im V[i, j], Re V[i, j]) along j
cudaError_t launch_oz_slice_v_fwd(const void *V, int64_t ldv, int64_t rows, OzOperand &out, cudaStream_t st);
// B rows for C -= V Z: row c = (Re Z[j, c], Im Z[j, c]) along j (Z: 32 x cols complex, column-major, ldz)
cudaError_t launch_oz_slice_z(const void *Z, int64_t ldz, int64_t cols, OzOperand &out, cudaStream_t st);
// W^H = C^H V (the adjoint product): D[c][j] (cols x 64 real: Re then Im of (C^H V)[c, j]) into
// FP64 partial sums over K splits, then W[j, c] = conj(...) (32 x cols complex, column-major, ldw)
struct OzAdjArgs {
  OzOperand a, b;
  double *part;           // splits x cols_pad x 64
  size_t part_bytes;      // its capacity (oz_adj_partial_bytes)
  void *W;
  int64_t ldw, cols;
  int *err;
  uint64_t limit_ns;
};
cudaError_t launch_oz_adj(const OzAdjArgs &a, cudaStream_t st);
size_t oz_adj_partial_bytes(int64_t l, int64_t m, int sms);
// C[i, c] -= (V Z)[i, c] for i < rows, c < cols (C complex column-major, ldc)
struct OzFwdArgs {
  OzOperand a, b;
  void *C;
  int64_t ldc, rows, cols;
  int *err;
  uint64_t limit_ns;
};
cudaError_t launch_oz_fwd(const OzFwdArgs &a, cudaStream_t st);

// ---- qrblk.cu ----------------------------------------------------------------------
// Workspace of the blocked Householder QR (sizes for l x m sketches): the operand slices and
// exponents of both trailing products, their FP64 partial sums, W = V^H C and Z = T^H W.
struct QrBlkWork {
  int64_t l = 0, m = 0;
  void *sA = nullptr, *sB = nullptr, *sV = nullptr, *sZ = nullptr;
  int32_t *eA = nullptr, *eB = nullptr, *eV = nullptr, *eZ = nullptr;
  double *part = nullptr;
  size_t part_bytes = 0;
  void *W = nullptr, *Z = nullptr, *T = nullptr;   // 32 x m, 32 x m, 32 x 32 complex, column-major
  void *tau = nullptr;                             // m complex: the reflectors' tau
  void *Vb = nullptr;                              // l x 32 complex: a panel's reflectors (unit diagonal)
  void *R1 = nullptr;                              // m x m complex: the triangle of the unpivoted QR
  void *ppart = nullptr;                           // 2 x sms x 32 complex: a panel's posted slots
  void *rowb = nullptr;                            // 2 x 32 complex: a panel's posted rows
  GridBarrier *bar = nullptr;
  cudaStream_t side = nullptr;                     // a panel's T, beside its adjoint product
  cudaEvent_t ev_panel = nullptr, ev_t = nullptr;
};
// bytes of each buffer: sA, sB, sV, sZ, eA, eB, eV, eZ, part, W, Z, T, tau, Vb, R1, ppart, rowb, bar
void qrblk_sizes(int64_t l, int64_t m, int sms, size_t (&bytes)[18]);
// Y P = Q R (Step 2) for l x m sketches, l >= m: blocked unpivoted QR, then the pivoted QR of
// its m x m triangle (launch_qrp with the arguments of q); the pivots and R are those of the
// pivoted QR of Y (R up to a unit diagonal)
cudaError_t launch_qr_blocked(QrBlkWork &w, const QrArgs &q, int sms, cudaStream_t st);
// its two parts: the blocked QR of Y without pivoting (R1 into the workspace), and the pivoted
// QR of the m x m triangle R1
cudaError_t launch_qr_tall(QrBlkWork &w, const QrArgs &q, int sms, cudaStream_t st);
cudaError_t launch_qr_triangle(QrBlkWork &w, const QrArgs &q, cudaStream_t st);
// P R^{-1} (Wp = P R^{-1} and WpH = Wp^*, row-major, the layout of launch_prinv) by blocks of 32
// rows with the K = 32 updates on the tensor cores; R: m x m complex column-major, upper
// triangular with a real diagonal; uses the workspace's triangle buffer (free after
// launch_qr_triangle) and its update slices. For kPinvBlockedMinM <= m <= the workspace's m.
constexpr int kPinvBlockedMinM = 256;
cudaError_t launch_prinv_blocked(QrBlkWork &w, const void *R, const int32_t *piv, int m, void *Wp, void *WpH,
                                 int *err, uint64_t limit_ns, cudaStream_t st);
// rows of a panel one CTA may hold in shared memory; the blocked QR needs l <= kPanelMaxRows * sms
constexpr int kPanelMaxRows = 384;
int qrblk_panel_grid(int64_t L, int sms);
// W = V^H C (when W is set; 32 x cols, ldw 32) and then C -= V Z (when Z is set; Z 32 x cols,
// column-major, ldz): V rows x 32 (ldv), C rows x cols (ldc), all complex FP64 column-major;
// rows <= l, cols <= m of the workspace
cudaError_t launch_trailing_products(QrBlkWork &w, const void *V, int64_t ldv, void *C, int64_t ldc, int64_t rows,
                                     int64_t cols, const void *Z, int64_t ldz, void *W, int *err, uint64_t limit_ns,
                                     cudaStream_t st);

// ---- blockcg.cu -------------------------------------------------------------------
// block CG over kBlockRhs right-hand sides (block vectors row-major m x kBlockRhs)
constexpr int kBlockRhs = 32;
struct BlockProductArgs {
  const void *A;           // complex64, row-major m x n, leading dimension lda
  int64_t m, n, lda;
  const void *W32;         // m x KB complex64: Wp P
  void *Q;                 // n x KB complex64: A^* W
  float *qqp;              // block_adj_parts(n) x KB partial |Q|^2
  const double *gam;       // KB
  const int *active;       // KB
  double *alpha;           // KB (out)
  void *tpart;             // nsplit x m x KB complex64
  int nsplit;
  void *T;                 // m x KB complex128: A Q
  const int *alldone;
  void *Bsplit;            // tc_split_bytes(m): BF16 pieces of W for the tensor-core product (or NULL)
  void *Bsplit2;           // tc_split2_bytes(n): BF16 pieces of Q for the tensor-core product (or NULL)
  int nsplit_tc;           // K ranges of the tensor-core T = A Q (tpart holds that many partials)
  int *err;                // set to 1 when a bounded wait of the tensor-core kernel expired
  uint64_t limit_ns;
  int sms;
};
int block_adj_parts(int64_t n);
int block_fwd_splits(int64_t m, int64_t n, int sms);
int block_col_parts(int64_t m);
cudaError_t launch_block_mm(const void *M, int m, const void *V, void *out, void *out32, const int *alldone,
                            cudaStream_t st);
cudaError_t launch_block_adj(const BlockProductArgs &a, cudaStream_t st);   // Q = A^* W, qq, alpha
// tcblock.cu: Q = A^* W and T = A Q on the tensor cores (split BF16, FP32 accumulation)
size_t tc_split_bytes(int64_t m);
size_t tc_split2_bytes(int64_t n);
int tc_fwd_splits(int64_t m, int64_t n, int sms);
bool tc_block_supported(int64_t m, int64_t n, int64_t lda, const void *A);
cudaError_t launch_tc_block_fwd(const void *A, int64_t m, int64_t n, int64_t lda, const void *Q32, void *Bsplit2,
                                void *tpart, int nsplit, const int *alldone, int *err, uint64_t limit_ns,
                                cudaStream_t st);
cudaError_t launch_tc_block_adj(const void *A, int64_t m, int64_t n, int64_t lda, const void *W32, void *Bsplit,
                                void *Q, float *qqp, const int *alldone, int *err, uint64_t limit_ns, int sms,
                                cudaStream_t st);
cudaError_t launch_block_fwd(const BlockProductArgs &a, cudaStream_t st);   // T = A Q
cudaError_t launch_block_get_col(int m, const void *Bk, int c, void *v, cudaStream_t st);
cudaError_t launch_block_set_col(int m, const void *v, int c, void *Bk, cudaStream_t st);
cudaError_t launch_block_load_rhs(int m, int kc, const void *B, int64_t ldb, void *R, cudaStream_t st);
cudaError_t launch_block_dd_acc(int m, const int *use, void *Yh, void *Yl, const void *dY, cudaStream_t st);
cudaError_t launch_block_colnorms(int m, const void *X, double *part, cudaStream_t st);
cudaError_t launch_block_cg_init(int m, const void *G, void *U, void *S, void *P, double *part, const int *use,
                                 double *gam, double *gam0, int *active, int *alldone, cudaStream_t st);
cudaError_t launch_block_cg_update(int m, const double *alpha, void *P, const void *Np, void *U, void *S,
                                   double *part, double tol2, double *gam, const double *gam0, int *active,
                                   double *beta, int *iters, int *alldone, cudaStream_t st);

// small dense m x m FP64 products: out = M v (M row-major), optionally also an FP32 copy
cudaError_t launch_small_gemv(const void *M, int m, const void *v, void *out, void *out32, const int *skip,
                              cudaStream_t st);

}  // namespace mn
