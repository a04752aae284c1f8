// vec.h -- launchers of the length-m vector kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mn {

struct CgScalars {
  double gamma;    // ||s||^2 of the current iterate
  double gamma0;   // ||s_0||^2
  int done;        // stopping test fired (or a zero curvature)
  int iters;       // iterations performed
};

// State of an asynchronous solve (minnorm_solve with info == NULL): the refinement's stopping
// test runs on the device, and every later step of the enqueued loop returns at once once
// `done` is set.
struct SolveState {
  int done;        // the loop has stopped (all later steps skip)
  int status;      // minnorm_status of the solve
  int outer;       // refinement steps taken
  int stagnant;    // consecutive steps that reduced the bound by less than half
  int cg_total;    // CG iterations summed over the inner solves
  int pad;
  double err;      // the certified bound of the last test
  double prev;     // the bound of the step before
};
// constants of the certificate (see solver.cu)
struct CertConsts {
  double delta;    // sigma_min(A^* P R^{-1}) >= 1 - delta
  double factor;   // 1 + the rounding of P R^{-1} and of g
  double eps;      // the requested accuracy
};

cudaError_t launch_cg_init(int m, const void *g, void *u, void *s, void *p, CgScalars *sc, cudaStream_t st,
                           const int *skip = nullptr);
cudaError_t launch_solve_state_init(SolveState *ss, cudaStream_t st);
// *dst = c (by a kernel: no host buffer has to outlive the call)
cudaError_t launch_set_cert(CertConsts *dst, CertConsts c, cudaStream_t st);
// the condition of a CUDA graph's WHILE node around a chunk of CG iterations: keep looping
// while the CG has neither met its test nor run maxit iterations
cudaError_t launch_cg_continue(cudaGraphConditionalHandle h, const CgScalars *sc, int maxit, cudaStream_t st);
// the refinement's stopping test on the device: norms[0] = ||g||^2, norms[1] = ||x||^2; step
// `outer` (0: before any inner solve); final: the loop's last test (ENOCONV unless within eps);
// sc: the CG scalars of the inner solve just finished (or NULL); c: device copy of the constants
cudaError_t launch_solve_stop(SolveState *ss, const double *norms, int outer, bool final, const CertConsts *c,
                              const CgScalars *sc, cudaStream_t st);
cudaError_t launch_cg_update(int m, const double *qq, int nqq, const void *np, void *u, void *s, void *p,
                             CgScalars *sc, double tol2, cudaStream_t st);
cudaError_t launch_dd_accumulate(int64_t len, void *yh, void *yl, const void *d, cudaStream_t st,
                                 const int *skip = nullptr);
cudaError_t launch_resid_finish(int64_t len, const void *b, const void *vh, const void *vl, void *r,
                                cudaStream_t st);
cudaError_t launch_sub(int64_t len, void *r, const void *t, cudaStream_t st);
cudaError_t launch_sumsq(int64_t len, const void *v, double *part, double *out, cudaStream_t st);
int sumsq_partials(int64_t len);
// *out = sum of the len doubles of v (one block)
cudaError_t launch_sum(int len, const double *v, double *out, cudaStream_t st);

}  // namespace mn
