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

cudaError_t launch_cg_init(int m, const void *g, void *u, void *s, void *p, CgScalars *sc, cudaStream_t st);
cudaError_t launch_cg_update(int m, const double *qq, int nqq, const void *np, void *u, void *s, void *p,
                             CgScalars *sc, double tol2, cudaStream_t st);
cudaError_t launch_dd_accumulate(int64_t len, void *yh, void *yl, const void *d, cudaStream_t st);
cudaError_t launch_resid_finish(int64_t len, const void *b, const void *vh, const void *vl, void *r,
                                cudaStream_t st);
cudaError_t launch_sub(int64_t len, void *r, const void *t, cudaStream_t st);
cudaError_t launch_sumsq(int64_t len, const void *v, double *part, double *out, cudaStream_t st);
int sumsq_partials(int64_t len);
// *out = sum of the len doubles of v (one block)
cudaError_t launch_sum(int len, const double *v, double *out, cudaStream_t st);

}  // namespace mn
