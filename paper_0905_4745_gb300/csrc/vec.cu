// vec.cu -- kernels on vectors of length m (the CG state of Step 4 and the
// refinement's y) and norms of length-n vectors. Every kernel that runs inside
// the CG loop takes `done`: once the loop's stopping test has fired, the
// remaining (already enqueued) iterations return immediately.
#include "common.cuh"
#include "kernels.h"
#include "vec.h"

namespace mn {

// CG scalars live in one small device array (see CgScalars in vec.h).

__global__ void __launch_bounds__(1024)
cg_init_kernel(int m, const zd *__restrict__ g, zd *__restrict__ u, zd *__restrict__ s, zd *__restrict__ p,
               CgScalars *sc, const int *__restrict__ skip) {
  __shared__ double red[32];
  if (skip && *skip) {  // the solve has stopped: the inner loop's kernels return at once
    if (threadIdx.x == 0) { sc->done = 1; sc->iters = 0; }
    return;
  }
  double loc = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const zd v = g[i];
    s[i] = v;
    p[i] = v;
    u[i] = {0.0, 0.0};
    loc = fma(v.re, v.re, fma(v.im, v.im, loc));
  }
  const double gam = block_sum(loc, red);
  if (threadIdx.x == 0) {
    sc->gamma = gam;
    sc->gamma0 = gam;
    sc->done = (gam == 0.0) ? 1 : 0;
    sc->iters = 0;
  }
}

// alpha = gamma / ||q||^2; u += alpha p; s -= alpha Np; gamma' = ||s||^2;
// p = s + (gamma'/gamma) p; stop when gamma' <= tol2 * gamma0.
__global__ void __launch_bounds__(1024)
cg_update_kernel(int m, const double *__restrict__ qq_part, int nqq, const zd *__restrict__ np,
                 zd *__restrict__ u, zd *__restrict__ s, zd *__restrict__ p, CgScalars *sc, double tol2) {
  __shared__ double red[32];
  if (sc->done) return;
  double q = 0.0;
  for (int i = threadIdx.x; i < nqq; i += blockDim.x) q += qq_part[i];
  const double qq = block_sum(q, red);
  const double gam = sc->gamma;
  const double alpha = qq > 0.0 ? gam / qq : 0.0;
  double loc = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const zd pi = p[i], ni = np[i];
    zd ui = u[i], si = s[i];
    ui.re = fma(alpha, pi.re, ui.re);
    ui.im = fma(alpha, pi.im, ui.im);
    si.re = fma(-alpha, ni.re, si.re);
    si.im = fma(-alpha, ni.im, si.im);
    u[i] = ui;
    s[i] = si;
    loc = fma(si.re, si.re, fma(si.im, si.im, loc));
  }
  const double gnew = block_sum(loc, red);
  const double beta = gam > 0.0 ? gnew / gam : 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const zd si = s[i];
    zd pi = p[i];
    pi.re = fma(beta, pi.re, si.re);
    pi.im = fma(beta, pi.im, si.im);
    p[i] = pi;
  }
  if (threadIdx.x == 0) {
    sc->gamma = gnew;
    sc->iters += 1;
    if (gnew <= tol2 * sc->gamma0 || !(qq > 0.0)) sc->done = 1;
  }
}

// (yh, yl) += d   componentwise, double-double
__global__ void dd_accumulate_kernel(int64_t len, zd *__restrict__ yh, zd *__restrict__ yl,
                                     const zd *__restrict__ d, const int *__restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const zd h = yh[i], l = yl[i], v = d[i];
    double s1, e1, s2, e2;
    two_sum(h.re, v.re, s1, e1);
    two_sum(h.im, v.im, s2, e2);
    double h1, l1, h2, l2;
    two_sum(s1, __dadd_rn(e1, l.re), h1, l1);
    two_sum(s2, __dadd_rn(e2, l.im), h2, l2);
    yh[i] = {h1, h2};
    yl[i] = {l1, l2};
  }
}

// r = b - (vh + vl), rounded to FP64
__global__ void resid_finish_kernel(int64_t len, const zd *__restrict__ b, const zd *__restrict__ vh,
                                    const zd *__restrict__ vl, zd *__restrict__ r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const zd bi = b[i], h = vh[i], l = vl[i];
    double s1, e1, s2, e2;
    two_sum(bi.re, -h.re, s1, e1);
    two_sum(bi.im, -h.im, s2, e2);
    r[i] = {__dadd_rn(s1, __dsub_rn(e1, l.re)), __dadd_rn(s2, __dsub_rn(e2, l.im))};
  }
}

// r -= t
__global__ void sub_kernel(int64_t len, zd *__restrict__ r, const zd *__restrict__ t) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    zd v = r[i];
    const zd w = t[i];
    v.re -= w.re;
    v.im -= w.im;
    r[i] = v;
  }
}

// partial sums of |v|^2 over blocks; out[block]
__global__ void __launch_bounds__(256)
sumsq_kernel(int64_t len, const zd *__restrict__ v, double *__restrict__ out) {
  __shared__ double red[8];
  double loc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const zd a = v[i];
    loc = fma(a.re, a.re, fma(a.im, a.im, loc));
  }
  const double t = block_sum(loc, red);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

__global__ void __launch_bounds__(256)
finish_sum_kernel(const double *__restrict__ part, int n, double *__restrict__ out) {
  __shared__ double red[8];
  double loc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) loc += part[i];
  const double t = block_sum(loc, red);
  if (threadIdx.x == 0) *out = t;
}

static int blocks_for(int64_t len) {
  int64_t b = (len + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

cudaError_t launch_cg_init(int m, const void *g, void *u, void *s, void *p, CgScalars *sc, cudaStream_t st,
                           const int *skip) {
  note_launch();
  cg_init_kernel<<<1, 1024, 0, st>>>(m, (const zd *)g, (zd *)u, (zd *)s, (zd *)p, sc, skip);
  return cudaGetLastError();
}

__global__ void solve_state_init_kernel(SolveState *ss) {
  ss->done = 0;
  ss->status = 6;  // MINNORM_ENOCONV until a test passes
  ss->outer = 0;
  ss->stagnant = 0;
  ss->cg_total = 0;
  ss->err = __longlong_as_double(0x7ff0000000000000LL);   // +inf
  ss->prev = ss->err;
}

// The same stopping rule as the host loop of a synchronous solve: stop with OK once the
// certified bound ||g|| factor / ((1 - delta) ||x||) + 2^-52 is within eps, with EFLOOR after two
// steps in a row that did not halve it, with ENOCONV after the last step.
__global__ void solve_stop_kernel(SolveState *ss, const double *norms, int outer, int final, const CertConsts *cp,
                                  const CgScalars *sc) {
  const CertConsts c = *cp;
  if (ss->done) return;
  if (sc && outer > 0) ss->cg_total += sc->iters;
  const double gn = sqrt(norms[0]);
  if (outer == 0 && !final) {
    if (gn == 0.0) { ss->done = 1; ss->status = 0; ss->err = 0.0; }
    return;
  }
  const double xn = sqrt(norms[1]);
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  const double err = (xn > 0.0 && c.delta < 0.5) ? gn * c.factor / ((1.0 - c.delta) * xn) + 0x1.0p-52 : inf;
  ss->err = err;
  ss->outer = outer;
  if (err <= c.eps) { ss->done = 1; ss->status = 0; return; }
  if (final) { ss->done = 1; ss->status = 6; return; }   // ENOCONV
  ss->stagnant = (err > 0.5 * ss->prev) ? ss->stagnant + 1 : 0;
  ss->prev = err;
  if (ss->stagnant >= 2) { ss->done = 1; ss->status = 7; }  // EFLOOR
}

__global__ void set_cert_kernel(CertConsts *dst, CertConsts c) { *dst = c; }

__global__ void cg_continue_kernel(cudaGraphConditionalHandle h, const CgScalars *sc, int maxit) {
  cudaGraphSetConditional(h, (sc->done || sc->iters >= maxit) ? 0u : 1u);
}

cudaError_t launch_set_cert(CertConsts *dst, CertConsts c, cudaStream_t st) {
  note_launch();
  set_cert_kernel<<<1, 1, 0, st>>>(dst, c);
  return cudaGetLastError();
}

cudaError_t launch_cg_continue(cudaGraphConditionalHandle h, const CgScalars *sc, int maxit, cudaStream_t st) {
  note_launch();
  cg_continue_kernel<<<1, 1, 0, st>>>(h, sc, maxit);
  return cudaGetLastError();
}

cudaError_t launch_solve_state_init(SolveState *ss, cudaStream_t st) {
  note_launch();
  solve_state_init_kernel<<<1, 1, 0, st>>>(ss);
  return cudaGetLastError();
}

cudaError_t launch_solve_stop(SolveState *ss, const double *norms, int outer, bool final, const CertConsts *c,
                              const CgScalars *sc, cudaStream_t st) {
  note_launch();
  solve_stop_kernel<<<1, 1, 0, st>>>(ss, norms, outer, final ? 1 : 0, c, sc);
  return cudaGetLastError();
}

cudaError_t launch_cg_update(int m, const double *qq, int nqq, const void *np, void *u, void *s, void *p,
                             CgScalars *sc, double tol2, cudaStream_t st) {
  note_launch();
  cg_update_kernel<<<1, 1024, 0, st>>>(m, qq, nqq, (const zd *)np, (zd *)u, (zd *)s, (zd *)p, sc, tol2);
  return cudaGetLastError();
}

cudaError_t launch_dd_accumulate(int64_t len, void *yh, void *yl, const void *d, cudaStream_t st,
                                 const int *skip) {
  note_launch();
  dd_accumulate_kernel<<<blocks_for(len), 256, 0, st>>>(len, (zd *)yh, (zd *)yl, (const zd *)d, skip);
  return cudaGetLastError();
}

cudaError_t launch_resid_finish(int64_t len, const void *b, const void *vh, const void *vl, void *r,
                                cudaStream_t st) {
  note_launch();
  resid_finish_kernel<<<blocks_for(len), 256, 0, st>>>(len, (const zd *)b, (const zd *)vh, (const zd *)vl,
                                                       (zd *)r);
  return cudaGetLastError();
}

cudaError_t launch_sub(int64_t len, void *r, const void *t, cudaStream_t st) {
  note_launch();
  sub_kernel<<<blocks_for(len), 256, 0, st>>>(len, (zd *)r, (const zd *)t);
  return cudaGetLastError();
}

cudaError_t launch_sumsq(int64_t len, const void *v, double *part, double *out, cudaStream_t st) {
  const int nb = blocks_for(len);
  note_launch();
  sumsq_kernel<<<nb, 256, 0, st>>>(len, (const zd *)v, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launch();
  finish_sum_kernel<<<1, 256, 0, st>>>(part, nb, out);
  return cudaGetLastError();
}

int sumsq_partials(int64_t len) { return blocks_for(len); }

cudaError_t launch_sum(int len, const double *v, double *out, cudaStream_t st) {
  note_launch();
  finish_sum_kernel<<<1, 256, 0, st>>>(v, len, out);
  return cudaGetLastError();
}

}  // namespace mn
