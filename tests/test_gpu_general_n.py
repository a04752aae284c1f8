"""GPU parity for lengths n that are not powers of two: the sketch's DFT then runs as
Bluestein's chirp convolution (two FFTs of the power-of-two length L >= 2n - 1), checked
against the oracle's transform (which takes Bluestein's identity too, but with its own
radix-2 code, in FP64) and, through full solves, against the oracle's p.

Tolerances: FP64 sketches 1e-12 relative, as for powers of two. Double-word sketches
(mixed precision) (40 + 12 log2 L) 2^-46: twice the power-of-two bound, since each
element now passes two FFTs of length L and two chirp products."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_0905_4745_gb300 import minnorm
    return minnorm


def _dev():
    import torch
    return torch.device("cuda:0")


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(_dev())


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _sketch(mn, m, n, prec, seed, A):
    import torch
    l = min(4 * m, n)
    plan = mn.minnorm_plan_create(m, n, 0, mn.C128, prec, seed=seed, flags=mn.FLAG_KEEP_SKETCH)
    try:
        mn.minnorm_sketch(plan, _t(A), allow=(mn.OK, mn.ERANK))
        Y = torch.empty((m, l), dtype=torch.complex128, device=_dev())
        mn.minnorm_get_sketch(plan, Y)
        torch.cuda.synchronize()
        return Y.cpu().numpy().T
    finally:
        mn.minnorm_plan_destroy(plan)


# single pass (L <= 4096 / 8192) and four-step (larger L); odd, prime and composite n
@pytest.mark.parametrize("m,n", [(4, 3), (5, 100), (8, 1000), (7, 2039), (6, 3000), (9, 24576), (3, 100003)])
def test_sketch_fp64_general_n(mn, m, n):
    if m >= n:
        m = n - 1
    s = synth.make_system(m, n, exponent=2, seed=500 + n)
    Y = _sketch(mn, m, n, mn.FP64, 13, s.A)
    Yref = oracle.sketch(oracle.draw_params(n, min(4 * m, n), 13), s.A)
    assert _rel(Y, Yref) <= 1e-12
    assert np.abs(Y - Yref).max() <= 1e-12 * np.abs(Yref).max()


@pytest.mark.parametrize("m,n", [(5, 100), (8, 3000), (6, 5000), (4, 40000)])
def test_sketch_dw_general_n(mn, m, n):
    s = synth.make_system(m, n, exponent=2, seed=600 + n)
    Y = _sketch(mn, m, n, mn.MIXED, 23, s.A)
    Yref = oracle.sketch(oracle.draw_params(n, 4 * m, 23), s.A)
    L = 1 << int(np.ceil(np.log2(2 * n - 1)))
    tol = (40 + 12 * np.log2(L)) * 2.0 ** -46
    assert _rel(Y, Yref) <= tol
    assert np.abs(Y - Yref).max() <= tol * np.abs(Yref).max()


@pytest.mark.parametrize("m,k,prec", [(48, 21, 0), (48, 21, 1), (100, 37, 1), (37, 9, 0)])
def test_solve_general_n(mn, m, k, prec):
    # the batching workload's shapes: n = m k with k in [8, 64], singular values 1 .. 1e-4
    import torch
    n = m * k
    s = synth.make_system(m, n, exponent=4, seed=900 + n)
    p = oracle.minnorm_direct(s.A, s.b, steps=5)["p"]
    plan = mn.minnorm_plan_create(m, n, 0, mn.C128, prec, seed=5)
    try:
        A = _t(s.A)
        mn.minnorm_sketch(plan, A)
        x = torch.empty(n, dtype=torch.complex128, device=_dev())
        st, info = mn.minnorm_solve(plan, A, _t(s.b), 1e-10, x)
        torch.cuda.synchronize()
    finally:
        mn.minnorm_plan_destroy(plan)
    assert st == mn.OK, info
    assert _rel(x.cpu().numpy(), p) <= 1e-10
