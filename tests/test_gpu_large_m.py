"""Solves with m > 512 against the oracle's O1, element by element: the code paths the
precision (2048 x 262144) and block right-hand-side (4096 x 131072) workloads take at full
size, on systems small enough for O1 on the host:
  - the mixed CG's one-pass product by clusters of CTAs (m > 512; the fused kernel serves
    m <= 512) and the FP64 CG's two passes, checked to be the paths taken (the plan's
    per-kernel counters),
  - the pivoted QR's general kernel (l = 4m > 2048),
  - the block CG on the tensor cores in 32-column chunks with a ragged last chunk,
in mixed precision and in FP64. Each x must be within eps of O1's p in the 2-norm (the
guarantee ||x - p|| <= eps ||p||) and per element within eps ||p||_inf (no single entry
off), and the library's own a-posteriori bound must also hold against p."""
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


def _check(x, p, eps, info):
    d = x - p
    rel = np.linalg.norm(d) / np.linalg.norm(p)
    assert rel <= eps, (rel, info)
    assert np.max(np.abs(d)) <= eps * np.max(np.abs(p)), (np.max(np.abs(d)), info)
    # the bound the library reports is a true bound (relative to ||x||), and its ingredients are
    # consistent: sigma_min(R) >= 1 / ||R^{-1}||_F <= |R_mm|, ||R||_F >= |R_11|, delta small
    assert rel * np.linalg.norm(p) <= info["err_bound"] * np.linalg.norm(x), (rel, info)
    assert info["cert_delta"] < 0.1, info
    assert info["sigma_min_R"] <= info["rdiag_min"] * (1 + 1e-12), info
    assert info["sigma_max_R"] >= info["rdiag_max"] * (1 - 1e-12), info


def _solve(mn, A, b, prec, eps, seed):
    import torch
    m, n = A.shape
    dev = torch.device("cuda:0")
    plan = mn.minnorm_plan_create(m, n, 0, mn.C64, prec, seed=seed, flags=mn.FLAG_TIMING)
    try:
        At = torch.from_numpy(A).to(dev)
        mn.minnorm_sketch(plan, At)
        x = torch.empty(n, dtype=torch.complex128, device=dev)
        st, info = mn.minnorm_solve(plan, At, torch.from_numpy(b).to(dev), eps, x)
        torch.cuda.synchronize()
        fused = mn.minnorm_kernel_stats(plan, 5)[0]
        adj, fwd = mn.minnorm_kernel_stats(plan, 0)[0], mn.minnorm_kernel_stats(plan, 1)[0]
        # mixed precision: both products in one pass (class 0 only); FP64: two passes
        two = prec != mn.MIXED
        assert fused == 0 and adj >= info["cg_iters"] and (fwd >= info["cg_iters"] if two else fwd == 0), \
            (fused, adj, fwd, info)
        return st, info, x.cpu().numpy()
    finally:
        mn.minnorm_plan_destroy(plan)


@pytest.fixture(scope="module")
def sys_2048():
    # 2048 x 16384 complex64, singular values 1 .. 1e-5: the precision workload's m and spectrum
    s = synth.make_system(2048, 16384, exponent=5, seed=8101, dtype="c64")
    p = oracle.minnorm_direct(s.A.astype(np.complex128), s.b, steps=5)["p"]
    return s, p


@pytest.mark.parametrize("prec", [1, 0])
def test_solve_2048x16384_kappa_1e5(mn, sys_2048, prec):
    s, p = sys_2048
    st, info, x = _solve(mn, s.A, s.b, prec, 1e-10, seed=3)
    assert st == mn.OK, info
    _check(x, p, 1e-10, info)


@pytest.mark.parametrize("prec", [1, 0])
def test_solve_1024x16384_kappa_1e6(mn, prec):
    # the block workload's spectrum (1 .. 1e-6) at m = 1024
    s = synth.make_system(1024, 16384, exponent=6, seed=8102, dtype="c64")
    p = oracle.minnorm_direct(s.A.astype(np.complex128), s.b, steps=6)["p"]
    st, info, x = _solve(mn, s.A, s.b, prec, 1e-10, seed=4)
    assert st == mn.OK, info
    _check(x, p, 1e-10, info)


def test_block_1024x8192_33_rhs(mn):
    # 33 right-hand sides: one full 32-column chunk of the tensor-core block CG and a ragged
    # chunk of one column; O1 on the chunks' first and last columns and the ragged one
    import torch
    m, n, k, eps = 1024, 8192, 33, 1e-10
    s = synth.make_system(m, n, exponent=6, seed=8103, dtype="c64", nrhs=k)
    dev = torch.device("cuda:0")
    plan = mn.minnorm_plan_create(m, n, 0, mn.C64, mn.MIXED, seed=6)
    try:
        At = torch.from_numpy(s.A).to(dev)
        mn.minnorm_sketch(plan, At)
        B = torch.from_numpy(s.b).to(dev).T.contiguous().T           # column-major m x k
        X = torch.empty((k, n), dtype=torch.complex128, device=dev).T
        st, infos = mn.minnorm_solve_many(plan, At, B, eps, X)
        torch.cuda.synchronize()
        X = X.cpu().numpy()
    finally:
        mn.minnorm_plan_destroy(plan)
    assert st == mn.OK
    A64 = s.A.astype(np.complex128)
    for j in (0, 31, 32):
        p = oracle.minnorm_direct(A64, np.ascontiguousarray(s.b[:, j]), steps=6)["p"]
        assert infos[j]["status"] == mn.OK
        _check(X[:, j], p, eps, infos[j])
