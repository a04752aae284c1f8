"""Full-size solves of the two large workloads, built on the GPU: 2048 x 262144
complex64 with singular values 1 .. 1e-5 (mixed precision), and 4096 x 131072
complex64 with singular values 1 .. 1e-6 and 64 right-hand sides (block entry
point), both to eps = 1e-10. The oracle's O1 solution would take tens of minutes
on the host, so each x is checked by the oracle's own a-posteriori certificate
(oracle.error_certificate: the oracle's FP64 sketch of A with its own T, a LAPACK
QR of it, and the double-double residual b - A x), a rigorous bound on
||x - p|| / ||x|| computed without the library: it must be within eps. (A plain
residual check is not enough: ||b - A x|| / sigma_min(A) is looser than the error by
up to the condition number, 1e5 .. 1e6 here.)"""
import numpy as np
import pytest

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


def _certified(A, b, X, eps):
    """The oracle's certificate for the columns of X (numpy, host), against eps."""
    import oracle
    bounds, delta = oracle.error_certificate(A, b, X, seed=17)
    assert delta < 0.1, delta
    return bounds


def test_precision_workload_2048x262144(mn):
    import torch
    dev = torch.device("cuda:0")
    w = synth.WORKLOADS["c3_precision_2048x262144"]
    m, n = w["m"], w["n"]
    s = synth.make_system(m, n, w["exponent"], w["seed"], dtype="c64", device="cuda:0")
    plan = mn.minnorm_plan_create(m, n, 0, mn.C64, mn.MIXED, seed=3)
    try:
        mn.minnorm_sketch(plan, s.A)
        x = torch.empty(n, dtype=torch.complex128, device=dev)
        st, info = mn.minnorm_solve(plan, s.A, s.b, w["eps"], x)
        torch.cuda.synchronize()
    finally:
        mn.minnorm_plan_destroy(plan)
    assert st == mn.OK and info["err_bound"] <= w["eps"], info
    A_np, b_np, x_np = s.A.cpu().numpy(), s.b.cpu().numpy(), x.cpu().numpy()
    del s
    bounds = _certified(A_np, b_np, x_np, w["eps"])
    assert bounds[0] <= w["eps"], (bounds, info)


def test_block_rhs_workload_4096x131072x64(mn):
    import torch
    dev = torch.device("cuda:0")
    w = synth.WORKLOADS["c5_blockrhs_4096x131072"]
    m, n, k = w["m"], w["n"], w["nrhs"]
    s = synth.make_system(m, n, w["exponent"], w["seed"], dtype="c64", nrhs=k, device="cuda:0")
    plan = mn.minnorm_plan_create(m, n, 0, mn.C64, mn.MIXED, seed=5)
    try:
        mn.minnorm_sketch(plan, s.A)
        B = s.b.T.contiguous().T                    # column-major m x k
        X = torch.empty((k, n), dtype=torch.complex128, device=dev).T
        st, infos = mn.minnorm_solve_many(plan, s.A, B, w["eps"], X)
        torch.cuda.synchronize()
    finally:
        mn.minnorm_plan_destroy(plan)
    assert st == mn.OK
    assert all(i["status"] == mn.OK and i["err_bound"] <= w["eps"] for i in infos)
    cols = [0, 31, 32, 63]                 # both ends of both 32-column chunks
    A_np = s.A.cpu().numpy()
    B_np, X_np = B[:, cols].cpu().numpy(), X[:, cols].cpu().numpy()
    del s
    bounds = _certified(A_np, B_np, X_np, w["eps"])
    assert np.all(bounds <= w["eps"]), (bounds, [infos[j] for j in cols])
