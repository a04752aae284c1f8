"""Full-size solves of the two large workloads, built on the GPU (their oracle
solutions would take hours on the host): 2048 x 262144 complex64 with singular
values 1 .. 1e-5 (mixed precision), and 4096 x 131072 complex64 with singular
values 1 .. 1e-6 and 64 right-hand sides (block entry point), both to eps = 1e-10.

Every solve must return OK with its a-posteriori bound <= eps, and its residual
b - A x, formed by torch in complex128 independently of the library, must be
within eps ||x|| (since sigma_max(A) = 1 and x - p is bounded by eps ||p||) plus
the rounding bound of torch's own product, 2 n 2^-53 || |A| |x| ||. The solution
lies in range(A^*) by construction (Step 5 forms x = A^* y)."""
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


def _check_residual(A64, b, x, eps):
    import torch
    r = b - A64 @ x
    n = A64.shape[1]
    bound = 2.0 * n * 2.0 ** -53 * torch.linalg.norm(A64.abs() @ x.abs(), dim=0)
    ok = torch.linalg.norm(r, dim=0) <= 1.01 * eps * torch.linalg.norm(x, dim=0) + bound
    return bool(ok.all())


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
    A64 = s.A.to(torch.complex128)
    assert _check_residual(A64, s.b[:, None], x[:, None], w["eps"])


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
    A64 = s.A.to(torch.complex128)
    assert _check_residual(A64, B, X, w["eps"])
