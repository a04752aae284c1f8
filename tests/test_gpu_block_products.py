"""Parity of the block-CG products (Step 4 for 32 right-hand sides sharing A):
Q = A^* W and T = A Q on the tensor cores (exact three-way BF16 splits of both
operands, FP32 accumulation), against the FP64 definitions on the same inputs.

W enters the kernels rounded to complex64, so the reference uses that W; T is
checked against A times the Q the library returned. The bound 2e-6 (relative,
Frobenius) is FP32-level accuracy for these sums; a product of single BF16
pieces would be off by ~4e-3 and fail it. Sizes span several 64-row K-blocks
and 64-column tiles with ragged ends (the tiles read zeros outside A)."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("m,n", [(200, 4000), (64, 4096), (512, 65536), (37, 1000)])
def test_block_products_tensor_core(mn, m, n):
    import torch
    rng = np.random.default_rng(1000 + m)
    A = ((rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(2)).astype(np.complex64)
    W = (rng.standard_normal((m, 32)) + 1j * rng.standard_normal((m, 32))) * np.exp(rng.uniform(-3, 3, (m, 1)))
    dev = torch.device("cuda:0")
    Ad = torch.from_numpy(A).to(dev)
    Wd = torch.from_numpy(W).to(dev)
    Q = torch.empty((n, 32), dtype=torch.complex128, device=dev)
    T = torch.empty((m, 32), dtype=torch.complex128, device=dev)
    plan = mn.minnorm_plan_create(m, n, 0, mn.C64, mn.MIXED, seed=1)
    try:
        mn.minnorm_block_products(plan, Ad, Wd, Q, T)
        torch.cuda.synchronize()
    finally:
        mn.minnorm_plan_destroy(plan)
    A64 = A.astype(np.complex128)
    W32 = W.astype(np.complex64).astype(np.complex128)
    Qref = A64.conj().T @ W32
    Qk = Q.cpu().numpy()
    eq = np.linalg.norm(Qk - Qref) / np.linalg.norm(Qref)
    assert eq <= 2e-6, eq
    # every column separately (columns of very different scale)
    ec = np.linalg.norm(Qk - Qref, axis=0) / np.linalg.norm(Qref, axis=0)
    assert ec.max() <= 4e-6, ec.max()
    Tref = A64 @ Qk
    et = np.linalg.norm(T.cpu().numpy() - Tref) / np.linalg.norm(Tref)
    assert et <= 2e-6, et
