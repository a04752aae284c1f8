"""The preconditioner P R^{-1} of Steps 3-4, as the plan keeps it after Step 2, against the
mathematics that defines it: X = P^T W must be upper triangular (exact zeros below the diagonal)
and R X = I. The residual F = R X - I is formed in double-double (the oracle's Dot2 products, so
that its own rounding is far below what is checked) and held to the a priori bound of the method
that computed X:
  column-by-column back substitution (sketches of up to 2048 rows):  ||F||_F <= 4 m 2^-53 ||R||_F ||X||_F
  blocks of 32 rows with the rank-32 updates on the tensor cores (taller sketches, m >= 256):
                                                  ||F||_F <= (160 + 2 ceil(m / 32)) 2^-53 ||R||_F ||X||_F
(the second derived from the update products' bound, tested element by element in
test_gpu_qr_products.py, and from the FP64 back substitution of the 32 x 32 diagonal blocks).
Cases: both methods; m a multiple of 32 and m with a ragged top block (600 = 18 x 32 + 24,
1100 = 34 x 32 + 12); complex128 and complex64 storage; both precisions."""
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


def _factors(mn, s, m, n, l, prec, dtype):
    import torch
    dev = torch.device("cuda:0")
    plan = mn.minnorm_plan_create(m, n, l, dtype, prec, seed=29)
    try:
        mn.minnorm_sketch(plan, torch.from_numpy(s.A).to(dev))
        R = torch.empty((m, m), dtype=torch.complex128, device=dev)
        W = torch.empty((m, m), dtype=torch.complex128, device=dev)
        piv = torch.empty(m, dtype=torch.int64, device=dev)
        mn.minnorm_get_factor(plan, R, piv)
        mn.minnorm_get_preconditioner(plan, W)
        torch.cuda.synchronize()
    finally:
        mn.minnorm_plan_destroy(plan)
    return R.cpu().numpy().T, W.cpu().numpy().T, piv.cpu().numpy()


def _residual_dd(R, X):
    """||R X - I||_F with every column's product in double-double"""
    m = R.shape[0]
    Rc = np.ascontiguousarray(R)
    tot = 0.0
    for k in range(m):
        h, lo = oracle.matvec_dd(Rc, np.ascontiguousarray(X[:, k]))
        h[k] -= 1.0
        tot += float(np.sum(np.abs(h + lo) ** 2))
    return np.sqrt(tot)


@pytest.mark.parametrize("m,n,l,prec,dtype", [(600, 16384, 0, 0, "c128"), (1100, 16384, 0, 1, "c64"),
                                              (256, 8192, 2112, 1, "c128"), (300, 8192, 0, 1, "c128"),
                                              (96, 4096, 2400, 0, "c128")])
def test_preconditioner_is_r_inverse(mn, m, n, l, prec, dtype):
    s = synth.make_system(m, n, exponent=4, seed=8800 + m, dtype=dtype)
    R, W, piv = _factors(mn, s, m, n, l, prec, mn.C64 if dtype == "c64" else mn.C128)
    X = W[piv, :]                      # row piv[k] of P R^{-1} is row k of R^{-1}
    assert np.all(np.tril(X, -1) == 0)
    assert np.all(np.diag(X).imag == 0) and np.all(np.diag(X).real * np.diag(R).real > 0)
    lr = l if l else 4 * m
    blocked = lr > 2048 and m >= 256
    c = (160 + 2 * ((m + 31) // 32)) if blocked else 4 * m
    F = _residual_dd(R, X)
    bound = c * 2.0 ** -53 * np.linalg.norm(R) * np.linalg.norm(X)
    assert F <= bound, (F, bound, blocked)
    # and the inverse itself against LAPACK's triangular solve, to the accuracy both residual bounds
    # imply (X - Xref = R^{-1} (F - Fref))
    from scipy.linalg import solve_triangular
    Xref = solve_triangular(R, np.eye(m, dtype=np.complex128))
    tol = (c + 4 * m) * 2.0 ** -53 * np.linalg.norm(R) * np.linalg.norm(Xref) * np.linalg.norm(Xref, 2)
    assert np.linalg.norm(X - Xref) <= tol
