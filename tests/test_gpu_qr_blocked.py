"""Step 2 for tall sketches (l = 4m > 2048): the blocked Householder QR of Y without
pivoting (panels of 32 columns; trailing updates on the tensor cores with FP64 accuracy),
then the pivoted QR of its m x m triangle. Against the oracle's pivoted Householder QR of the
same sketch (the GPU's own Y): the same pivots, and R equal up to a unit diagonal (each row
of R is fixed up to the sign the reflectors' convention gives it: R1 P = Q2 R and Y P = Q R
determine R only up to D R with D diagonal unitary, and both sides take a real diagonal),
to the QR tolerance of the other tests (1e-12 relative). Also the factorization's own
invariants on the GPU's R: upper triangular, real diagonal of non-increasing magnitude,
R^H R = (Y P)^H (Y P) to FP64 accuracy; and the certificate's premise for such a plan:
sigma_min(A^* P R^{-1}) >= 1 - delta. Sizes with a ragged last panel (600 = 18 x 32 + 24) and
with split K in the tensor-core products (2 l > 4096)."""
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


def _factor(mn, s, m, n, prec, dtype):
    import torch
    dev = torch.device("cuda:0")
    l = 4 * m
    plan = mn.minnorm_plan_create(m, n, 0, dtype, prec, seed=23, flags=mn.FLAG_KEEP_SKETCH)
    try:
        A = torch.from_numpy(s.A).to(dev)
        mn.minnorm_sketch(plan, A)
        Y = torch.empty((m, l), dtype=torch.complex128, device=dev)
        R = torch.empty((m, m), dtype=torch.complex128, device=dev)
        piv = torch.empty(m, dtype=torch.int64, device=dev)
        mn.minnorm_get_sketch(plan, Y)
        mn.minnorm_get_factor(plan, R, piv)
        x = torch.empty(n, dtype=torch.complex128, device=dev)
        st, info = mn.minnorm_solve(plan, A, torch.from_numpy(s.b).to(dev), 1e-10, x)
        torch.cuda.synchronize()
    finally:
        mn.minnorm_plan_destroy(plan)
    return Y.cpu().numpy().T, R.cpu().numpy().T, piv.cpu().numpy(), st, info


@pytest.mark.parametrize("m,n,prec,dtype", [(600, 16384, 0, "c128"), (1100, 16384, 1, "c64")])
def test_blocked_qr_matches_oracle(mn, m, n, prec, dtype):
    s = synth.make_system(m, n, exponent=4, seed=6600 + m, dtype=dtype)
    Y, R, piv, st, info = _factor(mn, s, m, n, prec, mn.C64 if dtype == "c64" else mn.C128)
    assert st == mn.OK, info
    # invariants of Y P = Q R
    assert np.array_equal(np.sort(piv), np.arange(m))
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R).imag == 0)
    d = np.abs(np.diag(R))
    assert np.all(d[:-1] >= d[1:] * (1 - 1e-10))
    G = Y[:, piv].conj().T @ Y[:, piv]
    assert np.linalg.norm(R.conj().T @ R - G) <= 1e-13 * np.linalg.norm(G)
    # against the oracle's pivoted QR of the same sketch
    f = oracle.qrp(Y)
    assert np.array_equal(piv, f.piv)
    D = np.sign(np.diag(R).real) * np.sign(np.diag(f.R).real)
    assert np.linalg.norm(D[:, None] * R - f.R) <= 1e-12 * np.linalg.norm(f.R)


def test_blocked_qr_certificate_premise(mn):
    m, n = 600, 8192
    s = synth.make_system(m, n, exponent=5, seed=6700)
    Y, R, piv, st, info = _factor(mn, s, m, n, 1, mn.C128)
    W = np.zeros((m, m), np.complex128)
    W[piv, :] = np.linalg.inv(R)
    sv = np.linalg.svd(s.A.conj().T @ W, compute_uv=False)
    assert 0.0 < info["cert_delta"] < 0.1, info
    assert sv.min() >= 1.0 - info["cert_delta"], (sv.min(), info)
