"""The trailing-update products of the blocked pivoted QR (Step 2) on the tensor cores,
W = V^H C and C - V Z, against double-double references from the oracle (Dot2 sums:
oracle.adj_matvec_dd / matvec_dd), element by element.

Tolerance, from the arithmetic. The adjoint product truncates every operand entry to 63 bits
below its row's scale 2^e (the least power of two above the row's largest entry component):
an absolute error below 2^(e - 63) <= 2^-62 max|row| per real component. A complex result is
two real products of the interleaved real forms, whose sums of moduli are at most sqrt 2 times
the complex ones, so the truncation adds at most 2^-61 (max|V_:j| sum|C_:c| + max|C_:c|
sum|V_:j|). The slice pairs beyond level 8 are dropped: at most 6.02 2^-72 2^(e+f) <= 2^-67.4
max|v| max|c| per real term, so (2 K real terms, sqrt 2 for the modulus) 2^-65.9 K max|V_:j|
max|C_:c| for complex length K. The kept levels are summed exactly and rounded once to FP64 per
K split, and the splits added by a compensated sum (their exact sum rounded once): at most
2^-53 (|V|^T|C| + |W|) <= 2^-52 |V|^T|C| per component. So
  |W_jc - W_ref| <= 2^-61 (max|V_:j| sum|C_:c| + max|C_:c| sum|V_:j|) + 2^-65 K max|V_:j| max|C_:c|
                    + 2^-51 |V|^T|C|,
checked with a factor 2 of slack: as accurate as an FP64 dot product at any K. The update
(K = 32) truncates to 55 bits and drops the levels beyond 7: 2^-53 (max|V_i:| sum|Z_:c| +
max|Z_:c| sum|V_i:|) + 2^-57 32 max|V_i:| max|Z_:c|, plus the low 15 bits of its level sums
dropped before the one conversion (below 2^-53 max|V_i:| max|Z_:c|, within the first term) and
the roundings of the product and of the subtraction. Cases: one K range and several (split K; odd K-block counts), ragged tile edges,
rows and columns of very different scales, zero rows and columns."""
import numpy as np
import pytest

import oracle

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


def _cm(a):
    """complex128 numpy array -> column-major CUDA tensor of the same shape"""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda:0").T


def _inputs(rows, cols, seed):
    rng = np.random.default_rng(seed)
    g = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)
    V = g(rows, 32) * 10.0 ** rng.uniform(-2, 2, size=(1, 32))
    V[:, 5] = 0.0                       # a zero reflector column
    V[3, :] = 0.0                       # a zero row
    C = g(rows, cols) * 10.0 ** rng.uniform(-3, 3, size=(1, cols)) * 10.0 ** rng.uniform(-1, 1, size=(rows, 1))
    C[:, 7 % cols] = 0.0
    Z = g(32, cols) * 10.0 ** rng.uniform(-3, 3, size=(1, cols))
    return V, C, Z


@pytest.mark.parametrize("rows,cols,m,n", [(1200, 300, 300, 8192), (1000, 257, 300, 8192), (4400, 1100, 1100, 16384),
                                           (33, 70, 300, 8192)])
def test_trailing_products_against_double_double(mn, rows, cols, m, n):
    import torch
    V, C, Z = _inputs(rows, cols, seed=rows + cols)
    plan = mn.minnorm_plan_create(m, n, 0, mn.C128, mn.FP64, seed=1)
    try:
        Vt, Ct, Zt = _cm(V), _cm(C), _cm(Z)
        Wt = torch.empty((cols, 32), dtype=torch.complex128, device="cuda:0").T   # 32 x cols, ld 32
        mn.minnorm_trailing_products(plan, Vt, Ct, Z=Zt, W=Wt)
        torch.cuda.synchronize()
        W, Cn = Wt.cpu().numpy(), Ct.cpu().numpy()
    finally:
        mn.minnorm_plan_destroy(plan)
    # W = V^H C against Dot2 sums (the library's K splits are added by a compensated sum)
    absV, absC = np.abs(V), np.abs(C)
    mV, sV = absV.max(axis=0), absV.sum(axis=0)      # per reflector column j
    for c in range(cols):
        xh, xl = oracle.adj_matvec_dd(V, np.ascontiguousarray(C[:, c]))
        ref = xh + xl
        mC, sC = absC[:, c].max(), absC[:, c].sum()
        tol = 2.0 * (2.0 ** -61 * (mV * sC + mC * sV) + 2.0 ** -65 * rows * mV * mC
                     + 2.0 ** -51 * (absV.T @ absC[:, c]))
        err = np.abs(W[:, c] - ref)
        assert np.all(err <= tol), (c, np.max(err / np.maximum(tol, 1e-300)))
    # C - V Z against Dot2 sums
    absZ = np.abs(Z)
    mVr, sVr = absV.max(axis=1), absV.sum(axis=1)      # per row i of V (the update's operand rows)
    for c in range(0, cols, 7):
        vh, vl = oracle.matvec_dd(V, np.ascontiguousarray(Z[:, c]))
        ref = (C[:, c] - vh) - vl
        mZ, sZ = absZ[:, c].max(), absZ[:, c].sum()
        tol = 2.0 * (2.0 ** -53 * (mVr * sZ + mZ * sVr) + 2.0 ** -57 * 32 * mVr * mZ
                     + 2.0 ** -52 * ((absV @ absZ[:, c]) + np.abs(ref) + absC[:, c]))
        err = np.abs(Cn[:, c] - ref)
        assert np.all(err <= tol), (c, np.max(err / np.maximum(tol, 1e-300)))


def test_trailing_products_argument_checks(mn):
    import torch
    plan = mn.minnorm_plan_create(16, 256, 0, mn.C128, mn.FP64, seed=1)
    try:
        V = torch.zeros((70, 32), dtype=torch.complex128, device="cuda:0").T.contiguous().T
        C = torch.zeros((70, 20), dtype=torch.complex128, device="cuda:0").T.contiguous().T
        with pytest.raises(mn.MinnormError) as e:      # rows beyond l = 64
            mn.minnorm_trailing_products(plan, V, C)
        assert e.value.status == mn.EINVAL
    finally:
        mn.minnorm_plan_destroy(plan)
