"""GPU parity of the block right-hand-side entry point (minnorm_solve_many): several
right-hand sides sharing one A, one SRFT realization and one pivoted QR, each
checked against the oracle's double-double-refined minimal-norm solution p. In mixed
precision the columns run through the block CG (32-column chunks; the 37-column case
spans two chunks, the second partly filled)."""
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


def _colmajor(a):
    """device tensor of shape a.shape holding `a` column-major (column j contiguous)"""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(_dev()).T


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("m,n,nrhs,prec", [(128, 8192, 5, 1), (96, 4096, 3, 0), (64, 2048, 8, 1), (48, 1000, 37, 1)])
def test_solve_many_matches_oracle(mn, m, n, nrhs, prec):
    import torch
    s = synth.make_system(m, n, exponent=6, seed=8100 + m, nrhs=nrhs)
    assert s.b.shape == (m, nrhs)
    plan = mn.minnorm_plan_create(m, n, 0, mn.C128, prec, seed=17)
    try:
        A = torch.from_numpy(s.A).to(_dev())
        mn.minnorm_sketch(plan, A)
        B = _colmajor(s.b)
        X = _colmajor(np.zeros((n, nrhs), np.complex128))
        st, infos = mn.minnorm_solve_many(plan, A, B, 1e-12, X)
        torch.cuda.synchronize()
        assert st == mn.OK, infos
        Xh = X.cpu().numpy()
        for j in range(nrhs):
            p = oracle.minnorm_direct(s.A, s.b[:, j], steps=6)["p"]
            assert _rel(Xh[:, j], p) <= 1e-12, (j, infos[j])
            assert infos[j]["err_bound"] <= 1e-12
        # the same plan, one column at a time: the same solutions (in mixed precision the block
        # CG takes different iterates, so both are only within eps of p)
        for j in (0, nrhs - 1):
            x = torch.empty(n, dtype=torch.complex128, device=_dev())
            mn.minnorm_solve(plan, A, B[:, j].contiguous(), 1e-12, x)
            torch.cuda.synchronize()
            assert _rel(Xh[:, j], x.cpu().numpy()) <= (1e-14 if prec == 0 else 2e-12)
    finally:
        mn.minnorm_plan_destroy(plan)


def test_solve_many_strided_and_errors(mn):
    import torch
    m, n, nrhs = 16, 512, 3
    s = synth.make_system(m, n, exponent=3, seed=8200, nrhs=nrhs)
    plan = mn.minnorm_plan_create(m, n, 0, mn.C128, mn.MIXED, seed=2)
    try:
        A = torch.from_numpy(s.A).to(_dev())
        # column-major with padding: ldb = m + 5, ldx = n + 3
        Bbuf = torch.zeros((nrhs, m + 5), dtype=torch.complex128, device=_dev())
        Bbuf[:, :m] = torch.from_numpy(np.ascontiguousarray(s.b.T)).to(_dev())
        Xbuf = torch.zeros((nrhs, n + 3), dtype=torch.complex128, device=_dev())
        B, X = Bbuf[:, :m].T, Xbuf[:, :n].T
        with pytest.raises(mn.MinnormError) as e:            # before the sketch
            mn.minnorm_solve_many(plan, A, B, 1e-10, X)
        assert e.value.status == mn.ESTATE
        mn.minnorm_sketch(plan, A)
        st, infos = mn.minnorm_solve_many(plan, A, B, 1e-12, X)
        torch.cuda.synchronize()
        assert st == mn.OK
        Xh = Xbuf.cpu().numpy()
        assert np.all(Xh[:, n:] == 0)                        # padding untouched
        for j in range(nrhs):
            p = oracle.minnorm_direct(s.A, s.b[:, j], steps=4)["p"]
            assert _rel(Xh[j, :n], p) <= 1e-12
        L = mn.lib()
        for args in ((m - 1, n, nrhs), (m, n - 1, nrhs), (m, n, 0)):   # ldb < m, ldx < n, nrhs < 1
            ldb, ldx, k = args
            st = L.minnorm_solve_many(plan, A.data_ptr(), n, B.data_ptr(), ldb, k, 1e-10, X.data_ptr(), ldx, None)
            assert st == mn.EINVAL, args
    finally:
        mn.minnorm_plan_destroy(plan)
