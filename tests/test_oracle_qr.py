"""Pins for the oracle's pivoted Householder QR (Section 7 / Step 2; GVL ch. 5)
and its triangular solves."""
import numpy as np
import pytest
import scipy.linalg

import oracle


def _rand(rows, cols, seed, scale_cols=None):
    rng = np.random.default_rng(seed)
    Y = rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))
    if scale_cols is not None:
        Y = Y * scale_cols[None, :]
    return Y


@pytest.mark.parametrize("rows,cols", [(8, 3), (40, 10), (256, 64), (33, 33)])
def test_qrp_factorisation_properties(rows, cols):
    Y = _rand(rows, cols, rows + cols, scale_cols=10.0 ** -np.linspace(0, 4, cols))
    f = oracle.qrp(Y)
    R, piv = f.R, f.piv
    assert np.array_equal(np.sort(piv), np.arange(cols))
    Q = f.Q()
    k = min(rows, cols)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(k)) < 1e-13
    assert np.linalg.norm(Y[:, piv] - Q @ R) < 1e-13 * np.linalg.norm(Y)
    d = np.abs(np.diag(R))
    assert np.all(np.abs(np.diag(R).imag) == 0)          # real diagonal (zlarfg convention)
    assert np.all(d[:-1] >= d[1:] * (1 - 1e-12))          # column pivoting: non-increasing |R_kk|
    assert np.array_equal(R, np.triu(R))


@pytest.mark.parametrize("rows,cols,seed", [(12, 5, 0), (64, 16, 1), (300, 75, 2)])
def test_qrp_matches_lapack(rows, cols, seed):
    # an independent implementation of the same algorithm: LAPACK zgeqp3 via scipy
    Y = _rand(rows, cols, seed, scale_cols=10.0 ** -np.linspace(0, 3, cols))
    f = oracle.qrp(Y)
    R2, piv2 = scipy.linalg.qr(Y, mode="r", pivoting=True)
    assert np.array_equal(f.piv, piv2)
    assert np.linalg.norm(f.R - R2[: f.R.shape[0]]) < 1e-12 * np.linalg.norm(R2)


def test_qrp_rank_deficient_and_trivial():
    Y = _rand(20, 4, 3)
    Y[:, 2] = Y[:, 0]                                     # rank 3
    f = oracle.qrp(Y)
    assert abs(f.R[3, 3]) < 1e-13 * abs(f.R[0, 0])
    Z = np.zeros((6, 3), complex)
    g = oracle.qrp(Z)
    assert np.all(g.R == 0) and np.all(g.tau == 0)


def test_triangular_solves_and_q_application():
    Y = _rand(50, 12, 4)
    f = oracle.qrp(Y)
    R = f.R
    rng = np.random.default_rng(5)
    x = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    assert np.allclose(oracle.solve_r(R, x), np.linalg.solve(R, x), atol=1e-13)
    assert np.allclose(oracle.solve_rh(R, x), np.linalg.solve(R.conj().T, x), atol=1e-13)
    v = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    Q = f.Q()
    full = oracle.qrp(Y)
    assert np.allclose(full.apply_q(v, conj=True)[:12], Q.conj().T @ v, atol=1e-13)
    w = np.zeros(50, complex); w[:12] = x
    assert np.allclose(full.apply_q(w), Q @ x, atol=1e-13)
