"""Pins for the oracle's SRFT (Section 3, Eqs. SRFT, SRFT2, Rokhlin_trans, big_def)
and its Step 1 sketch (Eq. randmat)."""
import numpy as np
import pytest

import oracle


def _givens_product(theta):
    """Theta = G_0 G_1 ... G_{n-2} as an explicit matrix product, G_k carrying the
    printed block [[cos, sin], [-sin, cos]] on rows/columns (k, k+1)."""
    n = theta.size + 1
    M = np.eye(n)
    for k in range(n - 1):
        G = np.eye(n)
        c, s = np.cos(theta[k]), np.sin(theta[k])
        G[k, k], G[k, k + 1], G[k + 1, k], G[k + 1, k + 1] = c, s, -s, c
        M = M @ G
    return M


def _perm_matrix(p):
    n = p.size
    M = np.zeros((n, n))
    M[np.arange(n), p] = 1.0          # (P v)[j] = v[p[j]]
    return M


def _dense_T(P):
    n = P.n
    H = (_givens_product(P.theta) @ _perm_matrix(P.pi) @ np.diag(P.zeta)
         @ _givens_product(P.theta_t) @ _perm_matrix(P.pi_t) @ np.diag(P.zeta_t))
    jk = np.outer(np.arange(n), np.arange(n))
    F = np.exp(-2j * np.pi * jk / n) / np.sqrt(n)
    return (F @ np.diag(P.d) @ H)[P.s, :], H


def test_chain_special_cases():
    rng = np.random.default_rng(0)
    v = rng.standard_normal(9) + 1j * rng.standard_normal(9)
    # theta = 0: every G_k is the identity
    assert np.array_equal(oracle.chain(v, np.zeros(8)), v)
    # theta = pi/2: G_k swaps with a sign, and the chain (G_{n-2} first) is the signed
    # cyclic shift out_0 = v_{n-1}, out_{k+1} = -v_k
    out = oracle.chain(v, np.full(8, np.pi / 2))
    expect = np.concatenate([[v[-1]], -v[:-1]])
    assert np.allclose(out, expect, atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 5, 16, 33])
def test_chain_matches_matrix_product(n):
    rng = np.random.default_rng(n)
    theta = rng.uniform(0, 2 * np.pi, n - 1)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    M = _givens_product(theta)
    assert np.allclose(oracle.chain(v, theta), M @ v, atol=1e-14)
    assert np.allclose(oracle.chain_adjoint(v, theta), M.T @ v, atol=1e-14)


@pytest.mark.parametrize("n,l", [(8, 3), (24, 6), (64, 16)])
def test_srft_matches_dense_definition(n, l):
    P = oracle.draw_params(n, l, seed=99 + n)
    T_ref, H_ref = _dense_T(P)
    rng = np.random.default_rng(n)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.allclose(oracle.apply_H(P, v), H_ref @ v, atol=1e-13)
    assert np.allclose(oracle.srft_dense(P), T_ref, atol=1e-13)


@pytest.mark.parametrize("n,l", [(64, 16), (100, 30), (256, 64)])
def test_srft_orthonormal_rows_and_adjoint(n, l):
    P = oracle.draw_params(n, l, seed=5)
    T = oracle.srft_dense(P)
    # T has orthonormal rows: F, D, H unitary and S picks distinct rows (Section 3)
    assert np.linalg.norm(T @ T.conj().T - np.eye(l)) < 1e-13
    rng = np.random.default_rng(1)
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w = rng.standard_normal(l) + 1j * rng.standard_normal(l)
    lhs = np.vdot(w, oracle.srft_apply(P, u))
    rhs = np.vdot(oracle.srft_adjoint(P, w), u)
    assert abs(lhs - rhs) < 1e-12 * np.linalg.norm(u) * np.linalg.norm(w)
    assert np.allclose(oracle.srft_adjoint(P, w), T.conj().T @ w, atol=1e-13)
    assert np.linalg.norm(oracle.srft_apply(P, u)) <= np.linalg.norm(u) * (1 + 1e-14)


def test_srft_without_H_is_subsampled_fft():
    # theta = 0, identity permutations, unit zetas: T = S F D, an FFT of d*v
    n, l = 128, 20
    P = oracle.draw_params(n, l, seed=8)
    Q = oracle.Params(n, l, np.ones(n), np.arange(n), np.zeros(n - 1), np.ones(n), np.arange(n),
                      np.zeros(n - 1), P.d, P.s)
    v = np.random.default_rng(2).standard_normal(n) + 0j
    assert np.allclose(oracle.srft_apply(Q, v), (np.fft.fft(P.d * v) / np.sqrt(n))[P.s], atol=1e-14)


@pytest.mark.parametrize("n", [96, 1000])
def test_srft_general_n(n):
    # non-power-of-two n goes through Bluestein; still orthonormal rows
    P = oracle.draw_params(n, 24, seed=n)
    T = oracle.srft_dense(P) if n <= 128 else None
    if T is not None:
        assert np.linalg.norm(T @ T.conj().T - np.eye(24)) < 1e-13
    rng = np.random.default_rng(0)
    w = rng.standard_normal(24) + 1j * rng.standard_normal(24)
    # T T^* w = w
    assert np.allclose(oracle.srft_apply(P, oracle.srft_adjoint(P, w)), w, atol=1e-13)


def test_sketch_is_T_times_A_adjoint():
    m, n, l = 5, 64, 20
    P = oracle.draw_params(n, l, seed=3)
    rng = np.random.default_rng(4)
    A = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    Y = oracle.sketch(P, A)
    assert Y.shape == (l, m)
    assert np.allclose(Y, oracle.srft_dense(P) @ A.conj().T, atol=1e-13)
