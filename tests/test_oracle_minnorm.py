"""Pins for the oracle's minimal-norm solvers: O1 (direct pivoted QR + double-double
refinement) and O2 (the randomized algorithm of Section 4, literally)."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _closed_form(sysm, b):
    # A = U diag(sigma) V^*  =>  p = V diag(1/sigma) U^* b   (Eqs. matrix_definition, exact_solution)
    return sysm.V @ ((sysm.U.conj().T @ b) / sysm.sigma)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_residual_dd_is_exact_to_double_rounding():
    # brute force in exact rational arithmetic on a small case
    rng = np.random.default_rng(0)
    m, n = 3, 7
    A = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    y = (rng.standard_normal(m) + 1j * rng.standard_normal(m)) * 1e6
    b = A @ (A.conj().T @ y) + 1e-9 * (rng.standard_normal(m) + 1j * rng.standard_normal(m))
    r, xh, xl = oracle.residual_dd(A, y, None, b)

    def fr(z):
        return Fraction(z.real), Fraction(z.imag)

    for i in range(m):
        er, ei = fr(b[i])
        for j in range(n):
            xr, xi = Fraction(0), Fraction(0)
            for k in range(m):
                ar, ai = fr(A[k, j]); yr, yi = fr(y[k])
                xr += ar * yr + ai * yi
                xi += ar * yi - ai * yr
            ar, ai = fr(A[i, j])
            er -= ar * xr - ai * xi
            ei -= ar * xi + ai * xr
        exact = complex(float(er), float(ei))
        scale = np.abs(A).sum() * np.abs(y).max() * np.abs(A).max() * n
        # double-double: error ~ 2^-104 of the summed magnitudes plus the final rounding
        assert abs(r[i] - exact) <= 2.0 ** -52 * abs(exact) + 2.0 ** -98 * scale


def test_direct_matches_closed_form_well_conditioned():
    s = synth.make_system(16, 200, exponent=1, seed=1, keep_factors=True)
    out = oracle.minnorm_direct(s.A, s.b, steps=3)
    assert out["rc"] == 0
    p_cf = _closed_form(s, s.b)
    assert _rel(out["p"], p_cf) < 1e-13
    assert _rel(out["x0"], p_cf) < 1e-13                  # the classical direct solution


def test_direct_matches_lapack_lstsq():
    s = synth.make_system(30, 120, exponent=3, seed=2)
    out = oracle.minnorm_direct(s.A, s.b, steps=4)
    ref = np.linalg.lstsq(s.A, s.b, rcond=None)[0]          # LAPACK zgelsd minimal-norm solution
    assert _rel(out["p"], ref) < 1e3 * 1e-15 * 10


def test_direct_refinement_beats_fp64_at_high_kappa():
    # kappa = 1e8: FP64 alone is good to ~1e-8; the double-double-refined p must match
    # an exact high-precision solve (mpmath, 60 digits) to ~1e-14
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    s = synth.make_system(4, 9, exponent=8, seed=3)
    A, b = s.A, s.b
    out = oracle.minnorm_direct(A, b, steps=8)
    Am = mpmath.matrix([[mpmath.mpc(complex(A[i, j])) for j in range(9)] for i in range(4)])
    bm = mpmath.matrix([mpmath.mpc(complex(b[i])) for i in range(4)])
    AH = Am.transpose_conj()
    pm = AH * mpmath.lu_solve(Am * AH, bm)
    p_exact = np.array([complex(pm[j]) for j in range(9)])
    assert _rel(out["p"], p_exact) < 1e-14
    assert _rel(out["x0"], p_exact) > 1e-12          # plain FP64 is visibly worse here


def test_direct_solution_properties():
    s = synth.make_system(24, 300, exponent=6, seed=4)
    out = oracle.minnorm_direct(s.A, s.b, steps=6)
    p = out["p"]
    r, _, _ = oracle.residual_dd(s.A, out["y"], None, s.b)
    assert np.linalg.norm(s.A @ p - s.b) < 1e-12 * np.linalg.norm(s.b) * 1e3
    # p lies in range(A^*): its component orthogonal to range(A^*) vanishes, up to the
    # ~kappa * 2^-53 error of this FP64 projector itself (the mpmath test above checks exactly)
    Q, _ = np.linalg.qr(s.A.conj().T)
    assert np.linalg.norm(p - Q @ (Q.conj().T @ p)) < 1e6 * 2.0 ** -53 * 10 * np.linalg.norm(p)


def test_direct_rank_deficient_reports():
    s = synth.make_system(6, 40, exponent=1, seed=5)
    A = s.A.copy()
    A[3] = A[1]
    out = oracle.minnorm_direct(A, s.b, steps=2)
    assert out["rc"] != 0 and not out["info"]["rank_ok"]


def _randomized(m, n, exponent, seed, tseed, eps, alpha=4.0, rhs="gaussian"):
    s = synth.make_system(m, n, exponent=exponent, seed=seed, rhs=rhs, keep_factors=True)
    l = 4 * m
    P = oracle.draw_params(n, l, tseed)
    delta = eps ** 2 * l / (alpha * n)
    out = oracle.minnorm_randomized(P, s.A, s.b, delta, maxit=2000)
    return s, P, out


def test_randomized_lemma_identities():
    s, P, out = _randomized(16, 512, 4, seed=6, tseed=1, eps=1e-10)
    assert out["rc"] == 0
    c, z = out["c"], out["z"]
    # Lemma 5.1, Eq. easy: A c = b
    assert np.linalg.norm(s.A @ c - s.b) < 1e-12 * np.linalg.norm(s.b) * 1e2
    # Eq. intermed1: ||z|| = ||c|| (T^* has orthonormal columns)
    assert np.isclose(np.linalg.norm(z), np.linalg.norm(c), rtol=1e-13)
    p = oracle.minnorm_direct(s.A, s.b, steps=6)["p"]
    x = out["x"]
    # Eq. first (Pythagorean identity)
    lhs = np.linalg.norm(c - p) ** 2 + np.linalg.norm(p - x) ** 2
    assert np.isclose(lhs, np.linalg.norm(c - x) ** 2, rtol=1e-10)
    # Lemma 5.2, Eq. energy, alpha = 4: ||c|| <= sqrt(alpha n / l) ||p||
    assert np.linalg.norm(c) <= np.sqrt(4 * 512 / 64) * np.linalg.norm(p)
    # Theorem 5.4: ||x - p|| <= eps ||p||
    assert _rel(x, p) <= 1e-10


def test_randomized_start_vector_reading():
    # u0 = Q^* T c equals R^{-*} P^T b because T T^* = I (Steps 2-4)
    m, n = 12, 256
    s = synth.make_system(m, n, exponent=2, seed=7)
    P = oracle.draw_params(n, 4 * m, 2)
    out = oracle.minnorm_randomized(P, s.A, s.b, 1e-20, maxit=0)
    f = oracle.qrp(oracle.sketch(P, s.A))
    u0 = oracle.solve_rh(f.R, s.b[f.piv])
    assert np.allclose(out["u0"], u0, atol=1e-12 * np.linalg.norm(u0))


def test_preconditioned_operator_bounds():
    # M = A^* P R^{-1}: T M = Q has orthonormal columns and ||T|| <= 1, so sigma_min(M) >= 1;
    # with alpha = 4, kappa(M) <= sqrt(alpha n / l) with high probability (Lemma 3.1)
    m, n = 20, 800
    s = synth.make_system(m, n, exponent=6, seed=8)
    P = oracle.draw_params(n, 4 * m, 3)
    f = oracle.qrp(oracle.sketch(P, s.A))
    M = s.A.conj().T[:, f.piv] @ np.linalg.inv(f.R)
    sv = np.linalg.svd(M, compute_uv=False)
    assert sv[-1] >= 1 - 1e-9
    assert sv[0] / sv[-1] <= np.sqrt(4 * n / (4 * m))


def test_normal_form_reproduces_literal_iterates():
    # the GPU path runs CG on R^{-*} P^T A A^* P R^{-1} u = R^{-*} P^T b (it needs only b);
    # from the same start it must give the literal CGLS iterates (A c = b, Lemma 5.1)
    m, n = 10, 300
    s = synth.make_system(m, n, exponent=3, seed=9)
    P = oracle.draw_params(n, 4 * m, 4)
    f = oracle.qrp(oracle.sketch(P, s.A))
    for k in (1, 3, 6):
        lit = oracle.minnorm_randomized(P, s.A, s.b, 0.0, maxit=k)
        _, y = oracle.pcg_normal(s.A, s.b, f.R, f.piv, k, u_start=lit["u0"])
        assert np.allclose(y, lit["y"], rtol=0, atol=1e-9 * np.linalg.norm(lit["y"]))


def _paper_rows():
    rows = []
    for line in open(os.path.join(GOLDEN, "paper_tables.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        rows.append(dict(m=int(f[1]), n=int(f[2]), l=int(f[3]), eps0=float(f[6]), epsr=float(f[7])))
    return rows


@pytest.mark.slow
def test_paper_table4_error_level():
    # Tables 3/4, first row (m = 256, n = 4096, l = 1024, kappa = 1e6, the paper's b):
    # the kappa-normalised errors of the classical and the randomized FP64 methods are a
    # few 1e-16 .. 1e-15. Ten trials, worst error, as in Section 7.
    row = [r for r in _paper_rows() if r["m"] == 256 and r["n"] == 4096][0]
    m, n, l = row["m"], row["n"], row["l"]
    s = synth.make_system(m, n, exponent=6, seed=2009, rhs="paper")
    kappa = 1e6
    delta = (1e-14 * kappa) ** 2 * m / n
    errs = []
    for t in range(1, 4):
        P = oracle.draw_params(n, l, t)
        out = oracle.minnorm_randomized(P, s.A, s.b, delta, maxit=500)
        errs.append(_rel(out["x"], s.p) / kappa)
    eps_r = max(errs)
    d = oracle.minnorm_direct(s.A, s.b, steps=0)
    eps_0 = _rel(d["x0"], s.p) / kappa
    assert row["epsr"] / 30 < eps_r < row["epsr"] * 10
    assert row["eps0"] / 30 < eps_0 < max(row["eps0"], row["epsr"]) * 10
