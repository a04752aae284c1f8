"""Pins of the oracle's a posteriori error certificate (oracle.error_certificate), which the
full-size GPU tests and the benchmark use where the oracle's O1 solve would take too long.

It must be an upper bound of the true error ||x - p|| / ||x|| (p from O1), also for an error
along the smallest singular direction, where the plain residual ||b - A x|| underestimates
the error by the condition number; and it must not be loose by more than the conditioning of
the preconditioned operator (a factor ~3 here), so that a transposed or dropped R^{-*}
fails one side or the other."""
import numpy as np

import oracle
import synth


def _setup(m=32, n=1024, exponent=4, seed=55):
    s = synth.make_system(m, n, exponent, seed, keep_factors=True)
    p = oracle.minnorm_direct(s.A, s.b, steps=5)["p"]
    return s, p


def test_certificate_of_the_exact_solution_is_tiny():
    s, p = _setup()
    bound, delta = oracle.error_certificate(s.A, s.b, p, seed=3)
    assert delta < 1e-6
    assert bound[0] < 1e-13


def test_certificate_bounds_errors_in_every_direction():
    s, p = _setup()
    m, n = s.A.shape
    V = s.V                                    # right singular vectors: range(A^*)
    # the premise, checked directly: M = A^* R^{-1} for the R of the same seed's sketch has
    # sigma_min(M) >= 1 (T has orthonormal rows); the certificate lies between sigma_min(M) and
    # sigma_max(M) times the true error
    Y = oracle.sketch(oracle.draw_params(n, 4 * m, 5), s.A)
    R = np.linalg.qr(np.ascontiguousarray(Y), mode="r")
    sv = np.linalg.svd(s.A.conj().T @ np.linalg.inv(R), compute_uv=False)
    assert sv.min() >= 1 - 1e-10
    for k, scale in ((0, 1e-6), (31, 1e-6), (31, 1e-9), (15, 1e-7)):
        e = scale * np.linalg.norm(p) * V[:, k]
        x = p + e
        true = np.linalg.norm(x - p) / np.linalg.norm(x)
        bound, _ = oracle.error_certificate(s.A, s.b, x, seed=5)
        assert bound[0] >= true * (1 - 1e-9), (k, scale, bound[0], true)
        assert bound[0] <= sv.max() * true * (1 + 1e-6) + 1e-13, (k, scale, bound[0], true, sv.max())
        # the plain residual misses an error along the smallest singular direction by kappa
        if k == 31:
            r = np.linalg.norm(s.A @ x - s.b) / np.linalg.norm(x)
            assert r < 1e-3 * true


def test_certificate_per_column():
    s, p = _setup(m=24, n=512, exponent=3, seed=9)
    X = np.stack([p, p + 1e-8 * np.linalg.norm(p) * s.V[:, 0]], axis=1)
    B = np.stack([s.b, s.b], axis=1)
    bound, _ = oracle.error_certificate(s.A, B, X, seed=2)
    assert bound[0] < 1e-13 and 0.9e-8 < bound[1] < 3e-8
