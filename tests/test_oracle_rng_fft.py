"""Pins for the oracle's random parameters (Section 3) and its DFT (Eq. DFT)."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_splitmix():
    vals = []
    for line in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            vals.append(int(line, 16))
    return vals


def test_splitmix64_published_vector():
    # kind 0 of seed 0 is the published generator's own stream
    for j, v in enumerate(_golden_splitmix()):
        assert oracle.draw(0, 0, j) == v


def test_streams_are_distinct_and_seeded():
    a = [oracle.draw(7, k, 0) for k in range(8)]
    assert len(set(a)) == 8
    assert oracle.draw(7, 0, 0) != oracle.draw(8, 0, 0)


@pytest.mark.parametrize("n,l", [(2, 1), (16, 4), (1000, 37), (4096, 1024)])
def test_params_are_valid(n, l):
    P = oracle.draw_params(n, l, seed=12345)
    for perm in (P.pi, P.pi_t):
        assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.all(np.diff(P.s) > 0) and P.s[0] >= 0 and P.s[-1] < n and P.s.size == l
    for ph in (P.d, P.zeta, P.zeta_t):
        assert np.allclose(np.abs(ph), 1.0, atol=1e-15)
    for th in (P.theta, P.theta_t):
        assert th.size == n - 1
        assert np.all(th >= 0) and np.all(th < 2 * np.pi)


def test_params_distribution():
    # uniform permutations: each position's value is uniform on [0, n)
    n, trials = 8, 4000
    counts = np.zeros((n, n))
    for t in range(trials):
        P = oracle.draw_params(n, 2, seed=t)
        counts[np.arange(n), P.pi] += 1
    expected = trials / n
    chi2 = ((counts - expected) ** 2 / expected).sum()
    # 49 degrees of freedom after the row/column constraints; 99.9% quantile ~ 86
    assert chi2 < 100
    # angles uniform on [0, 2pi): mean pi, phases mean 0
    P = oracle.draw_params(200000, 10, seed=3)
    assert abs(P.theta.mean() - np.pi) < 0.02
    assert abs(P.d.mean()) < 0.01
    # sample without replacement covers [0, n) uniformly
    hits = np.zeros(64)
    for t in range(3000):
        hits[oracle.draw_params(64, 16, seed=10_000 + t).s] += 1
    assert abs(hits.mean() - 3000 * 16 / 64) < 1e-9
    assert hits.min() > 0.8 * 750 and hits.max() < 1.2 * 750


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 8, 12, 16, 17, 60, 64, 97, 100, 128, 243, 1000])
def test_dft_matches_definition(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, +1):
        fast = oracle.dft(x, sign)
        brute = oracle.dft_brute(x, sign)
        assert np.linalg.norm(fast - brute) <= 1e-13 * np.linalg.norm(x) * max(1, np.log2(n))
    # an independent library FFT (numpy's pocketfft)
    assert np.allclose(oracle.dft(x, -1), np.fft.fft(x) / np.sqrt(n), atol=1e-13 * np.linalg.norm(x))


def test_dft_closed_forms():
    n = 48
    # F e_0 is the constant vector n^{-1/2}; F of a pure frequency is a spike
    e0 = np.zeros(n, complex); e0[0] = 1
    assert np.allclose(oracle.dft(e0), np.full(n, n ** -0.5), atol=1e-15)
    k = 5
    wave = np.exp(2j * np.pi * k * np.arange(n) / n)
    spike = oracle.dft(wave)
    expect = np.zeros(n, complex); expect[k] = np.sqrt(n)
    assert np.allclose(spike, expect, atol=1e-12)
    # unitary: Parseval and F^* F = I
    rng = np.random.default_rng(1)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.isclose(np.linalg.norm(oracle.dft(x)), np.linalg.norm(x), rtol=1e-14)
    assert np.allclose(oracle.dft(oracle.dft(x, -1), +1), x, atol=1e-14 * np.linalg.norm(x))
