"""GPU parity: every step of the hot path, called through the C ABI, against the
CPU oracle on the same seeded inputs.

Tolerances:
  - FP64 sketch: 1e-12 relative (Frobenius and per element, relative to the largest
    entry), the bound the solver's specification sets for Step 1.
  - double-word sketch (mixed precision): (20 + 6 log2 n) 2^-46 relative. Per
    element the transform is ~16 double-word operations in the two Givens chains
    and phases plus at most 6 per radix-2 stage of the FFT, each within 2^-46
    relative (products) or 2^-47 of its operands (sums); ~2e-12 at n = 65536.
  - products: FP64 1e-13 relative; FP32 products of a complex64 A (exact inputs)
    are within ~sqrt(k) u32 of the FP64 result: 2e-6 relative for the configs here.
  - solves: the requested eps against the oracle's double-double-refined p.
"""
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


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(_dev())


def _plan(mn, m, n, prec, seed, dtype=None, flags=0, l=0):
    dtype = mn.C128 if dtype is None else dtype
    return mn.minnorm_plan_create(m, n, l, dtype, prec, seed=seed, flags=flags)


def _sketch(mn, plan, A, m, l):
    import torch
    mn.minnorm_sketch(plan, A, allow=(mn.OK, mn.ERANK))
    Y = torch.empty((m, l), dtype=torch.complex128, device=_dev())
    mn.minnorm_get_sketch(plan, Y)
    torch.cuda.synchronize()
    return Y.cpu().numpy().T


def _factor(mn, plan, m):
    import torch
    R = torch.empty((m, m), dtype=torch.complex128, device=_dev())
    piv = torch.empty(m, dtype=torch.int64, device=_dev())
    mn.minnorm_get_factor(plan, R, piv)
    torch.cuda.synchronize()
    return R.cpu().numpy().T, piv.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------- Step 1 ----
@pytest.mark.parametrize("m,n", [(8, 1024), (5, 4096), (12, 8192), (3, 65536), (7, 2)])
def test_sketch_fp64_matches_oracle(mn, m, n):
    if m >= n:
        m = n - 1
    s = synth.make_system(m, n, exponent=2, seed=100 + n)
    l = min(4 * m, n)
    plan = _plan(mn, m, n, mn.FP64, seed=11, flags=mn.FLAG_KEEP_SKETCH)
    try:
        Y = _sketch(mn, plan, _t(s.A), m, l)
    finally:
        mn.minnorm_plan_destroy(plan)
    Yref = oracle.sketch(oracle.draw_params(n, l, 11), s.A)
    assert _rel(Y, Yref) <= 1e-12
    assert np.abs(Y - Yref).max() <= 1e-12 * np.abs(Yref).max()


@pytest.mark.parametrize("m,n", [(6, 2048), (9, 16384), (4, 131072)])
def test_sketch_fp64_complex64_storage(mn, m, n):
    s = synth.make_system(m, n, exponent=2, seed=200 + n, dtype="c64")
    l = 4 * m
    plan = _plan(mn, m, n, mn.FP64, seed=5, dtype=mn.C64, flags=mn.FLAG_KEEP_SKETCH)
    try:
        Y = _sketch(mn, plan, _t(s.A), m, l)
    finally:
        mn.minnorm_plan_destroy(plan)
    Yref = oracle.sketch(oracle.draw_params(n, l, 5), s.A.astype(np.complex128))
    assert _rel(Y, Yref) <= 1e-12


def dw_sketch_tol(n):
    """Relative tolerance of a double-word sketch of a length-n (power of two) row."""
    return (20 + 6 * np.log2(n)) * 2.0 ** -46


@pytest.mark.parametrize("m,n", [(8, 1024), (10, 16384), (3, 65536)])
def test_sketch_dw_matches_oracle(mn, m, n):
    s = synth.make_system(m, n, exponent=2, seed=300 + n)
    l = 4 * m
    plan = _plan(mn, m, n, mn.MIXED, seed=21, flags=mn.FLAG_KEEP_SKETCH)
    try:
        Y = _sketch(mn, plan, _t(s.A), m, l)
    finally:
        mn.minnorm_plan_destroy(plan)
    Yref = oracle.sketch(oracle.draw_params(n, l, 21), s.A)
    assert _rel(Y, Yref) <= dw_sketch_tol(n)
    assert np.abs(Y - Yref).max() <= dw_sketch_tol(n) * np.abs(Yref).max()


def test_export_params_round_trip(mn):
    # the exported realization is the one the plan drew (the oracle's streams for the same seed),
    # setting it back leaves the sketch bit for bit unchanged, and the oracle ingests it
    m, n = 5, 2048
    l = 4 * m
    s = synth.make_system(m, n, exponent=1, seed=5)
    plan = _plan(mn, m, n, mn.FP64, seed=29, flags=mn.FLAG_KEEP_SKETCH)
    try:
        E = mn.minnorm_plan_export_params(plan, n, l)
        P = oracle.draw_params(n, l, 29)
        for got, want in zip(E, (P.zeta_t, P.pi_t, P.theta_t, P.zeta, P.pi, P.theta, P.d, P.s)):
            assert got.shape == want.shape
            if got.dtype == np.int64:
                assert np.array_equal(got, want)
            else:      # phases and angles: libm on either side, within an ulp or two
                assert np.max(np.abs(got - want)) <= 1e-15 * max(1.0, np.max(np.abs(want)))
        Y0 = _sketch(mn, plan, _t(s.A), m, l)
        mn.minnorm_plan_set_params(plan, *E)
        Y1 = _sketch(mn, plan, _t(s.A), m, l)
        assert np.array_equal(Y0, Y1)
        assert _rel(Y1, oracle.sketch(oracle.Params(n, l, *E), s.A)) <= 1e-12
    finally:
        mn.minnorm_plan_destroy(plan)


def test_sketch_with_injected_parameters(mn):
    # the same plan with parameters set from the oracle's streams of another seed,
    # and with a degenerate transform (no H): both must match the oracle's T
    m, n = 6, 4096
    l = 4 * m
    s = synth.make_system(m, n, exponent=1, seed=4)
    plan = _plan(mn, m, n, mn.FP64, seed=1, flags=mn.FLAG_KEEP_SKETCH)
    try:
        P = oracle.draw_params(n, l, 777)
        mn.minnorm_plan_set_params(plan, P.zeta_t, P.pi_t, P.theta_t, P.zeta, P.pi, P.theta, P.d, P.s)
        Y = _sketch(mn, plan, _t(s.A), m, l)
        assert _rel(Y, oracle.sketch(P, s.A)) <= 1e-12
        Q = oracle.Params(n, l, np.ones(n), np.arange(n), np.zeros(n - 1), np.ones(n), np.arange(n),
                          np.zeros(n - 1), P.d, P.s)
        mn.minnorm_plan_set_params(plan, Q.zeta_t, Q.pi_t, Q.theta_t, Q.zeta, Q.pi, Q.theta, Q.d, Q.s)
        Y2 = _sketch(mn, plan, _t(s.A), m, l)
        # no H: column i of Y is the subsampled unitary FFT of d * conj(a_i)
        ref = (np.fft.fft(P.d[None, :] * s.A.conj(), axis=1) / np.sqrt(n))[:, P.s].T
        assert _rel(Y2, ref) <= 1e-12
        bad_pi = P.pi.copy()
        bad_pi[0] = bad_pi[1]
        with pytest.raises(mn.MinnormError):
            mn.minnorm_plan_set_params(plan, P.zeta_t, P.pi_t, P.theta_t, P.zeta, bad_pi, P.theta, P.d, P.s)
    finally:
        mn.minnorm_plan_destroy(plan)


# ---------------------------------------------------------------- Step 2 ----
@pytest.mark.parametrize("m,n,prec", [(16, 1024, 0), (48, 4096, 0), (200, 2048, 0), (40, 8192, 1)])
def test_pivoted_qr_matches_oracle(mn, m, n, prec):
    s = synth.make_system(m, n, exponent=2, seed=400 + m)
    l = 4 * m
    plan = _plan(mn, m, n, prec, seed=31, flags=mn.FLAG_KEEP_SKETCH)
    try:
        Y = _sketch(mn, plan, _t(s.A), m, l)
        R, piv = _factor(mn, plan, m)
    finally:
        mn.minnorm_plan_destroy(plan)
    # invariants of Y P = Q R on the GPU's own sketch
    assert np.array_equal(np.sort(piv), np.arange(m))
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R).imag == 0)
    d = np.abs(np.diag(R))
    assert np.all(d[:-1] >= d[1:] * (1 - 1e-10))
    G = Y[:, piv].conj().T @ Y[:, piv]
    assert np.linalg.norm(R.conj().T @ R - G) <= 1e-13 * np.linalg.norm(G)
    # against the oracle's QR of the same sketch
    f = oracle.qrp(Y)
    assert np.array_equal(piv, f.piv)
    assert _rel(R, f.R) <= 1e-12


@pytest.mark.parametrize("m,n,prec,dtype", [(64, 1024, 1, "c128"), (64, 1024, 0, "c128"), (48, 4096, 1, "c64")])
def test_certificate_premise(mn, m, n, prec, dtype):
    # the error bound divides by 1 - delta on the premise sigma_min(A^* P R^{-1}) >= 1 - delta for
    # the R of the GPU's own sketch and QR; check it with the singular values of A^* P R^{-1}
    # formed on the host, and the Frobenius norms the library reports
    import torch
    s = synth.make_system(m, n, exponent=5, seed=4400 + m, dtype=dtype)
    A = _t(s.A)
    plan = _plan(mn, m, n, prec, seed=19, dtype=mn.C64 if dtype == "c64" else mn.C128)
    try:
        mn.minnorm_sketch(plan, A)
        R, piv = _factor(mn, plan, m)
        x = torch.empty(n, dtype=torch.complex128, device=_dev())
        st, info = mn.minnorm_solve(plan, A, _t(s.b), 1e-10, x)
    finally:
        mn.minnorm_plan_destroy(plan)
    A64 = s.A.astype(np.complex128)
    W = np.zeros((m, m), np.complex128)
    W[piv, :] = np.linalg.inv(R)                       # P R^{-1}: row piv[k] of W is row k of R^{-1}
    sv = np.linalg.svd(A64.conj().T @ W, compute_uv=False)
    delta = info["cert_delta"]
    assert 0.0 < delta < 1e-3, info
    assert sv.min() >= 1.0 - delta, (sv.min(), delta)
    assert info["sigma_max_R"] >= np.linalg.norm(R, 2)
    assert info["sigma_min_R"] <= np.linalg.svd(R, compute_uv=False).min()
    assert abs(info["sigma_min_R"] * np.linalg.norm(np.linalg.inv(R)) - 1.0) <= 1e-9


# ---------------------------------------------------------------- Step 4 ----
# pad: row stride n + pad. The complex64 forward product reads two entries per 16-byte load only
# for an even stride and column count; odd ones (pad 1 or 3, n = 3001) take the 8-byte form.
# m = 700 leaves a ragged last block of rows (8 per CTA).
@pytest.mark.parametrize("m,n,prec,dtype,pad", [(32, 4096, 0, "c128", 0), (64, 65536, 0, "c128", 0),
                                                (17, 8192, 1, "c128", 0), (96, 16384, 1, "c64", 0),
                                                (40, 8192, 0, "c64", 0), (96, 16384, 1, "c64", 1),
                                                (40, 8192, 0, "c64", 3), (700, 8192, 1, "c64", 0),
                                                (21, 3001, 1, "c64", 0)])
def test_cg_products_match_oracle(mn, m, n, prec, dtype, pad):
    import torch
    s = synth.make_system(m, n, exponent=3, seed=500 + m, dtype=dtype)
    A64 = s.A.astype(np.complex128)
    rng = np.random.default_rng(m)
    w = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    plan = _plan(mn, m, n, prec, seed=2, dtype=mn.C64 if dtype == "c64" else mn.C128)
    try:
        Ap = np.zeros((m, n + pad), s.A.dtype)
        Ap[:, :n] = s.A
        A = _t(Ap)
        mn.minnorm_sketch(plan, A)
        q = torch.empty(n, dtype=torch.complex128, device=_dev())
        t = torch.empty(m, dtype=torch.complex128, device=_dev())
        mn.minnorm_cg_products(plan, A, _t(w), q, t)
        torch.cuda.synchronize()
        q, t = q.cpu().numpy(), t.cpu().numpy()
    finally:
        mn.minnorm_plan_destroy(plan)
    qref = oracle.adj_matvec(A64, w)
    tol = 1e-13 if prec == 0 else 2e-6
    if prec == 1 and dtype == "c128":
        tol = 4e-6                     # A rounded to complex64 first
    assert _rel(q, qref) <= tol
    assert _rel(t, oracle.matvec(A64, q)) <= tol


# The mixed CG's one-pass product for 512 < m <= 4096 (clusters of ceil(m / 512) CTAs, the
# partial q of each CTA's rows added through distributed shared memory): t = A (A^* w) against the
# oracle's FP64 products. Its FP32 sums run over at most a few thousand terms per thread, so the
# error is held to 2e-5 of |A| (|A|^H |w|), the scale of every rounding in them; a lost sub-panel,
# row block or rank would be off by O(1) of it. Cluster sizes 2, 3 and 4 with ragged row blocks
# (700 = 512 + 188, 1100 = 2 x 512 + 76), and a ragged last 16-column sub-panel (n = 8200).
@pytest.mark.parametrize("m,n", [(700, 8192), (1100, 16384), (2048, 8200)])
def test_cg_one_pass_product_matches_oracle(mn, m, n):
    import torch
    s = synth.make_system(m, n, exponent=3, seed=900 + m, dtype="c64")
    A64 = s.A.astype(np.complex128)
    rng = np.random.default_rng(m)
    w = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    plan = _plan(mn, m, n, 1, seed=2, dtype=mn.C64)
    try:
        A = _t(s.A)
        mn.minnorm_sketch(plan, A)
        t = torch.empty(m, dtype=torch.complex128, device=_dev())
        mn.minnorm_cg_products(plan, A, _t(w), None, t)
        torch.cuda.synchronize()
        t = t.cpu().numpy()
    finally:
        mn.minnorm_plan_destroy(plan)
    w32 = w.astype(np.complex64).astype(np.complex128)      # the kernel's w is complex64
    tref = oracle.matvec(A64, oracle.adj_matvec(A64, w32))
    scale = np.abs(A64) @ (np.abs(A64).T @ np.abs(w32))
    assert np.linalg.norm(t - tref) <= 2e-5 * np.linalg.norm(scale), (np.linalg.norm(t - tref), np.linalg.norm(scale))


@pytest.mark.parametrize("m,n,dtype", [(24, 4096, "c128"), (128, 65536, "c128"), (50, 8192, "c64")])
def test_residual_dd_matches_oracle(mn, m, n, dtype):
    import torch
    s = synth.make_system(m, n, exponent=6, seed=600 + m, dtype=dtype)
    A64 = s.A.astype(np.complex128)
    y = oracle.minnorm_direct(A64, s.b, steps=1)["y"]        # large entries: strong cancellation
    rng = np.random.default_rng(1)
    y_lo = (rng.standard_normal(m) + 1j * rng.standard_normal(m)) * np.abs(y) * 2.0 ** -60
    r_ref, xh_ref, xl_ref = oracle.residual_dd(A64, y, y_lo, s.b)
    plan = _plan(mn, m, n, 0, seed=2, dtype=mn.C64 if dtype == "c64" else mn.C128)
    try:
        A = _t(s.A)
        r = torch.empty(m, dtype=torch.complex128, device=_dev())
        xh = torch.empty(n, dtype=torch.complex128, device=_dev())
        xl = torch.empty(n, dtype=torch.complex128, device=_dev())
        mn.minnorm_residual_dd(plan, A, _t(y), _t(y_lo), _t(s.b), r, xh, xl)
        torch.cuda.synchronize()
        r, xh, xl = r.cpu().numpy(), xh.cpu().numpy(), xl.cpu().numpy()
    finally:
        mn.minnorm_plan_destroy(plan)
    absA = np.abs(A64)
    ay = np.abs(y) + np.abs(y_lo)
    xmag = absA.T @ ay
    rmag = absA @ xmag + np.abs(s.b)
    # the library holds A in 62-bit fixed point per row: exact for complex64, and for
    # complex128 a component more than 2^9 below its row's largest is rounded at
    # 2^(E_i - 62); dA is that representation error, computed exactly here
    E = np.frexp(np.maximum(np.abs(A64.real), np.abs(A64.imag)).max(axis=1))[1]
    k = (62 - E)[:, None].astype(float)
    dA = (A64.real - np.rint(np.ldexp(A64.real, k.astype(int))) * np.ldexp(1.0, -k.astype(int))) + \
        1j * (A64.imag - np.rint(np.ldexp(A64.imag, k.astype(int))) * np.ldexp(1.0, -k.astype(int)))
    if dtype == "c64":
        assert np.all(dA == 0)
    bx = 1.001 * (np.abs(dA).T @ ay)          # tight when a column has one rounded entry
    br = 1.001 * (np.abs(dA) @ np.abs(xh_ref) + absA @ bx)
    dx = (xh - xh_ref) + (xl - xl_ref)          # double-double difference, not rounded sums
    assert np.all(np.abs(dx) <= bx + 2.0 ** -100 * 8 * m * xmag + 2.0 ** -104 * np.abs(xh_ref))
    assert np.all(np.abs(r - r_ref) <= br + 2.0 ** -98 * 8 * n * rmag + 2.0 ** -52 * np.abs(r_ref))


# --------------------------------------------------------------- Steps 1-5 --
def _solve(mn, s, prec, eps, seed=3, dtype=None):
    import torch
    m, n = s.A.shape
    plan = _plan(mn, m, n, prec, seed=seed, dtype=dtype)
    try:
        A = _t(s.A)
        mn.minnorm_sketch(plan, A)
        x = torch.empty(n, dtype=torch.complex128, device=_dev())
        st, info = mn.minnorm_solve(plan, A, _t(s.b), eps, x, allow=(mn.OK, mn.EFLOOR, mn.ENOCONV))
        torch.cuda.synchronize()
        return st, info, x.cpu().numpy()
    finally:
        mn.minnorm_plan_destroy(plan)


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_small_plain_workload(mn, prec):
    # m = 64, n = 1024, singular values 1 .. 1e-3, eps = 1e-12
    s = synth.make_system(64, 1024, exponent=3, seed=1001)
    p = oracle.minnorm_direct(s.A, s.b, steps=4)["p"]
    st, info, x = _solve(mn, s, prec, 1e-12)
    assert st == mn.OK, info
    assert _rel(x, p) <= 1e-12
    assert info["err_bound"] <= 1e-12


@pytest.mark.parametrize("m,n,prec", [(128, 8192, 0), (128, 8192, 1), (256, 4096, 1), (33, 16384, 0)])
def test_solve_kappa_1e6(mn, m, n, prec):
    s = synth.make_system(m, n, exponent=6, seed=7000 + m)
    p = oracle.minnorm_direct(s.A, s.b, steps=6)["p"]
    st, info, x = _solve(mn, s, prec, 1e-12)
    assert st == mn.OK, info
    assert _rel(x, p) <= 1e-12, info


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_complex64_storage(mn, prec):
    s = synth.make_system(100, 16384, exponent=5, seed=3003, dtype="c64")
    p = oracle.minnorm_direct(s.A.astype(np.complex128), s.b, steps=6)["p"]
    st, info, x = _solve(mn, s, prec, 1e-10, dtype=mn.C64)
    assert st == mn.OK, info
    assert _rel(x, p) <= 1e-10


def test_solve_paper_right_hand_side(mn):
    # the paper's workload (Section 7): kappa = 1e6, b = A p, p = sum eps_j v_j / sqrt(m)
    s = synth.make_system(128, 4096, exponent=6, seed=2009, rhs="paper")
    p = oracle.minnorm_direct(s.A, s.b, steps=6)["p"]
    st, info, x = _solve(mn, s, 1, 1e-12)
    assert st == mn.OK
    assert _rel(x, p) <= 1e-12


def test_solve_edge_shapes(mn):
    # m = 1 (l = 4), and l = n for a tiny system
    for m, n in ((1, 64), (3, 8), (2, 4)):
        s = synth.make_system(m, n, exponent=1, seed=m * 100 + n)
        p = oracle.minnorm_direct(s.A, s.b, steps=3)["p"]
        for prec in (0, 1):
            st, info, x = _solve(mn, s, prec, 1e-12)
            assert st == mn.OK and _rel(x, p) <= 1e-12, (m, n, prec, info)


def test_error_paths(mn):
    import torch
    s = synth.make_system(8, 256, exponent=1, seed=1)
    A = _t(s.A)
    x = torch.empty(256, dtype=torch.complex128, device=_dev())
    plan = _plan(mn, 8, 256, 0, seed=1)
    try:
        with pytest.raises(mn.MinnormError) as e:          # solve before sketch
            mn.minnorm_solve(plan, A, _t(s.b), 1e-10, x)
        assert e.value.status == mn.ESTATE
        mn.minnorm_sketch(plan, A)
        for eps in (0.0, 1.0, -1.0):
            with pytest.raises(mn.MinnormError) as e:
                mn.minnorm_solve(plan, A, _t(s.b), eps, x)
            assert e.value.status == mn.EINVAL
        with pytest.raises(mn.MinnormError):
            mn.minnorm_sketch(plan, A, lda=100)
        # rank deficiency (Remark 4.1): two equal rows
        B = s.A.copy()
        B[5] = B[2]
        assert mn.minnorm_sketch(plan, _t(B), allow=(mn.OK, mn.ERANK)) == mn.ERANK
    finally:
        mn.minnorm_plan_destroy(plan)


def test_solve_host_buffers(mn):
    s = synth.make_system(32, 2048, exponent=4, seed=77)
    p = oracle.minnorm_direct(s.A, s.b, steps=4)["p"]
    plan = _plan(mn, 32, 2048, 1, seed=9)
    try:
        x = np.empty(2048, np.complex128)
        st, info = mn.minnorm_solve_host(plan, s.A, s.b, 1e-12, x)
        assert st == mn.OK
        assert _rel(x, p) <= 1e-12
        st, info = mn.minnorm_solve_host(plan, s.A, s.b, 1e-12, x)   # second call reuses staging
        assert _rel(x, p) <= 1e-12
    finally:
        mn.minnorm_plan_destroy(plan)


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_plain_workload(mn, prec):
    # the 512 x 65536 complex128 workload with singular values 1 .. 1e-6 and eps = 1e-12,
    # in the launch configuration the benchmark times; sampled rows of the sketch and the
    # whole solution against the oracle
    import torch
    m, n, eps = 512, 65536, 1e-12
    s = synth.make_system(m, n, exponent=6, seed=1002, device="cuda:0")
    A, b = s.A, s.b
    A_np, b_np = A.cpu().numpy(), b.cpu().numpy()
    l = 4 * m
    plan = _plan(mn, m, n, prec, seed=1, flags=mn.FLAG_KEEP_SKETCH)
    try:
        st = mn.minnorm_sketch(plan, A)
        Y = torch.empty((m, l), dtype=torch.complex128, device=_dev())
        mn.minnorm_get_sketch(plan, Y)
        x = torch.empty(n, dtype=torch.complex128, device=_dev())
        st, info = mn.minnorm_solve(plan, A, b, eps, x)
        torch.cuda.synchronize()
        Y, x = Y.cpu().numpy().T, x.cpu().numpy()
    finally:
        mn.minnorm_plan_destroy(plan)
    P = oracle.draw_params(n, l, 1)
    rows = [0, 1, 255, 511]
    Yref = np.stack([oracle.srft_apply(P, A_np[i].conj()) for i in rows], axis=1)
    tol = 1e-12 if prec == 0 else dw_sketch_tol(n)
    assert _rel(Y[:, rows], Yref) <= tol
    ref = oracle.minnorm_direct(A_np, b_np, steps=5)["p"]
    assert st == mn.OK
    assert _rel(x, ref) <= eps, info
