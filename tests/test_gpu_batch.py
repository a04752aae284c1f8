"""GPU parity of the batch entry points (minnorm_batch_*): independent systems of uneven
m and n = m k (mostly not powers of two, so the sketch runs Bluestein's transform),
complex64 storage, singular values 1 .. 1e-4, eps = 1e-10 -- the batching workload.

Small batches are checked system by system against the oracle's p and against a
standalone plan with the same SRFT seed. The full workload (256 systems, m in
[32, 512], k in [8, 64]) is too large for the oracle on every system; there each
system must return OK with its a-posteriori bound <= eps, its residual b - A x
(computed by torch in complex128, independent of the library) must be within
eps ||x|| plus the rounding bound of that product, and a sample of systems is
compared with the oracle."""
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


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,dtype", [(1, "c64"), (0, "c128")])
def test_batch_small_matches_oracle(mn, prec, dtype):
    import torch
    shapes = [(m, m * k) for m, k in ((8, 9), (33, 8), (17, 64), (40, 13), (64, 16), (21, 50), (5, 11))]
    systems = [synth.make_system(m, n, exponent=4, seed=4100 + i, dtype=dtype) for i, (m, n) in enumerate(shapes)]
    cdt = mn.C64 if dtype == "c64" else mn.C128
    batch = mn.minnorm_batch_create([m for m, _ in shapes], [n for _, n in shapes], cdt, prec, seed=40)
    try:
        As = [_t(s.A) for s in systems]
        bs = [_t(s.b) for s in systems]
        xs = [torch.empty(n, dtype=torch.complex128, device=_dev()) for _, n in shapes]
        st, infos = mn.minnorm_batch_solve(batch, As, bs, 1e-10, xs)
        torch.cuda.synchronize()
        assert st == mn.OK, infos
        for i, s in enumerate(systems):
            assert infos[i]["status"] == mn.OK
            p = oracle.minnorm_direct(s.A.astype(np.complex128), s.b, steps=5)["p"]
            assert _rel(xs[i].cpu().numpy(), p) <= 1e-10, (i, shapes[i], infos[i])
        # system i is the system a plan with SRFT seed 40 + i solves
        for i in (0, 3, 6):
            m, n = shapes[i]
            plan = mn.minnorm_plan_create(m, n, 0, cdt, prec, seed=40 + i)
            try:
                mn.minnorm_sketch(plan, As[i])
                x = torch.empty(n, dtype=torch.complex128, device=_dev())
                mn.minnorm_solve(plan, As[i], bs[i], 1e-10, x)
                torch.cuda.synchronize()
            finally:
                mn.minnorm_plan_destroy(plan)
            assert _rel(xs[i].cpu().numpy(), x.cpu().numpy()) <= 1e-14
    finally:
        mn.minnorm_batch_destroy(batch)


def test_batch_statuses_and_errors(mn):
    import torch
    L = mn.lib()
    import ctypes
    h = ctypes.c_void_p()
    ms = (ctypes.c_int64 * 2)(8, 16)
    bad = (ctypes.c_int64 * 2)(64, 16)                   # m >= n for the second system
    assert L.minnorm_batch_create(ctypes.byref(h), 2, ms, bad, mn.C128, 0, 1, 0, None) == mn.EINVAL
    assert L.minnorm_batch_create(ctypes.byref(h), 0, ms, bad, mn.C128, 0, 1, 0, None) == mn.EINVAL
    # a rank-deficient system is reported in its own info and does not stop the others
    shapes = [(8, 100), (6, 90), (10, 120)]
    systems = [synth.make_system(m, n, exponent=2, seed=4200 + i) for i, (m, n) in enumerate(shapes)]
    A1 = systems[1].A.copy()
    A1[4] = A1[1]
    batch = mn.minnorm_batch_create([m for m, _ in shapes], [n for _, n in shapes], mn.C128, mn.MIXED, seed=3)
    try:
        As = [_t(systems[0].A), _t(A1), _t(systems[2].A)]
        bs = [_t(s.b) for s in systems]
        xs = [torch.empty(n, dtype=torch.complex128, device=_dev()) for _, n in shapes]
        st, infos = mn.minnorm_batch_solve(batch, As, bs, 1e-12, xs, allow=(mn.ERANK,))
        torch.cuda.synchronize()
        assert st == mn.ERANK
        assert [i["status"] for i in infos] == [mn.OK, mn.ERANK, mn.OK]
        for i in (0, 2):
            p = oracle.minnorm_direct(systems[i].A, systems[i].b, steps=4)["p"]
            assert _rel(xs[i].cpu().numpy(), p) <= 1e-12
        with pytest.raises(mn.MinnormError):
            mn.minnorm_batch_solve(batch, As, bs, 0.0, xs)
    finally:
        mn.minnorm_batch_destroy(batch)


def test_batch_full_workload(mn):
    # 256 systems: m uniform in [32, 512], n = m k with k uniform in [8, 64] (seed 4000),
    # system i built with seed 4000 + i, complex64 storage, singular values 1 .. 1e-4
    import torch
    shapes = synth.batch_shapes(256, seed=4000)
    systems = [synth.make_system(m, n, exponent=4, seed=4000 + i, dtype="c64", device="cuda")
               for i, (m, n) in enumerate(shapes)]
    batch = mn.minnorm_batch_create([m for m, _ in shapes], [n for _, n in shapes], mn.C64, mn.MIXED, seed=4000)
    try:
        xs = [torch.empty(n, dtype=torch.complex128, device=_dev()) for _, n in shapes]
        st, infos = mn.minnorm_batch_solve(batch, [s.A for s in systems], [s.b for s in systems], 1e-10, xs)
        torch.cuda.synchronize()
        assert st == mn.OK
        for i, s in enumerate(systems):
            assert infos[i]["status"] == mn.OK and infos[i]["err_bound"] <= 1e-10, (i, infos[i])
            # ||A (x - p)|| <= sigma_max ||x - p|| <= eps ||p|| (sigma_max = 1 up to the storage
            # rounding), plus the rounding of torch's own product: n u || |A| |x| ||
            A64 = s.A.to(torch.complex128)
            r = s.b - A64 @ xs[i]
            n = A64.shape[1]
            round_bound = 2.0 * n * 2.0 ** -53 * float(torch.linalg.norm(A64.abs() @ xs[i].abs()))
            assert float(torch.linalg.norm(r)) <= 1.01e-10 * float(torch.linalg.norm(xs[i])) + round_bound, i
        # the oracle on a sample: the three smallest systems and one large one
        order = sorted(range(len(shapes)), key=lambda i: shapes[i][0] * shapes[i][1])
        for i in order[:3] + [order[len(order) // 2]]:
            A = systems[i].A.cpu().numpy().astype(np.complex128)
            p = oracle.minnorm_direct(A, systems[i].b.cpu().numpy(), steps=5)["p"]
            assert _rel(xs[i].cpu().numpy(), p) <= 1e-10, (i, shapes[i])
    finally:
        mn.minnorm_batch_destroy(batch)
