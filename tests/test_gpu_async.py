"""The asynchronous form of minnorm_solve (info == NULL): the whole refinement loop is
enqueued with its stopping test on the device, so the call makes no host round trip.

Shown two ways: (1) with the stream held busy by a long spin kernel enqueued just before,
the call returns while the stream is still running (a host synchronisation inside it would
have waited for the spin); (2) minnorm_solve_wait then reports the same status, step counts
and bound as the synchronous form, and x is bit for bit the synchronous x (the same kernels
and the same stopping rule, only decided on the device). Both CG forms are covered: the
one-pass fused kernel (m <= 512, mixed) and the two-pass products (m > 512, and FP64)."""
import time

import numpy as np
import pytest

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


def _solve(mn, A, b, prec, eps, dtype, asynchronous, spin=False):
    import torch
    m, n = A.shape
    dev = torch.device("cuda:0")
    plan = mn.minnorm_plan_create(m, n, 0, dtype, prec, seed=8)
    try:
        mn.minnorm_sketch(plan, A)
        x = torch.empty(n, dtype=torch.complex128, device=dev)
        torch.cuda.synchronize()
        if not asynchronous:
            st, info = mn.minnorm_solve(plan, A, b, eps, x)
            return st, info, x.cpu().numpy(), None
        stream = torch.cuda.current_stream()
        if spin:
            torch.cuda._sleep(int(2e9))            # ~1 s of device time ahead of the solve
        t0 = time.perf_counter()
        st = mn.minnorm_solve(plan, A, b, eps, x, info=False)[0]
        t_call = time.perf_counter() - t0
        busy = not stream.query()
        st_wait, info = mn.minnorm_solve_wait(plan, allow=(mn.OK, mn.EFLOOR, mn.ENOCONV))
        assert st == mn.OK
        return st_wait, info, x.cpu().numpy(), (t_call, busy)
    finally:
        mn.minnorm_plan_destroy(plan)


@pytest.mark.parametrize("m,n,prec,dtype", [(96, 8192, 1, "c128"), (600, 8192, 1, "c64"), (96, 4096, 0, "c128")])
def test_async_solve_matches_sync(mn, m, n, prec, dtype):
    import torch
    s = synth.make_system(m, n, exponent=5, seed=5100 + m, dtype=dtype)
    dev = torch.device("cuda:0")
    A = torch.from_numpy(s.A).to(dev)
    b = torch.from_numpy(s.b).to(dev)
    dt = mn.C64 if dtype == "c64" else mn.C128
    st0, info0, x0, _ = _solve(mn, A, b, prec, 1e-10, dt, asynchronous=False)
    st1, info1, x1, (t_call, busy) = _solve(mn, A, b, prec, 1e-10, dt, asynchronous=True, spin=True)
    assert busy, "the asynchronous call waited for its stream"
    assert t_call < 0.5, t_call
    assert st0 == st1 == mn.OK
    assert np.array_equal(x0, x1)
    for k in ("outer_steps", "cg_iters", "status", "err_bound", "cert_delta"):
        assert info0[k] == info1[k], (k, info0, info1)
    assert abs(info0["resid_rel"] - info1["resid_rel"]) <= 1e-12 * info0["resid_rel"]


def test_wait_without_a_pending_solve(mn):
    import torch
    m, n = 8, 256
    s = synth.make_system(m, n, exponent=1, seed=3)
    dev = torch.device("cuda:0")
    plan = mn.minnorm_plan_create(m, n, 0, mn.C128, mn.MIXED, seed=1)
    try:
        with pytest.raises(mn.MinnormError) as e:
            mn.minnorm_solve_wait(plan)
        assert e.value.status == mn.ESTATE
        A = torch.from_numpy(s.A).to(dev)
        mn.minnorm_sketch(plan, A)
        x = torch.empty(n, dtype=torch.complex128, device=dev)
        mn.minnorm_solve(plan, A, torch.from_numpy(s.b).to(dev), 1e-12, x, info=False)
        st, info = mn.minnorm_solve_wait(plan)
        assert st == mn.OK and info["err_bound"] <= 1e-12
        with pytest.raises(mn.MinnormError) as e:      # consumed
            mn.minnorm_solve_wait(plan)
        assert e.value.status == mn.ESTATE
    finally:
        mn.minnorm_plan_destroy(plan)
