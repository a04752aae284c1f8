"""The bounded device-side waits run out cleanly. A test hook of the plan makes one CTA of
the next fused CG launch leave without arriving at the grid barrier (a flag no kernel will
ever satisfy); with a 20 ms wait limit the other CTAs give up, wait for their own copies in
flight and return. The solve must report MINNORM_ETIMEOUT (synchronous and asynchronous
forms), the failed plan must refuse further work and still be destroyable, and the CUDA
context must stay usable: a fresh plan then solves to its bound. No fault, trap or endless
wait is involved."""
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


@pytest.mark.parametrize("asynchronous", [False, True])
def test_withheld_arrival_times_out(mn, asynchronous):
    import torch
    m, n = 64, 8192                    # mixed precision, m <= 512: the fused CG kernel
    s = synth.make_system(m, n, exponent=4, seed=77)
    dev = torch.device("cuda:0")
    A = torch.from_numpy(s.A).to(dev)
    b = torch.from_numpy(s.b).to(dev)
    x = torch.empty(n, dtype=torch.complex128, device=dev)
    plan = mn.minnorm_plan_create(m, n, 0, mn.C128, mn.MIXED, seed=4)
    try:
        mn.minnorm_sketch(plan, A)
        with pytest.raises(mn.MinnormError) as e:
            mn.minnorm_plan_set_wait_limit(plan, 1000)          # below 1 ms: refused
        assert e.value.status == mn.EINVAL
        mn.minnorm_plan_set_wait_limit(plan, 20_000_000, withhold=1)
        if asynchronous:
            st = mn.minnorm_solve(plan, A, b, 1e-10, x, info=False)[0]
            assert st == mn.OK                                  # enqueued
            st, _ = mn.minnorm_solve_wait(plan, allow=(mn.ETIMEOUT,))
        else:
            st, _ = mn.minnorm_solve(plan, A, b, 1e-10, x, allow=(mn.ETIMEOUT,))
        assert st == mn.ETIMEOUT
        with pytest.raises(mn.MinnormError) as e:                # the failed plan refuses work
            mn.minnorm_solve(plan, A, b, 1e-10, x)
        assert e.value.status == mn.ESTATE
    finally:
        mn.minnorm_plan_destroy(plan)
    torch.cuda.synchronize()                                     # the context is healthy
    plan = mn.minnorm_plan_create(m, n, 0, mn.C128, mn.MIXED, seed=4)
    try:
        mn.minnorm_sketch(plan, A)
        st, info = mn.minnorm_solve(plan, A, b, 1e-10, x)
    finally:
        mn.minnorm_plan_destroy(plan)
    p = oracle.minnorm_direct(s.A, s.b, steps=4)["p"]
    assert st == mn.OK
    assert np.linalg.norm(x.cpu().numpy() - p) <= 1e-10 * np.linalg.norm(p)
