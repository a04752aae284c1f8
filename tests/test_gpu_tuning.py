"""The exact residual's work split is chosen by timing candidates on a plan's
first residual. The residual is computed exactly in 128-bit fixed point, so the
tuned split must give the same bits as the default one: checked here on a
system large enough to be tuned, before and after the plan's first solve."""
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


def test_tuned_split_gives_identical_residual(mn):
    import torch
    m, n = 256, 32768
    s = synth.make_system(m, n, exponent=4, seed=77, dtype="c64", device="cuda:0")
    rng = np.random.default_rng(5)
    y = torch.from_numpy(rng.standard_normal(m) + 1j * rng.standard_normal(m)).to("cuda:0")
    y_lo = torch.zeros_like(y)
    outs = []
    plan = mn.minnorm_plan_create(m, n, 0, mn.C64, mn.MIXED, seed=4)
    try:
        c0, r0, k0, tuned0 = mn.minnorm_plan_tuning(plan)
        assert not tuned0
        for stage in range(2):
            r = torch.empty(m, dtype=torch.complex128, device="cuda:0")
            xh = torch.empty(n, dtype=torch.complex128, device="cuda:0")
            xl = torch.empty(n, dtype=torch.complex128, device="cuda:0")
            mn.minnorm_residual_dd(plan, s.A, y, y_lo, s.b, r, xh, xl)
            torch.cuda.synchronize()
            outs.append((r.cpu().numpy(), xh.cpu().numpy(), xl.cpu().numpy()))
            if stage == 0:   # a solve runs the first residual of the plan: the split is tuned there
                mn.minnorm_sketch(plan, s.A)
                x = torch.empty(n, dtype=torch.complex128, device="cuda:0")
                st, info = mn.minnorm_solve(plan, s.A, s.b, 1e-10, x)
                assert st == mn.OK
        c1, r1, k1, tuned1 = mn.minnorm_plan_tuning(plan)
        assert tuned1 and c1 >= 1 and r1 >= 1 and 0 <= k1 <= 100
    finally:
        mn.minnorm_plan_destroy(plan)
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
