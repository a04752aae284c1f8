"""The allocation-free pivoted QR (minnorm_qr_noalloc) against the plan's QR.

minnorm_qr_noalloc serves callers that cannot allocate device memory: it runs
the same pivoted Householder QR kernel as minnorm_sketch, with its scratch in a
fixed array inside the library instead of plan workspace. Two calls in a row,
on two different sketches, must each reproduce what the plan path
(minnorm_sketch + minnorm_get_factor) gives for the same matrix: the same
pivots and R within the QR parity tolerance of the other tests (1e-12
relative). The calls run a larger system, then a smaller one, then the larger
one again, so a smaller call meets the flags, posts and partial norms a larger
call left in the shared scratch (each call must clear what has to start at
zero); one call is enqueued on a side stream instead of the current one.
This file is collected last on purpose.
"""
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


def _plan_factor(mn, A, m, n, seed):
    """Sketch through a plan and return (Y, R, piv) of the existing entry points."""
    import torch
    dev = torch.device("cuda:0")
    l = 4 * m
    plan = mn.minnorm_plan_create(m, n, 0, mn.C128, mn.FP64, seed=seed, flags=mn.FLAG_KEEP_SKETCH)
    try:
        mn.minnorm_sketch(plan, A)
        Y = torch.empty((m, l), dtype=torch.complex128, device=dev)   # column i of Y = row i here
        R = torch.empty((m, m), dtype=torch.complex128, device=dev)
        piv = torch.empty(m, dtype=torch.int64, device=dev)
        mn.minnorm_get_sketch(plan, Y)
        mn.minnorm_get_factor(plan, R, piv)
        torch.cuda.synchronize()
    finally:
        mn.minnorm_plan_destroy(plan)
    return Y, R, piv


def test_qr_noalloc_matches_plan_path_twice(mn):
    import torch
    dev = torch.device("cuda:0")
    side = torch.cuda.Stream(device=dev)
    cases = [(200, 2048, 6, None), (48, 4096, 5, side), (200, 2048, 7, None)]
    for m, n, seed, stream in cases:               # calls in a row: large, small, large
        s = synth.make_system(m, n, exponent=2, seed=900 + m)
        A = torch.from_numpy(s.A).to(dev)
        Y, R_ref, piv_ref = _plan_factor(mn, A, m, n, seed)
        Yw = Y.clone()                              # overwritten by the call
        R = torch.full((m, m), complex(np.nan, np.nan), dtype=torch.complex128, device=dev)
        piv = torch.full((m,), -1, dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        st = mn.minnorm_qr_noalloc(Yw, 4 * m, m, R, piv, stream=stream)
        torch.cuda.synchronize()
        assert st == mn.OK
        assert torch.equal(piv, piv_ref)
        R, R_ref = R.cpu().numpy(), R_ref.cpu().numpy()
        assert np.linalg.norm(R - R_ref) <= 1e-12 * np.linalg.norm(R_ref)


def test_qr_noalloc_rejects_sizes_beyond_its_scratch(mn):
    import torch
    dev = torch.device("cuda:0")
    Y = torch.zeros(8, dtype=torch.complex128, device=dev)
    with pytest.raises(mn.MinnormError) as e:
        mn.minnorm_qr_noalloc(Y, 5000, 4097, Y, Y)
    assert e.value.status == mn.ENOTSUP
    with pytest.raises(mn.MinnormError) as e:
        mn.minnorm_qr_noalloc(Y, 3, 4, Y, Y)          # l < m
    assert e.value.status == mn.EINVAL
