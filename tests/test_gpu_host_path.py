"""minnorm_solve_host copies A in row blocks on a second stream and sketches each
block as it arrives. Every kernel of Step 1 is row-local, so the solution must
equal the one of minnorm_sketch + minnorm_solve on device buffers with the same
plan seed, including ragged blocks (m not a multiple of the block count, and
fewer rows than blocks) and both storage types and precisions."""
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


@pytest.mark.parametrize("m,n,dtype,prec", [(37, 4096, "c128", 1), (20, 2048, "c64", 1), (5, 1024, "c128", 0),
                                            (64, 8192, "c128", 0)])
def test_host_path_matches_device_path(mn, m, n, dtype, prec):
    import torch
    s = synth.make_system(m, n, exponent=4, seed=900 + m, dtype=dtype)
    cdt = mn.C64 if dtype == "c64" else mn.C128
    dev = torch.device("cuda:0")
    plan = mn.minnorm_plan_create(m, n, 0, cdt, prec, seed=11)
    try:
        A = torch.from_numpy(s.A).to(dev)
        b = torch.from_numpy(s.b).to(dev)
        xd = torch.empty(n, dtype=torch.complex128, device=dev)
        mn.minnorm_sketch(plan, A)
        st_d, _ = mn.minnorm_solve(plan, A, b, 1e-12, xd)
        x_dev = xd.cpu().numpy()
    finally:
        mn.minnorm_plan_destroy(plan)
    plan = mn.minnorm_plan_create(m, n, 0, cdt, prec, seed=11)
    try:
        x_host = np.empty(n, np.complex128)
        st_h, _ = mn.minnorm_solve_host(plan, s.A, s.b, 1e-12, x_host)
        x_host2 = np.empty(n, np.complex128)
        mn.minnorm_solve_host(plan, s.A, s.b, 1e-12, x_host2)      # staging reused
    finally:
        mn.minnorm_plan_destroy(plan)
    assert st_d == st_h == mn.OK
    rel = np.linalg.norm(x_host - x_dev) / np.linalg.norm(x_dev)
    assert rel <= 1e-14, rel
    assert np.linalg.norm(x_host2 - x_dev) / np.linalg.norm(x_dev) <= 1e-14
