"""Pivoted QR parity for sketches longer than 2048 rows, where Step 2 runs the
general kernel (any number of own columns per CTA) instead of the register/shared
tiled one; called through minnorm_qr_noalloc, which takes any Y. Shapes chosen so
that the widest per-CTA column share is 2, 5 and 9 (the 2-, 8- and 16-column
instantiations). Same bar as the other QR tests: equal pivots, R within 1e-12."""
import numpy as np
import pytest

import oracle

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


@pytest.mark.parametrize("l,m", [(2400, 600), (2600, 1300), (2560, 2500)])
def test_general_qr_matches_oracle(mn, l, m):
    import torch
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(l + m)
    # graded columns in shuffled order, so that pivoting reorders them
    Y = (rng.standard_normal((l, m)) + 1j * rng.standard_normal((l, m))) / np.sqrt(2)
    Y *= (10.0 ** (-4.0 * rng.permutation(m) / m))[None, :]
    Yt = torch.from_numpy(np.ascontiguousarray(Y.T)).to(dev)     # column-major l x m
    R = torch.empty((m, m), dtype=torch.complex128, device=dev)    # column-major m x m
    piv = torch.empty(m, dtype=torch.int64, device=dev)
    assert mn.minnorm_qr_noalloc(Yt, l, m, R, piv) == mn.OK
    torch.cuda.synchronize()
    R = R.cpu().numpy().T
    piv = piv.cpu().numpy()
    assert np.array_equal(np.sort(piv), np.arange(m))
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R).imag == 0)
    f = oracle.qrp(Y)
    assert np.array_equal(piv, f.piv)
    assert np.linalg.norm(R - f.R) <= 1e-12 * np.linalg.norm(f.R)
