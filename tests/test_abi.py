"""The C ABI library loads and exports every entry point include/*.h declares
(no GPU needed: nothing is called that touches a device)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(minnorm_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__ as g
    g.build()
    from paper_0905_4745_gb300 import minnorm
    return minnorm.LIB_PATH


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("minnorm_plan_create", "minnorm_sketch", "minnorm_solve", "minnorm_plan_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_0905_4745_gb300 import minnorm
    assert sorted(minnorm.EXPORTS) == _declared()
    for n in _declared():
        assert hasattr(minnorm, n) or n == "minnorm_status_string"


def test_status_strings_without_gpu(libpath):
    from paper_0905_4745_gb300 import minnorm
    assert minnorm.status_string(minnorm.OK) == "MINNORM_OK"
    assert "rank" in minnorm.status_string(minnorm.ERANK)


def test_plan_create_validates_before_touching_the_device(libpath):
    # argument checks run before any CUDA call, so they are testable on CPU
    from paper_0905_4745_gb300 import minnorm
    L = minnorm.lib()
    h = ctypes.c_void_p()
    c128 = minnorm.C128
    bad = [(5, 5, 0), (0, 8, 0), (8, 4, 0), (4, 64, 4), (4, 64, 65)]
    for m, n, l in bad:
        st = L.minnorm_plan_create(ctypes.byref(h), m, n, l, c128, 0, 1, 0, None)
        assert st == minnorm.EINVAL, (m, n, l, st)
    # storage kinds: MINNORM_C64 = 1, MINNORM_C128 = 2 (0 and others are invalid)
    assert (minnorm.C64, minnorm.C128) == (1, 2)
    for dt in (0, 3, 7):
        assert L.minnorm_plan_create(ctypes.byref(h), 4, 64, 0, dt, 0, 1, 0, None) == minnorm.EINVAL
    assert L.minnorm_plan_create(ctypes.byref(h), 4, 64, 0, c128, 9, 1, 0, None) == minnorm.EINVAL
    # n above 2^30 is beyond the transform's tables (any other n >= 2, power of two or not, is planned)
    assert L.minnorm_plan_create(ctypes.byref(h), 4, (1 << 30) + 1, 0, c128, 0, 1, 0, None) == minnorm.ENOTSUP
    assert L.minnorm_plan_create(None, 4, 64, 0, c128, 0, 1, 0, None) == minnorm.EINVAL
    assert L.minnorm_plan_export_params(None, *([None] * 8)) == minnorm.EINVAL
    # null plan handles
    assert L.minnorm_sketch(None, None, 64) == minnorm.EINVAL
    assert L.minnorm_solve(None, None, 64, None, 1e-3, None, None) == minnorm.EINVAL
    assert L.minnorm_plan_destroy(None) == minnorm.OK


def test_qr_noalloc_refuses_unaligned_buffers_before_any_launch(libpath):
    # offset views of complex128 / int64 buffers would fault inside the kernels; the entry point
    # returns EINVAL from its argument checks, which run before any CUDA call (so on CPU too)
    from paper_0905_4745_gb300 import minnorm
    L = minnorm.lib()
    good, odd8, odd4 = 0x10000, 0x10008, 0x10004
    l, m = 64, 16
    assert L.minnorm_qr_noalloc(odd8, l, l, m, good, good, None) == minnorm.EINVAL   # Y offset by 8 bytes
    assert L.minnorm_qr_noalloc(good, l, l, m, odd8, good, None) == minnorm.EINVAL   # R offset by 8 bytes
    assert L.minnorm_qr_noalloc(good, l, l, m, good, odd4, None) == minnorm.EINVAL   # pivots offset by 4 bytes
