"""C ABI checks that need no GPU: the library loads, exports every function
declared in include/cglbm.h, and rejects invalid arguments before touching
the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2608_15781_b300 import build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cglbm.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(lbm_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbm.load_library()


def test_header_and_binding_agree():
    assert _declared() == sorted(lbm.SYMBOLS)


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(lbm.LIB_PATH)
    for name in _declared():
        assert hasattr(raw, name), name


def test_strerror(lib):
    for code in (0, -1, -2, -3, -4):
        assert lib.lbm_strerror(code).decode()
    assert "unknown" in lib.lbm_strerror(7).decode()


def test_invalid_arguments_rejected_on_host(lib):
    solid = np.zeros((4, 4, 4), np.uint8)
    for bad in (lbm.Params(tau=0.5), lbm.Params(diffusivity=0.0), lbm.Params(reaction_mode=2),
                lbm.Params(storage=3), lbm.Params(storage=-1), lbm.Params(rho_out=0.0)):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(solid, bad)
        assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(np.ones((3, 3, 3), np.uint8), lbm.Params())      # no fluid node
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(np.zeros((1, 4, 4), np.uint8), lbm.Params(), bc_z=1)   # column needs nz >= 2
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(np.zeros((4, 4, 4), np.uint8), lbm.Params(), bc_z=2)
    # the allocation-free step takes FP32 populations only; checked before any device call
    dummy = ctypes.c_void_p(16)
    for st in (1,):
        prm = lbm.Params(storage=st).to_c()
        assert lib.lbm_step_static(4, 4, 4, dummy, None, dummy, ctypes.c_void_p(1 << 20), None,
                                   ctypes.byref(prm)) == lbm.LBM_EINVAL
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_observables(None, None) == lbm.LBM_EINVAL
    lib.lbm_destroy(None)
