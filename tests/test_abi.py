"""The C-ABI library: it loads, exports every symbol that include/nedner.h
declares, and its host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "nedner.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nedner(?:2d)?_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1510_01078_gb300 import build as b
    b.build()
    from paper_1510_01078_gb300 import nedner
    return nedner.library()


def test_header_and_binding_agree():
    from paper_1510_01078_gb300 import nedner
    assert _declared_symbols() == sorted(nedner.SIGNATURES)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_strerror(lib):
    for st in range(6):
        assert isinstance(lib.nedner_strerror(st), bytes)
    assert b"aperture" in lib.nedner_strerror(2)


def _try_plan(lib, xy, Nt=64, grid=(16, 16, 32, 1e-4, 1e-4, 1e-4), window=(0, 12), sigma=2.0, opts=None):
    from paper_1510_01078_gb300 import nedner
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1, 2))
    g = nedner._Grid(*grid)
    w = nedner._Window(*window)
    handle = ctypes.c_void_p()
    st = lib.nedner_plan(xy.ctypes.data if len(xy) else None, len(xy), Nt, 1e-8, 1500.0, ctypes.byref(g), w,
                         sigma, opts, None, ctypes.byref(handle))
    if st == 0:
        lib.nedner_destroy(handle)
    return st


def test_argument_checks_without_gpu(lib):
    """Bad sizes give EINVAL and off-aperture sensors ERANGE before any CUDA call."""
    xy = [[0.0, 0.0], [1e-4, -2e-4]]
    assert _try_plan(lib, xy, Nt=63) == 1                       # Nt not a power of two
    assert _try_plan(lib, xy, Nt=4) == 1                        # too short
    assert _try_plan(lib, xy, grid=(12, 16, 32, 1e-4, 1e-4, 1e-4)) == 1
    assert _try_plan(lib, xy, grid=(16, 16, 32, -1e-4, 1e-4, 1e-4)) == 1
    assert _try_plan(lib, xy, window=(0, 11)) == 1              # odd width
    assert _try_plan(lib, xy, window=(2, 12)) == 1              # unknown window
    assert _try_plan(lib, xy, sigma=1.5) == 1                   # unsupported oversampling
    X = 16 * 1e-4
    assert _try_plan(lib, [[0.5 * X, 0.0]]) == 2                # on the aperture edge
    assert _try_plan(lib, [[0.0, -0.7 * X]]) == 2
    assert _try_plan(lib, [[np.nan, 0.0]]) == 1
    assert lib.nedner_destroy(None) == 0
    assert lib.nedner_workspace_bytes(None) == 0
