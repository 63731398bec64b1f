"""The C-ABI library loads and exports every symbol include/lbm.h declares, and its host-side
argument checks reject bad calls before touching a GPU (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2010_11751_b300 import build
    from paper_2010_11751_b300 import lbm
    build.build()
    return lbm


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(r"LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = _declared("lbm.h")
    assert "lbm_create" in names and "lbm_step" in names and "lbm_macroscopic" in names and "lbm_destroy" in names
    so = ctypes.CDLL(L.LIBRARY)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_debug_library_exports_every_symbol(L):
    """liblbm_debug.so (the bounds-checked build) has the same C ABI."""
    from paper_2010_11751_b300 import build
    build.build(debug=True)
    so = ctypes.CDLL(L.LIBRARY_DEBUG)
    missing = [n for n in _declared("lbm.h") if not hasattr(so, n)]
    assert not missing, missing


def test_invalid_arguments_rejected(L):
    fl = np.zeros(27, np.uint8)
    bad = [
        (5, 3, 3, 3, L.TWOPOP, L.BGK_W2, 1.0, fl),      # unknown lattice
        (19, 0, 3, 3, L.TWOPOP, L.BGK_W2, 1.0, fl),     # empty dimension
        (19, 3, 3, 3, 9, L.BGK_W2, 1.0, fl),            # unknown scheme
        (19, 3, 3, 3, L.AA, 42, 1.0, fl),               # unknown model
        (19, 3, 3, 3, L.AA, L.TRT, 2.0, fl),            # omega out of (0, 2)
        (19, 3, 3, 3, L.AA, L.TRT, -0.5, fl),
        (19, 3, 3, 3, L.AA, L.TRT, 1.0, np.full(27, 9, np.uint8)),  # flag value > 7
        # larger than LBM_MAX_CELLS = 2^31 - 2^22 (rejected before the flags are read)
        (19, 1024, 1024, 2048, L.AA, L.TRT, 1.0, fl),
        (27, 2047, 1024, 1024, L.AA, L.TRT, 1.0, fl),
        (19, 1 << 20, 1 << 20, 1 << 20, L.AA, L.TRT, 1.0, fl),  # 2^60 cells: far beyond
    ]
    for args in bad:
        with pytest.raises(L.LBMError) as ei:
            L.lbm_create(*args)
        assert ei.value.code == L.ERR_INVALID_ARG, args
        assert L.lbm_last_error()


def test_null_handles_rejected(L):
    so = L.lib()
    assert so.lbm_step(None, 1) == L.ERR_INVALID_ARG
    assert so.lbm_macroscopic(None, None, None) == L.ERR_INVALID_ARG
    assert so.lbm_destroy(None) == L.OK


def test_supported_combinations(L):
    for Q in (19, 27):
        for s in range(4):
            for m in range(12):  # ten models, plus BGK-W2 in its two educational forms
                assert L.lbm_supported(Q, s, m, L.SOA, L.F64)
                assert L.lbm_supported(Q, s, m, L.AOS, L.F64)
                assert L.lbm_supported(Q, s, m, L.SOA, L.F32)
                assert L.lbm_supported(Q, s, m, L.SOA, L.F16)
                assert not L.lbm_supported(Q, s, m, L.AOS, L.F32)
    assert not L.lbm_supported(21, 0, 0, 0, 0)
    assert not L.lbm_supported(19, 0, 12, 0, 0)
