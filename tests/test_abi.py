"""The C ABI library loads and exports every symbol include/stokes.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "stokes.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stk_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_abi():
    names = _declared()
    for n in ("stk_create", "stk_destroy", "stk_set_coefficients", "stk_apply_operator",
              "stk_apply_preconditioner", "stk_solve"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib_path = os.path.join(ROOT, "paper_1308_4605_gb300", "libstokes_gb300.so")
    if not os.path.exists(lib_path):
        pytest.skip("library not built (run __graft_entry__.build())")
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1308_4605_gb300 import stokes
    assert set(stokes.EXPORTED) <= set(_declared())


def test_create_rejects_bad_sizes_without_gpu():
    lib_path = os.path.join(ROOT, "paper_1308_4605_gb300", "libstokes_gb300.so")
    if not os.path.exists(lib_path):
        pytest.skip("library not built")
    from paper_1308_4605_gb300 import stokes
    with pytest.raises(stokes.StokesError) as e:
        stokes.stk_create(2, (12, 16), 1.0, (0, 0, 0, 0))
    assert e.value.code == stokes.STK_ERR_SIZE
    with pytest.raises(stokes.StokesError) as e:
        stokes.stk_create(4, (16, 16), 1.0, (0, 0, 0, 0))
    assert e.value.code == stokes.STK_ERR_ARG
