"""CPU checks of the C ABI library: it loads, exports every function that
include/tdvp.h declares, and reports errors (no compute call needs a GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "tdvp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tdvp_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("tdvp_create", "tdvp_step", "tdvp_measure", "tdvp_heff_apply", "tdvp_destroy", "tdvp_strerror",
              "tdvp_bond_create", "tdvp_block_list"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2606_04771_b300 import lib

    L = lib()
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing


def test_error_reporting_without_gpu():
    import torch

    from paper_2606_04771_b300 import Chain, TdvpError, lib

    assert lib().tdvp_strerror(-1) == b"invalid argument"
    assert lib().tdvp_strerror(0) == b"ok"
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(TdvpError) as e:
        Chain(8, 1.0, 4.0)
    assert e.value.code == -6  # ECUDA: no device, no CPU fallback


def test_invalid_arguments_rejected_before_any_device_call():
    from paper_2606_04771_b300 import TdvpError, lib
    import paper_2606_04771_b300._lib as B

    h = ctypes.c_void_p()
    assert lib().tdvp_create(8, 1.0, 4.0, 7, None, ctypes.byref(h)) == -1  # unknown symmetry
    assert lib().tdvp_step(None, 0.1, 8, 0.0) == -1
    assert lib().tdvp_destroy(None) == 0
