"""Host-side checks that need no GPU: the library builds and exports every
declared entry point, the binding matches the header, and the product's
parameter-table helper agrees with the oracle's mixing rule."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W


def test_library_exports_declared_symbols():
    import paper_1607_02904_gb300 as T
    lib = T.load()
    declared = T.declared_symbols()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    # the binding knows every declared symbol
    from paper_1607_02904_gb300 import _lib
    assert set(declared) <= set(_lib._SIG)


def test_header_constants_match_binding():
    import re
    import os
    import paper_1607_02904_gb300 as T
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "include",
                            "tersoff.h")).read()
    consts = dict(re.findall(r"#define (TERSOFF_\w+) (\d+)", hdr))
    assert int(consts["TERSOFF_NPARAM"]) == T.NPARAM
    assert int(consts["TERSOFF_FP64"]) == T.FP64
    assert int(consts["TERSOFF_MIXED"]) == T.MIXED
    assert int(consts["TERSOFF_NOALLOC_MAX_ATOMS"]) == T.NOALLOC_MAX_ATOMS
    for name in ("NO_SHORT", "GENERAL", "FP32_SUMS", "FASTFWD", "COMP_ATOM_SUMS"):
        assert int(consts["TERSOFF_ABLATE_" + name]) == getattr(T, "ABLATE_" + name)
    order = ["M", "GAMMA", "LAMBDA3", "C", "D", "H", "N", "BETA", "LAMBDA2", "B", "R", "D_CUT",
             "LAMBDA1", "A"]
    for q, name in enumerate(order):
        assert int(consts["TERSOFF_P_" + name]) == q


@pytest.mark.parametrize("names", [["Si"], ["C"], ["Si", "C"], ["C", "Si"]])
def test_product_mixing_matches_oracle(names):
    import paper_1607_02904_gb300 as T
    elem, chi = W.element_records(names)
    a = T.mix_tersoff89(elem, chi)
    b = oracle.mix_tersoff89(elem, chi)
    assert a.shape == b.shape
    assert np.allclose(a, b, rtol=1e-15, atol=0)


def test_create_without_gpu_reports_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_1607_02904_gb300 as T
    lib = T.load()
    h = ctypes.c_void_p()
    st = lib.tersoff_create(ctypes.byref(h), 1)
    assert st == 6  # TERSOFF_E_CUDA
    assert lib.tersoff_create(None, 1) == 1
    assert lib.tersoff_destroy(None) == 0
