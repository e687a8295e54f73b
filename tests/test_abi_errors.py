"""Error behaviour of the C ABI that needs no GPU: every entry point rejects a
null context with TERSOFF_E_INVALID_ARG before any CUDA call, tersoff_create
checks its arguments, the null-context queries return their fixed text, and,
on a machine without a GPU, context creation fails with TERSOFF_E_CUDA
instead of falling back to anything.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")

E_INVALID_ARG = 1
E_CUDA = 6


@pytest.fixture(scope="module")
def lib():
    from paper_1607_02904_gb300 import _lib
    return _lib.load(), _lib._SIG


def _null_args(argtypes):
    out = []
    for t in argtypes[1:]:
        if t in (ctypes.c_int, ctypes.c_longlong):
            out.append(0)
        elif t is ctypes.c_double:
            out.append(0.0)
        else:
            out.append(None)
    return out


def test_every_entry_point_rejects_a_null_context(lib):
    L, sig = lib
    special = {"tersoff_create", "tersoff_destroy", "tersoff_last_error",
               "tersoff_autotune_summary"}
    checked = 0
    for name, (argtypes, restype) in sig.items():
        if name in special:
            continue
        st = getattr(L, name)(None, *_null_args(argtypes))
        assert st == E_INVALID_ARG, (name, st)
        checked += 1
    assert checked == len(sig) - len(special)
    from paper_1607_02904_gb300._lib import declared_symbols
    assert set(sig) == set(declared_symbols())  # every declared entry point is covered


def test_null_context_queries_and_destroy(lib):
    L, _ = lib
    assert L.tersoff_destroy(None) == 0
    assert L.tersoff_last_error(None) == b"null context"
    assert L.tersoff_autotune_summary(None) == b"null context"


def test_create_checks_its_arguments(lib):
    L, _ = lib
    assert L.tersoff_create(None, 1) == E_INVALID_ARG
    h = ctypes.c_void_p(1234)
    assert L.tersoff_create(ctypes.byref(h), 7) == E_INVALID_ARG  # no such precision
    assert h.value is None  # the output is cleared on failure


def test_create_without_a_gpu_fails_loudly(lib):
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L, _ = lib
    h = ctypes.c_void_p()
    assert L.tersoff_create(ctypes.byref(h), 1) == E_CUDA
    assert h.value is None
    from paper_1607_02904_gb300 import Context, TersoffError
    with pytest.raises(TersoffError):
        Context(1)
