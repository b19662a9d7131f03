"""The C ABI library builds for sm_103a, loads, and exports what include/prop.h declares.
Argument validation that happens before any CUDA call is checked here on CPU."""
import ctypes as ct
import os
import re

import pytest

from paper_2410_17446_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_2410_17446_gb300 import prop as P
    return P


def declared_functions():
    text = open(os.path.join(ROOT, "include", "prop.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(prop_[a-z0-9_]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_every_declared_symbol_is_exported(lib):
    L = lib.lib()
    names = declared_functions()
    assert "prop_create" in names and "prop_step" in names and "prop_run" in names
    for n in names:
        assert hasattr(L, n), n


def test_error_strings(lib):
    L = lib.lib()
    for s in range(7):
        assert L.prop_error_string(s)


def test_argument_errors_before_any_cuda_call(lib):
    P = lib
    o = P.prop_default_opts(1, P.PROP_FP32)
    assert o.restart == 20 and o.tol == 1e-7
    n = ct.c_size_t()
    bad = (P.prop_grid * 1)(P.prop_grid(100, 64, 0.25, 0.25))
    assert P.lib().prop_workspace_size(1, bad, 12, ct.byref(o), ct.byref(n)) == P.PROP_E_UNSUPPORTED
    good = (P.prop_grid * 1)(P.prop_grid(64, 64, 0.25, 0.25))
    assert P.lib().prop_workspace_size(1, good, 12, ct.byref(o), ct.byref(n)) == P.PROP_OK
    assert n.value > 64 * 64 * 8 * 21 * 12
    o2 = P.prop_default_opts(1, P.PROP_FP32)
    o2.restart = 0
    assert P.lib().prop_workspace_size(1, good, 12, ct.byref(o2), ct.byref(n)) == P.PROP_E_ARG
    o3 = P.prop_default_opts(3, P.PROP_FP32)
    assert P.lib().prop_workspace_size(1, good, 12, ct.byref(o3), ct.byref(n)) != P.PROP_OK
    h = ct.c_void_p()
    d = (ct.c_double * 2)(0.0, 0.0)
    # null workspace is rejected before any device work
    assert P.lib().prop_create(1, good, 6.28, 1.0, 0.5, 1, d, d, d, ct.byref(o), None, 0, None,
                               ct.byref(h)) == P.PROP_E_WORKSPACE
    assert P.lib().prop_create(1, good, -1.0, 1.0, 0.5, 1, d, d, d, ct.byref(o), None, 0, None,
                               ct.byref(h)) == P.PROP_E_ARG
    assert P.lib().prop_step(None) == P.PROP_E_ARG
