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
    o4 = P.prop_default_opts(1, P.PROP_FP32)
    assert o4.multigroup == 1                        # lockstep grids by default
    o4.multigroup = 2
    assert P.lib().prop_workspace_size(1, good, 12, ct.byref(o4), ct.byref(n)) == P.PROP_E_ARG
    h = ct.c_void_p()
    d = (ct.c_double * 2)(0.0, 0.0)
    # null workspace is rejected before any device work
    assert P.lib().prop_create(1, good, 6.28, 1.0, 0.5, 1, d, d, d, ct.byref(o), None, 0, None,
                               ct.byref(h)) == P.PROP_E_WORKSPACE
    assert P.lib().prop_create(1, good, -1.0, 1.0, 0.5, 1, d, d, d, ct.byref(o), None, 0, None,
                               ct.byref(h)) == P.PROP_E_ARG
    assert P.lib().prop_step(None) == P.PROP_E_ARG


def test_workspace_holds_m_plus_2_basis_slots(lib):
    """The Krylov basis keeps m + 2 vectors per system (slot j+1 takes w up to
    step j = m): one more restart step adds exactly one vector per system."""
    P = lib
    grids = (P.prop_grid * 2)(P.prop_grid(256, 256, 0.25, 0.25), P.prop_grid(256, 256, 0.25, 0.25))
    npoles = 12
    sizes = {}
    for prec, cs in ((P.PROP_FP32, 8), (P.PROP_FP64, 16)):
        for m in (20, 21):
            o = P.prop_default_opts(1, prec)
            o.restart = m
            n = ct.c_size_t()
            assert P.lib().prop_workspace_size(2, grids, npoles, ct.byref(o), ct.byref(n)) == P.PROP_OK
            sizes[(prec, m)] = n.value
        assert sizes[(prec, 21)] - sizes[(prec, 20)] == 2 * npoles * 256 * 256 * cs
    o = P.prop_default_opts(1, P.PROP_FP32)
    o.restart = 65                                    # above the compiled maximum restart length
    n = ct.c_size_t()
    assert P.lib().prop_workspace_size(2, grids, npoles, ct.byref(o), ct.byref(n)) == P.PROP_E_ARG
