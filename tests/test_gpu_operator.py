"""The device operator Z (Eq. Z_bar_eq) and free-space solve (Sec. 4.2.1)
against the oracle, through the C ABI."""
import math

import numpy as np
import pytest

from util import rel_l2, table_json

pytestmark = pytest.mark.gpu

K0 = 2 * math.pi


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2410_17446_gb300 import build, prop
    build.build()
    return prop


def make(P, prec, nx=64, ny=32, dx=0.25, dy=0.2, seed=0):
    import torch
    from paper_2410_17446_gb300 import workloads as wl
    g = wl.Grid(nx, ny, dx, dy)
    rng = np.random.default_rng(seed)
    n2 = 1 + 0.05 * rng.standard_normal((ny, nx)) + 1j * wl.absorbing_sigma(g, 6, 0.2)
    pr = P.Propagator.from_table([(nx, ny, dx, dy)], K0, 1.0, 0.5, table_json("plain_scalar_64"),
                                 precision=P.PROP_FP64 if prec == "fp64" else P.PROP_FP32)
    pr.set_medium(0, n2)
    v = rng.standard_normal((1, ny, nx)) + 1j * rng.standard_normal((1, ny, nx))
    return pr, g, n2, v


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_operator_matches_oracle(P, prec, tol):
    import torch
    from oracle import operators as ops
    pr, g, n2, v = make(P, prec)
    dv = torch.tensor(v, device="cuda")
    out = torch.empty_like(dv)
    pr.apply_operator(0, dv, out)
    med = ops.Medium(n2, g.dx, g.dy, K0, 1.0, 1)
    assert rel_l2(out.cpu().numpy(), med.apply_Z(v)) < tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_freespace_inverse_matches_oracle(P, prec, tol):
    import torch
    from oracle import operators as ops
    pr, g, n2, v = make(P, prec)
    med = ops.Medium(n2, g.dx, g.dy, K0, 1.0, 1)
    T = table_json("plain_scalar_64")
    dv = torch.tensor(v, device="cuda")
    out = torch.empty_like(dv)
    for k in [0, 3, 11]:
        p = complex(*T["poles"][k])
        pr.apply_freespace_inverse(0, k, dv, out)
        assert rel_l2(out.cpu().numpy(), med.freespace_solve(v, p)) < tol


def make_vec(P, prec, nx=64, ny=32, dx=0.25, dy=0.2, seed=3):
    from paper_2410_17446_gb300 import workloads as wl
    g = wl.Grid(nx, ny, dx, dy)
    rng = np.random.default_rng(seed)
    n2 = 1 + 0.04 * wl.gaussian_random_field(g, 0.6, rng) + 1j * wl.absorbing_sigma(g, 5, 0.2)
    pr = P.Propagator.from_table([(nx, ny, dx, dy)], K0, 1.0, 0.5, table_json("vector_random_512"), ncomp=2,
                                 precision=P.PROP_FP64 if prec == "fp64" else P.PROP_FP32)
    pr.set_medium(0, n2)
    v = rng.standard_normal((2, ny, nx)) + 1j * rng.standard_normal((2, ny, nx))
    return pr, g, n2, v


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 5e-6)])
def test_vector_operator_matches_oracle(P, prec, tol):
    """All terms of Eq. (Z_bar_eq): Laplacian, delta, the psi terms and the
    cross-polarisation coupling, with psi = Log n^2 differentiated spectrally."""
    import torch
    from oracle import operators as ops
    pr, g, n2, v = make_vec(P, prec)
    dv = torch.tensor(v, device="cuda")
    out = torch.empty_like(dv)
    pr.apply_operator(0, dv, out)
    med = ops.Medium(n2, g.dx, g.dy, K0, 1.0, 2)
    assert rel_l2(out.cpu().numpy(), med.apply_Z(v)) < tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_vector_freespace_inverse_matches_oracle(P, prec, tol):
    import torch
    from oracle import operators as ops
    pr, g, n2, v = make_vec(P, prec)
    med = ops.Medium(n2, g.dx, g.dy, K0, 1.0, 2)
    T = table_json("vector_random_512")
    dv = torch.tensor(v, device="cuda")
    out = torch.empty_like(dv)
    for k in [0, 7]:
        pr.apply_freespace_inverse(0, k, dv, out)
        assert rel_l2(out.cpu().numpy(), med.freespace_solve(v, complex(*T["poles"][k]))) < tol
