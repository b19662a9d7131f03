"""The pseudo-differential propagator (Sec. 3.2; PROP_FORM_PSEUDODIFF) through
the C ABI: RK4 substeps of dw/dz = i k0 n0 (S(Z) - I) w with the Cauchy-integral
square root (N = 25, alpha = 1) as the handle's table, against the oracle's
RK4 with GMRES solves of the auxiliary systems (Eq. eq:Auxiliary_W), and in a
homogeneous medium against the Fourier closed form."""
import math

import numpy as np
import pytest

from util import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "the GPU tests need a CUDA device"
    from paper_2410_17446_gb300 import build, prop
    build.build()
    return prop


def _prop(P, g, dz, prec, substeps, ncomp=1, n0=1.0):
    from paper_2410_17446_gb300 import prop as Pm, tables
    return Pm.Propagator.from_table([(g.nx, g.ny, g.dx, g.dy)], 2 * math.pi, n0, dz, tables.load("cauchy_sqrt_25"),
                                    ncomp=ncomp, precision=prec, form=P.PROP_FORM_PSEUDODIFF, substeps=substeps,
                                    **({"tol": 1e-12} if prec == P.PROP_FP64 else {}))


@pytest.mark.parametrize("prec,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_homogeneous_against_fourier_closed_form(P, prec, bar):
    from oracle import aaa_lawson as al
    from oracle import cauchy as ca
    from paper_2410_17446_gb300 import tables, workloads as wl
    g = wl.Grid(128, 128, 0.25, 0.25)
    w0 = wl.gaussian_beam(g, 2.0)[None]
    pr = _prop(P, g, 0.5, P.PROP_FP64 if prec == "fp64" else P.PROP_FP32, 0)
    pr.set_field(0, w0)
    pr.set_medium(0, np.ones((g.ny, g.nx), np.complex128))
    for _ in range(3):
        pr.step()
    M = pr.substeps
    assert M >= 1
    T = al.PoleTable.from_json(tables.load("cauchy_sqrt_25"))
    ref = ca.homogeneous_pseudodiff(w0, g.dx, g.dy, 2 * math.pi, T, 0.5, M, 3)
    assert rel_l2(pr.get_field(0), ref) < bar


def test_auto_substeps_follow_the_stability_rule(P):
    """substeps = 0: the fewest M with (dz/M) k0 n0 (1 + sqrt(1.5 + |zeta_min|)) <= 2.5."""
    from paper_2410_17446_gb300 import workloads as wl
    for dx, dz in ((0.25, 0.5), (0.125, 0.5), (0.25, 1.0)):
        g = wl.Grid(32, 32, dx, dx)
        pr = _prop(P, g, dz, P.PROP_FP64, 0)
        pr.set_field(0, wl.gaussian_beam(g, 1.0)[None])
        pr.step()
        lam = 2 * math.pi * (1 + math.sqrt(1.5 + 2 * (math.pi / dx) ** 2 / (2 * math.pi) ** 2))
        assert pr.substeps == max(1, math.ceil(dz * lam / 2.5)), (dx, dz)


@pytest.mark.parametrize("prec,unit", [("fp64", 1e-12), ("fp32", 1e-7)])
def test_inhomogeneous_against_oracle(P, prec, unit):
    """32^2, dx = lambda/4, sine-product medium with an absorbing border, two
    steps of dz = lambda/2 (the handle's automatic substeps).

    The bar is derived: one application of S(Z) carries a relative error of
    about unit * sum_j |s_j| / |Im q_j| (~51 for this table, whose constant
    c_alpha + sum wt_j ~ 51 cancels against the auxiliary terms), and the
    Runge-Kutta sums feed it into the field scaled by h k0 n0 per substep, so
    over a range Z the field error stays below about 4 unit amp k0 n0 Z.  FP32
    therefore holds the pseudo-differential form to ~1e-4, against ~1e-6 for
    the exponential form on the same grid."""
    from oracle import aaa_lawson as al
    from oracle import cauchy as ca
    from oracle import operators as ops
    from paper_2410_17446_gb300 import tables, workloads as wl
    g = wl.Grid(32, 32, 0.25, 0.25)
    n2 = wl.sine_product_n2(g, 0.05, 2.0, None, 4, 0.2)
    w0 = wl.gaussian_beam(g, 1.5)[None]
    pr = _prop(P, g, 0.5, P.PROP_FP64 if prec == "fp64" else P.PROP_FP32, 0)
    pr.set_field(0, w0)
    pr.set_medium(0, n2)
    pr.step()
    pr.step()
    M = pr.substeps
    T = al.PoleTable.from_json(tables.load("cauchy_sqrt_25"))
    med = ops.Medium(n2, g.dx, g.dy, 2 * math.pi, 1.0, 1)
    ref = ca.pseudodiff_step(med, ca.pseudodiff_step(med, w0, T, 2 * math.pi, 0.5, M), T, 2 * math.pi, 0.5, M)
    amp = float(np.sum(np.abs(T.residues) / np.abs(T.poles.imag)))
    bar = max(1e-10, 4 * unit * amp * 2 * math.pi * (2 * 0.5))
    err = rel_l2(pr.get_field(0), ref)
    print(f"{prec}: rel L2 {err:.2e}, derived bar {bar:.2e} (amplification {amp:.1f}, {M} substeps)")
    assert err < bar
    assert pr.stats().total_iters > 0
