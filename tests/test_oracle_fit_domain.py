"""Pins of the fit range (oracle.aaa_lawson.fit_domain) to the operator's spectrum.

Sec. 3 (Eq. eq_spectra_operators): the propagator is accurate on spec Z only
where the scalar rational fit is accurate, so the fit range must cover spec Z.
Two independent facts fix it:

* the free-space symbol's most evanescent value, -(kx_max^2 + ky_max^2)/(k0 n0)^2
  with kx_max = pi/dx (the Nyquist wavenumber), computed here by hand for the
  grid spacings of the workloads (lambda/4: -8, lambda/6: -18, lambda/8: -32);
* the eigenvalues of the dense operator matrix (Kronecker products of 1-D
  spectral matrices, not the FFT application) on 16 x 16 grids with each
  workload's spacing, medium amplitude and absorbing border.

A slip in fit_domain (2 pi/dx for the Nyquist wavenumber, a lost ky term, the
wrong sign on min Re delta) moves lo away from these values or leaves an
eigenvalue outside the range, and fails here.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import aaa_lawson as al
from oracle import operators as ops
from paper_2410_17446_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
TABLES = os.path.join(os.path.dirname(HERE), "paper_2410_17446_gb300", "tables")
K0N0 = 2 * math.pi          # lambda = 1, n0 = 1


@pytest.mark.parametrize("dx,zeta_min", [(0.25, -8.0), (1 / 6, -18.0), (0.125, -32.0)])
def test_zeta_min_by_hand(dx, zeta_min):
    """(pi/dx)^2 * 2/(2 pi)^2 = 1/(2 dx^2): 8, 18, 32 for dx = 1/4, 1/6, 1/8.
    fit_domain adds min Re delta and a 0.5 margin, and never goes above -4
    (the paper's default lower end)."""
    assert al.fit_domain(16, 16, dx, dx, K0N0, 0.0) == pytest.approx(zeta_min - 0.5, abs=1e-12)
    assert al.fit_domain(64, 32, dx, dx, K0N0, -0.07) == pytest.approx(zeta_min - 0.57, abs=1e-12)
    # a positive min Re delta does not raise the range (the spectrum still reaches zeta_min)
    assert al.fit_domain(16, 16, dx, dx, K0N0, 0.3) == pytest.approx(zeta_min - 0.5, abs=1e-12)
    # a coarse grid's spectrum ends above -4: the paper's default range is kept
    assert al.fit_domain(16, 16, 1.0, 1.0, K0N0, 0.0) == -4.0


def test_anisotropic_grid_uses_both_axes():
    """dx != dy: zeta_min = -((pi/dx)^2 + (pi/dy)^2)/(k0 n0)^2 = -(1/(4 dx^2) + 1/(4 dy^2))
    = -(4 + 1) for dx = 1/4, dy = 1/2."""
    assert al.fit_domain(16, 8, 0.25, 0.5, K0N0, 0.0) == pytest.approx(-5.5, abs=1e-12)


def decaying_target(z, K):
    """g on the decaying branch Im sqrt(1 + z) >= 0 (Eq. exp_prop_planewave), for
    z on either side of the real axis; below the cut this is minus the principal
    root, the continuation from above."""
    s = np.sqrt(1.0 + np.asarray(z, np.complex128))
    s = np.where(s.imag < 0, -s, s)
    return np.exp(1j * K * (s - 1.0))


def _media():
    """16 x 16 analogues of each workload family: spacing, amplitude, border."""
    g4 = wl.Grid(16, 16, 0.25, 0.25)
    g6 = wl.Grid(16, 16, 1 / 6, 1 / 6)
    g8 = wl.Grid(16, 16, 0.125, 0.125)
    rng = np.random.Generator(np.random.PCG64(5))
    out = [
        ("plain_scalar_64", g8, wl.sine_product_n2(g8, 0.1, 2.0, None, 4, 0.2), 1),
        ("batched_scalar_1024", g4, wl.sine_product_n2(g4, 0.05, 1.5, 0.25, 4, 0.2), 1),
        ("uneven_batch", g4, wl.sine_product_n2(g4, 0.1, 1.0, 0.4, 4, 0.2), 1),
        ("vector_random_512", g6, (1 + 0.03 * wl.gaussian_random_field(g6, 1.0, rng))
         + 1j * wl.absorbing_sigma(g6, 4, 0.2), 2),
    ]
    return out


@pytest.mark.parametrize("name,grid,n2,ncomp", _media(), ids=lambda v: v if isinstance(v, str) else "")
def test_dense_spectrum_inside_fit_range(name, grid, n2, ncomp):
    """Every eigenvalue of the dense Z lies in [lo, 2] x [0, 2 sigma], where lo
    comes from fit_domain for this grid and medium and 2 sigma is the largest
    absorbing shift the tables sample (corners carry sigma_x + sigma_y).

    The scalar Z is the Hermitian Laplacian plus diag(delta), so its numerical
    range, and with it the spectrum, lies in [zeta_min + min Re delta, max Re delta]
    x [min Im delta, max Im delta].  The vector Z adds the first-derivative psi
    terms, which are not dissipative: with a complex border one eigenvalue sits
    about 0.015 below the real axis (seen for every seed tried); the bound
    checked for it is -0.05."""
    med = ops.Medium(n2, grid.dx, grid.dy, 1.0 * K0N0, 1.0, ncomp)
    lam = np.linalg.eigvals(ops.dense_Z(med))
    lo = al.fit_domain(grid.nx, grid.ny, grid.dx, grid.dy, K0N0, float(med.delta.real.min()))
    assert lam.real.min() >= lo, (lam.real.min(), lo)
    assert lam.real.max() <= 2.0
    assert lam.imag.min() >= (-1e-9 if ncomp == 1 else -0.05)
    assert lam.imag.max() <= 0.4 + 1e-9
    # the margin is not slack that hides a wrong zeta_min: the spectrum reaches within
    # 0.5 + max|Re delta| + 0.1 of lo (the Nyquist corner mode is nearly an eigenvector)
    reach = 0.5 + float(np.abs(med.delta.real).max()) + 0.1
    assert lam.real.min() <= lo + reach, (lam.real.min(), lo)


@pytest.mark.parametrize("name,grid,n2,ncomp", _media(), ids=lambda v: v if isinstance(v, str) else "")
def test_committed_table_covers_and_fits_the_spectrum(name, grid, n2, ncomp):
    """The committed table for the family covers the dense spectrum at its
    spacing, and r(lambda) matches g(lambda) = exp(iK(-1+sqrt(1+lambda))) on
    every eigenvalue to within a few times the table's sampled fit error (the
    accuracy of Eq. eq_spectra_operators on spec Z).  g is taken on the decaying
    branch, which matters for the vector operator's eigenvalue just below the
    negative real axis: the principal root there would be the growing branch."""
    T = al.PoleTable.from_json(json.load(open(os.path.join(TABLES, name + ".json"))))
    med = ops.Medium(n2, grid.dx, grid.dy, K0N0, 1.0, ncomp)
    lam = np.linalg.eigvals(ops.dense_Z(med))
    assert lam.real.min() >= T.lo and lam.real.max() <= T.hi
    assert lam.imag.max() <= max(T.im_shifts) + 1e-9
    err = np.abs(T(lam) - decaying_target(lam, T.K))
    assert err.max() <= 5 * T.fit_max_err, (err.max(), T.fit_max_err)
