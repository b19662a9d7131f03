"""Pins of the Cauchy-integral square root and the pseudo-differential
propagator oracle (Sec. 3.2, App. A) to facts fixed outside them."""
import cmath
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import cauchy as ca
from oracle import operators as ops
from oracle import propagator as orp
from paper_2410_17446_gb300 import workloads as wl


@pytest.mark.parametrize("alpha", [1.0, 0.1])
def test_cauchy_integral_representation_is_the_square_root(alpha):
    """App. A: c_alpha (1 - (1/pi) int sqrt((1+eta)/(1-eta))/(eta - w) d eta)
    with w the Möbius image of zeta equals sqrt(1 + zeta) on the principal
    branch (i sqrt|1+zeta| for zeta < -1), the integral done by adaptive
    quadrature, not by the Gauss-Jacobi rule."""
    c = math.sqrt(alpha) * cmath.exp(1j * math.pi / 4)
    for z in (0.7, -0.4, -2.5, 1.2 + 0.3j, -6.0 + 0.1j):
        w = (z + 1 + 1j * alpha) / (z + 1 - 1j * alpha)
        f = lambda e: np.sqrt((1 + e) / (1 - e)) / (e - w)
        re = integrate.quad(lambda e: f(e).real, -1, 1, limit=400)[0]
        im = integrate.quad(lambda e: f(e).imag, -1, 1, limit=400)[0]
        g = c * (1 - (re + 1j * im) / math.pi)
        assert abs(g - np.sqrt(1 + complex(z))) < 1e-9, z


def test_gauss_jacobi_rule_is_exact_for_polynomials():
    eta, om = ca.gauss_jacobi(12)
    for deg in range(0, 23):
        ref = integrate.quad(lambda e: e ** deg * np.sqrt((1 + e) / (1 - e)), -1, 1, limit=200)[0]
        assert abs(np.sum(om * eta ** deg) - ref) < 1e-10, deg
    assert abs(np.sum(om) - math.pi) < 1e-13          # int sqrt((1+e)/(1-e)) = pi


def test_partial_fractions_equal_the_quadrature_form():
    """Eq. pf_sqrt_exp is the synthetic division of Eq. prime_sqrt_exp."""
    T = ca.cauchy_sqrt_table(25, 1.0)
    z = np.concatenate([np.linspace(-4, 2, 301), np.linspace(-4, 2, 31) + 0.2j])
    assert np.max(np.abs(T(z) - ca.sqrt_quadrature_form(z, 25, 1.0))) < 1e-12
    assert np.all(T.poles.imag < 0) and np.allclose(T.poles.real, -1.0)


def test_paper_accuracy_statements():
    """Sec. 3.2: with N = 25 and alpha = 1 the expansion is accurate on [-4, 2]
    except a narrow band around zeta = -1; alpha = 0.1 costs accuracy away from
    the branch point, and N = 45 with alpha = 0.1 then narrows the band."""
    z = np.linspace(-4, 2, 6001)
    s = np.sqrt(1 + z + 0j)
    err = lambda N, a: np.abs(ca.cauchy_sqrt_table(N, a)(z) - s)
    e1, e01, e45 = err(25, 1.0), err(25, 0.1), err(45, 0.1)
    far = np.abs(z + 1) > 0.2
    assert e1[far].max() < 1e-8
    assert e1[np.argmin(np.abs(z + 1))] > 1e-3
    assert e01[far].max() > 100 * e1[far].max()
    band = lambda e: np.ptp(z[e > 1e-6]) if np.any(e > 1e-6) else 0.0
    assert band(e45) < band(e1)
    assert e45[far].max() < 1e-8


def test_rk4_amplification_is_fourth_order():
    lam = np.array([-3.0 + 2.0j, 0.5j, -1.0])
    for h in (0.05, 0.025):
        err = np.abs(ca.rk4_amplification(lam, h) - np.exp(h * lam))
        assert np.all(err < 1.0 * np.abs(h * lam) ** 5)


def test_homogeneous_pseudodiff_step_matches_fourier_closed_form_and_converges():
    """In a homogeneous medium the RK4 pseudo-differential step (GMRES path) is
    diagonal in Fourier space.  Refining the substeps converges at fourth order
    to exp(i k0 n0 dz (S(zeta) - 1)), and that differs from the exact angular
    spectrum only by the square root's error (Eq. exp_prop_planewave)."""
    g = wl.Grid(32, 32, 0.25, 0.25)
    w = wl.gaussian_beam(g, 1.2)[None]
    med = ops.Medium(np.ones((32, 32), np.complex128), g.dx, g.dy, 2 * math.pi, 1.0, 1)
    T = ca.cauchy_sqrt_table(25, 1.0)
    k0n0, dz = 2 * math.pi, 0.5
    a = ca.pseudodiff_step(med, w, T, k0n0, dz, 4)
    b = ca.homogeneous_pseudodiff(w, g.dx, g.dy, k0n0, T, dz, 4)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10
    z = ops.zeta_fs(32, 32, g.dx, g.dy, k0n0)
    limit = ops.ifft2(np.exp(1j * k0n0 * dz * (T(z) - 1)) * ops.fft2(w[0]))[None]
    # M = 4 keeps h |lambda| <= 2.3 on the whole spectrum, inside RK4's stability region
    e = {M: np.linalg.norm(ca.homogeneous_pseudodiff(w, g.dx, g.dy, k0n0, T, dz, M) - limit) for M in (4, 8, 16)}
    assert 12 < e[4] / e[8] < 20 and 12 < e[8] / e[16] < 20
    exact = orp.angular_spectrum(w, g.dx, g.dy, 2 * math.pi, 1.0, dz)
    assert np.linalg.norm(limit - exact) / np.linalg.norm(exact) < 1e-6
