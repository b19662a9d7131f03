"""Pins of the operator oracle (Eqs. Z_bar_eq, Z_bar_fs_def, fs_sylvester)."""
import math

import numpy as np
import pytest

from oracle import operators as ops
from paper_2410_17446_gb300 import workloads as wl

K0 = 2 * math.pi


def _grid(nx=16, ny=12, dx=0.25, dy=0.2):
    return wl.Grid(nx, ny, dx, dy)


def test_plane_wave_is_eigenvector_scalar():
    """Sec. 3 below Eq. exp_prop_planewave: on a plane wave exp(i(kx x + ky y))
    in a uniform medium, Z acts as the number -(kx^2+ky^2)/(k0 n0)^2 + (n^2-n0^2)/n0^2."""
    g = _grid()
    n0 = 1.1
    n2 = (1.3 + 0.05j) * np.ones((g.ny, g.nx))
    med = ops.Medium(n2, g.dx, g.dy, K0, n0, 1)
    X, Y = g.mesh()
    for (mx, my) in [(0, 0), (3, -2), (-5, 4), (7, 5)]:
        kx = 2 * math.pi * mx / (g.nx * g.dx)
        ky = 2 * math.pi * my / (g.ny * g.dy)
        v = np.exp(1j * (kx * X + ky * Y))[None]
        lam = -(kx ** 2 + ky ** 2) / (K0 * n0) ** 2 + (1.3 + 0.05j - n0 ** 2) / n0 ** 2
        np.testing.assert_allclose(med.apply_Z(v), lam * v, atol=1e-12)


def test_first_derivative_nyquist_convention():
    s = ops.first_derivative_symbol(8, 0.5)
    assert s[4] == 0
    np.testing.assert_allclose(s[1], 1j * 2 * math.pi / 4.0)
    np.testing.assert_allclose(s[7], -1j * 2 * math.pi / 4.0)


def _analytic_case(g, a=0.04):
    """n^2 = exp(psi) with psi = a cos(al x) cos(be y) periodic on the grid."""
    X, Y = g.mesh()
    al_ = 2 * math.pi * 2 / (g.nx * g.dx)
    be = 2 * math.pi * 1 / (g.ny * g.dy)
    psi = a * np.cos(al_ * X) * np.cos(be * Y)
    d = {
        "x": -a * al_ * np.sin(al_ * X) * np.cos(be * Y),
        "y": -a * be * np.cos(al_ * X) * np.sin(be * Y),
        "xx": -a * al_ ** 2 * np.cos(al_ * X) * np.cos(be * Y),
        "yy": -a * be ** 2 * np.cos(al_ * X) * np.cos(be * Y),
        "xy": a * al_ * be * np.sin(al_ * X) * np.sin(be * Y),
    }
    return np.exp(psi), psi, d


def test_psi_terms_match_analytic_derivatives():
    g = _grid(24, 20, 0.25, 0.3)
    n0 = 1.05
    n2, psi, d = _analytic_case(g)
    p = ops.psi_terms(n2, g.dx, g.dy, K0 * n0)
    for k in d:
        np.testing.assert_allclose(p[k], d[k] / (K0 * n0) ** 2, atol=1e-13)


def test_vector_operator_on_analytic_fields():
    """Every term of Eq. (Z_bar_eq), evaluated by hand with analytic derivatives
    of psi and of trigonometric test fields, against Medium.apply_Z."""
    g = _grid(24, 20, 0.25, 0.3)
    n0 = 1.05
    s = 1.0 / (K0 * n0) ** 2
    n2, psi, d = _analytic_case(g)
    X, Y = g.mesh()
    p1 = 2 * math.pi * 3 / (g.nx * g.dx)
    q1 = 2 * math.pi * 1 / (g.ny * g.dy)
    p2 = 2 * math.pi * 1 / (g.nx * g.dx)
    q2 = 2 * math.pi * 2 / (g.ny * g.dy)
    v1 = np.exp(1j * (p1 * X + q1 * Y))
    v2 = np.cos(p2 * X) * np.sin(q2 * Y)
    v1x, v1y = 1j * p1 * v1, 1j * q1 * v1
    lap1 = -(p1 ** 2 + q1 ** 2) * v1
    v2x = -p2 * np.sin(p2 * X) * np.sin(q2 * Y)
    v2y = q2 * np.cos(p2 * X) * np.cos(q2 * Y)
    lap2 = -(p2 ** 2 + q2 ** 2) * v2
    dn = n2 - n0 ** 2
    # Eq. (Z_bar_eq) written out, then scaled by (k0 n0)^-2
    z1 = s * (lap1 + K0 ** 2 * dn * v1 + d["xx"] * v1 + d["x"] * v1x + d["xy"] * v2 + d["y"] * v2x)
    z2 = s * (d["xy"] * v1 + d["x"] * v1y + lap2 + K0 ** 2 * dn * v2 + d["yy"] * v2 + d["y"] * v2y)
    med = ops.Medium(n2, g.dx, g.dy, K0, n0, 2)
    out = med.apply_Z(np.stack([v1, v2]))
    np.testing.assert_allclose(out[0], z1, atol=1e-12)
    np.testing.assert_allclose(out[1], z2, atol=1e-12)


@pytest.mark.parametrize("ncomp", [1, 2])
def test_dense_matrix_equals_fft_application(ncomp):
    g = _grid(10, 8, 0.25, 0.2)
    rng = np.random.default_rng(1)
    n2 = 1 + 0.05 * rng.standard_normal((g.ny, g.nx)) + 0.02j * rng.uniform(0, 1, (g.ny, g.nx))
    med = ops.Medium(n2, g.dx, g.dy, K0, 1.0, ncomp)
    v = rng.standard_normal((ncomp, g.ny, g.nx)) + 1j * rng.standard_normal((ncomp, g.ny, g.nx))
    np.testing.assert_allclose(ops.dense_Z(med) @ v.ravel(), med.apply_Z(v).ravel(), atol=1e-12)


def test_freespace_solve_equals_sylvester_solution():
    """Eq. (fs_sylvester), solved by Bartels-Stewart, equals the FFT-diagonal
    free-space solve; the grid is not square so a transposed operand fails."""
    g = _grid(12, 10, 0.25, 0.2)
    rng = np.random.default_rng(2)
    rhs = rng.standard_normal((g.ny, g.nx)) + 1j * rng.standard_normal((g.ny, g.nx))
    med = ops.Medium(np.ones((g.ny, g.nx)), g.dx, g.dy, K0, 1.0, 1)
    for pole in [-0.99 - 0.01j, 0.3 - 1.2j]:
        xs = ops.sylvester_freespace_solve(rhs, g.dx, g.dy, K0, pole)
        xf = med.freespace_solve(rhs[None], pole)[0]
        np.testing.assert_allclose(xs, xf, atol=1e-10 * np.abs(xf).max())


def test_freespace_solve_on_plane_wave():
    g = _grid()
    med = ops.Medium(np.ones((g.ny, g.nx)), g.dx, g.dy, K0, 1.2, 1)
    X, Y = g.mesh()
    kx = 2 * math.pi * 3 / (g.nx * g.dx)
    ky = 2 * math.pi * -1 / (g.ny * g.dy)
    v = np.exp(1j * (kx * X + ky * Y))[None]
    p = -0.5 - 0.3j
    lam = -(kx ** 2 + ky ** 2) / (K0 * 1.2) ** 2
    np.testing.assert_allclose(med.freespace_solve(v, p), v / (lam - p), atol=1e-13)
