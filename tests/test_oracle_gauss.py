"""Pins of the E3 recovery oracle (Sec. 2, Gauss's law) to Gauss's law itself.

In a homogeneous medium the transverse field at z - h, z, z + h is propagated
exactly by the angular spectrum (Eq. exp_prop_planewave); the recovered E3 at
the three planes then makes the full field E = w exp(i k0 n0 z) divergence
free: d_x E1 + d_y E2 + d_z E3 = 0, with d_z taken by a central difference in
z (error O(h^2)) and d_x, d_y spectrally.  This checks the sign, the branch of
kz and the placement of n0 without restating the formula."""
import math

import numpy as np
import pytest

from oracle import gauss
from oracle import operators as ops
from oracle import propagator as orp


def _field(n, dx, rng):
    """A random two-component field with propagating and evanescent content."""
    x = (np.arange(n) - n // 2) * dx
    X, Y = np.meshgrid(x, x)
    env = np.exp(-(X ** 2 + Y ** 2) / 1.5 ** 2)
    w = np.stack([env * (1 + 0.3 * rng.standard_normal((n, n))),
                  env * (0.5j + 0.3 * rng.standard_normal((n, n)))]).astype(np.complex128)
    return w


@pytest.mark.parametrize("n0", [1.0, 1.2])
def test_recovered_e3_makes_the_field_divergence_free(n0):
    n, dx, k0, h = 64, 0.2, 2 * math.pi, 1e-3
    rng = np.random.default_rng(4)
    w = _field(n, dx, rng)
    n2 = np.full((n, n), n0 ** 2, np.complex128)
    z = 0.7

    def full(wz, zz):          # E1, E2, E3 of the full field at plane zz
        e3 = gauss.e3_from_transverse(wz, n2, dx, dx, k0, n0)
        ph = np.exp(1j * k0 * n0 * zz)
        return wz[0] * ph, wz[1] * ph, e3 * ph

    wm = orp.angular_spectrum(w, dx, dx, k0, n0, z - h)
    w0 = orp.angular_spectrum(w, dx, dx, k0, n0, z)
    wp = orp.angular_spectrum(w, dx, dx, k0, n0, z + h)
    E1, E2, _ = full(w0, z)
    _, _, E3m = full(wm, z - h)
    _, _, E3p = full(wp, z + h)
    ikx = ops.first_derivative_symbol(n, dx)[None, :]
    iky = ops.first_derivative_symbol(n, dx)[:, None]
    dxE1 = ops.ifft2(ikx * ops.fft2(E1))
    dyE2 = ops.ifft2(iky * ops.fft2(E2))
    dzE3 = (E3p - E3m) / (2 * h)
    div = dxE1 + dyE2 + dzE3
    scale = np.linalg.norm(dxE1) + np.linalg.norm(dyE2)
    assert np.linalg.norm(div) / scale < 1e-4
    # and E3 is not negligible: the check is not passed by a zero E3
    assert np.linalg.norm(dzE3) > 0.1 * scale


def test_uniform_transverse_field_has_no_e3():
    """A plane wave along z (kx = ky = 0) is purely transverse."""
    n = 16
    w = np.zeros((2, n, n), np.complex128)
    w[0] = 1.0 + 0.5j
    w[1] = -0.3
    e3 = gauss.e3_from_transverse(w, np.ones((n, n), np.complex128), 0.25, 0.25, 2 * math.pi, 1.0)
    assert np.max(np.abs(e3)) < 1e-14


def test_e3_is_linear_in_the_field():
    n = 32
    rng = np.random.default_rng(1)
    n2 = 1 + 0.05 * rng.standard_normal((n, n)) + 0.01j
    a, b = _field(n, 0.25, rng), _field(n, 0.25, rng)
    f = lambda v: gauss.e3_from_transverse(v, n2, 0.25, 0.25, 2 * math.pi, 1.0)
    np.testing.assert_allclose(f(2 * a - 1j * b), 2 * f(a) - 1j * f(b), atol=1e-12)
