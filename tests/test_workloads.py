"""Input generators (not the method): the Sec. 5.3 rotated sine product."""
import math

import numpy as np

from paper_2410_17446_gb300 import workloads as wl


def test_axis_angle_matrix_is_a_rotation_about_the_axis():
    u = np.array(wl.SINEPROD_AXIS) / np.linalg.norm(wl.SINEPROD_AXIS)
    R = wl.axis_angle_matrix(wl.SINEPROD_AXIS, wl.SINEPROD_ANGLE)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-15)
    assert abs(np.linalg.det(R) - 1) < 1e-14
    np.testing.assert_allclose(R @ u, u, atol=1e-15)
    # the angle: trace = 1 + 2 cos(a)
    assert abs((np.trace(R) - 1) / 2 - math.cos(wl.SINEPROD_ANGLE)) < 1e-14
    # a quarter turn about z takes x to y
    np.testing.assert_allclose(wl.axis_angle_matrix((0, 0, 1), math.pi / 2) @ [1, 0, 0], [0, 1, 0], atol=1e-15)


def test_sineprod_medium_matches_the_direct_formula():
    for q in (2.0, 0.5):
        W = wl.sineprod_helmholtz(q, 3, 64)
        b = W.beams[0]
        for s in (0, 2):
            direct = wl.rotated_sine_product_n2(b.grid, q, (s + 0.5) * W.dz, b.border, 0.2)
            np.testing.assert_allclose(b.medium(s), direct, rtol=0, atol=1e-13)


def test_sineprod_steps_cover_240_wavelengths():
    for q in (2.0, 1.0, 0.5):
        W = wl.sineprod_helmholtz(q)
        ks = wl.K0 * 1.2 / (math.sqrt(3) * q)
        assert abs(W.dz - (2 * math.pi / ks) / 4) < 1e-12
        assert abs(W.nsteps * W.dz - 240) <= W.dz / 2
        n2 = W.beams[0].medium(0)
        nn = np.sqrt(n2.real[W.beams[0].border + 1:-W.beams[0].border - 1])
        assert 1.2 - 0.025 - 1e-9 <= nn.min() and nn.max() <= 1.2 + 0.025 + 1e-9
