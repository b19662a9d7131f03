"""Pins of the one-step propagator oracle (Eqs. approx_prop, approx_fs_prop,
exp_prop_planewave, eq_spectra_operators) and its invariants."""
import json
import math
import os

import numpy as np
import pytest

from oracle import aaa_lawson as al, operators as ops, propagator as pr
from paper_2410_17446_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
TABLES = os.path.join(os.path.dirname(HERE), "paper_2410_17446_gb300", "tables")
K0 = 2 * math.pi


def table(name):
    return al.PoleTable.from_json(json.load(open(os.path.join(TABLES, name + ".json"))))


def test_homogeneous_step_equals_fourier_multiplier():
    """Eq. (approx_fs_prop): in a homogeneous medium the GMRES step is IFFT[r(zeta_fs) FFT w]."""
    T = table("plain_scalar_64")
    g = wl.Grid(32, 24, 0.125, 0.125)
    w = (wl.gaussian_beam(g, 0.7) * np.exp(1j * 3.0 * g.mesh()[0]))[None]
    med = ops.Medium(np.ones((g.ny, g.nx)), g.dx, g.dy, K0, 1.0, 1)
    out = w
    for _ in range(3):
        out, st = pr.step(med, out, T, tol=1e-13)
        assert all(i == 1 for i in st.iterations)
    ref = pr.homogeneous_rational_step(w, g.dx, g.dy, K0, T, 3)
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-11


def test_angular_spectrum_two_writings_agree():
    """exp(i(kz - k0 n0) dz) from the dispersion relation equals
    g(zeta_fs) = exp(iK(-1+sqrt(1+zeta_fs))) (Eq. exp_prop_planewave), evanescent part included."""
    g = wl.Grid(64, 48, 0.125, 0.2)
    rng = np.random.default_rng(0)
    w = (rng.standard_normal((g.ny, g.nx)) + 1j * rng.standard_normal((g.ny, g.nx)))[None]
    n0, dz = 1.2, 0.35
    a = pr.angular_spectrum(w, g.dx, g.dy, K0, n0, dz, 2)
    z = ops.zeta_fs(g.nx, g.ny, g.dx, g.dy, K0 * n0)
    b = np.fft.ifft2(al.target(z, K0 * n0 * dz) ** 2 * np.fft.fft2(w[0]))[None]
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_rational_step_close_to_exact_angular_spectrum():
    """The rational propagator differs from the exact one by exactly
    ||(r^s - g^s) w_hat|| (Parseval), which is small for the fitted table."""
    T = table("homogeneous_aperture_1024")
    W = wl.homogeneous_aperture_1024(5, n=128)
    g = W.beams[0].grid
    w0 = W.beams[0].w0
    s = 5
    approx = pr.homogeneous_rational_step(w0, g.dx, g.dy, K0, T, s)
    exact = pr.angular_spectrum(w0, g.dx, g.dy, K0, 1.0, W.dz, s)
    z = ops.zeta_fs(g.nx, g.ny, g.dx, g.dy, K0)
    bound = np.linalg.norm((T(z) ** s - al.target(z, T.K) ** s) * np.fft.fft2(w0[0])) / math.sqrt(z.size)
    diff = np.linalg.norm(approx - exact)
    assert abs(diff - bound) <= 1e-9 * np.linalg.norm(exact)
    # soft: the hard-edged aperture excites the modes next to zeta = -1 where the fit is weakest
    assert diff / np.linalg.norm(exact) < 1e-2


def test_spectral_mapping_of_the_step_matrix():
    """Eq. (eq_spectra_operators): r0 I + sum r_k (Z - p_k)^-1 has eigenvalues
    r(lambda_i) on the eigenvectors of Z (dense, 12x12 scalar, lossy medium)."""
    T = table("plain_scalar_64")
    W = wl.small_scalar(12, dx=0.125, border=2)
    b = W.beams[0]
    g = b.grid
    med = ops.Medium(b.medium(0), g.dx, g.dy, K0, 1.0, 1)
    Z = ops.dense_Z(med)
    n = Z.shape[0]
    S = T.r0 * np.eye(n)
    for p, r in zip(T.poles, T.residues):
        S = S + r * np.linalg.inv(Z - p * np.eye(n))
    lam, Q = np.linalg.eig(Z)
    D = np.linalg.solve(Q, S @ Q)
    np.testing.assert_allclose(np.diag(D), T(lam), atol=1e-9)
    assert np.abs(D - np.diag(np.diag(D))).max() < 1e-8


@pytest.mark.parametrize("maker", [wl.small_scalar, wl.small_vector])
def test_dense_step_equals_gmres_step(maker):
    W = maker(16)
    T = table("plain_scalar_64")
    b = W.beams[0]
    g = b.grid
    med = ops.Medium(b.medium(0), g.dx, g.dy, W.k0, W.n0, W.ncomp)
    a, _ = pr.step(med, b.w0, T, solver="dense")
    c, st = pr.step(med, b.w0, T, solver="gmres", tol=1e-13)
    assert np.linalg.norm(a - c) / np.linalg.norm(a) < 1e-10


def test_step_is_linear():
    W = wl.small_scalar(16)
    T = table("plain_scalar_64")
    g = W.beams[0].grid
    med = ops.Medium(W.beams[0].medium(0), g.dx, g.dy, K0, 1.0, 1)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((1, g.ny, g.nx)) + 0j
    v = rng.standard_normal((1, g.ny, g.nx)) * 1j
    a, b = 0.3 - 1.1j, 2.0 + 0.5j
    su = pr.step(med, u, T, solver="dense")[0]
    sv = pr.step(med, v, T, solver="dense")[0]
    suv = pr.step(med, a * u + b * v, T, solver="dense")[0]
    np.testing.assert_allclose(suv, a * su + b * sv, atol=1e-11)


def test_homogeneous_step_commutes_with_translation():
    T = table("plain_scalar_64")
    g = wl.Grid(32, 32, 0.125, 0.125)
    w = wl.gaussian_beam(g, 0.5)[None]
    med = ops.Medium(np.ones((32, 32)), g.dx, g.dy, K0, 1.0, 1)
    a = pr.step(med, np.roll(w, (3, -5), axis=(1, 2)), T, tol=1e-13)[0]
    b = np.roll(pr.step(med, w, T, tol=1e-13)[0], (3, -5), axis=(1, 2))
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_lossless_step_does_not_amplify():
    """Real n^2 and no border: Z is Hermitian (scalar), so ||r(Z) w|| <= max|r| on
    its real spectrum <= 1 + fit error, since |g| <= 1 on the real axis."""
    T = table("plain_scalar_64")
    g = wl.Grid(16, 16, 0.125, 0.125)
    rng = np.random.default_rng(9)
    n2 = 1 + 0.08 * rng.uniform(-1, 1, (16, 16))
    med = ops.Medium(n2, g.dx, g.dy, K0, 1.0, 1)
    w = (rng.standard_normal((1, 16, 16)) + 1j * rng.standard_normal((1, 16, 16)))
    lam = np.linalg.eigvalsh(ops.dense_Z(med))
    bound = np.abs(T(lam)).max()
    assert bound <= 1 + 1e-3
    out = pr.step(med, w, T, solver="dense")[0]
    assert np.linalg.norm(out) <= bound * np.linalg.norm(w) * (1 + 1e-12)
