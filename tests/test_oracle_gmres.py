"""Pins of the GMRES oracle (Sec. 4.2) against direct solves."""
import json
import math
import os

import numpy as np
import pytest

from oracle import aaa_lawson as al, gmres as gm, operators as ops, propagator as pr
from paper_2410_17446_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_numbers.json")))


def test_gmres_on_random_nonnormal_matrix_with_restarts():
    """Generic right-preconditioned restarted GMRES against numpy.linalg.solve."""
    rng = np.random.default_rng(0)
    n = 60
    A = np.eye(n) * 3 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    A[np.triu_indices(n, 1)] *= 2.0
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    d = np.diag(A).copy()
    res = gm.gmres(lambda v: A @ v, lambda v: v / d, b, restart=7, tol=1e-12, max_cycles=200)
    assert res.converged and res.cycles > 1
    np.testing.assert_allclose(res.x, np.linalg.solve(A, b), atol=1e-10)


def test_gmres_zero_rhs():
    res = gm.gmres(lambda v: 2 * v, lambda v: v, np.zeros(5, complex))
    assert res.converged and res.iterations == 0 and np.all(res.x == 0)


@pytest.mark.parametrize("maker", [wl.small_scalar, wl.small_vector])
def test_gmres_matches_dense_lu(maker):
    """Eq. (W_k_def) solved by preconditioned GMRES equals its dense LU solution."""
    W = maker(16)
    b = W.beams[0]
    g = b.grid
    med = ops.Medium(b.medium(0), g.dx, g.dy, W.k0, W.n0, W.ncomp)
    for pole in [-0.98 - 0.02j, -0.5 - 0.6j, 1.5 - 1.0j]:
        xd = pr.solve_shifted_dense(med, b.w0, pole)
        r = pr.solve_shifted_gmres(med, b.w0, pole, tol=1e-13, max_cycles=100)
        assert r.converged
        assert np.linalg.norm(r.x - xd) / np.linalg.norm(xd) < 1e-10


def test_homogeneous_medium_needs_one_iteration():
    """Sec. 4.2: in a homogeneous medium the free-space preconditioner is exact,
    and the solve takes one GMRES iteration and equals the free-space solve."""
    g = wl.Grid(32, 24, 0.25, 0.25)
    w = wl.gaussian_beam(g, 1.5)[None]
    med = ops.Medium(np.ones((g.ny, g.nx)), g.dx, g.dy, 2 * math.pi, 1.0, 1)
    for pole in [-0.999 - 0.001j, 0.4 - 1.6j]:
        r = pr.solve_shifted_gmres(med, w, pole, tol=1e-12)
        assert r.iterations == GOLD["gmres_homogeneous_iterations"]["iterations"]
        np.testing.assert_allclose(r.x, med.freespace_solve(w, pole), atol=1e-13)


def test_least_squares_qr_branch_matches_lstsq():
    """The QR fallback of the Hessenberg least-squares solve gives lstsq's y."""
    import numpy as np
    from oracle import gmres as gm
    rng = np.random.default_rng(5)
    for k in (1, 4, 19):
        H = np.triu(rng.standard_normal((k + 1, k)) + 1j * rng.standard_normal((k + 1, k)), -1)
        g = np.zeros(k + 1, complex)
        g[0] = 2.5
        y_ref = np.linalg.lstsq(H, g, rcond=None)[0]
        assert np.allclose(gm._lsq_qr(H, g), y_ref, rtol=1e-12, atol=1e-12)
        assert np.allclose(gm._lsq(H, g), y_ref, rtol=1e-12, atol=1e-12)


def test_reflector_with_subnormal_leading_entry():
    """A subnormal leading entry still gives a unit reflector mapping z to alpha e_j."""
    import numpy as np
    from oracle import gmres as gm
    z = np.array([0.3 + 0.1j, 5e-320 + 3e-320j, 1.0 - 2.0j, 0.5j])
    u, alpha = gm._reflector(z, 1)
    assert np.isfinite(u).all() and abs(np.linalg.norm(u) - 1.0) < 1e-14
    r = gm._apply_P(u, z)
    assert np.allclose(r[2:], 0.0, atol=1e-14) and abs(r[1] - alpha) < 1e-14 and r[0] == z[0]
    assert abs(abs(alpha) - np.linalg.norm(z[1:])) < 1e-14
