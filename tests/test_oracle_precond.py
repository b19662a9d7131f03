"""The constant-index preconditioner (Sec. 4.2) against facts fixed outside it.

Right preconditioning changes only the path GMRES takes: for any fixed
invertible M, GMRES on (Z - p) M^-1 y = w with x = M^-1 y converges to the
unique x = (Z - p)^-1 w.  So the solution with M = Z_fs + mean(delta) - p must
equal dense LU of Z - p (the plain definition, no iteration), exactly as the
paper's free-space M = Z_fs - p does.  The iteration counts are the reason for
the choice: with an absorbing border the mean medium carries the border's
average loss, as the paper's preconditioner carries its PML.
"""
import math

import numpy as np
import pytest

from oracle import operators as ops
from oracle import propagator as pr
from paper_2410_17446_gb300 import workloads as wl


def _case(n=16, ncomp=1):
    W = wl.small_scalar(n) if ncomp == 1 else wl.small_vector(n)
    b = W.beams[0]
    med = ops.Medium(b.medium(0), b.grid.dx, b.grid.dy, W.k0, W.n0, ncomp)
    return med, b.w0


@pytest.mark.parametrize("ncomp", [1, 2])
def test_mean_preconditioner_reaches_the_dense_solution(ncomp):
    med, w = _case(16, ncomp)
    for p in (-1.0007 - 0.0018j, -0.4 - 0.01j, -3.2 - 0.2j):
        x_lu = pr.solve_shifted_dense(med, w, p)
        for precond in ("freespace", "mean"):
            r = pr.solve_shifted_gmres(med, w, p, tol=1e-13, max_cycles=200, precond=precond)
            assert r.converged
            assert np.linalg.norm(r.x - x_lu) / np.linalg.norm(x_lu) < 1e-9, (precond, p)


def test_mean_shift_is_the_mean_of_delta():
    """dbar = mean((n^2 - n0^2)/n0^2); for a homogeneous n != n0 it is exact, and
    GMRES then needs one step (the preconditioner is the operator)."""
    g = wl.Grid(16, 16, 0.25, 0.25)
    n2 = np.full((16, 16), 1.1 + 0.02j)
    med = ops.Medium(n2, g.dx, g.dy, 2 * math.pi, 1.0, 1)
    assert pr.preconditioner_shift(med, "mean") == pytest.approx(0.1 + 0.02j, abs=1e-15)
    assert pr.preconditioner_shift(med, "freespace") == 0.0
    w = wl.gaussian_beam(g, 1.0)[None]
    r = pr.solve_shifted_gmres(med, w, -1.0 - 0.001j, tol=1e-12, precond="mean")
    assert r.converged and r.iterations == 1
    r0 = pr.solve_shifted_gmres(med, w, -1.0 - 0.001j, tol=1e-12, precond="freespace")
    assert r0.iterations > 1


def test_mean_preconditioner_cuts_iterations_with_a_border():
    """Sine-product medium (eps 0.05, period 1.5) with the 0.2 quadratic border
    at 64^2: the hardest pole next to the branch point needs several times fewer
    Arnoldi steps, and the total over the poles drops."""
    from util import oracle_table
    W = wl.batched_scalar_1024(1, n=64)
    b = W.beams[0]
    med = ops.Medium(b.medium(0), b.grid.dx, b.grid.dy, W.k0, W.n0, 1)
    T = oracle_table("batched_scalar_1024")
    its = {}
    for precond in ("freespace", "mean"):
        its[precond] = [pr.solve_shifted_gmres(med, b.w0, p, tol=1e-10, max_cycles=100, precond=precond).iterations
                        for p in T.poles[:4]]
    assert its["mean"][0] * 2 <= its["freespace"][0], its
    assert sum(its["mean"]) < sum(its["freespace"]), its
