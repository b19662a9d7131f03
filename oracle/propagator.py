"""One z-step of the exponential one-way propagator, and runs of steps.

Oracle (test infrastructure).

Sec. 2, Eqs. (Wk_define), (approx_prop), (W_k_def): with the rational
approximation in partial fractions r(zeta) = r0 + sum_k r_k/(zeta - p_k)
(the e^{-iK} factor folded into r0 and r_k),

    w(z + dz) = r0 w(z) + sum_k r_k x_k,     (Z - p_k I) x_k = w(z).

Each x_k is found either by dense LU of the shifted matrix (small grids: the
plain definition, no iteration) or by right-preconditioned GMRES with the
free-space preconditioner (Sec. 4.2).  Sec. 2 also updates n (hence delta and
psi) between steps: step s uses the slab the workload gives for s.

The exact propagator in a homogeneous medium (Eq. exp_prop_planewave) is
diagonal in Fourier space: w(dz) = IFFT[exp(iK(-1 + sqrt(1 + zeta_fs))) FFT w],
and the rational approximation's homogeneous step (Eq. approx_fs_prop) is
IFFT[r(zeta_fs) FFT w].
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.linalg

from . import aaa_lawson, gmres as gm, operators as ops


@dataclasses.dataclass
class StepStats:
    iterations: List[int]        # Arnoldi steps per pole
    rel_residuals: List[float]   # true relative residual per pole


def solve_shifted_dense(med: ops.Medium, w: np.ndarray, pole: complex) -> np.ndarray:
    """x = (Z - p I)^-1 w by dense LU (Eq. W_k_def)."""
    A = ops.dense_Z(med) - pole * np.eye(med.ncomp * med.nx * med.ny)
    x = scipy.linalg.lu_solve(scipy.linalg.lu_factor(A), w.ravel())
    return x.reshape(w.shape)


def preconditioner_shift(med: ops.Medium, precond: str) -> complex:
    """Constant medium of the preconditioner, as delta = (n^2 - n0^2)/n0^2.

    "freespace": the n = n0 problem of Eq. Z_bar_fs_def (delta = 0).
    "mean": the constant-index problem whose n^2 is the mean of the slab's n^2
    over the grid, so delta = mean(delta).  Sec. 4.2 builds its free-space
    preconditioner from the same difference matrices as Z, PML included; on the
    periodic grid the absorber lives in Im n^2, and the mean carries its
    average loss while keeping the solve diagonal in Fourier space.
    """
    if precond == "freespace":
        return 0.0
    if precond == "mean":
        return complex(med.delta.mean())
    raise ValueError(precond)


def solve_shifted_gmres(med: ops.Medium, w: np.ndarray, pole: complex, restart: int = 20,
                        tol: float = 1e-12, max_cycles: int = 50,
                        x0: Optional[np.ndarray] = None, precond: str = "freespace") -> gm.GmresResult:
    """x = (Z - p I)^-1 w by GMRES right-preconditioned with (Z_fs + dbar - p I),
    dbar = preconditioner_shift(med, precond) (0 for the paper's free-space solve)."""
    dbar = preconditioner_shift(med, precond)
    return gm.gmres(lambda v: med.apply_shifted(v, pole),
                    lambda v: med.freespace_solve(v, pole - dbar),
                    w, x0=x0, restart=restart, tol=tol, max_cycles=max_cycles)


def step(med: ops.Medium, w: np.ndarray, table: aaa_lawson.PoleTable, solver: str = "gmres",
         restart: int = 20, tol: float = 1e-12, max_cycles: int = 50, precond: str = "freespace"):
    """w(z+dz) = r0 w + sum_k r_k (Z - p_k)^-1 w  (Eq. approx_prop).  w: (ncomp, ny, nx).
    ``precond`` only changes how GMRES reaches each (Z - p_k)^-1 w."""
    out = table.r0 * w
    its, rels = [], []
    for p, r in zip(table.poles, table.residues):
        if solver == "dense":
            x = solve_shifted_dense(med, w, p)
            its.append(0)
            rels.append(float(np.linalg.norm(med.apply_shifted(x, p) - w) / np.linalg.norm(w)))
        else:
            res = solve_shifted_gmres(med, w, p, restart, tol, max_cycles, precond=precond)
            if not res.converged:
                raise RuntimeError(f"GMRES did not converge for pole {p}: {res.rel_residual:.3e}")
            x = res.x
            its.append(res.iterations)
            rels.append(res.rel_residual)
        out = out + r * x
    return out, StepStats(its, rels)


def run(beam, k0: float, n0: float, table: aaa_lawson.PoleTable, ncomp: int, nsteps: int,
        solver: str = "gmres", restart: int = 20, tol: float = 1e-12, first_step: int = 0,
        w: Optional[np.ndarray] = None, return_stats: bool = False):
    """March ``nsteps`` steps from ``w`` (default: the beam's initial field)."""
    g = beam.grid
    w = beam.w0.copy() if w is None else w.copy()
    med = None
    stats = []
    for s in range(first_step, first_step + nsteps):
        if med is None or beam.medium_changes(s):
            med = ops.Medium(beam.medium(s), g.dx, g.dy, k0, n0, ncomp)
        w, st = step(med, w, table, solver, restart, tol)
        stats.append(st)
    return (w, stats) if return_stats else w


def homogeneous_rational_step(w: np.ndarray, dx: float, dy: float, k0n0: float,
                              table: aaa_lawson.PoleTable, nsteps: int = 1) -> np.ndarray:
    """IFFT[r(zeta_fs)^s FFT w]: the rational propagator in a homogeneous medium (Eq. approx_fs_prop)."""
    ny, nx = w.shape[-2:]
    z = ops.zeta_fs(nx, ny, dx, dy, k0n0)
    R = table(z) ** nsteps
    return np.stack([ops.ifft2(R * ops.fft2(c)) for c in w.reshape(-1, ny, nx)]).reshape(w.shape)


def angular_spectrum(w: np.ndarray, dx: float, dy: float, k0: float, n0: float, dz: float,
                     nsteps: int = 1) -> np.ndarray:
    """Exact envelope propagation in a homogeneous medium (Eq. exp_prop_planewave):
    each plane wave gains exp(i (kz - k0 n0) s dz) with kz = sqrt((k0 n0)^2 - kx^2 - ky^2),
    Im kz >= 0 (evanescent waves decay)."""
    ny, nx = w.shape[-2:]
    kx = ops.wavenumbers(nx, dx)[None, :]
    ky = ops.wavenumbers(ny, dy)[:, None]
    kz = np.sqrt((k0 * n0) ** 2 - kx ** 2 - ky ** 2 + 0j)
    G = np.exp(1j * (kz - k0 * n0) * dz * nsteps)
    return np.stack([ops.ifft2(G * ops.fft2(c)) for c in w.reshape(-1, ny, nx)]).reshape(w.shape)
