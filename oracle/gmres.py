"""Right-preconditioned restarted GMRES with Householder Arnoldi (Sec. 4.2).

Oracle (test infrastructure).  The paper joins a generic right-preconditioned
GMRES (Saad's algorithm) to the free-space preconditioner and keeps the
Krylov basis orthogonal with Householder transformations.  Read as:

  solve A x = b, A = Z - b_k I, preconditioner M = Z_fs - b_k I, applied on the
  right: minimise ||b - A(x0 + M^-1 V y)|| over the Krylov space of A M^-1
  started from r0 = b - A x0.

Householder Arnoldi: reflectors P_j = I - 2 u_j u_j^H (u_j zero above index j)
are chosen so that P_j ... P_0 r0 and P_j ... P_0 (A M^-1 v_{j-1}) are zero
below index j; the basis vectors are v_j = P_0 ... P_j e_j and the Hessenberg
column is the first j+1 entries of the reflected vector.  The small least
squares problem min || beta e_0 - H y || is solved each step (numpy lstsq);
its residual decides when a cycle ends, and the true residual
||b - A x|| / ||b|| <= tol decides convergence.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np


@dataclasses.dataclass
class GmresResult:
    x: np.ndarray
    iterations: int          # total Arnoldi steps over all cycles
    cycles: int
    rel_residual: float      # true ||b - A x|| / ||b||
    converged: bool


def _reflector(z: np.ndarray, j: int):
    """Unit u (zero above j) and alpha with (I - 2uu^H) z = [z[:j], alpha, 0, ...]."""
    tail = z[j:]
    nrm = np.linalg.norm(tail)
    u = np.zeros_like(z)
    if nrm == 0.0:
        return u, 0.0 + 0.0j
    # alpha = -exp(i arg z_j) ||tail|| (the sign that avoids cancellation); the
    # phase from the angle stays exact when z_j is subnormal, where z_j/|z_j| overflows
    phase = np.exp(1j * np.angle(tail[0])) if tail[0] != 0 else 1.0
    alpha = -phase * nrm
    u[j:] = tail
    u[j] -= alpha
    un = np.linalg.norm(u)
    if un == 0.0:
        return np.zeros_like(z), alpha
    return u / un, alpha


def _apply_P(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    return v - 2.0 * u * np.vdot(u, v)


def _lsq_qr(Hk: np.ndarray, g: np.ndarray) -> np.ndarray:
    """min ||g - Hk y|| by a Householder QR of Hk (full column rank)."""
    Q, R = np.linalg.qr(Hk)
    return np.linalg.solve(R, Q.conj().T @ g)


def _lsq(Hk: np.ndarray, g: np.ndarray) -> np.ndarray:
    """The GMRES least-squares problem min ||beta e_1 - Hbar y|| (Saad & Schultz,
    1986): LAPACK's SVD-based driver, or the QR solve when that driver reports
    that its SVD did not converge (seen with some BLAS builds).  Hbar has full
    column rank before a breakdown, where both give the same y."""
    try:
        return np.linalg.lstsq(Hk, g, rcond=None)[0]
    except np.linalg.LinAlgError:
        return _lsq_qr(Hk, g)


def gmres(apply_A: Callable[[np.ndarray], np.ndarray],
          apply_Minv: Callable[[np.ndarray], np.ndarray],
          b: np.ndarray, x0: Optional[np.ndarray] = None, restart: int = 20,
          tol: float = 1e-12, max_cycles: int = 50) -> GmresResult:
    shape = b.shape
    bf = b.ravel().astype(np.complex128)
    n = bf.size
    bnorm = np.linalg.norm(bf)
    x = np.zeros(n, np.complex128) if x0 is None else x0.ravel().astype(np.complex128).copy()
    A = lambda v: apply_A(v.reshape(shape)).ravel()
    Minv = lambda v: apply_Minv(v.reshape(shape)).ravel()
    if bnorm == 0.0:
        return GmresResult(x.reshape(shape), 0, 0, 0.0, True)

    iters = 0
    for cycle in range(max_cycles + 1):
        r = bf - A(x)
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol or cycle == max_cycles:
            return GmresResult(x.reshape(shape), iters, cycle, float(rel), rel <= tol)
        m = min(restart, n)
        U = []
        H = np.zeros((m + 1, m), np.complex128)
        z = r
        beta = 0.0
        k = 0                                  # columns of H filled
        for j in range(m + 1):
            u, alpha = _reflector(z, j)
            U.append(u)
            if j == 0:
                beta = alpha
            else:
                H[:j, j - 1] = z[:j]
                H[j, j - 1] = alpha
                k = j
                g = np.zeros(k + 1, np.complex128)
                g[0] = beta
                y = _lsq(H[:k + 1, :k], g)
                est = np.linalg.norm(g - H[:k + 1, :k] @ y)
                if est <= tol * bnorm or j == m or alpha == 0.0:
                    break
            # v_j = P_0 ... P_j e_j
            v = np.zeros(n, np.complex128)
            v[j] = 1.0
            for i in range(j, -1, -1):
                v = _apply_P(U[i], v)
            z = A(Minv(v))
            iters += 1
            for i in range(j + 1):
                z = _apply_P(U[i], z)
        # s = sum_i y_i v_i, v_i = P_0..P_i e_i, by Horner from the innermost reflector
        s = np.zeros(n, np.complex128)
        for i in range(k - 1, -1, -1):
            s[i] += y[i]
            s = _apply_P(U[i], s)
        x = x + Minv(s)
    raise AssertionError("unreachable")
