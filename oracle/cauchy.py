"""The pseudo-differential propagator with the Cauchy-integral square root (Sec. 3.2, App. A).

Oracle (test infrastructure).

Square root.  The Möbius map w = (zeta + 1 + i alpha)/(zeta + 1 - i alpha)
(Eq. eq:Mobius) sends the branch point at zeta = -infinity to w = 1; with the
cut of g(w) = sqrt(1 + zeta(w)) on [-1, 1], Cauchy's formula on a contour
around the cut (App. A) gives

    g(w) = c_alpha (1 - (1/pi) int_{-1}^{1} sqrt((1+eta)/(1-eta)) / (eta - w) d eta),
    c_alpha = sqrt(alpha) e^{i pi/4}.

An N-point Gauss-Jacobi rule for the weight (1 - eta)^{-1/2} (1 + eta)^{1/2}
(nodes eta_j, weights omega_j) and the map back to zeta give partial fractions
(Eq. pf_sqrt_exp):

    sqrt(1 + zeta) ~ (c_alpha + sum_j wt_j) - sum_j i alpha wt_j (1 + sigma_j) / ((1 + i alpha sigma_j) + zeta),
    wt_j = (c_alpha/pi) omega_j/(1 - eta_j),   sigma_j = (1 + eta_j)/(1 - eta_j),

i.e. S(zeta) = s0 + sum_j s_j/(zeta - q_j) with q_j = -(1 + i alpha sigma_j),
s_j = -i alpha wt_j (1 + sigma_j), s0 = c_alpha + sum_j wt_j.

Propagator (Eqs. eq_barZfactor2, eq:ApproxPropagator_W): the envelope obeys

    dw/dz = i k0 n0 (S(Z) - I) w,

where S(Z) w = s0 w + sum_j W_j and (Z - q_j) W_j = s_j w: the auxiliary
systems of Eq. eq:Auxiliary_W, shifted solves of the same kind as Eq. W_k_def,
solved by the same preconditioned GMRES.  The paper names no z-integrator;
the reading here is the classical fourth-order Runge-Kutta method with M equal
substeps of h = dz/M per step.
"""
from __future__ import annotations

import cmath
import math

import numpy as np
import scipy.special

from . import aaa_lawson as al
from . import propagator as pr


def gauss_jacobi(N: int):
    """Nodes and weights of the N-point rule for int_{-1}^{1} f(eta) sqrt((1+eta)/(1-eta)) d eta."""
    x, w = scipy.special.roots_jacobi(N, -0.5, 0.5)
    return x, w


def cauchy_sqrt_table(N: int = 25, alpha: float = 1.0) -> al.PoleTable:
    """S(zeta) ~ sqrt(1 + zeta) in partial fractions (Eq. pf_sqrt_exp); K is unused (0)."""
    eta, om = gauss_jacobi(N)
    c = math.sqrt(alpha) * cmath.exp(1j * math.pi / 4)
    wt = (c / math.pi) * om / (1 - eta)
    sig = (1 + eta) / (1 - eta)
    poles = -(1 + 1j * alpha * sig)
    res = -1j * alpha * wt * (1 + sig)
    s0 = c + wt.sum()
    order = np.argsort(poles.real)
    return al.PoleTable(0.0, poles[order], res[order], complex(s0), -4.0, 2.0, (), float("nan"))


def sqrt_quadrature_form(z, N: int = 25, alpha: float = 1.0):
    """The Gauss-Jacobi sum written as in the paper before the synthetic division
    (Eq. prime_sqrt_exp, scalar form):
    c (1 + (1/pi) sum_j omega_j/(1 - eta_j) (1 - i alpha + z)/(1 + i alpha sigma_j + z))."""
    eta, om = gauss_jacobi(N)
    c = math.sqrt(alpha) * cmath.exp(1j * math.pi / 4)
    sig = (1 + eta) / (1 - eta)
    z = np.asarray(z, np.complex128)[..., None]
    return c * (1 + (1 / math.pi) * np.sum(om / (1 - eta) * (1 - 1j * alpha + z) / (1 + 1j * alpha * sig + z), -1))


def rk4_step(apply_L, w: np.ndarray, h: float) -> np.ndarray:
    """One classical Runge-Kutta step of dw/dz = L w."""
    k1 = apply_L(w)
    k2 = apply_L(w + 0.5 * h * k1)
    k3 = apply_L(w + 0.5 * h * k2)
    k4 = apply_L(w + h * k3)
    return w + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)


def apply_S(med, v: np.ndarray, table: al.PoleTable, tol: float = 1e-12, precond: str = "freespace") -> np.ndarray:
    """S(Z) v = s0 v + sum_j s_j (Z - q_j)^-1 v, each solve by preconditioned GMRES."""
    out = table.r0 * v
    for q, s in zip(table.poles, table.residues):
        r = pr.solve_shifted_gmres(med, v, q, tol=tol, max_cycles=200, precond=precond)
        if not r.converged:
            raise RuntimeError(f"GMRES did not converge for the shift {q}")
        out = out + s * r.x
    return out


def pseudodiff_step(med, w: np.ndarray, table: al.PoleTable, k0n0: float, dz: float, substeps: int,
                    tol: float = 1e-12) -> np.ndarray:
    """Advance w by dz: `substeps` RK4 steps of dw/dz = i k0 n0 (S(Z) - I) w."""
    h = dz / substeps
    L = lambda v: 1j * k0n0 * (apply_S(med, v, table, tol) - v)
    for _ in range(substeps):
        w = rk4_step(L, w, h)
    return w


def rk4_amplification(lam: np.ndarray, h: float) -> np.ndarray:
    """The RK4 growth factor 1 + x + x^2/2 + x^3/6 + x^4/24, x = h lam, of dw/dz = lam w."""
    x = h * lam
    return 1 + x + x ** 2 / 2 + x ** 3 / 6 + x ** 4 / 24


def homogeneous_pseudodiff(w: np.ndarray, dx: float, dy: float, k0n0: float, table: al.PoleTable, dz: float,
                           substeps: int, nsteps: int = 1) -> np.ndarray:
    """The pseudo-differential RK4 step in a homogeneous medium, diagonal in Fourier
    space: each plane wave is multiplied by rk4_amplification(i k0 n0 (S(zeta_fs) - 1), h)^M."""
    from . import operators as ops
    ny, nx = w.shape[-2:]
    z = ops.zeta_fs(nx, ny, dx, dy, k0n0)
    G = rk4_amplification(1j * k0n0 * (table(z) - 1), dz / substeps) ** (substeps * nsteps)
    return np.stack([ops.ifft2(G * ops.fft2(c)) for c in w.reshape(-1, ny, nx)]).reshape(w.shape)
