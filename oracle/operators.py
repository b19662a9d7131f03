"""The operator matrix Z of the envelope equation and its free-space part.

Oracle (test infrastructure).  Discretisation: Fourier pseudo-spectral on the
periodic transverse grid (x fastest; arrays ``[y, x]``), with the absorbing
border carried by Im n^2.

Sec. 2, Eq. (Z_bar_eq):
    Z = (k0 n0)^-2 [[D + k0^2 (n^2-n0^2) + psi_xx + psi_x d_x,  psi_xy + psi_y d_x],
                    [psi_xy + psi_x d_y,  D + k0^2 (n^2-n0^2) + psi_yy + psi_y d_y]]
with D the transverse Laplacian and psi = ln n^2.  Written with the scaled
quantities of Sec. 4.2 (Eq. Z_bar_fs_def): Dt = D/(k0 n0)^2,
delta = (n^2 - n0^2)/n0^2 and psit_* = psi_*/(k0 n0)^2,
    (Z v)_1 = Dt v1 + delta v1 + psit_xx v1 + psit_x d_x v1 + psit_xy v2 + psit_y d_x v2
    (Z v)_2 = psit_xy v1 + psit_x d_y v1 + Dt v2 + delta v2 + psit_yy v2 + psit_y d_y v2
The scalar operator drops the psi terms (Sec. 2, the reduction to scalar
Helmholtz).  The free-space operator Z_fs is Dt on each component (Eq.
Z_bar_fs_def); on a plane wave exp(i(kx x + ky y)) it is the number
zeta_fs = -(kx^2 + ky^2)/(k0 n0)^2 (Sec. 3, below Eq. exp_prop_planewave).

Spectral derivatives: d/dx -> i kx with the Nyquist entry set to 0 for first
derivatives of an even-length grid; the Laplacian keeps -kx^2 at Nyquist.
"""
from __future__ import annotations

import numpy as np
import scipy.fft
import scipy.linalg

# Threads of the 2-D transforms (scipy.fft's ``workers``); 1 unless a caller
# that times the oracle on all host cores sets it.  Results do not depend on it
# beyond rounding order.
FFT_WORKERS = 1


def fft2(v: np.ndarray) -> np.ndarray:
    return scipy.fft.fft2(v, workers=FFT_WORKERS)


def ifft2(v: np.ndarray) -> np.ndarray:
    return scipy.fft.ifft2(v, workers=FFT_WORKERS)


def wavenumbers(n: int, d: float) -> np.ndarray:
    """Angular wavenumbers of an n-point periodic grid of spacing d (FFT order)."""
    return 2.0 * np.pi * np.fft.fftfreq(n, d)


def first_derivative_symbol(n: int, d: float) -> np.ndarray:
    """i*k for d/dx, with the unpaired Nyquist mode of an even grid set to zero."""
    k = 1j * wavenumbers(n, d)
    if n % 2 == 0:
        k[n // 2] = 0.0
    return k


def zeta_fs(nx: int, ny: int, dx: float, dy: float, k0n0: float) -> np.ndarray:
    """Symbol of Z_fs = Dt: -(kx^2 + ky^2)/(k0 n0)^2, shape (ny, nx)."""
    kx = wavenumbers(nx, dx)
    ky = wavenumbers(ny, dy)
    return -(ky[:, None] ** 2 + kx[None, :] ** 2) / k0n0 ** 2


def delta_of(n2: np.ndarray, n0: float) -> np.ndarray:
    """delta = (n^2 - n0^2)/n0^2, i.e. k0^2 (n^2 - n0^2) scaled by (k0 n0)^-2 (Eq. Z_bar_eq)."""
    return (n2 - n0 ** 2) / n0 ** 2


def psi_terms(n2: np.ndarray, dx: float, dy: float, k0n0: float) -> dict:
    """psi = Log n^2 (principal) and its spectral derivatives scaled by (k0 n0)^-2.

    Returns dict with keys x, y, xx, yy, xy (each (ny, nx) complex128).
    """
    ny, nx = n2.shape
    psi = np.log(n2.astype(np.complex128))
    P = fft2(psi)
    ikx = first_derivative_symbol(nx, dx)[None, :]
    iky = first_derivative_symbol(ny, dy)[:, None]
    kx = wavenumbers(nx, dx)[None, :]
    ky = wavenumbers(ny, dy)[:, None]
    s = 1.0 / k0n0 ** 2
    return {
        "x": s * ifft2(ikx * P),
        "y": s * ifft2(iky * P),
        "xx": s * ifft2(-(kx ** 2) * P),
        "yy": s * ifft2(-(ky ** 2) * P),
        "xy": s * ifft2(ikx * iky * P),
    }


class Medium:
    """Pointwise coefficients of Z for one slab: delta and (vector only) psi terms."""

    def __init__(self, n2: np.ndarray, dx: float, dy: float, k0: float, n0: float, ncomp: int):
        self.n2 = np.asarray(n2, np.complex128)
        self.ny, self.nx = self.n2.shape
        self.dx, self.dy = dx, dy
        self.k0n0 = k0 * n0
        self.ncomp = ncomp
        self.delta = delta_of(self.n2, n0)
        self.zfs = zeta_fs(self.nx, self.ny, dx, dy, self.k0n0)
        self.psi = psi_terms(self.n2, dx, dy, self.k0n0) if ncomp == 2 else None
        self.ikx = first_derivative_symbol(self.nx, dx)[None, :]
        self.iky = first_derivative_symbol(self.ny, dy)[:, None]

    # --- derivative helpers (spectral) ---
    def dxf(self, v):
        return ifft2(self.ikx * fft2(v))

    def dyf(self, v):
        return ifft2(self.iky * fft2(v))

    def lap_t(self, v):
        """Scaled transverse Laplacian Dt v."""
        return ifft2(self.zfs * fft2(v))

    def apply_Z(self, v: np.ndarray) -> np.ndarray:
        """Z v for v of shape (ncomp, ny, nx), Eq. (Z_bar_eq)."""
        out = np.empty_like(v, dtype=np.complex128)
        if self.ncomp == 1:
            out[0] = self.lap_t(v[0]) + self.delta * v[0]
            return out
        p = self.psi
        v1, v2 = v[0], v[1]
        out[0] = (self.lap_t(v1) + self.delta * v1 + p["xx"] * v1 + p["x"] * self.dxf(v1)
                  + p["xy"] * v2 + p["y"] * self.dxf(v2))
        out[1] = (p["xy"] * v1 + p["x"] * self.dyf(v1)
                  + self.lap_t(v2) + self.delta * v2 + p["yy"] * v2 + p["y"] * self.dyf(v2))
        return out

    def apply_shifted(self, v: np.ndarray, pole: complex) -> np.ndarray:
        """(Z - b I) v, the coefficient matrix of Eq. (W_k_def)."""
        return self.apply_Z(v) - pole * v

    def freespace_solve(self, v: np.ndarray, pole: complex) -> np.ndarray:
        """(Z_fs - b I)^-1 v per component: the preconditioner of Sec. 4.2.1.

        On the periodic grid Dt is diagonal in Fourier space, so the solve is
        FFT -> divide by (zeta_fs - b) -> inverse FFT.
        """
        out = np.empty_like(v, dtype=np.complex128)
        for c in range(v.shape[0]):
            out[c] = ifft2(fft2(v[c]) / (self.zfs - pole))
        return out


# ---------------------------------------------------------------------------
# Dense forms (small grids only): used as independent checks.
# ---------------------------------------------------------------------------

def dft_matrix(n: int) -> np.ndarray:
    j = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(j, j) / n)


def spectral_matrix(n: int, symbol: np.ndarray) -> np.ndarray:
    """Dense F^-1 diag(symbol) F for an n-point grid."""
    F = dft_matrix(n)
    return (F.conj().T / n) @ (symbol[:, None] * F)


def dense_second_derivative(n: int, d: float, k0n0: float) -> np.ndarray:
    """Scaled dense second-derivative matrix: (k0 n0)^-2 d^2/dx^2."""
    return spectral_matrix(n, -(wavenumbers(n, d) ** 2) / k0n0 ** 2)


def dense_first_derivative(n: int, d: float) -> np.ndarray:
    return spectral_matrix(n, first_derivative_symbol(n, d))


def dense_Z(med: Medium) -> np.ndarray:
    """Dense matrix of Z (ncomp*ny*nx square), unknowns ordered [comp, y, x].

    Built from Kronecker products of 1-D spectral matrices, independently of
    the FFT application in Medium.apply_Z.
    """
    nx, ny = med.nx, med.ny
    Ix, Iy = np.eye(nx), np.eye(ny)
    Dxx = dense_second_derivative(nx, med.dx, med.k0n0)
    Dyy = dense_second_derivative(ny, med.dy, med.k0n0)
    lap = np.kron(Iy, Dxx) + np.kron(Dyy, Ix)
    D = np.diag(med.delta.ravel())
    if med.ncomp == 1:
        return lap + D
    Dx = np.kron(Iy, dense_first_derivative(nx, med.dx))
    Dy = np.kron(dense_first_derivative(ny, med.dy), Ix)
    p = {k: np.diag(v.ravel()) for k, v in med.psi.items()}
    Z11 = lap + D + p["xx"] + p["x"] @ Dx
    Z12 = p["xy"] + p["y"] @ Dx
    Z21 = p["xy"] + p["x"] @ Dy
    Z22 = lap + D + p["yy"] + p["y"] @ Dy
    return np.block([[Z11, Z12], [Z21, Z22]])


def sylvester_freespace_solve(rhs: np.ndarray, dx: float, dy: float, k0n0: float,
                              pole: complex) -> np.ndarray:
    """Free-space solve written as the Sylvester equation of Eq. (fs_sylvester).

    (Dy - b/2 I) W + W (Dx - b/2 I)^T = rhs for one (ny, nx) component, with
    the symmetric split alpha = beta = b/2 of Eq. (shift_identity), solved by
    Bartels-Stewart (scipy.linalg.solve_sylvester).
    """
    ny, nx = rhs.shape
    A = dense_second_derivative(ny, dy, k0n0) - 0.5 * pole * np.eye(ny)
    B = (dense_second_derivative(nx, dx, k0n0) - 0.5 * pole * np.eye(nx)).T
    return scipy.linalg.solve_sylvester(A, B, rhs)
