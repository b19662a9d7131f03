"""Recovery of the longitudinal field E3 from Gauss's law (Sec. 2).

Oracle (test infrastructure).  Sec. 2 propagates only the transverse envelope
(w1, w2) and notes that E3 can be recovered from Gauss's law, div D = 0 with
D = eps0 n^2 E, without giving a formula.  Reading used here:

* Within one step n^2 = n^2(x, y), so div D = 0 reads
  d_x (n^2 E1) + d_y (n^2 E2) + n^2 d_z E3 = 0.
* The z-derivative of the one-way field is taken from the reference medium:
  each plane-wave component of D exp(i(kx x + ky y)) advances as exp(i kz z)
  with kz = sqrt((k0 n0)^2 - kx^2 - ky^2) on the branch Im kz >= 0 (Eq.
  exp_prop_planewave; the envelope factor exp(i k0 n0 z) of Eq. vec_envelop
  is part of it).  Then i kx D1^ + i ky D2^ + i kz D3^ = 0, i.e.

      D3^ = -(kx D1^ + ky D2^) / kz,      E3 = D3 / n^2.

  Working with D' = (n^2/n0^2) E keeps the numbers at the field's scale:
  E3 = (n0^2/n^2) IFFT[-(kx FFT(D1') + ky FFT(D2'))/kz].
* kx, ky are the grid's angular wavenumbers (the unpaired Nyquist entry of a
  first derivative is zero, as for every first derivative here).  A mode with
  kz = 0 exactly (on the evanescent boundary) has no finite E3; it is set to 0.

In a homogeneous medium this is exact Gauss's law for the one-way field; in an
inhomogeneous one it is the stated approximation (parity with the CUDA path is
then checked against this definition).
"""
from __future__ import annotations

import numpy as np

from . import operators as ops


def e3_from_transverse(w: np.ndarray, n2: np.ndarray, dx: float, dy: float, k0: float, n0: float) -> np.ndarray:
    """E3 envelope (ny, nx) from the transverse envelope w = (w1, w2) (2, ny, nx)."""
    ny, nx = n2.shape
    ratio = np.asarray(n2, np.complex128) / n0 ** 2
    d1 = ops.fft2(ratio * w[0])
    d2 = ops.fft2(ratio * w[1])
    kx = (ops.first_derivative_symbol(nx, dx) / 1j)[None, :]
    ky = (ops.first_derivative_symbol(ny, dy) / 1j)[:, None]
    kxf = ops.wavenumbers(nx, dx)[None, :]
    kyf = ops.wavenumbers(ny, dy)[:, None]
    kz = np.sqrt((k0 * n0) ** 2 - kxf ** 2 - kyf ** 2 + 0j)
    kz = np.where(kz.imag < 0, -kz, kz)
    num = -(kx * d1 + ky * d2)
    d3 = np.divide(num, kz, out=np.zeros_like(num), where=kz != 0)
    return ops.ifft2(d3) / ratio
