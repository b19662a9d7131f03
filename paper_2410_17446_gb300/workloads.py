"""Seeded synthetic inputs for the propagator: grids, media and initial fields.

This module is shared by the CUDA path (bench, binding tests) and by the CPU
oracle.  It builds only the *inputs* of the method -- coordinates, the complex
n^2 slab with its absorbing border, the initial envelope -- and none of the
method's arithmetic (no operator, no rational approximation, no solve).  It
imports nothing from the rest of the package, so loading it never loads the
CUDA library.

Conventions (the paper's Sec. 2 notation, lambda = 1 is the unit of length):

* A field or slab is a complex128 array indexed ``[y, x]`` (x fastest), shape
  ``(ny, nx)``; a vector field is ``[comp, y, x]`` with comp = (w1, w2).
* Grid coordinates are ``x_i = (i - nx//2) * dx`` so the beam / aperture centre
  sits on index ``nx//2`` (likewise y).
* The absorbing border is an imaginary part added to n^2: for a border of
  ``W`` cells, a cell ``d`` cells deep (d = 1 at the inner edge, d = W at the
  outermost cell) gets ``sigma_max * (d / W)**2``; x and y contributions add
  in the corners.  It replaces the finite-difference PML of Sec. 4.1 on the
  periodic pseudo-spectral grid.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np

LAMBDA = 1.0
K0 = 2.0 * math.pi / LAMBDA


@dataclasses.dataclass(frozen=True)
class Grid:
    """One transverse grid: ``nx`` x ``ny`` cells of size ``dx`` x ``dy``."""
    nx: int
    ny: int
    dx: float
    dy: float

    @property
    def x(self) -> np.ndarray:
        return (np.arange(self.nx) - self.nx // 2) * self.dx

    @property
    def y(self) -> np.ndarray:
        return (np.arange(self.ny) - self.ny // 2) * self.dy

    def mesh(self):
        """(X, Y) arrays of shape (ny, nx)."""
        return np.meshgrid(self.x, self.y, indexing="xy")


def border_depth(n: int, width: int) -> np.ndarray:
    """Cells into the border for each of ``n`` cells: 0 inside, 1..width in the border."""
    d = np.zeros(n)
    if width <= 0:
        return d
    i = np.arange(n)
    left = i < width
    right = i >= n - width
    d[left] = width - i[left]
    d[right] = i[right] - (n - width) + 1
    return d


def absorbing_sigma(grid: Grid, width: int, sigma_max: float) -> np.ndarray:
    """Imaginary part added to n^2 by the absorbing border, shape (ny, nx)."""
    if width <= 0 or sigma_max == 0.0:
        return np.zeros((grid.ny, grid.nx))
    sx = sigma_max * (border_depth(grid.nx, width) / width) ** 2
    sy = sigma_max * (border_depth(grid.ny, width) / width) ** 2
    return sy[:, None] + sx[None, :]


def gaussian_beam(grid: Grid, waist: float) -> np.ndarray:
    """exp(-(x^2+y^2)/w^2), the beam of Eq. (eq_ft_gaussian) in Sec. 5.2."""
    X, Y = grid.mesh()
    return np.exp(-(X ** 2 + Y ** 2) / waist ** 2).astype(np.complex128)


def aperture_plane_wave(grid: Grid, radius: float) -> np.ndarray:
    """Unit normal plane wave through a hard circular aperture r <= a (Sec. 5.1)."""
    X, Y = grid.mesh()
    return (X ** 2 + Y ** 2 <= radius ** 2).astype(np.complex128)


def sine_product_n2(grid: Grid, eps: float, period: float, z: Optional[float],
                    border: int, sigma_max: float) -> np.ndarray:
    """n^2 = 1 + eps sin(2 pi x/L) sin(2 pi y/L) [sin(2 pi z/L)] + i sigma."""
    X, Y = grid.mesh()
    f = np.sin(2 * math.pi * X / period) * np.sin(2 * math.pi * Y / period)
    if z is not None:
        f = f * math.sin(2 * math.pi * z / period)
    return (1.0 + eps * f) + 1j * absorbing_sigma(grid, border, sigma_max)


def gaussian_random_field(grid: Grid, corr_len: float, rng: np.random.Generator) -> np.ndarray:
    """Unit-variance periodic Gaussian random field with covariance exp(-r^2/l^2).

    White noise from ``rng`` is filtered in Fourier space by exp(-k^2 l^2/8)
    (the square root of the Gaussian covariance's spectral density), then the
    sample is normalised to zero mean and unit variance.
    """
    noise = rng.standard_normal((grid.ny, grid.nx))
    kx = 2 * math.pi * np.fft.fftfreq(grid.nx, grid.dx)
    ky = 2 * math.pi * np.fft.fftfreq(grid.ny, grid.dy)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    g = np.fft.ifft2(np.fft.fft2(noise) * np.exp(-k2 * corr_len ** 2 / 8.0)).real
    g = g - g.mean()
    return g / g.std()


# ---------------------------------------------------------------------------
# The five workloads.  Each returns a Workload: grid(s), physical constants,
# the initial field(s), and a callable giving the n^2 slab used by step s.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Beam:
    grid: Grid
    w0: np.ndarray                               # (ncomp, ny, nx) complex128
    medium: Callable[[int], np.ndarray]           # step -> (ny, nx) complex128 n^2
    medium_changes: Callable[[int], bool]         # step -> does n^2 differ from step-1?
    border: int
    sigma_max: float


@dataclasses.dataclass
class Workload:
    name: str
    k0: float
    n0: float
    dz: float
    nsteps: int
    npoles: int
    ncomp: int
    precision: str                               # "fp64" | "fp32"
    restart: int
    tol: float
    beams: List[Beam]
    description: str = ""

    @property
    def K(self) -> float:
        return self.k0 * self.n0 * self.dz

    @property
    def points(self) -> int:
        return sum(b.grid.nx * b.grid.ny for b in self.beams)


def _constant(n2: np.ndarray):
    return (lambda s: n2), (lambda s: s == 0)


def plain_scalar_64(nsteps: int = 16) -> Workload:
    """64^2, dx=lambda/8, 8-cell border (0 -> 0.2 quadratic), static sine product."""
    g = Grid(64, 64, LAMBDA / 8, LAMBDA / 8)
    n2 = sine_product_n2(g, 0.1, 2 * LAMBDA, None, 8, 0.2)
    med, ch = _constant(n2)
    beam = Beam(g, gaussian_beam(g, 2 * LAMBDA)[None], med, ch, 8, 0.2)
    return Workload("plain_scalar_64", K0, 1.0, LAMBDA / 2, nsteps, 12, 1, "fp64", 20, 1e-10,
                    [beam], "64x64 scalar, static sine-product n^2, Gaussian w=2, dz=1/2")


def homogeneous_aperture_1024(nsteps: int = 100, n: int = 1024) -> Workload:
    """n^2 = 1, no border, plane wave through an r <= 64 lambda hard aperture, dz = lambda."""
    g = Grid(n, n, LAMBDA / 4, LAMBDA / 4)
    n2 = np.ones((n, n), np.complex128)
    med, ch = _constant(n2)
    radius = 64 * LAMBDA * (n / 1024)
    beam = Beam(g, aperture_plane_wave(g, radius)[None], med, ch, 0, 0.0)
    return Workload(f"homogeneous_aperture_{n}", K0, 1.0, LAMBDA, nsteps, 12, 1, "fp32", 20, 1e-7,
                    [beam], f"{n}^2 homogeneous, aperture r={radius:g}, dz=1")


def batched_scalar_1024(nsteps: int = 200, n: int = 1024) -> Workload:
    """Sine product with z factor, eps=0.05, period 1.5, Gaussian w=8, 16 poles."""
    g = Grid(n, n, LAMBDA / 4, LAMBDA / 4)
    width = max(8, n // 16)
    dz = LAMBDA / 2

    def med(s):
        return sine_product_n2(g, 0.05, 1.5 * LAMBDA, (s + 0.5) * dz, width, 0.2)

    beam = Beam(g, gaussian_beam(g, 8 * LAMBDA)[None], med, lambda s: True, width, 0.2)
    return Workload(f"batched_scalar_{n}", K0, 1.0, dz, nsteps, 16, 1, "fp32", 20, 1e-7,
                    [beam], f"{n}^2 scalar, z-varying sine product, Gaussian w=8, dz=1/2")


def vector_random_512(nsteps: int = 150, n: int = 512, seed: int = 7) -> Workload:
    """Two-component (w1, w2) field, n^2 = 1 + 0.03 g + i sigma, g refreshed every 8 lambda."""
    g = Grid(n, n, LAMBDA / 6, LAMBDA / 6)
    width = max(8, n // 16)
    dz = LAMBDA / 2
    refresh = int(round(8 * LAMBDA / dz))
    rng = np.random.Generator(np.random.PCG64(seed))
    sigma = absorbing_sigma(g, width, 0.2)
    slabs = []
    for _ in range((nsteps + refresh - 1) // refresh):
        slabs.append((1.0 + 0.03 * gaussian_random_field(g, LAMBDA, rng)) + 1j * sigma)

    w0 = np.zeros((2, n, n), np.complex128)
    w0[0] = gaussian_beam(g, 4 * LAMBDA)
    beam = Beam(g, w0, lambda s: slabs[s // refresh], lambda s: s % refresh == 0, width, 0.2)
    return Workload(f"vector_random_{n}", K0, 1.0, dz, nsteps, 14, 2, "fp32", 20, 1e-7,
                    [beam], f"{n}^2 vector, Gaussian random n^2 (l=1, seed {seed}), x-pol w=4")


def uneven_batch(nbeams: int = 48, nsteps: int = 64, seed: int = 11,
                 sizes=(128, 256, 384, 512, 768)) -> Workload:
    """Independent scalar beams of uneven grid sizes, each with its own sine product."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dz = LAMBDA / 2
    beams = []
    for _ in range(nbeams):
        n = int(sizes[int(rng.integers(0, len(sizes)))])
        eps = float(rng.uniform(0.02, 0.1))
        period = float(rng.uniform(1.0, 3.0)) * LAMBDA
        waist = float(rng.uniform(2.0, 8.0)) * LAMBDA
        g = Grid(n, n, LAMBDA / 4, LAMBDA / 4)
        width = max(8, n // 16)

        def med(s, g=g, eps=eps, period=period, width=width):
            return sine_product_n2(g, eps, period, (s + 0.5) * dz, width, 0.2)

        beams.append(Beam(g, gaussian_beam(g, waist)[None], med, lambda s: True, width, 0.2))
    return Workload("uneven_batch", K0, 1.0, dz, nsteps, 12, 1, "fp32", 20, 1e-7, beams,
                    f"{nbeams} beams, sizes {sizes}, 12 poles")


def multiwave_scalar_64(nsteps: int = 4) -> Workload:
    """Multiple-wavelength steps (Sec. 3.1): dz = 5 lambda, 28 poles, on a 64^2
    grid at dx = lambda/4 with an 8-cell border and a static sine product
    (eps 0.05, period 2 lambda), Gaussian w = 2; FP64."""
    g = Grid(64, 64, LAMBDA / 4, LAMBDA / 4)
    n2 = sine_product_n2(g, 0.05, 2 * LAMBDA, None, 8, 0.2)
    med, ch = _constant(n2)
    beam = Beam(g, gaussian_beam(g, 2 * LAMBDA)[None], med, ch, 8, 0.2)
    return Workload("multiwave_scalar_64", K0, 1.0, 5 * LAMBDA, nsteps, 28, 1, "fp64", 20, 1e-10,
                    [beam], "64x64 scalar, dz = 5 lambda, 28 poles")


def axis_angle_matrix(axis, angle: float) -> np.ndarray:
    """Rotation by `angle` about the unit vector along `axis` (Rodrigues' formula):
    R = cos(a) I + sin(a) [u]_x + (1 - cos(a)) u u^T."""
    u = np.asarray(axis, float)
    u = u / np.linalg.norm(u)
    K = np.array([[0.0, -u[2], u[1]], [u[2], 0.0, -u[0]], [-u[1], u[0], 0.0]])
    return math.cos(angle) * np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * np.outer(u, u)


SINEPROD_AXIS = (0.258, 0.312, 0.914)   # Sec. 5.3: rotation axis (normalised here) and angle
SINEPROD_ANGLE = 0.128
SINEPROD_N0, SINEPROD_DN = 1.2, 0.025


def rotated_sine_product_n2(grid: Grid, q: float, z: float, border: int, sigma_max: float,
                            n0: float = SINEPROD_N0, dn: float = SINEPROD_DN) -> np.ndarray:
    """n^2 of Eq. eq_sineprod at plane z: n = n0 + dn sin(ks x~) sin(ks y~) sin(ks z~),
    ks = k0 n0 / (sqrt(3) q), (x~, y~, z~) = R (x, y, z) with R the axis-angle
    rotation of Sec. 5.3; plus i sigma of the absorbing border."""
    X, Y = grid.mesh()
    R = axis_angle_matrix(SINEPROD_AXIS, SINEPROD_ANGLE)
    ks = K0 * n0 / (math.sqrt(3.0) * q)
    xt = R[0, 0] * X + R[0, 1] * Y + R[0, 2] * z
    yt = R[1, 0] * X + R[1, 1] * Y + R[1, 2] * z
    zt = R[2, 0] * X + R[2, 1] * Y + R[2, 2] * z
    n = n0 + dn * np.sin(ks * xt) * np.sin(ks * yt) * np.sin(ks * zt)
    return (n * n).astype(np.complex128) + 1j * absorbing_sigma(grid, border, sigma_max)


def sineprod_helmholtz(q: float, nsteps: Optional[int] = None, n: Optional[int] = None,
                       range_lambda: float = 240.0) -> Workload:
    """Sec. 5.3: a collimated Gaussian beam (1/e amplitude width 25 lambda, read as
    the diameter: exp(-r^2/w^2), w = 12.5 lambda) through the rotated sine product
    with n0 = 1.2, dn = 0.025, q in {0.5, 1, 2}; dz = a quarter of the index
    field's wavelength 2 pi/ks; 240 lambda of range.  The paper's 481^2 and
    961^2 grids over 120 lambda (dx = lambda/4, lambda/8) with 60- and
    120-point PMLs become 512^2 and 1024^2 at the same dx (128 lambda) with
    64- and 128-cell absorbing borders (16 lambda).  The medium is sampled at
    the step midpoints.  `n` shrinks the grid at the same dx (tests)."""
    fine = q < 0.75
    dx = LAMBDA / 8 if fine else LAMBDA / 4
    N = n or (1024 if fine else 512)
    g = Grid(N, N, dx, dx)
    width = max(8, N // 8)
    ks = K0 * SINEPROD_N0 / (math.sqrt(3.0) * q)
    dz = (2 * math.pi / ks) / 4
    steps = nsteps if nsteps is not None else int(round(range_lambda / dz))

    # sin(ks (R_i0 x + R_i1 y + R_i2 z)) = sin(A_i) cos(c_i) + cos(A_i) sin(c_i): the
    # z-independent parts A_i are evaluated once (the same n^2 as rotated_sine_product_n2)
    X, Y = g.mesh()
    R = axis_angle_matrix(SINEPROD_AXIS, SINEPROD_ANGLE)
    A = [ks * (R[i, 0] * X + R[i, 1] * Y) for i in range(3)]
    SA, CA = [np.sin(a) for a in A], [np.cos(a) for a in A]
    sig = absorbing_sigma(g, width, 0.2)

    def med(s):
        z = (s + 0.5) * dz
        f = None
        for i in range(3):
            c = ks * R[i, 2] * z
            t = SA[i] * math.cos(c) + CA[i] * math.sin(c)
            f = t if f is None else f * t
        nn = SINEPROD_N0 + SINEPROD_DN * f
        return (nn * nn) + 1j * sig

    beam = Beam(g, gaussian_beam(g, 12.5 * LAMBDA)[None], med, lambda s: True, width, 0.2)
    tag = {0.5: "05", 1.0: "1", 2.0: "2"}.get(float(q), str(q))
    return Workload(f"sineprod_q{tag}", K0, SINEPROD_N0, dz, steps, 16, 1, "fp32", 20, 1e-7, [beam],
                    f"Sec. 5.3 rotated sine product, q = {q}, {N}^2, dx = {dx:g}, dz = {dz:.4f}")


def small_scalar(n: int = 16, dx: float = LAMBDA / 4, border: int = 3, eps: float = 0.1,
                 seed: int = 0, waist: float = 1.0) -> Workload:
    """Tiny random-medium scalar case (dense-LU sized) for unit tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = Grid(n, n, dx, dx)
    n2 = (1.0 + eps * rng.uniform(-1, 1, (n, n))) + 1j * absorbing_sigma(g, border, 0.2)
    med, ch = _constant(n2)
    w0 = gaussian_beam(g, waist) * (1 + 0.1 * rng.standard_normal((n, n)))
    return Workload(f"small_scalar_{n}", K0, 1.0, LAMBDA / 2, 2, 6, 1, "fp64", 20, 1e-12,
                    [Beam(g, w0[None].astype(np.complex128), med, ch, border, 0.2)])


def small_vector(n: int = 16, dx: float = LAMBDA / 4, border: int = 3, eps: float = 0.05,
                 seed: int = 0, waist: float = 1.0) -> Workload:
    """Tiny smooth random-medium vector case for unit tests (periodic n^2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = Grid(n, n, dx, dx)
    n2 = (1.0 + eps * gaussian_random_field(g, 2 * dx, rng)) + 1j * absorbing_sigma(g, border, 0.2)
    med, ch = _constant(n2)
    w0 = np.zeros((2, n, n), np.complex128)
    w0[0] = gaussian_beam(g, waist)
    w0[1] = 0.3 * gaussian_beam(g, waist) * rng.standard_normal((n, n))
    return Workload(f"small_vector_{n}", K0, 1.0, LAMBDA / 2, 2, 6, 2, "fp64", 20, 1e-12,
                    [Beam(g, w0, med, ch, border, 0.2)])


WORKLOADS = {
    "plain_scalar_64": plain_scalar_64,
    "homogeneous_aperture_1024": homogeneous_aperture_1024,
    "batched_scalar_1024": batched_scalar_1024,
    "vector_random_512": vector_random_512,
    "uneven_batch": uneven_batch,
    "multiwave_scalar_64": multiwave_scalar_64,
    "sineprod_q2": lambda nsteps=None, n=None: sineprod_helmholtz(2.0, nsteps, n),
    "sineprod_q1": lambda nsteps=None, n=None: sineprod_helmholtz(1.0, nsteps, n),
    "sineprod_q05": lambda nsteps=None, n=None: sineprod_helmholtz(0.5, nsteps, n),
}
