"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle, the tests and the bench.

This module only draws numbers: point-spread functions (PSFs), piecewise-constant true
images, Gaussian vectors (noise directions, the GKB start vector, the RSVD test matrix)
and the noise scaling of the paper's experiments.  It holds none of the method's
arithmetic (no blur, no rearrangement, no SVD, no split Bregman) and imports neither
the oracle nor the CUDA binding.

The paper's own test images and speckle PSFs (IR Tools `pattern2`, `satellite`, `hst`,
the Mild/Medium speckle PSFs of Sec. 5.2) are not available; these generators stand in
for them with the same shapes: square n x n images with sharp-edged piecewise-constant
content, odd-sized non-separable PSFs normalised to sum 1, zero or reflexive boundary
conditions, and white Gaussian noise at a stated level (Sec. 5.3.2, noise model of the
SNR definition).

Conventions: images are n x n float64 arrays indexed [row, col]; vec() is column-major
(Fortran order), as in the paper's vec/array notation (Sec. 1).  A PSF is an s x s array
whose centre tap is at index (s // 2, s // 2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BC_ZERO = 0
BC_REFLEXIVE = 1


def rng(seed: int) -> np.random.Generator:
    """Counter-based generator (Philox4x32-10) with a fixed seed."""
    return np.random.Generator(np.random.Philox(int(seed)))


def _grid(s: int):
    c = s // 2
    off = np.arange(s, dtype=np.float64) - c
    dy, dx = np.meshgrid(off, off, indexing="ij")  # dy = row offset, dx = column offset
    return dy, dx


def _normalise(p: np.ndarray) -> np.ndarray:
    return p / p.sum()


def psf_gaussian(s: int, sigma_u: float, sigma_v: float, angle_deg: float) -> np.ndarray:
    """Rotated anisotropic Gaussian exp(-(u^2/su^2 + v^2/sv^2)/2), normalised to sum 1."""
    th = math.radians(angle_deg)
    dy, dx = _grid(s)
    u = math.cos(th) * dx + math.sin(th) * dy
    v = -math.sin(th) * dx + math.cos(th) * dy
    return _normalise(np.exp(-0.5 * (u * u / sigma_u**2 + v * v / sigma_v**2)))


def psf_gaussian_mixture(s: int, g: np.random.Generator) -> np.ndarray:
    """Sum of two rotated Gaussians (weights 1/2, widths U[1,6] px, angles U[0,180) deg)."""
    p = np.zeros((s, s))
    for _ in range(2):
        su, sv = g.uniform(1.0, 6.0, size=2)
        ang = g.uniform(0.0, 180.0)
        p += 0.5 * psf_gaussian(s, su, sv, ang)
    return _normalise(p)


def psf_turbulence(s: int, g: np.random.Generator) -> np.ndarray:
    """Turbulence-like speckle PSF: envelope exp(-(rho/r0)^(5/3)) with anisotropic, rotated
    rho (a/b in [1,2], r0 in [2, s/6]) times a pixelwise speckle factor 1 + 0.5 U[-1,1]
    (non-separable, slowly decaying Kronecker spectrum like the paper's speckle PSFs)."""
    th = g.uniform(0.0, math.pi)
    ratio = g.uniform(1.0, 2.0)
    r0 = g.uniform(2.0, max(2.0, s / 6.0))
    dy, dx = _grid(s)
    u = math.cos(th) * dx + math.sin(th) * dy
    v = -math.sin(th) * dx + math.cos(th) * dy
    rho = np.sqrt((u / ratio) ** 2 + v**2)
    speckle = 1.0 + 0.5 * g.uniform(-1.0, 1.0, size=(s, s))
    return _normalise(np.exp(-((rho / r0) ** (5.0 / 3.0))) * speckle)


def psf_separable(s: int, g: np.random.Generator) -> np.ndarray:
    """Outer product of two positive 1-D profiles: its R(A) has rank 1."""
    a = g.uniform(0.1, 1.0, size=s)
    b = g.uniform(0.1, 1.0, size=s)
    return _normalise(np.outer(a, b))


def psf_random(s: int, g: np.random.Generator) -> np.ndarray:
    """Dense positive random PSF (no structure), normalised to sum 1."""
    return _normalise(g.uniform(0.05, 1.0, size=(s, s)))


def image_piecewise_constant(n: int, g: np.random.Generator) -> np.ndarray:
    """3 + n//16 random axis-aligned rectangles and disks, values U[0,1], on zero background."""
    x = np.zeros((n, n))
    rows, cols = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    lo, hi = max(1.0, n / 16.0), max(2.0, n / 3.0)
    for _ in range(3 + n // 16):
        val = g.uniform(0.0, 1.0)
        if g.uniform() < 0.5:
            h, w = g.uniform(lo, hi, size=2)
            r0 = g.uniform(0, n - h)
            c0 = g.uniform(0, n - w)
            m = (rows >= r0) & (rows < r0 + h) & (cols >= c0) & (cols < c0 + w)
        else:
            rad = 0.5 * g.uniform(lo, hi)
            rc, cc = g.uniform(rad, n - rad, size=2)
            m = (rows - rc) ** 2 + (cols - cc) ** 2 <= rad * rad
        x[m] = val
    return x


def gaussian(shape, g: np.random.Generator, dtype=np.float64) -> np.ndarray:
    """Standard normal draws (mean 0, variance 1), like MATLAB randn."""
    return g.standard_normal(size=shape).astype(dtype)


def noise_vector(b_true: np.ndarray, eta: float, zeta: np.ndarray) -> np.ndarray:
    """Noise eta * (||b_true|| / ||zeta||) * zeta of the paper's experiments (Sec. 5.3.2)."""
    return eta * (np.linalg.norm(b_true) / np.linalg.norm(zeta)) * zeta


@dataclass
class Problem:
    """One deblurring request: inputs only (the blurred data b is made by a blur operator)."""

    n: int
    psf: np.ndarray
    bc: int
    x_true: np.ndarray
    zeta: np.ndarray  # noise direction, n x n
    eta: float  # noise level
    start: np.ndarray  # GKB start vector y (length n^2, float64 draws; a FP32 build rounds them)
    k: int = 5  # target rank (fixed-rank mode) or cap (auto mode)
    p: int = 2
    tau: float = 0.0  # > 0: automatic rank with relative tolerance tau
    iso: bool = False
    seed: int = 0
    extra: dict = field(default_factory=dict)


def problem_small(index: int = 0) -> Problem:
    """n = 32, 9x9 rotated anisotropic Gaussian (sigma 1.5/3.0, 30 deg), zero boundary,
    1% noise, rank 5 enlarged to 10, anisotropic TV."""
    g = rng(1000 + index)
    n = 32
    psf = psf_gaussian(9, 1.5, 3.0, 30.0)
    return Problem(n=n, psf=psf, bc=BC_ZERO, x_true=image_piecewise_constant(n, g),
                   zeta=gaussian((n, n), g), eta=0.01, start=gaussian(n * n, g),
                   k=5, p=5, tau=0.0, iso=False, seed=1000 + index)


def problem_medium(index: int = 0, eta: float | None = None) -> Problem:
    """n = 128, 31x31 two-Gaussian mixture, reflexive boundary, automatic rank (cap 30),
    isotropic TV, noise 1% (even index) or 5% (odd index)."""
    g = rng(2000 + index)
    n = 128
    psf = psf_gaussian_mixture(31, g)
    if eta is None:
        eta = 0.01 if index % 2 == 0 else 0.05
    return Problem(n=n, psf=psf, bc=BC_REFLEXIVE, x_true=image_piecewise_constant(n, g),
                   zeta=gaussian((n, n), g), eta=eta, start=gaussian(n * n, g),
                   k=30, p=4, tau=1e-3, iso=True, seed=2000 + index)


def problem_large(index: int = 0) -> Problem:
    """n = 512, 63x63 turbulence-like PSF, zero boundary, rank 20, 1% noise."""
    g = rng(3000 + index)
    n = 512
    psf = psf_turbulence(63, g)
    return Problem(n=n, psf=psf, bc=BC_ZERO, x_true=image_piecewise_constant(n, g),
                   zeta=gaussian((n, n), g), eta=0.01, start=gaussian(n * n, g),
                   k=20, p=20, tau=0.0, iso=True, seed=3000 + index)


def problem_batched(index: int) -> Problem:
    """One of 96 uneven problems: n = (64, 128, 256, 384)[index % 4]; boundary, TV type and
    PSF family alternate with index // 4, index // 8 and index // 16, so every size carries
    every combination (zero / reflexive, aniso / iso, Gaussian mixture / turbulence); odd
    s in [15, 63], k in [5, 20], noise 1-5%."""
    g = rng(4000 + index)
    n = (64, 128, 256, 384)[index % 4]
    s = int(g.integers(7, 32)) * 2 + 1  # odd in [15, 63]
    s = min(s, n - 1 if n % 2 == 0 else n)
    psf = psf_gaussian_mixture(s, g) if (index // 16) % 2 == 0 else psf_turbulence(s, g)
    k = int(g.integers(5, 21))
    return Problem(n=n, psf=psf, bc=(index // 4) % 2, x_true=image_piecewise_constant(n, g),
                   zeta=gaussian((n, n), g), eta=float(g.uniform(0.01, 0.05)),
                   start=gaussian(n * n, g), k=k, p=max(2, (k + 3) // 4), tau=0.0,
                   iso=bool((index // 8) % 2), seed=4000 + index)
