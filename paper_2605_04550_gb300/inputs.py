"""Seeded synthetic inputs for the sigma_min grid engine.

This module builds inputs only: band storage of the test matrices, grid extents
and epsilon levels. It holds none of the method's arithmetic (no factorisation,
no solve, no singular values of zI - A), so both the CUDA path and the CPU
oracle can take their inputs from it.

Band storage (shared by every consumer): a complex128 array ``bands`` of shape
``(kl + ku + 1, n)`` with ``bands[d + kl, i] = A[i, i + d]`` for
``d in [-kl, ku]``; entries whose column ``i + d`` falls outside ``[0, n)`` are
ignored by every consumer and are set to zero here.

Workloads (all synthetic, seeded):

* ``grcar(n)`` -- the Grcar matrix: -1 on the subdiagonal, +1 on the diagonal
  and the first three superdiagonals (kl = 1, ku = 3).
* ``random_toeplitz(n, kl, ku, seed, super_scale)`` -- a banded Toeplitz matrix
  with complex coefficients a_d = N(0,1) + i N(0,1), the superdiagonal ones
  (d >= 1) multiplied by ``super_scale``.
* ``paper_class(seed)`` -- the random banded training/test class of the paper
  (Sec. 3.3, Eq. (matrix)): n = 64, beta uniform in {1,2,3,4}, entries uniform
  in {-1, 0, 1} for |i - j| <= beta, redrawn while A == A^T or
  cond(A) >= 1e8 (best-conditioned draw when no draw qualifies).
* ``batch_workload(nmat, seed)`` -- a batch of Grcar-type and random-Toeplitz
  matrices of log-uniform order and random band shape, with 1e-3 band noise,
  each on its own grid.
* normal matrices with known spectra, used by the closed-form checks.
"""
from __future__ import annotations

import dataclasses
from typing import Tuple

import numpy as np

__all__ = [
    "Grid",
    "EPS_LEVELS_8",
    "grcar",
    "random_toeplitz",
    "toeplitz_symbol_grid",
    "paper_class",
    "diagonal_normal",
    "hermitian_toeplitz_tridiag",
    "shifted_hermitian_band",
    "jordan_block",
    "grcar_grid_100",
    "paper_grid_100",
    "grcar_type",
    "batch_workload",
    "restriction_matrices",
    "restriction_test_matrix",
]


@dataclasses.dataclass(frozen=True)
class Grid:
    """Rectangular grid of the complex plane (paper Sec. 2.1).

    Row i (0 <= i < ny) holds Im z = y_i, column j (0 <= j < nx) holds
    Re z = x_j; points are stored row-major ``[ny][nx]``, row 0 = ``im_min``.
    """

    re_min: float
    re_max: float
    im_min: float
    im_max: float
    nx: int
    ny: int

    @property
    def npoints(self) -> int:
        return int(self.nx) * int(self.ny)


#: epsilon levels 1e-1 ... 1e-8 (one mask bit per level).
EPS_LEVELS_8 = tuple(10.0 ** (-k) for k in range(1, 9))


def _empty_bands(n: int, kl: int, ku: int) -> np.ndarray:
    return np.zeros((kl + ku + 1, n), dtype=np.complex128)


def _zero_outside(bands: np.ndarray, n: int, kl: int, ku: int) -> np.ndarray:
    for d in range(-kl, ku + 1):
        row = bands[d + kl]
        i = np.arange(n)
        row[(i + d < 0) | (i + d >= n)] = 0.0
    return bands


def grcar(n: int) -> Tuple[np.ndarray, int, int]:
    """Grcar matrix of order n: A[i,i-1] = -1, A[i,i+d] = +1 for d = 0..3."""
    kl, ku = 1, 3
    b = _empty_bands(n, kl, ku)
    b[-1 + kl, :] = -1.0
    for d in range(0, 4):
        b[d + kl, :] = 1.0
    return _zero_outside(b, n, kl, ku), kl, ku


def toeplitz_coefficients(kl: int, ku: int, seed: int, super_scale: float = 4.0) -> np.ndarray:
    """Complex coefficients a_d, d = -kl..ku (index d + kl); Re, Im ~ N(0,1).

    The superdiagonal coefficients (d >= 1) are multiplied by ``super_scale``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal(kl + ku + 1) + 1j * rng.standard_normal(kl + ku + 1)
    a[kl + 1:] *= super_scale
    return a.astype(np.complex128)


def random_toeplitz(n: int, kl: int, ku: int, seed: int, super_scale: float = 4.0):
    """Banded Toeplitz matrix A[i, i+d] = a_d with seeded complex a_d."""
    a = toeplitz_coefficients(kl, ku, seed, super_scale)
    b = _empty_bands(n, kl, ku)
    for d in range(-kl, ku + 1):
        b[d + kl, :] = a[d + kl]
    return _zero_outside(b, n, kl, ku), kl, ku, a


def toeplitz_symbol_grid(a: np.ndarray, kl: int, ku: int, nx: int, ny: int,
                         pad: float = 0.2, samples: int = 4096, min_aspect: float = 0.0) -> Grid:
    """Grid over the bounding box of the symbol curve, widened by ``pad``.

    The symbol is f(t) = sum_d a_d exp(i d t) sampled at ``samples`` points of
    [0, 2 pi); the box keeps its centre and its width and height grow by the
    factor 1 + pad. With ``min_aspect`` > 0 the shorter side is widened to at
    least min_aspect times the longer one (a symbol curve that is a segment,
    as for kl = ku Grcar-type bands, still gets a two-dimensional box).
    """
    t = np.arange(samples) * (2.0 * np.pi / samples)
    d = np.arange(-kl, ku + 1)
    f = (a[None, :] * np.exp(1j * np.outer(t, d))).sum(axis=1)
    cx = 0.5 * (f.real.min() + f.real.max())
    cy = 0.5 * (f.imag.min() + f.imag.max())
    hw = 0.5 * (f.real.max() - f.real.min()) * (1.0 + pad)
    hh = 0.5 * (f.imag.max() - f.imag.min()) * (1.0 + pad)
    hw, hh = max(hw, min_aspect * hh), max(hh, min_aspect * hw)
    return Grid(float(cx - hw), float(cx + hw), float(cy - hh), float(cy + hh), nx, ny)


def dense_to_bands(A: np.ndarray, kl: int, ku: int) -> np.ndarray:
    """Copy the band of a dense matrix into band storage (format conversion)."""
    n = A.shape[0]
    b = _empty_bands(n, kl, ku)
    for d in range(-kl, ku + 1):
        for i in range(n):
            j = i + d
            if 0 <= j < n:
                b[d + kl, i] = A[i, j]
    return b


def paper_class(seed: int, n: int = 64, max_tries: int = 200):
    """One matrix of the paper's random banded class (Sec. 3.3, Eq. (matrix)).

    beta ~ uniform{1,2,3,4} is drawn once; A_ij ~ uniform{-1,0,1} for
    |i-j| <= beta, else 0, redrawn (same beta) while A == A^T or
    cond_2(A) >= 1e8, so that beta stays uniform over the class. For beta = 1
    almost no draw meets cond_2(A) < 1e8 (tridiagonal {-1,0,1} matrices are
    near-singular), so after ``max_tries`` draws the non-symmetric draw with
    the smallest condition number is returned.
    Returns (bands, kl, ku, A) with kl = ku = beta and A dense complex128.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    beta = int(rng.integers(1, 5))
    i, j = np.indices((n, n))
    outside = np.abs(i - j) > beta
    best, best_c = None, np.inf
    for _ in range(max_tries):
        A = rng.integers(-1, 2, size=(n, n)).astype(np.float64)
        A[outside] = 0.0
        if np.array_equal(A, A.T):
            continue
        c = np.linalg.cond(A)
        if not np.isfinite(c):
            c = np.inf
        if c < best_c or best is None:
            best, best_c = A, c
        if c < 1e8:
            break
    Ac = best.astype(np.complex128)
    return dense_to_bands(Ac, beta, beta), beta, beta, Ac


def diagonal_normal(n: int, seed: int):
    """Diagonal A (kl = ku = 0) with distinct complex entries; normal."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = rng.uniform(-2, 2, n) + 1j * rng.uniform(-2, 2, n)
    b = lam.reshape(1, n).astype(np.complex128)
    return b, 0, 0, lam


def hermitian_toeplitz_tridiag(n: int, a: float, b: complex):
    """tridiag(conj(b), a, b) with real a: Hermitian, eigenvalues known in closed form."""
    bands = _empty_bands(n, 1, 1)
    bands[0, :] = np.conj(b)   # d = -1: A[i, i-1] = conj(b)
    bands[1, :] = a            # d = 0
    bands[2, :] = b            # d = +1: A[i, i+1] = b
    return _zero_outside(bands, n, 1, 1), 1, 1


def shifted_hermitian_band(n: int, k: int, alpha: complex, shift: complex, seed: int):
    """A = alpha * H + shift * I with H a random Hermitian band matrix (kl = ku = k).

    A is normal for any complex alpha and shift. Returns (bands, kl, ku, H).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    H = np.zeros((n, n), dtype=np.complex128)
    for d in range(0, k + 1):
        v = rng.standard_normal(n - d) + (1j * rng.standard_normal(n - d) if d > 0 else 0.0)
        H[np.arange(n - d), np.arange(d, n)] = v
    H = np.triu(H) + np.triu(H, 1).conj().T
    A = alpha * H + shift * np.eye(n)
    return dense_to_bands(A, k, k), k, k, H


def jordan_block(n: int = 32):
    """Jordan block with ones on the subdiagonal (paper Sec. 2 example): kl = 1, ku = 0."""
    bands = _empty_bands(n, 1, 0)
    bands[0, :] = 1.0
    return _zero_outside(bands, n, 1, 0), 1, 0


def grcar_perturbed(n: int, seed: int, scale: float = 1e-2):
    """Grcar-type band (kl = 1, ku = 3) with every band entry perturbed by seeded
    real Gaussian noise of standard deviation `scale`."""
    b, kl, ku = grcar(n)
    rng = np.random.Generator(np.random.PCG64(seed))
    b = b + scale * rng.standard_normal(b.shape)
    return _zero_outside(b.astype(np.complex128), n, kl, ku), kl, ku


def grcar_type(n: int, kl: int, ku: int) -> np.ndarray:
    """Grcar-type band: -1 on the kl subdiagonals, +1 on the diagonal and the ku
    superdiagonals (the Grcar matrix is kl = 1, ku = 3)."""
    b = _empty_bands(n, kl, ku)
    b[:kl, :] = -1.0
    b[kl:, :] = 1.0
    return _zero_outside(b, n, kl, ku)


def batch_workload(nmat: int = 256, seed: int = 0, n_min: int = 200, n_max: int = 8000,
                   nx: int = 128, ny: int = 128, noise: float = 1e-3):
    """Seeded batch of banded matrices of uneven order and band shape, each with its grid.

    Per matrix m (one PCG64 stream per batch): n = round(exp(U(log n_min, log n_max)))
    (log-uniform), kl uniform in {1..4}, ku uniform in {1..8}, the type Grcar-type or
    random Toeplitz (``toeplitz_coefficients`` with seed ``seed * 100003 + m``) with
    probability 1/2 each, then every band entry plus complex Gaussian noise
    noise * (N(0,1) + i N(0,1)). The grid is nx x ny over the bounding box of the
    coefficient symbol widened by 20 %, its shorter side at least half the
    longer (``toeplitz_symbol_grid`` with min_aspect = 0.5).
    Returns a list of (bands, kl, ku, grid, kind).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for m in range(nmat):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        kl = int(rng.integers(1, 5))
        ku = int(rng.integers(1, 9))
        if rng.random() < 0.5:
            kind = "grcar"
            a = np.concatenate([-np.ones(kl), np.ones(ku + 1)]).astype(np.complex128)
            b = grcar_type(n, kl, ku)
        else:
            kind = "toeplitz"
            b, _, _, a = random_toeplitz(n, kl, ku, seed=seed * 100003 + m)
        b = b + noise * (rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape))
        b = _zero_outside(b.astype(np.complex128), n, kl, ku)
        out.append((b, kl, ku, toeplitz_symbol_grid(a, kl, ku, nx, ny, min_aspect=0.5), kind))
    return out


def restriction_matrices(nmat: int, seed: int, n_min: int = 500, n_max: int = 5000, nx: int = 32, ny: int = 32,
                         noise: float = 1e-3):
    """Training / validation matrices of the learned restriction: the families of
    ``batch_workload`` (Grcar-type or random Toeplitz with complex band noise,
    kl 1..4, ku 1..8), n log-uniform in [n_min, n_max], each on an nx x ny grid
    over its symbol box +20 % (shorter side at least half the longer).
    Returns a list of (bands, kl, ku, grid, kind)."""
    return batch_workload(nmat=nmat, seed=seed, n_min=n_min, n_max=n_max, nx=nx, ny=ny, noise=noise)


def restriction_test_matrix(n: int = 20000, kl: int = 3, ku: int = 6, nx: int = 1024, ny: int = 1024,
                            seed: int = 2024, noise: float = 1e-3):
    """The test matrix of the learned restriction: random banded Toeplitz
    (``toeplitz_coefficients`` with this seed) plus complex Gaussian band noise
    of standard deviation ``noise``, on an nx x ny grid over its symbol box
    +20 % (shorter side at least half the longer). Returns (bands, kl, ku, grid)."""
    b, _, _, a = random_toeplitz(n, kl, ku, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    b = b + noise * (rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape))
    b = _zero_outside(b.astype(np.complex128), n, kl, ku)
    return b, kl, ku, toeplitz_symbol_grid(a, kl, ku, nx, ny, min_aspect=0.5)


def grcar_grid_100() -> Grid:
    """100 x 100 grid over Re z in [-1, 3], Im z in [-3.5, 3.5]."""
    return Grid(-1.0, 3.0, -3.5, 3.5, 100, 100)


def paper_grid_100() -> Grid:
    """100 x 100 grid over [-4, 4] x [-4, 4] (paper Sec. 3.3)."""
    return Grid(-4.0, 4.0, -4.0, 4.0, 100, 100)
