"""CPU oracle for sigma_min(zI - A) over a complex grid.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
product path (the CUDA library and its binding) never calls it; the two share
no code. Inputs come from the seeded generators in
``paper_2605_04550_gb300.inputs``, which hold none of the method's arithmetic.

Two tiers:

* ``sigma_min_dense`` -- the paper's own method (Sec. 2.1): a dense complex
  FP64 SVD of zI - A per point, sigma_min = sigma_n. Used for small n and for
  sampled points of larger problems.
* ``sigma_min_banded`` -- the banded LU + inverse Lanczos reading of the same
  quantity, in plain C (``psa_oracle.c``), run to convergence. Its steps are
  exposed one by one (``band_lu``, ``band_solve``, ``tridiag_top``,
  ``lanczos_coeffs``) so that each can be checked on its own.

``masks`` gives the epsilon-level bits of the sensitive zone
S_eps = {z : sigma_min(z) <= eps} (paper Sec. 2.1, Eq. (sensitive_zone)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psa_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# status codes of the oracle (same meaning as the library's per-point codes)
OK, SINGULAR, NOT_CONVERGED, NONFINITE, UNDERFLOW = 0, 1, 2, 3, 5

#: converged-mode settings of the exact tier
EXACT_TOL = 1e-15
EXACT_KMAX = 5000


def build(force: bool = False) -> str:
    """Compile ``psa_oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i8p = ctypes.POINTER(ctypes.c_int8)
            lib.oracle_grid_coord.restype = ctypes.c_double
            lib.oracle_grid_coord.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32]
            lib.oracle_grid_points.restype = None
            lib.oracle_grid_points.argtypes = [ctypes.c_double] * 4 + [ctypes.c_int32] * 2 + [dp]
            lib.oracle_splitmix64.restype = ctypes.c_uint64
            lib.oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_start_vector.restype = None
            lib.oracle_start_vector.argtypes = [ctypes.c_int32, ctypes.c_uint64, dp]
            lib.oracle_tridiag_top.restype = None
            lib.oracle_tridiag_top.argtypes = [ctypes.c_int32, dp, dp, dp, dp]
            lib.oracle_sigma_min_points.restype = ctypes.c_int
            lib.oracle_sigma_min_points.argtypes = [
                ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, dp, ctypes.c_int64, dp,
                ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64,
                dp, i8p, i32p, ctypes.c_int32]
            lib.oracle_band_lu.restype = ctypes.c_int
            lib.oracle_band_lu.argtypes = [ctypes.c_int32] * 3 + [dp, ctypes.c_double, ctypes.c_double, dp, i32p]
            lib.oracle_band_solve.restype = None
            lib.oracle_band_solve.argtypes = [ctypes.c_int32] * 3 + [dp, i32p, ctypes.c_int32, dp]
            lib.oracle_lanczos_coeffs.restype = ctypes.c_int32
            lib.oracle_lanczos_coeffs.argtypes = [ctypes.c_int32] * 3 + [dp, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_int32, ctypes.c_uint64, dp, dp, i32p]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


# ---------------------------------------------------------------- grid
def grid_points(grid) -> np.ndarray:
    """Complex grid points z[i, j] = x_j + i y_i, shape (ny, nx) (paper Sec. 2.1).

    x_j = re_min + j (re_max - re_min)/(nx - 1) as one fused multiply-add.
    """
    lib = _load()
    z = np.empty((grid.ny, grid.nx), dtype=np.complex128)
    lib.oracle_grid_points(grid.re_min, grid.re_max, grid.im_min, grid.im_max,
                           grid.nx, grid.ny, _dp(z.view(np.float64)))
    return z


def grid_coord(lo: float, hi: float, count: int, j: int) -> float:
    return _load().oracle_grid_coord(lo, hi, count, j)


# -------------------------------------------------------- start vector
def splitmix64(seed: int, c: int) -> int:
    return int(_load().oracle_splitmix64(seed & (2**64 - 1), c))


def start_vector(n: int, seed: int) -> np.ndarray:
    q = np.empty(n, dtype=np.complex128)
    _load().oracle_start_vector(n, seed & (2**64 - 1), _dp(q.view(np.float64)))
    return q


# ------------------------------------------------------- dense (paper)
def band_to_dense(bands: np.ndarray, kl: int, ku: int) -> np.ndarray:
    """Dense A from band storage bands[d + kl, i] = A[i, i + d]."""
    n = bands.shape[1]
    A = np.zeros((n, n), dtype=np.complex128)
    for d in range(-kl, ku + 1):
        for i in range(n):
            j = i + d
            if 0 <= j < n:
                A[i, j] = bands[d + kl, i]
    return A


def sigma_min_dense(A: np.ndarray, z: Sequence[complex]) -> np.ndarray:
    """sigma_min(zI - A) by dense SVD, the paper's method (Sec. 2.1)."""
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    eye = np.eye(n, dtype=np.complex128)
    z = np.asarray(z, dtype=np.complex128).ravel()
    out = np.empty(z.shape[0], dtype=np.float64)
    for k, zk in enumerate(z):
        out[k] = np.linalg.svd(zk * eye - A, compute_uv=False)[-1]
    return out


# ------------------------------------------------- banded LU + Lanczos
def sigma_min_banded(bands: np.ndarray, kl: int, ku: int, z: Sequence[complex], *,
                     k_min: int = 2, k_max: int = EXACT_KMAX, tol: float = EXACT_TOL,
                     seed: int = 0, nthreads: int = 0) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """sigma_min(zI - A) at the points z; returns (sigma, status, steps)."""
    lib = _load()
    b = _c128(bands)
    kl, ku = int(kl), int(ku)
    n = b.shape[1]
    assert b.shape == (kl + ku + 1, n)
    zz = _c128(z).ravel()
    sigma = np.empty(zz.shape[0], dtype=np.float64)
    status = np.empty(zz.shape[0], dtype=np.int8)
    steps = np.empty(zz.shape[0], dtype=np.int32)
    rc = lib.oracle_sigma_min_points(
        n, kl, ku, _dp(b.view(np.float64)), zz.shape[0], _dp(zz.view(np.float64)),
        int(k_min), int(k_max), float(tol), seed & (2**64 - 1),
        _dp(sigma), status.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
        steps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle_sigma_min_points failed")
    return sigma, status, steps


def band_lu(bands: np.ndarray, kl: int, ku: int, z: complex):
    """Banded LU of zI - A: (factor rows [n, 2kl+ku+1], piv [n], singular flag)."""
    lib = _load()
    b = _c128(bands)
    n = b.shape[1]
    w = 2 * kl + ku + 1
    factor = np.zeros((n, w), dtype=np.complex128)
    piv = np.zeros(n, dtype=np.int32)
    rc = lib.oracle_band_lu(n, kl, ku, _dp(b.view(np.float64)), complex(z).real, complex(z).imag,
                            _dp(factor.view(np.float64)), piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return factor, piv, rc


def band_solve(factor: np.ndarray, piv: np.ndarray, kl: int, ku: int, rhs: np.ndarray,
               adjoint: bool = False) -> np.ndarray:
    """Solve (zI - A) x = rhs, or its adjoint system, with a factor from ``band_lu``."""
    lib = _load()
    n = factor.shape[0]
    x = _c128(rhs).copy()
    f = _c128(factor)
    p = np.ascontiguousarray(piv, dtype=np.int32)
    lib.oracle_band_solve(n, kl, ku, _dp(f.view(np.float64)), p.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          1 if adjoint else 0, _dp(x.view(np.float64)))
    return x


def tridiag_top(alpha: np.ndarray, beta_off: np.ndarray) -> Tuple[float, float]:
    """Largest eigenvalue of tridiag(beta_off, alpha, beta_off) and |last eigvec component|."""
    lib = _load()
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta_off, dtype=np.float64)
    if b.size == 0:
        b = np.zeros(1)
    th = ctypes.c_double()
    s = ctypes.c_double()
    lib.oracle_tridiag_top(a.size, _dp(a), _dp(b), ctypes.byref(th), ctypes.byref(s))
    return th.value, s.value


def lanczos_coeffs(bands: np.ndarray, kl: int, ku: int, z: complex, k: int, seed: int = 0):
    """alpha_1..alpha_k, beta_1..beta_k of the Lanczos recurrence on (B B^*)^{-1} / 2^(2 e1)."""
    lib = _load()
    b = _c128(bands)
    n = b.shape[1]
    alpha = np.zeros(k)
    beta = np.zeros(k)
    e1 = ctypes.c_int32()
    done = lib.oracle_lanczos_coeffs(n, kl, ku, _dp(b.view(np.float64)), complex(z).real, complex(z).imag,
                                     k, seed & (2**64 - 1), _dp(alpha), _dp(beta), ctypes.byref(e1))
    return alpha[:done], beta[:done], int(e1.value)


# ---------------------------------------------------------------- masks
def masks(sigma: np.ndarray, eps: Sequence[float]) -> np.ndarray:
    """uint32 bits: bit l set iff sigma <= eps[l] (Eq. (sensitive_zone), inclusive)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    out = np.zeros(sigma.shape, dtype=np.uint32)
    for l, e in enumerate(eps):
        out |= (sigma <= e).astype(np.uint32) << np.uint32(l)
    return out


def sigma_min_grid(bands: np.ndarray, kl: int, ku: int, grid, eps: Sequence[float], **kw):
    """Full-grid oracle: (sigma[ny, nx], mask[ny, nx], status[ny, nx], steps[ny, nx])."""
    z = grid_points(grid)
    s, st, k = sigma_min_banded(bands, kl, ku, z.ravel(), **kw)
    shp = (grid.ny, grid.nx)
    return s.reshape(shp), masks(s, eps).reshape(shp), st.reshape(shp), k.reshape(shp)


# ------------------------------------------------------------ gradients
def sigma_min_grad_dense(A: np.ndarray, z: complex):
    """sigma_min(zI - A) and its first derivatives from a dense SVD.

    For a simple smallest singular value with B v = sigma u (B = zI - A),
    d sigma = Re(u^* dB v) (first-order perturbation of a singular value), so
      grad_z = d sigma / d Re z + i d sigma / d Im z = conj(u^* v)
      grad_A[i, j] = d sigma / d Re A_ij + i d sigma / d Im A_ij = -u_i conj(v_j).
    Returns (sigma, grad_z, grad_A) with grad_A dense (n x n).
    """
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    B = complex(z) * np.eye(n) - A
    U, s, Vh = np.linalg.svd(B)
    u = U[:, -1]
    v = Vh[-1].conj()
    gz = np.conj(np.vdot(u, v))
    gA = -np.outer(u, v.conj())
    return float(s[-1]), complex(gz), gA


def dense_grad_to_bands(gA: np.ndarray, kl: int, ku: int) -> np.ndarray:
    """The band part of a dense gradient, in band storage g[d + kl, i] = gA[i, i + d]."""
    n = gA.shape[0]
    g = np.zeros((kl + ku + 1, n), dtype=np.complex128)
    for d in range(-kl, ku + 1):
        for i in range(n):
            if 0 <= i + d < n:
                g[d + kl, i] = gA[i, i + d]
    return g
