"""Plain NumPy restatement of the learned restriction's features (TEST INFRASTRUCTURE).

Only ``tests/`` may use this module; the library computes the same quantities in
its own kernels (psa_matrix_stats, psa_global_features, psa_point_features) and
shares no code with it. Each function writes the definition out directly, entry by
entry, in FP64 (the library stores the point features in BF16).

The features follow the paper's tables of matrix features and its per-point
distances (Sec. 3.1, Tables "matrix", "matrixAdd" and "resolvent", Eq. (dist)).
With eigenvalues given (point_set_stats, point_features(closed=False)) they are
the paper's own; by default they take the readings this library uses in place of
dense eigenvalues:
the eigenvalue set is replaced by the symbol curve of the diagonal means,
f(t) = sum_d abar_d e^{i d t} at 256 points t_k = 2 pi k / 256, about the
centroid trace(A) / n (the eigenvalue mean, Table 3); g1 is the distance to the
closed polyline through the samples; distances are in units of the curve's radius
R = max_k |f(t_k) - centroid|.
"""
from __future__ import annotations

import numpy as np

SAMPLES = 256
STATS = 24
GLOBAL = 28
ROW = 128


def dense(bands: np.ndarray, kl: int, ku: int) -> np.ndarray:
    """The band as a dense matrix: A[i, i + d] = bands[d + kl, i]."""
    n = bands.shape[1]
    A = np.zeros((n, n), dtype=np.complex128)
    for d in range(-kl, ku + 1):
        for i in range(n):
            if 0 <= i + d < n:
                A[i, i + d] = bands[d + kl, i]
    return A


def symbol_samples(bands: np.ndarray, kl: int, ku: int, samples: int = SAMPLES) -> np.ndarray:
    """f(t_k) = sum_d abar_d exp(i d t_k) with abar_d the mean of the d-th diagonal."""
    A = dense(bands, kl, ku)
    abar = np.array([np.mean(np.diag(A, d)) for d in range(-kl, ku + 1)])
    t = 2.0 * np.pi * np.arange(samples) / samples
    return np.array([sum(abar[d + kl] * np.exp(1j * d * tk) for d in range(-kl, ku + 1)) for tk in t])


def matrix_stats(bands: np.ndarray, kl: int, ku: int):
    """The 24 statistics (layout PSA_STAT_* of the library's header) and the symbol samples."""
    A = dense(bands, kl, ku)
    n = A.shape[0]
    f = symbol_samples(bands, kl, ku)
    cen = np.trace(A) / n
    x = f - cen
    inband = np.zeros((n, n), dtype=bool)
    for d in range(-kl, ku + 1):
        inband |= np.eye(n, k=d, dtype=bool)
    offband = inband & ~np.eye(n, dtype=bool)
    mod = np.abs(A)
    st = np.zeros(STATS)
    st[0], st[1] = cen.real, cen.imag
    st[2] = np.abs(x).max()
    st[3] = np.linalg.norm(A)
    st[4] = mod.sum(axis=0).max()
    st[5] = mod.sum(axis=1).max()
    st[6] = np.linalg.norm(A - A.T)
    st[7] = np.linalg.norm(A - A.conj().T)
    dg = np.abs(np.diag(A))
    st[8], st[9] = dg.mean(), dg.std()
    od = mod[offband]
    st[10], st[11] = (od.mean(), od.std()) if od.size else (0.0, 0.0)
    st[12] = float(np.sum(mod[inband] > 1e-10))
    st[13], st[14], st[15], st[16] = x.real.mean(), x.real.std(), x.real.min(), x.real.max()
    st[17], st[18], st[19], st[20] = x.imag.mean(), x.imag.std(), x.imag.min(), x.imag.max()
    st[21] = np.abs(x).min()
    st[22] = n
    st[23] = 16 * kl + ku
    return st, f


def point_set_stats(st: np.ndarray, pts) -> np.ndarray:
    """The statistics with the spectrum entries taken over a point set (the paper's
    eigenvalue features f1-f10, Sec. 3.1, Table "matrix"): about the centroid st[0:2],
    R = max |p - c|, mean / std / min / max of Re and Im of (p - c), min |p - c|."""
    out = np.array(st, dtype=np.float64)
    x = np.asarray(pts, dtype=np.complex128).ravel() - complex(st[0], st[1])
    out[2] = np.abs(x).max()
    out[13], out[14], out[15], out[16] = x.real.mean(), x.real.std(), x.real.min(), x.real.max()
    out[17], out[18], out[19], out[20] = x.imag.mean(), x.imag.std(), x.imag.min(), x.imag.max()
    out[21] = np.abs(x).min()
    return out


def global_features(st: np.ndarray, sigma4, eps: float) -> np.ndarray:
    """28 scale-free global features. sigma4 = sigma_min(zI - A) at z = 0 and at the
    centroid + 0.5, + 1, + 2 (the resolvent norms of Table "resolvent" are their inverses)."""
    R, fro, n = max(st[2], 1e-300), max(st[3], 1e-300), st[22]
    rms = fro / np.sqrt(n)
    band = int(st[23])
    lg = lambda v: np.log10(max(v, 1e-300))
    g = np.zeros(GLOBAL)
    g[0:4] = st[13:17] / R                    # f1-f8: the spectrum stand-in about the centroid
    g[4:8] = st[17:21] / R
    g[8] = st[21] / R                         # f10 (f9 = 1 after scaling)
    g[9] = st[6] / fro                        # f11: departure from symmetry
    g[10] = st[7] / fro                       # f12: departure from Hermitian
    s1 = np.sqrt(st[4] * st[5])               # bound on sigma_1
    g[11] = lg(s1 / max(sigma4[0], 1e-300) + 1e-12)  # f13 with sigma_n = sigma_min at z = 0
    g[12] = st[4] / fro                       # f15, f16
    g[13] = st[5] / fro
    g[14], g[15] = st[8] / rms, st[9] / rms    # f17, f18
    g[16], g[17] = st[10] / rms, st[11] / rms  # f19, f20
    g[18] = st[12] / n / 16.0                 # f21
    g[19] = lg(st[7] / fro + 1e-12)           # f25
    for k in range(3):                        # f28-f30 (exact 2-norm) times R
        g[20 + k] = lg(R / max(sigma4[1 + k], 1e-300))
    g[23] = lg(R)
    g[24] = lg(eps / R)
    g[25] = (band >> 4) / 4.0
    g[26] = (band & 15) / 8.0
    g[27] = np.log10(n) / 4.0
    return g


def polyline_distance(f: np.ndarray, z: complex) -> float:
    """Distance from z to the closed polyline f[0] -> f[1] -> ... -> f[-1] -> f[0]."""
    best = np.inf
    for k in range(f.size):
        a, b = f[k - 1], f[k]
        e = b - a
        ee = abs(e) ** 2
        t = 0.0 if ee == 0 else min(max(np.real(np.conj(e) * (z - a)) / ee, 0.0), 1.0)
        best = min(best, abs(a + t * e - z))
    return best


def winding_number(f: np.ndarray, z: complex) -> int:
    """Winding number of the closed polyline f about z (sum of the turning angles)."""
    ang = 0.0
    for k in range(f.size):
        ang += np.angle(np.conj(f[k - 1] - z) * (f[k] - z))
    return int(np.rint(ang / (2.0 * np.pi)))


def point_features(grid, st: np.ndarray, f: np.ndarray, g: np.ndarray, flat_idx, closed: bool = True) -> np.ndarray:
    """Feature rows (FP64) of the flat grid indices: [0, 26) the Fourier encoding of Sec.
    3.2.1, [c, sin 2^k c, cos 2^k c] for k = 1..6 (sines and cosines of x and y
    interleaved as the library stores them) of the coordinates scaled to [-1, 1]^2;
    26..28 g1 (polyline), g2 (centroid), g3 (mean sample distance), in units of R;
    29, 30 log10 of g1 and g3; 31 the winding number; 32..59 the global features;
    60 log10 of the polyline distance over eps; zeros after.
    closed=False: f is a point set (the eigenvalues, Eq. (dist)): g1 is the distance
    to its nearest point, g3 the mean distance, column 31 is 0."""
    cen = st[0] + 1j * st[1]
    R = max(st[2], 1e-30)
    hx = (grid.re_max - grid.re_min) / (grid.nx - 1) if grid.nx > 1 else 0.0
    hy = (grid.im_max - grid.im_min) / (grid.ny - 1) if grid.ny > 1 else 0.0
    xc, yc = grid.re_min + 0.5 * hx * (grid.nx - 1), grid.im_min + 0.5 * hy * (grid.ny - 1)
    hw, hh = max(0.5 * hx * (grid.nx - 1), 1e-300), max(0.5 * hy * (grid.ny - 1), 1e-300)
    rows = []
    for fl in np.asarray(flat_idx).ravel():
        i, j = divmod(int(fl), grid.nx)
        z = complex(grid.re_min + j * hx, grid.im_min + i * hy)
        cx, cy = (z.real - xc) / hw, (z.imag - yc) / hh
        v = np.zeros(ROW)
        v[0], v[1] = cx, cy
        for k in range(1, 7):
            w = 2.0 ** k
            v[2 + 4 * (k - 1):6 + 4 * (k - 1)] = [np.sin(w * cx), np.sin(w * cy), np.cos(w * cx), np.cos(w * cy)]
        d = np.abs(f - z)
        g1 = (polyline_distance(f, z) if closed else d.min()) / R
        v[26], v[27], v[28] = g1, abs(z - cen) / R, d.mean() / R
        v[29], v[30] = np.log10(g1 + 1e-7), np.log10(d.mean() / R + 1e-7)
        v[31] = winding_number(f, z) if closed else 0
        v[32:32 + GLOBAL] = g
        v[32 + GLOBAL] = v[29] - g[24]
        rows.append(v)
    return np.array(rows)
