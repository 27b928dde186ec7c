"""Newton refinement of eps-contours along grid lines.

The eps-pseudospectrum boundary is the level set sigma_min(zI - A) = eps (paper
Sec. 2, Definition "Pseudospectrum"; the grid and the sensitive zone of Sec. 2.1).
On a grid, a row i crosses the contour between columns j and j+1 whenever the mask
bit (sigma <= eps) changes there. Each crossing is refined to a point x* on that
grid line with sigma(x* + i y_i) = eps by Newton's method on f(x) = sigma - eps,
f'(x) = d sigma / d Re z from the adjoint kernel, kept inside the bracket
[x_j, x_{j+1}] (a step that leaves the bracket, or a non-positive slope in the
wrong direction, is replaced by bisection).

All evaluations of one Newton iteration go to the GPU in one call of
``sigma_min_grad``; the host only keeps the brackets (plain arithmetic on a few
thousand numbers).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from . import LanczosOpts, sigma_min_grad
from .inputs import Grid


@dataclasses.dataclass
class ContourRefinement:
    x: np.ndarray            # refined abscissae
    y: np.ndarray            # ordinate of each crossing (its grid row)
    row: np.ndarray          # grid row i
    col: np.ndarray          # left grid column j of the bracket
    residual: np.ndarray     # |sigma(x* + i y) - eps| / eps at the final iterate
    iterations: int          # Newton iterations done (GPU calls)
    converged: np.ndarray    # bool per crossing


def grid_crossings(sigma: np.ndarray, eps: float):
    """(rows, cols) of the grid intervals [j, j+1] whose endpoints lie on opposite sides of eps."""
    s = np.asarray(sigma) <= eps
    rows, cols = np.nonzero(s[:, :-1] != s[:, 1:])
    return rows, cols


def refine_rows(bands, kl: int, ku: int, grid: Grid, sigma: np.ndarray, eps: float,
                max_iter: int = 40, rtol: float = 1e-12, opts: Optional[LanczosOpts] = None) -> ContourRefinement:
    """Refine every row crossing of the eps-contour of a computed grid field `sigma` (ny, nx)."""
    import torch

    rows, cols = grid_crossings(sigma, eps)
    hx = (grid.re_max - grid.re_min) / (grid.nx - 1)
    hy = (grid.im_max - grid.im_min) / max(grid.ny - 1, 1)
    lo = grid.re_min + cols * hx
    hi = grid.re_min + (cols + 1) * hx
    y = grid.im_min + rows * hy
    s_lo = np.asarray(sigma)[rows, cols]
    s_hi = np.asarray(sigma)[rows, cols + 1]
    # start from the interpolation of log(sigma) between the bracket ends
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (np.log(eps) - np.log(np.maximum(s_lo, 1e-300))) / (np.log(np.maximum(s_hi, 1e-300)) -
                                                                np.log(np.maximum(s_lo, 1e-300)))
    t = np.where(np.isfinite(t), np.clip(t, 0.05, 0.95), 0.5)
    x = lo + t * (hi - lo)
    f_lo_neg = s_lo <= eps          # sign of f = sigma - eps at the left end (<= 0 there)
    m = x.size
    done = np.zeros(m, dtype=bool)
    resid = np.full(m, np.inf)
    it = 0
    o = opts or LanczosOpts(tol=1e-15, k_max=4000)
    dev = bands.device
    for it in range(1, max_iter + 1):
        act = np.flatnonzero(~done)
        if act.size == 0:
            it -= 1
            break
        z = torch.as_tensor(x[act] + 1j * y[act], dtype=torch.complex128, device=dev)
        r = sigma_min_grad(bands, kl, ku, z, opts=o)
        s = r.sigma.cpu().numpy()
        g = r.grad_z.cpu().numpy().real          # d sigma / d Re z
        f = s - eps
        resid[act] = np.abs(f) / eps
        conv = resid[act] <= rtol
        done[act[conv]] = True
        # shrink the brackets: the left end keeps the sign it had on the grid
        same_as_lo = (f <= 0) == f_lo_neg[act]
        lo[act] = np.where(same_as_lo, x[act], lo[act])
        hi[act] = np.where(same_as_lo, hi[act], x[act])
        with np.errstate(divide="ignore", invalid="ignore"):
            xn = x[act] - f / g
        ok = np.isfinite(xn) & (xn > lo[act]) & (xn < hi[act])
        xn = np.where(ok, xn, 0.5 * (lo[act] + hi[act]))
        width = hi[act] - lo[act]
        done[act[width <= 4e-16 * np.maximum(np.abs(lo[act]), 1.0)]] = True
        x[act] = np.where(conv, x[act], xn)
    return ContourRefinement(x=x, y=y, row=rows, col=cols, residual=resid, iterations=it, converged=done & (resid <= rtol))
