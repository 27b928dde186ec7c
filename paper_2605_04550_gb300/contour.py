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
``sigma_min_grad``, and the iteration's arithmetic (first iterate, bracket update,
Newton or bisection step) runs in the library's psa_contour_init / psa_contour_step
kernels; the host finds the crossings on the grid, selects the running ones and
launches.
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
    import ctypes

    import torch
    from . import _native

    lib = _native.load()
    rows, cols = grid_crossings(sigma, eps)
    m = int(rows.size)
    dev = bands.device
    s_np = np.asarray(sigma)
    t32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32), device=dev)
    t64 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    r_t, c_t = t32(rows), t32(cols)
    s_lo, s_hi = t64(s_np[rows, cols]), t64(s_np[rows, cols + 1])
    x, lo, hi, y, resid = (torch.empty(max(m, 1), dtype=torch.float64, device=dev) for _ in range(5))
    flo_neg, done = (torch.empty(max(m, 1), dtype=torch.uint8, device=dev) for _ in range(2))
    z = torch.empty(max(m, 1), dtype=torch.complex128, device=dev)
    g = _native.PsaGrid(float(grid.re_min), float(grid.re_max), float(grid.im_min), float(grid.im_max),
                        int(grid.nx), int(grid.ny))
    st = torch.cuda.current_stream(dev).cuda_stream
    _native.check(lib.psa_contour_init(m, r_t.data_ptr(), c_t.data_ptr(), ctypes.byref(g), s_lo.data_ptr(),
                                       s_hi.data_ptr(), float(eps), x.data_ptr(), lo.data_ptr(), hi.data_ptr(),
                                       y.data_ptr(), flo_neg.data_ptr(), done.data_ptr(), resid.data_ptr(),
                                       z.data_ptr(), st), "psa_contour_init")
    o = opts or LanczosOpts(tol=1e-15, k_max=4000)
    it = 0
    for it in range(1, max_iter + 1):
        # the running crossings and their iterates, selected on the host (a few thousand
        # values; copies only, so no other kernels run on the device)
        act_h = np.flatnonzero(done[:m].cpu().numpy() == 0).astype(np.int32)
        if act_h.size == 0:
            it -= 1
            break
        act = torch.as_tensor(act_h, device=dev)
        z_act = torch.as_tensor(z[:m].cpu().numpy()[act_h], device=dev)
        r = sigma_min_grad(bands, kl, ku, z_act, opts=o)
        _native.check(lib.psa_contour_step(int(act.numel()), act.data_ptr(), r.sigma.data_ptr(),
                                           r.grad_z.data_ptr(), float(eps), float(rtol), x.data_ptr(),
                                           lo.data_ptr(), hi.data_ptr(), y.data_ptr(), flo_neg.data_ptr(),
                                           done.data_ptr(), resid.data_ptr(), z.data_ptr(), st),
                      "psa_contour_step")
    res = resid[:m].cpu().numpy()
    return ContourRefinement(x=x[:m].cpu().numpy(), y=y[:m].cpu().numpy(), row=rows, col=cols, residual=res,
                             iterations=it, converged=(done[:m].cpu().numpy() != 0) & (res <= rtol))
