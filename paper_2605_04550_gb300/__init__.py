"""GB300-native sigma_min(zI - A) grid engine for banded non-normal matrices.

Python binding of libpsa (include/psa.h): argument marshalling only. Every
step of the computation runs in the library's CUDA kernels; PyTorch provides
device memory and streams. There is no CPU fallback: calling into the
library without a built libpsa.so or without a CUDA device raises.

    import torch, paper_2605_04550_gb300 as psa
    from paper_2605_04550_gb300.inputs import grcar, grcar_grid_100, EPS_LEVELS_8
    bands, kl, ku = grcar(100)
    out = psa.sigma_min(torch.as_tensor(bands, device="cuda"), kl, ku,
                        grcar_grid_100(), eps=EPS_LEVELS_8)
    out.sigma   # (ny, nx) float64: sigma_min(zI - A) on the grid (paper Sec. 2.1)
    out.mask    # (ny, nx) int32 bit l <=> sigma <= eps[l]  (Eq. (sensitive_zone))
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional, Sequence

from . import _native
from ._native import (PT_NONFINITE, PT_NOT_CONVERGED, PT_NOT_EVALUATED, PT_OK, PT_SINGULAR,
                      PT_UNDERFLOW, PsaError)
from .inputs import Grid

__all__ = [
    "Grid", "LanczosOpts", "SigmaMinResult", "Workspace", "sigma_min", "workspace_bytes",
    "default_points_in_flight", "probe_dfma_rate", "library_path", "PsaError", "tile_order",
    "SigmaMinGradResult", "sigma_min_grad", "grad_workspace_bytes", "SigmaMinFunction", "sigma_min_autograd",
    "GradWorkspace", "band_grad_from_pairs", "release_workspaces",
    "PT_OK", "PT_SINGULAR", "PT_NOT_CONVERGED", "PT_NONFINITE", "PT_NOT_EVALUATED", "PT_UNDERFLOW",
]


@dataclasses.dataclass(frozen=True)
class LanczosOpts:
    """Lanczos controls (psa_lanczos_opts). Defaults = converged mode."""

    k_min: int = 2
    k_max: int = 1000
    tol: float = 1e-13
    seed: int = 0

    @staticmethod
    def fixed(k: int, seed: int = 0) -> "LanczosOpts":
        """Exactly k Lanczos steps (k_min = k_max = k)."""
        return LanczosOpts(k_min=k, k_max=k, tol=0.0, seed=seed)

    def _c(self) -> _native.PsaLanczosOpts:
        return _native.PsaLanczosOpts(int(self.k_min), int(self.k_max), float(self.tol),
                                      int(self.seed) & (2**64 - 1))


@dataclasses.dataclass
class SigmaMinResult:
    sigma: "object"   # torch.float64 (ny, nx)
    mask: "object"    # torch.int32 (ny, nx) (bits; reinterpret as uint32)
    status: "object"  # torch.int8 (ny, nx)
    steps: "object"   # torch.int32 (ny, nx)


def library_path() -> str:
    return _native.LIB


def _band(bands, kl: int, ku: int) -> _native.PsaBand:
    import torch
    if not isinstance(bands, torch.Tensor) or bands.dtype != torch.complex128 or not bands.is_cuda:
        raise TypeError("bands must be a CUDA torch.complex128 tensor of shape (kl + ku + 1, n)")
    if bands.dim() != 2 or bands.shape[0] != kl + ku + 1 or not bands.is_contiguous():
        raise ValueError("bands must be contiguous with shape (kl + ku + 1, n)")
    return _native.PsaBand(int(bands.shape[1]), int(kl), int(ku), bands.data_ptr())


def _band_shape(n: int, kl: int, ku: int) -> _native.PsaBand:
    return _native.PsaBand(int(n), int(kl), int(ku), None)


def workspace_bytes(n: int, kl: int, ku: int, points_in_flight: int,
                    opts: Optional[LanczosOpts] = None, npoints: int = 0) -> int:
    """Workspace bytes for `points_in_flight` points in flight and calls of up to
    `npoints` points (0: no work-order schedule)."""
    lib = _native.load()
    o = (opts or LanczosOpts())._c()
    out = ctypes.c_size_t()
    _native.check(lib.psa_workspace_bytes(ctypes.byref(_band_shape(n, kl, ku)), ctypes.byref(o),
                                          int(points_in_flight), int(npoints), ctypes.byref(out)),
                  "psa_workspace_bytes")
    return int(out.value)


def default_points_in_flight(n: int, kl: int, ku: int, npoints: int) -> int:
    """Points in flight that fill the device once for this band shape."""
    lib = _native.load()
    out = ctypes.c_int64()
    _native.check(lib.psa_default_points_in_flight(ctypes.byref(_band_shape(n, kl, ku)), int(npoints),
                                                   ctypes.byref(out)), "psa_default_points_in_flight")
    return int(out.value)


class Workspace:
    """Reusable device scratch for sigma_min (a torch uint8 buffer, 256-byte aligned)."""

    def __init__(self, n: int, kl: int, ku: int, points_in_flight: int,
                 opts: Optional[LanczosOpts] = None, device=None, npoints: int = 0):
        import torch
        self.nbytes = workspace_bytes(n, kl, ku, points_in_flight, opts, npoints)
        self.buffer = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device or "cuda")
        base = self.buffer.data_ptr()
        self.offset = (-base) % 256
        self.ptr = base + self.offset


# The workspace of the last sigma_min call made without one, per device: repeated calls
# on the same problem shape reuse it instead of allocating; release_workspaces() frees it.
_default_ws = {}


def _default_workspace(n: int, kl: int, ku: int, pif: int, o: "LanczosOpts", dev, npoints: int) -> Workspace:
    key = (n, kl, ku, pif, o.k_max, npoints)
    ent = _default_ws.get(str(dev))
    if ent is None or ent[0] != key:
        _default_ws.pop(str(dev), None)  # free the old buffer before taking the new one
        ent = (key, Workspace(n, kl, ku, pif, o, device=dev, npoints=npoints))
        _default_ws[str(dev)] = ent
    return ent[1]


def release_workspaces() -> None:
    """Free the workspaces that sigma_min keeps for calls made without one (the memory
    returns to torch's caching allocator)."""
    _default_ws.clear()


def _check_out(out, npoints: int, dev) -> None:
    """Caller-provided outputs: contiguous, on the device, one entry per grid point."""
    import torch
    for t, dt, name in ((out.sigma, torch.float64, "sigma"), (out.mask, torch.int32, "mask"),
                        (out.status, torch.int8, "status"), (out.steps, torch.int32, "steps")):
        if t.dtype != dt or t.device != dev or not t.is_contiguous() or t.numel() != npoints:
            raise ValueError(f"out.{name} must be a contiguous {dt} tensor of {npoints} entries on {dev}")


def sigma_min(bands, kl: int, ku: int, grid: Grid, eps: Sequence[float] = (), idx=None,
              opts: Optional[LanczosOpts] = None, workspace: Optional[Workspace] = None,
              points_in_flight: Optional[int] = None, out: Optional[SigmaMinResult] = None,
              stream=None) -> SigmaMinResult:
    """sigma_min(zI - A) and epsilon masks on ``grid`` (or at the flat indices ``idx``).

    bands: CUDA complex128 (kl + ku + 1, n), bands[d + kl, i] = A[i, i + d].
    idx:   optional CUDA int32 tensor of flat grid indices (restricted mode).
    workspace: a Workspace to use; without one, the binding keeps the workspace of the
    last such call per device and reuses it for calls of the same shape (the size fills
    the device once: up to tens of GB at large n; ``release_workspaces()`` frees it).
    Calls that may overlap on the GPU must not share a workspace: pass each its own.
    Asynchronous on ``stream`` (default: torch's current stream).
    """
    import torch
    lib = _native.load()
    A = _band(bands, kl, ku)
    n = A.n
    g = _native.PsaGrid(float(grid.re_min), float(grid.re_max), float(grid.im_min), float(grid.im_max),
                        int(grid.nx), int(grid.ny))
    dev = bands.device
    npts = grid.npoints if idx is None else int(idx.numel())
    if idx is not None:
        if idx.dtype != torch.int32 or not idx.is_cuda or not idx.is_contiguous():
            raise TypeError("idx must be a contiguous CUDA int32 tensor")
    o = opts or LanczosOpts()
    if workspace is None:
        pif = points_in_flight or default_points_in_flight(n, kl, ku, max(npts, 1))
        workspace = _default_workspace(n, kl, ku, pif, o, dev, npts)
    elif points_in_flight is not None:
        raise ValueError("pass either workspace or points_in_flight")
    if out is None:
        shape = (grid.ny, grid.nx)
        out = SigmaMinResult(torch.empty(shape, dtype=torch.float64, device=dev),
                             torch.empty(shape, dtype=torch.int32, device=dev),
                             torch.empty(shape, dtype=torch.int8, device=dev),
                             torch.empty(shape, dtype=torch.int32, device=dev))
    else:
        _check_out(out, grid.npoints, dev)
    eps_arr = (ctypes.c_double * max(len(eps), 1))(*[float(e) for e in eps])
    idx_ptr = None
    if idx is not None:
        # an empty list is still a list (restricted mode with no points), never NULL
        idx_ptr = idx.data_ptr() if idx.numel() > 0 else workspace.ptr
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    rc = lib.psa_sigma_min(ctypes.byref(A), ctypes.byref(g), eps_arr, len(eps),
                           idx_ptr, npts if idx is not None else 0,
                           out.sigma.data_ptr(), out.mask.data_ptr(), out.status.data_ptr(),
                           out.steps.data_ptr(), ctypes.byref(o._c()), workspace.ptr, workspace.nbytes,
                           s.cuda_stream)
    _native.check(rc, "psa_sigma_min")
    return out


@dataclasses.dataclass
class SigmaMinGradResult:
    sigma: "object"       # torch.float64 (npts,)
    grad_z: "object"      # torch.complex128 (npts,): d sigma / d Re z + i d sigma / d Im z
    grad_bands: "object"  # torch.complex128 (kl + ku + 1, n) or None
    status: "object"      # torch.int8 (npts,)
    steps: "object"       # torch.int32 (npts,)
    u: "object" = None    # torch.complex128 (n, npts) singular vectors (pairs=True), element-major
    v: "object" = None


def grad_workspace_bytes(n: int, kl: int, ku: int, points_in_flight: int,
                         opts: Optional[LanczosOpts] = None) -> int:
    lib = _native.load()
    o = (opts or LanczosOpts())._c()
    out = ctypes.c_size_t()
    _native.check(lib.psa_grad_workspace_bytes(ctypes.byref(_band_shape(n, kl, ku)), ctypes.byref(o),
                                               int(points_in_flight), ctypes.byref(out)), "psa_grad_workspace_bytes")
    return int(out.value)


class GradWorkspace:
    """Reusable device workspace of psa_sigma_min_grad / psa_sigma_min_pairs."""

    def __init__(self, n: int, kl: int, ku: int, points_in_flight: int, opts: Optional[LanczosOpts] = None,
                 device="cuda"):
        import torch
        self.nbytes = grad_workspace_bytes(n, kl, ku, points_in_flight, opts)
        self._buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        self.ptr = self._buf.data_ptr() + ((-self._buf.data_ptr()) % 256)
        self.shape = (int(n), int(kl), int(ku), (opts or LanczosOpts()).k_max)


def sigma_min_grad(bands, kl: int, ku: int, z, weight=None, opts: Optional[LanczosOpts] = None,
                   points_in_flight: Optional[int] = None, stream=None, workspace: Optional[GradWorkspace] = None,
                   pairs: bool = False) -> SigmaMinGradResult:
    """sigma_min(z I - A) at explicit points with its adjoint gradients (psa_sigma_min_grad).

    z: CUDA complex128 tensor of points. weight: optional CUDA float64 tensor of
    upstream weights; when given, grad_bands = sum_p weight_p d sigma_p / d bands.
    workspace: a GradWorkspace to reuse (else one is allocated for this call).
    pairs: also return the singular pair of every point (psa_sigma_min_pairs; then no
    weight): u, v as (n, npts) complex tensors, element-major.
    """
    import torch
    lib = _native.load()
    A = _band(bands, kl, ku)
    n = A.n
    dev = bands.device
    if not isinstance(z, torch.Tensor) or z.dtype != torch.complex128 or not z.is_cuda:
        raise TypeError("z must be a CUDA complex128 tensor")
    zc = z.contiguous().reshape(-1)
    npts = int(zc.numel())
    o = opts or LanczosOpts()
    if weight is not None:
        weight = weight.to(device=dev, dtype=torch.float64).contiguous().reshape(-1)
        if weight.numel() != npts:
            raise ValueError("weight must have one entry per point")
    if pairs and weight is not None:
        raise ValueError("pairs=True returns the singular pairs instead of a band gradient: pass no weight")
    if workspace is None:
        pif = points_in_flight or min(default_points_in_flight(n, kl, ku, max(npts, 1)),
                                      max(32, -(-npts // 32) * 32))
        workspace = GradWorkspace(n, kl, ku, pif, o, device=dev)
    elif points_in_flight is not None:
        raise ValueError("pass either workspace or points_in_flight")
    elif workspace.shape[:3] != (n, int(kl), int(ku)) or workspace.shape[3] < o.k_max:
        raise ValueError("workspace was sized for another problem")
    nbytes, ptr = workspace.nbytes, workspace.ptr
    sigma = torch.empty(npts, dtype=torch.float64, device=dev)
    gz = torch.empty(npts, dtype=torch.complex128, device=dev)
    gb = torch.empty((kl + ku + 1, n), dtype=torch.complex128, device=dev) if weight is not None else None
    status = torch.empty(npts, dtype=torch.int8, device=dev)
    steps = torch.empty(npts, dtype=torch.int32, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    if pairs:
        u = torch.empty((n, npts), dtype=torch.complex128, device=dev)
        v = torch.empty((n, npts), dtype=torch.complex128, device=dev)
        rc = lib.psa_sigma_min_pairs(ctypes.byref(A), zc.data_ptr() if npts else None, npts, sigma.data_ptr(),
                                     gz.data_ptr(), u.data_ptr() if npts else None, v.data_ptr() if npts else None,
                                     status.data_ptr(), steps.data_ptr(), ctypes.byref(o._c()), ptr, nbytes,
                                     s.cuda_stream)
        _native.check(rc, "psa_sigma_min_pairs")
        return SigmaMinGradResult(sigma, gz, None, status, steps, u, v)
    rc = lib.psa_sigma_min_grad(ctypes.byref(A), zc.data_ptr() if npts else None, npts,
                                weight.data_ptr() if weight is not None else None,
                                sigma.data_ptr(), gz.data_ptr(), gb.data_ptr() if gb is not None else None,
                                status.data_ptr(), steps.data_ptr(), ctypes.byref(o._c()), ptr, nbytes, s.cuda_stream)
    _native.check(rc, "psa_sigma_min_grad")
    return SigmaMinGradResult(sigma, gz, gb, status, steps)


def band_grad_from_pairs(n: int, kl: int, ku: int, u, v, weight, stream=None):
    """Weighted band gradient -sum_p w_p u_p[i] conj(v_p[i + d]) from stored singular pairs
    (psa_band_grad_from_pairs); u, v (n, npts) complex128, weight (npts,) float64."""
    import torch
    lib = _native.load()
    npts = int(u.shape[1])
    if u.shape != (n, npts) or v.shape != (n, npts) or weight.numel() != npts:
        raise ValueError("u, v must be (n, npts) and weight (npts,)")
    w = weight.to(dtype=torch.float64).contiguous().reshape(-1)
    gb = torch.empty((kl + ku + 1, n), dtype=torch.complex128, device=u.device)
    s = stream if stream is not None else torch.cuda.current_stream(u.device)
    _native.check(lib.psa_band_grad_from_pairs(ctypes.byref(_band_shape(n, kl, ku)), npts, u.data_ptr(),
                                               v.data_ptr(), w.data_ptr(), gb.data_ptr(), s.cuda_stream),
                  "psa_band_grad_from_pairs")
    return gb


def tile_order(flat_idx, nx: int):
    """Flat grid indices reordered into 8 x 4 tiles (the full-grid work order).

    Restricted mode hands the list to warps in chunks of 32 entries; in this
    order a chunk covers a compact patch of the grid whose points take similar
    Lanczos step counts. Returns an int32 numpy array.
    """
    import numpy as np
    f = np.asarray(flat_idx, dtype=np.int64).ravel()
    i, j = f // nx, f % nx
    key = ((i // 4) * ((nx + 7) // 8) + (j // 8)) * 32 + (i % 4) * 8 + (j % 8)
    return f[np.argsort(key, kind="stable")].astype(np.int32)


def probe_dfma_rate(iters: int = 4096, stream=None) -> float:
    """Measured DFMA lane-operations per second of the current device (synchronises)."""
    import torch
    lib = _native.load()
    out = ctypes.c_double()
    s = stream if stream is not None else torch.cuda.current_stream()
    _native.check(lib.psa_probe_dfma_rate(int(iters), ctypes.byref(out), s.cuda_stream), "psa_probe_dfma_rate")
    return float(out.value)


#: bytes of singular pairs (2 * 16 * n * points) the autograd forward keeps for its backward
PAIR_BUDGET = 2 << 30


def _make_autograd():
    import torch

    class SigmaMinFunction(torch.autograd.Function):
        """sigma_min(z I - A) as a differentiable function of the band entries and z.

        forward(bands, z, kl, ku, opts) -> sigma (float64, shape of z); backward forms
        d/d bands = sum_p g_p d sigma_p / d bands and d/d z_p = g_p d sigma_p / d z
        (PyTorch's convention for complex inputs: d/d Re + i d/d Im). When the bands
        need a gradient and the singular pairs of all points fit in PAIR_BUDGET bytes,
        the forward keeps them (psa_sigma_min_pairs) and the backward is one contraction
        (psa_band_grad_from_pairs); otherwise the backward reruns the adjoint kernel
        (psa_sigma_min_grad) with the upstream gradient as weights.
        """

        @staticmethod
        def forward(ctx, bands, z, kl, ku, opts=None):
            n, npts = int(bands.shape[1]), int(z.numel())
            keep = bands.requires_grad and 2 * 16 * n * npts <= PAIR_BUDGET
            r = sigma_min_grad(bands.detach(), kl, ku, z.detach(), weight=None, opts=opts, pairs=keep)
            if keep:
                ctx.save_for_backward(r.u, r.v, r.grad_z)
            else:
                ctx.save_for_backward(bands.detach(), z.detach(), r.grad_z)
            ctx.kl, ctx.ku, ctx.opts, ctx.keep, ctx.n = kl, ku, opts, keep, n
            return r.sigma.reshape(z.shape)

        @staticmethod
        def backward(ctx, g):
            a, b, gz = ctx.saved_tensors
            gflat = g.reshape(-1).to(torch.float64).contiguous()
            grad_bands = grad_z = None
            if ctx.needs_input_grad[0]:
                if ctx.keep:
                    grad_bands = band_grad_from_pairs(ctx.n, ctx.kl, ctx.ku, a, b, gflat)
                else:
                    grad_bands = sigma_min_grad(a, ctx.kl, ctx.ku, b, weight=gflat, opts=ctx.opts).grad_bands
            if ctx.needs_input_grad[1]:
                grad_z = (gz * gflat).reshape(g.shape)
            return grad_bands, grad_z, None, None, None

    return SigmaMinFunction


def __getattr__(name):
    if name == "SigmaMinFunction":
        return _make_autograd()
    raise AttributeError(name)


def sigma_min_autograd(bands, z, kl: int, ku: int, opts: Optional[LanczosOpts] = None):
    """Differentiable sigma_min(z I - A) (see SigmaMinFunction)."""
    return _make_autograd().apply(bands, z, kl, ku, opts)
