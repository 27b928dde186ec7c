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
        workspace = Workspace(n, kl, ku, pif, o, device=dev, npoints=npts)
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


def grad_workspace_bytes(n: int, kl: int, ku: int, points_in_flight: int,
                         opts: Optional[LanczosOpts] = None) -> int:
    lib = _native.load()
    o = (opts or LanczosOpts())._c()
    out = ctypes.c_size_t()
    _native.check(lib.psa_grad_workspace_bytes(ctypes.byref(_band_shape(n, kl, ku)), ctypes.byref(o),
                                               int(points_in_flight), ctypes.byref(out)), "psa_grad_workspace_bytes")
    return int(out.value)


def sigma_min_grad(bands, kl: int, ku: int, z, weight=None, opts: Optional[LanczosOpts] = None,
                   points_in_flight: Optional[int] = None, stream=None) -> SigmaMinGradResult:
    """sigma_min(z I - A) at explicit points with its adjoint gradients (psa_sigma_min_grad).

    z: CUDA complex128 tensor of points. weight: optional CUDA float64 tensor of
    upstream weights; when given, grad_bands = sum_p weight_p d sigma_p / d bands.
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
    pif = points_in_flight or min(default_points_in_flight(n, kl, ku, max(npts, 1)), max(32, -(-npts // 32) * 32))
    nbytes = grad_workspace_bytes(n, kl, ku, pif, o)
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    ptr = buf.data_ptr() + ((-buf.data_ptr()) % 256)
    sigma = torch.empty(npts, dtype=torch.float64, device=dev)
    gz = torch.empty(npts, dtype=torch.complex128, device=dev)
    gb = torch.empty((kl + ku + 1, n), dtype=torch.complex128, device=dev) if weight is not None else None
    status = torch.empty(npts, dtype=torch.int8, device=dev)
    steps = torch.empty(npts, dtype=torch.int32, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    rc = lib.psa_sigma_min_grad(ctypes.byref(A), zc.data_ptr() if npts else None, npts,
                                weight.data_ptr() if weight is not None else None,
                                sigma.data_ptr(), gz.data_ptr(), gb.data_ptr() if gb is not None else None,
                                status.data_ptr(), steps.data_ptr(), ctypes.byref(o._c()), ptr, nbytes, s.cuda_stream)
    _native.check(rc, "psa_sigma_min_grad")
    return SigmaMinGradResult(sigma, gz, gb, status, steps)


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


def _make_autograd():
    import torch

    class SigmaMinFunction(torch.autograd.Function):
        """sigma_min(z I - A) as a differentiable function of the band entries and z.

        forward(bands, z, kl, ku, opts) -> sigma (float64, shape of z); backward uses the
        adjoint kernel (psa_sigma_min_grad) with the upstream gradient as weights:
        d/d bands = sum_p g_p d sigma_p / d bands, d/d z_p = g_p d sigma_p / d z
        (PyTorch's convention for complex inputs: d/d Re + i d/d Im).
        """

        @staticmethod
        def forward(ctx, bands, z, kl, ku, opts=None):
            r = sigma_min_grad(bands.detach(), kl, ku, z.detach(), weight=None, opts=opts)
            ctx.save_for_backward(bands.detach(), z.detach(), r.grad_z)
            ctx.kl, ctx.ku, ctx.opts = kl, ku, opts
            return r.sigma.reshape(z.shape)

        @staticmethod
        def backward(ctx, g):
            bands, z, gz = ctx.saved_tensors
            gflat = g.reshape(-1).to(torch.float64).contiguous()
            grad_bands = grad_z = None
            if ctx.needs_input_grad[0]:
                r = sigma_min_grad(bands, ctx.kl, ctx.ku, z, weight=gflat, opts=ctx.opts)
                grad_bands = r.grad_bands
            if ctx.needs_input_grad[1]:
                grad_z = (gz * gflat).reshape(z.shape)
            return grad_bands, grad_z, None, None, None

    return SigmaMinFunction


def __getattr__(name):
    if name == "SigmaMinFunction":
        return _make_autograd()
    raise AttributeError(name)


def sigma_min_autograd(bands, z, kl: int, ku: int, opts: Optional[LanczosOpts] = None):
    """Differentiable sigma_min(z I - A) (see SigmaMinFunction)."""
    return _make_autograd().apply(bands, z, kl, ku, opts)
