"""Batches of matrices, each on its own grid, through psa_sigma_min_batched.

A batch plan (psa_batch_plan) groups the matrices into classes of equal band
shape (kl, ku); each class runs as one persistent launch of the sigma_min kernel
specialised for its shape, whose warps take 8 x 4 tiles of all the class's grids
from one counter. Results are bit-identical to one psa_sigma_min call per matrix.

The batched call allocates nothing and moves nothing between host and device,
so ``BatchGraph`` captures it once in a CUDA graph and replays it. ``autotune``
picks the launch controls (points in flight per class, work order, number of
streams) by timing replays of the captured batch itself.

With several streams the classes are split over the caller's stream and up to
seven auxiliary streams, so that several classes are in flight at once and the
tail of one class (its last few long tiles) runs beside the others.
"""
from __future__ import annotations

import ctypes
import dataclasses
import itertools
from typing import List, Optional, Sequence, Tuple

from . import LanczosOpts, _native
from .inputs import Grid

ORDER_AUTO = _native.BATCH_ORDER_AUTO
ORDER_PLAN = _native.BATCH_ORDER_PLAN
ORDER_ESTIMATE = _native.BATCH_ORDER_ESTIMATE

__all__ = ["BatchPlan", "BatchResult", "BatchConfig", "BatchGraph", "batch_workspace_bytes",
           "sigma_min_batched", "autotune", "ORDER_AUTO", "ORDER_PLAN", "ORDER_ESTIMATE"]


def _aligned(nbytes: int, device):
    import torch
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf, buf.data_ptr() + off


class BatchPlan:
    """Host and device copies of the plan of a batch; outputs are laid out in the
    order of ``mats``, matrix m's grid at ``offsets[m] .. offsets[m] + ny * nx``.

    mats: sequence of (bands, kl, ku, grid), bands a contiguous CUDA complex128
    tensor of shape (kl + ku + 1, n) on one device. The plan keeps references to
    the bands tensors (the plan holds their device pointers).
    """

    def __init__(self, mats: Sequence[Tuple[object, int, int, Grid]]):
        import torch
        lib = _native.load()
        if len(mats) == 0:
            raise ValueError("a batch needs at least one matrix")
        dev = mats[0][0].device
        entries = (_native.PsaBatchEntry * len(mats))()
        self.bands = []
        self.shapes: List[Tuple[int, int]] = []
        self.offsets: List[int] = []
        self.band_shapes: List[Tuple[int, int, int]] = []
        off = 0
        for m, (b, kl, ku, g) in enumerate(mats):
            if (not isinstance(b, torch.Tensor) or b.dtype != torch.complex128 or b.device != dev or
                    b.dim() != 2 or b.shape[0] != kl + ku + 1 or not b.is_contiguous()):
                raise ValueError(f"matrix {m}: bands must be a contiguous complex128 ({kl + ku + 1}, n) "
                                 f"tensor on {dev}")
            self.bands.append(b)
            entries[m].A = _native.PsaBand(int(b.shape[1]), int(kl), int(ku), b.data_ptr())
            entries[m].g = _native.PsaGrid(float(g.re_min), float(g.re_max), float(g.im_min), float(g.im_max),
                                           int(g.nx), int(g.ny))
            entries[m].out_offset = off
            self.shapes.append((int(g.ny), int(g.nx)))
            self.offsets.append(off)
            self.band_shapes.append((int(b.shape[1]), int(kl), int(ku)))
            off += int(g.nx) * int(g.ny)
        self.npoints = off
        self.nmat = len(mats)
        self.device = dev
        nb = ctypes.c_size_t()
        _native.check(lib.psa_batch_plan_bytes(self.nmat, ctypes.byref(nb)), "psa_batch_plan_bytes")
        self.nbytes = int(nb.value)
        self.host = ctypes.create_string_buffer(self.nbytes)
        _native.check(lib.psa_batch_plan(entries, self.nmat, self.host, self.nbytes), "psa_batch_plan")
        self._dbuf, self.dev_ptr = _aligned(self.nbytes, dev)
        hb = torch.frombuffer(bytearray(self.host.raw), dtype=torch.uint8)
        off = self.dev_ptr - self._dbuf.data_ptr()
        self._dbuf[off:off + self.nbytes].copy_(hb)

    def classes(self) -> List[Tuple[int, int]]:
        """Band shapes (kl, ku) of the batch, one per class."""
        return sorted({(kl, ku) for _, kl, ku in self.band_shapes})

    def split(self, flat) -> list:
        """Per-matrix (ny, nx) views of a flat batch output."""
        return [flat[o:o + ny * nx].view(ny, nx) for o, (ny, nx) in zip(self.offsets, self.shapes)]


def batch_workspace_bytes(plan: BatchPlan, points_in_flight: int, opts: Optional[LanczosOpts] = None,
                          streams: int = 4) -> int:
    lib = _native.load()
    out = ctypes.c_size_t()
    _native.check(lib.psa_batch_workspace_bytes(plan.host, ctypes.byref((opts or LanczosOpts())._c()),
                                                int(points_in_flight), int(streams), ctypes.byref(out)),
                  "psa_batch_workspace_bytes")
    return int(out.value)


MAX_STREAMS = 8
_aux_streams = {}


def _aux_stream_array(device, n: int):
    """The first n auxiliary streams of a device (created once per process and device)."""
    import torch
    key = torch.device(device).index
    pool = _aux_streams.setdefault(key, [])
    while len(pool) < n:
        pool.append(torch.cuda.Stream(device))
    return (ctypes.c_void_p * max(n, 1))(*[s.cuda_stream for s in pool[:n]])


def _full_points_in_flight(plan: BatchPlan) -> int:
    """Points in flight that fill the device once, for the class that allows most."""
    from . import default_points_in_flight
    return max(default_points_in_flight(n, kl, ku, 1 << 30) for n, kl, ku in plan.band_shapes)


@dataclasses.dataclass
class BatchResult:
    sigma: "object"   # torch.float64 (npoints,), matrix m at plan.offsets[m]
    mask: "object"    # torch.int32 (npoints,)
    status: "object"  # torch.int8 (npoints,)
    steps: "object"   # torch.int32 (npoints,)


@dataclasses.dataclass(frozen=True)
class BatchConfig:
    """Launch controls of a batched call: points in flight per class (0: as many as
    the workspace and one full occupancy allow), the work order, and the number of
    streams the classes are split over (1 to 8)."""
    points_in_flight: int = 0
    order: int = ORDER_AUTO
    streams: int = 4


class BatchWorkspace:
    """Device scratch of a batched call. ``max_bytes`` caps it (the classes then run
    with as many warps as fit); default: a full occupancy of the device for every
    class on each of ``streams`` streams, capped at half of the free device memory."""

    def __init__(self, plan: BatchPlan, opts: Optional[LanczosOpts] = None, max_bytes: Optional[int] = None,
                 streams: int = 4):
        import torch
        want = batch_workspace_bytes(plan, _full_points_in_flight(plan), opts, streams)
        if max_bytes is None:
            free, _ = torch.cuda.mem_get_info(plan.device)
            max_bytes = free // 2
        self.nbytes = int(min(want, max_bytes))
        self.buffer, self.ptr = _aligned(self.nbytes, plan.device)


def sigma_min_batched(plan: BatchPlan, eps: Sequence[float] = (), opts: Optional[LanczosOpts] = None,
                      workspace: Optional[BatchWorkspace] = None, config: BatchConfig = BatchConfig(),
                      out: Optional[BatchResult] = None, stream=None) -> BatchResult:
    """sigma_min and eps masks on every grid point of every matrix of the plan
    (asynchronous on ``stream``, default torch's current stream)."""
    import torch
    lib = _native.load()
    dev = plan.device
    o = opts or LanczosOpts()
    ws = workspace or BatchWorkspace(plan, o)
    if out is None:
        N = plan.npoints
        out = BatchResult(torch.empty(N, dtype=torch.float64, device=dev), torch.empty(N, dtype=torch.int32, device=dev),
                          torch.empty(N, dtype=torch.int8, device=dev), torch.empty(N, dtype=torch.int32, device=dev))
    else:
        from . import _check_out
        _check_out(out, plan.npoints, dev)
    eps_arr = (ctypes.c_double * max(len(eps), 1))(*[float(e) for e in eps])
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    if not 1 <= config.streams <= MAX_STREAMS:
        raise ValueError(f"streams must be in 1..{MAX_STREAMS}")
    aux = _aux_stream_array(dev, config.streams - 1)
    rc = lib.psa_sigma_min_batched(plan.host, plan.dev_ptr, eps_arr, len(eps), out.sigma.data_ptr(),
                                   out.mask.data_ptr(), out.status.data_ptr(), out.steps.data_ptr(),
                                   ctypes.byref(o._c()), int(config.points_in_flight), int(config.order),
                                   ws.ptr, ws.nbytes, s.cuda_stream, aux, config.streams - 1)
    _native.check(rc, "psa_sigma_min_batched")
    return out


class BatchGraph:
    """A batched call captured once in a CUDA graph; ``replay()`` re-runs it on the
    same plan, workspace and outputs (``out``)."""

    def __init__(self, plan: BatchPlan, eps: Sequence[float] = (), opts: Optional[LanczosOpts] = None,
                 config: BatchConfig = BatchConfig(), workspace: Optional[BatchWorkspace] = None):
        import torch
        self.plan = plan
        self.workspace = workspace or BatchWorkspace(plan, opts)
        N = plan.npoints
        dev = plan.device
        self.out = BatchResult(torch.empty(N, dtype=torch.float64, device=dev),
                               torch.empty(N, dtype=torch.int32, device=dev),
                               torch.empty(N, dtype=torch.int8, device=dev), torch.empty(N, dtype=torch.int32, device=dev))
        args = dict(eps=eps, opts=opts, workspace=self.workspace, config=config, out=self.out)
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            sigma_min_batched(plan, **args, stream=side)  # checks the arguments outside capture
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            sigma_min_batched(plan, **args, stream=torch.cuda.current_stream(dev))

    def replay(self) -> BatchResult:
        self.graph.replay()
        return self.out


def autotune(plan: BatchPlan, eps: Sequence[float] = (), opts: Optional[LanczosOpts] = None,
             candidates: Optional[Sequence[BatchConfig]] = None, reps: int = 1,
             workspace: Optional[BatchWorkspace] = None):
    """Times each candidate configuration on the batch itself (graph replays, CUDA
    events) and returns (best config, {config: ms}). Default candidates: 4, 6, 8
    and 12 warps per SM (where the occupancy allows them) x the three work orders
    x 1, 2, 4 or 8 streams."""
    import torch
    dev = plan.device
    ws = workspace or BatchWorkspace(plan, opts)
    if candidates is None:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        pifs = [w * 32 * sms for w in (4, 6, 8, 12)]
        candidates = [BatchConfig(p, o, st) for p, o, st in
                      itertools.product(pifs, (ORDER_AUTO, ORDER_PLAN, ORDER_ESTIMATE), (1, 2, 4, 8))]
    times = {}
    for cfg in candidates:
        g = BatchGraph(plan, eps, opts, cfg, workspace=ws)
        g.replay()  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(reps):
            e0.record()
            g.replay()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        times[cfg] = min(ms)
        del g
    best = min(times, key=times.get)
    return best, times
