"""The classifier network of the restricted method (psa_mlp_* through the C ABI).

A multilayer perceptron IN -> 256 -> 256 -> 256 -> 1 with SiLU hidden units and a
sigmoid output; its dense layers run as BF16 GEMMs on the tensor cores (FP32
accumulation), training is Adam on binary cross-entropy (paper Sec. 3.4). All
parameters live in one float32 device vector ``theta`` (layout in include/psa.h).
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _native

IN, HIDDEN, NPARAM = _native.MLP_IN, _native.MLP_HIDDEN, _native.MLP_PARAMS

# offsets of the parameter blocks in theta
OFF = {}
_o = 0
for _name, _size in (("W1", HIDDEN * IN), ("b1", HIDDEN), ("W2", HIDDEN * HIDDEN), ("b2", HIDDEN),
                     ("W3", HIDDEN * HIDDEN), ("b3", HIDDEN), ("w4", HIDDEN), ("b4", 1)):
    OFF[_name] = (_o, _size)
    _o += _size
assert _o == NPARAM


def init_theta(seed: int = 0, device="cuda"):
    """Seeded initial parameters: weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)) as for a
    default linear layer, biases zero."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    th = np.zeros(NPARAM, dtype=np.float32)
    for name, fan_in in (("W1", IN), ("W2", HIDDEN), ("W3", HIDDEN), ("w4", HIDDEN)):
        o, n = OFF[name]
        th[o:o + n] = rng.uniform(-1.0, 1.0, n) / np.sqrt(fan_in)
    return torch.as_tensor(th, device=device)


def _bf16_bits(x):
    import torch
    if x.dtype != torch.bfloat16 or not x.is_cuda or not x.is_contiguous():
        raise TypeError("expected a contiguous CUDA bfloat16 tensor")
    return x.data_ptr()


def gemm_bf16(A, B, stream=None):
    """C = A @ B.T on the tensor cores: A (M, K), B (N, K) bfloat16, C float32."""
    import torch
    lib = _native.load()
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    s = stream if stream is not None else torch.cuda.current_stream(A.device)
    _native.check(lib.psa_gemm_bf16(_bf16_bits(A), A.stride(0), _bf16_bits(B), B.stride(0), M, N, K,
                                    C.data_ptr(), N, s.cuda_stream), "psa_gemm_bf16")
    return C


def check_timeouts() -> None:
    """Raise if a tensor-core GEMM tile gave up on a bounded wait since the last check
    (its outputs were written as NaN). Synchronises the device."""
    lib = _native.load()
    n = ctypes.c_uint32()
    _native.check(lib.psa_mlp_timeouts(ctypes.byref(n)), "psa_mlp_timeouts")
    if n.value:
        raise _native.PsaError(_native.PSA_ECUDA, f"{n.value} GEMM tile(s) timed out waiting for the tensor cores")


def workspace_bytes(rows: int, training: bool) -> int:
    lib = _native.load()
    out = ctypes.c_size_t()
    _native.check(lib.psa_mlp_workspace_bytes(int(rows), int(bool(training)), ctypes.byref(out)),
                  "psa_mlp_workspace_bytes")
    return int(out.value)


def _aligned_buffer(nbytes: int, device):
    import torch
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    return buf, buf.data_ptr() + (-buf.data_ptr()) % 256


def forward(theta, x, out=None, workspace=None, stream=None):
    """Probabilities (float32, rows) of feature rows x (bfloat16, (rows, IN))."""
    import torch
    lib = _native.load()
    rows = int(x.shape[0])
    if x.dim() != 2 or x.shape[1] != IN:
        raise ValueError(f"x must have shape (rows, {IN})")
    if theta.dtype != torch.float32 or theta.numel() != NPARAM or not theta.is_contiguous():
        raise ValueError("theta must be a contiguous float32 vector of the parameter count")
    prob = out if out is not None else torch.empty(rows, dtype=torch.float32, device=x.device)
    if prob.dtype != torch.float32 or not prob.is_contiguous() or prob.numel() < rows or prob.device != x.device:
        raise ValueError("out must be a contiguous float32 tensor of at least `rows` values on x's device")
    if workspace is None:
        nb = workspace_bytes(rows, False)
        buf, ptr = _aligned_buffer(nb, x.device)
    else:
        buf, ptr, nb = workspace
    s = stream if stream is not None else torch.cuda.current_stream(x.device)
    _native.check(lib.psa_mlp_forward(theta.data_ptr(), _bf16_bits(x), rows, prob.data_ptr(), ptr, nb,
                                      s.cuda_stream), "psa_mlp_forward")
    return prob


class Trainer:
    """Adam on binary cross-entropy with fixed batch size ``batch`` (a multiple of
    128). ``step(x, y)`` takes one batch; ``graph_step`` replays a captured step
    whose inputs are the trainer's own ``x`` and ``y`` buffers."""

    def __init__(self, theta, batch: int = 512, lr: float = 1e-3):
        import torch
        if batch % 128:
            raise ValueError("batch must be a multiple of 128")
        self.theta = theta
        self.batch = batch
        self.lr = lr
        dev = theta.device
        self.m = torch.zeros_like(theta)
        self.v = torch.zeros_like(theta)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        nb = workspace_bytes(batch, True)
        self._buf, self._ptr = _aligned_buffer(nb, dev)
        self._nb = nb
        self.t = 0
        self.x = torch.zeros((batch, IN), dtype=torch.bfloat16, device=dev)
        self.y = torch.zeros(batch, dtype=torch.float32, device=dev)

    def _launch(self, x, y, t: int, stream):
        lib = _native.load()
        _native.check(lib.psa_mlp_train_step(self.theta.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), int(t),
                                             float(self.lr), _bf16_bits(x), y.data_ptr(), self.batch,
                                             self.loss.data_ptr(), self._ptr, self._nb, stream.cuda_stream),
                      "psa_mlp_train_step")

    def step(self, x, y, stream=None):
        """One Adam step on the batch (x bfloat16 (batch, IN), y float32 (batch,))."""
        import torch
        if x.shape != (self.batch, IN) or y.shape != (self.batch,):
            raise ValueError("batch shape")
        self.t += 1
        s = stream if stream is not None else torch.cuda.current_stream(self.theta.device)
        self._launch(x.contiguous(), y.contiguous(), self.t, s)
        return self.loss
