"""The classifier networks of the restricted method (psa_mlp_* and psa_dual_*
through the C ABI).

``net="mlp"``: a multilayer perceptron IN -> 256 -> 256 -> 256 -> 1 with SiLU hidden
units and a sigmoid output. ``net="dual"``: the paper's dual-path network (Sec.
3.2.2): a coordinate pathway on the Fourier encoding (26 -> 64 -> 64), a matrix
pathway on the other features (35 -> 128 -> 64), concatenation, a residual block
(128, h6 = h4 + h5), a 64-unit projection and a sigmoid output. Dense layers run as
BF16 GEMMs on the tensor cores (FP32 accumulation); training is Adam on binary
cross-entropy (paper Sec. 3.4). All parameters live in one float32 device vector
``theta`` (layouts in include/psa.h).
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


# the dual-path network's fused, padded layout (include/psa.h): name -> (offset, rows,
# cols) of each padded block, and the trainable sub-blocks (rows, cols, fan_in)
DUAL_NPARAM = _native.DUAL_PARAMS
DUAL_BLOCKS = {}
_o = 0
for _name, _r, _c in (("WA", 256, IN), ("bA", 256, 1), ("WB", 128, 256), ("bB", 128, 1), ("W4", 128, 128),
                      ("b4", 128, 1), ("W5", 128, 128), ("b5", 128, 1), ("W7", 128, 128), ("b7", 128, 1),
                      ("w8", 128, 1), ("b8", 1, 1)):
    DUAL_BLOCKS[_name] = (_o, _r, _c)
    _o += _r * _c
assert _o == DUAL_NPARAM
#: (block, row slice, column slice, fan_in) of every trainable weight block
DUAL_WEIGHTS = (("WA", slice(0, 64), slice(0, 26), 26),       # W_c1: Fourier columns -> h_c1
                ("WA", slice(64, 192), slice(26, 61), 35),    # W_m1: feature columns -> h_m1
                ("WB", slice(0, 64), slice(0, 64), 64),       # W_c2
                ("WB", slice(64, 128), slice(64, 192), 128),  # W_m2
                ("W4", slice(0, 128), slice(0, 128), 128),
                ("W5", slice(0, 128), slice(0, 128), 128),
                ("W7", slice(0, 64), slice(0, 128), 128),
                ("w8", slice(0, 64), slice(0, 1), 64))
DUAL_BIASES = (("bA", slice(0, 192)), ("bB", slice(0, 128)), ("b4", slice(0, 128)), ("b5", slice(0, 128)),
               ("b7", slice(0, 64)), ("b8", slice(0, 1)))


def dual_block(theta_np: np.ndarray, name: str) -> np.ndarray:
    """View of one padded block of a dual-path parameter vector (numpy) as (rows, cols)."""
    o, r, c = DUAL_BLOCKS[name]
    return theta_np[o:o + r * c].reshape(r, c)


def dual_param_mask() -> np.ndarray:
    """1 at the trainable entries of the dual-path parameter vector, 0 at its structural zeros."""
    m = np.zeros(DUAL_NPARAM, dtype=np.float32)
    for name, rs, cs, _ in DUAL_WEIGHTS:
        dual_block(m, name)[rs, cs] = 1.0
    for name, rs in DUAL_BIASES:
        dual_block(m, name)[rs, 0] = 1.0
    return m


def nparam(net: str = "mlp") -> int:
    return NPARAM if net == "mlp" else DUAL_NPARAM


def init_theta(seed: int = 0, device="cuda", net: str = "mlp"):
    """Seeded initial parameters: weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)) as for a
    default linear layer, biases zero (the dual-path network's structural zeros stay 0)."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    if net == "mlp":
        th = np.zeros(NPARAM, dtype=np.float32)
        for name, fan_in in (("W1", IN), ("W2", HIDDEN), ("W3", HIDDEN), ("w4", HIDDEN)):
            o, n = OFF[name]
            th[o:o + n] = rng.uniform(-1.0, 1.0, n) / np.sqrt(fan_in)
    elif net == "dual":
        th = np.zeros(DUAL_NPARAM, dtype=np.float32)
        for name, rs, cs, fan_in in DUAL_WEIGHTS:
            blk = dual_block(th, name)
            shape = blk[rs, cs].shape
            blk[rs, cs] = rng.uniform(-1.0, 1.0, shape) / np.sqrt(fan_in)
    else:
        raise ValueError(f"unknown network {net!r}")
    return torch.as_tensor(th, device=device)


def _fn(net: str, what: str):
    lib = _native.load()
    if net not in ("mlp", "dual"):
        raise ValueError(f"unknown network {net!r}")
    return getattr(lib, f"psa_{net}_{what}")


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


def workspace_bytes(rows: int, training: bool, net: str = "mlp") -> int:
    out = ctypes.c_size_t()
    _native.check(_fn(net, "workspace_bytes")(int(rows), int(bool(training)), ctypes.byref(out)),
                  f"psa_{net}_workspace_bytes")
    return int(out.value)


def _aligned_buffer(nbytes: int, device):
    import torch
    buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    return buf, buf.data_ptr() + (-buf.data_ptr()) % 256


def forward(theta, x, out=None, workspace=None, stream=None, net: str = "mlp"):
    """Probabilities (float32, rows) of feature rows x (bfloat16, (rows, IN))."""
    import torch
    fwd = _fn(net, "forward")
    rows = int(x.shape[0])
    if x.dim() != 2 or x.shape[1] != IN:
        raise ValueError(f"x must have shape (rows, {IN})")
    if theta.dtype != torch.float32 or theta.numel() != nparam(net) or not theta.is_contiguous():
        raise ValueError("theta must be a contiguous float32 vector of the parameter count")
    prob = out if out is not None else torch.empty(rows, dtype=torch.float32, device=x.device)
    if prob.dtype != torch.float32 or not prob.is_contiguous() or prob.numel() < rows or prob.device != x.device:
        raise ValueError("out must be a contiguous float32 tensor of at least `rows` values on x's device")
    if workspace is None:
        nb = workspace_bytes(rows, False, net)
        buf, ptr = _aligned_buffer(nb, x.device)
    else:
        buf, ptr, nb = workspace
    s = stream if stream is not None else torch.cuda.current_stream(x.device)
    _native.check(fwd(theta.data_ptr(), _bf16_bits(x), rows, prob.data_ptr(), ptr, nb, s.cuda_stream),
                  f"psa_{net}_forward")
    return prob


class Trainer:
    """Adam on binary cross-entropy with fixed batch size ``batch`` (a multiple of
    128) for the network ``net``. ``step(x, y)`` takes one batch; no call allocates,
    so a step can be captured in a CUDA graph whose inputs are the trainer's own
    ``x`` and ``y`` buffers."""

    def __init__(self, theta, batch: int = 512, lr: float = 1e-3, net: str = "mlp"):
        import torch
        if batch % 128:
            raise ValueError("batch must be a multiple of 128")
        if theta.numel() != nparam(net):
            raise ValueError("theta does not match the network")
        self.net = net
        self.theta = theta
        self.batch = batch
        self.lr = lr
        dev = theta.device
        self.m = torch.zeros_like(theta)
        self.v = torch.zeros_like(theta)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        nb = workspace_bytes(batch, True, net)
        self._buf, self._ptr = _aligned_buffer(nb, dev)
        self._nb = nb
        self.t = 0
        self.x = torch.zeros((batch, IN), dtype=torch.bfloat16, device=dev)
        self.y = torch.zeros(batch, dtype=torch.float32, device=dev)

    def _launch(self, x, y, t: int, stream):
        step = _fn(self.net, "train_step")
        _native.check(step(self.theta.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), int(t), float(self.lr),
                           _bf16_bits(x), y.data_ptr(), self.batch, self.loss.data_ptr(), self._ptr, self._nb,
                           stream.cuda_stream), f"psa_{self.net}_train_step")

    def step(self, x, y, stream=None):
        """One Adam step on the batch (x bfloat16 (batch, IN), y float32 (batch,))."""
        import torch
        if x.shape != (self.batch, IN) or y.shape != (self.batch,):
            raise ValueError("batch shape")
        self.t += 1
        s = stream if stream is not None else torch.cuda.current_stream(self.theta.device)
        self._launch(x.contiguous(), y.contiguous(), self.t, s)
        return self.loss
