"""GPU classifier kernels (tensor-core GEMM, MLP forward, Adam training step)
against plain PyTorch FP32 references of the same operations.

Bars: the GEMM equals the FP32 product of the same BF16 operands to 1e-5
relative (only the summation order differs); the forward pass matches a
reference that rounds the hidden activations to BF16 as the kernels do (1e-3 in
probability); the first Adam step's gradient (recovered from the first moment,
m_1 = 0.1 g) matches autograd of that reference to 2 % in norm per layer; a few
hundred steps learn a separable problem.
"""
import numpy as np
import pytest
import torch

from paper_2605_04550_gb300 import mlp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _ref_forward(theta, x, keep=False):
    """FP32 reference with the kernels' BF16 rounding of every hidden activation."""
    th = theta.float()

    def blk(name, shape):
        o, n = mlp.OFF[name]
        return th[o:o + n].view(*shape)

    W1, b1 = blk("W1", (mlp.HIDDEN, mlp.IN)), blk("b1", (mlp.HIDDEN,))
    W2, b2 = blk("W2", (mlp.HIDDEN, mlp.HIDDEN)), blk("b2", (mlp.HIDDEN,))
    W3, b3 = blk("W3", (mlp.HIDDEN, mlp.HIDDEN)), blk("b3", (mlp.HIDDEN,))
    w4, b4 = blk("w4", (mlp.HIDDEN,)), blk("b4", (1,))
    bf = lambda t: t.to(torch.bfloat16).float()
    h = x.float()
    for W, b in ((W1, b1), (W2, b2), (W3, b3)):
        h = bf(torch.nn.functional.silu(h @ bf(W).T + b))
    return h @ w4 + b4


def test_gemm_matches_fp32_product():
    g = torch.Generator(device=DEV).manual_seed(0)
    for M, N, K in ((300, 256, 192), (128, 128, 64), (1, 384, 128), (1000, 128, 512)):
        A = torch.randn(M, K, device=DEV, generator=g).to(torch.bfloat16)
        B = torch.randn(N, K, device=DEV, generator=g).to(torch.bfloat16)
        C = mlp.gemm_bf16(A, B)
        torch.cuda.synchronize()
        ref = A.double() @ B.double().T
        err = (C.double() - ref).abs().max().item()
        assert err <= 1e-5 * ref.abs().max().item(), (M, N, K, err)


def test_gemm_strided_operands():
    g = torch.Generator(device=DEV).manual_seed(1)
    big = torch.randn(200, 320, device=DEV, generator=g).to(torch.bfloat16)
    A = big[:, 64:256]           # lda = 320
    B = torch.randn(128, 192, device=DEV, generator=g).to(torch.bfloat16)
    lib = mlp._native.load()
    C = torch.empty(200, 128, dtype=torch.float32, device=DEV)
    rc = lib.psa_gemm_bf16(A.data_ptr(), 320, B.data_ptr(), 192, 200, 128, 192, C.data_ptr(), 128,
                           torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    ref = A.double() @ B.double().T
    assert (C.double() - ref).abs().max().item() <= 1e-5 * ref.abs().max().item()


@pytest.mark.parametrize("rows", [1, 130, 1000])
def test_forward_matches_reference(rows):
    theta = mlp.init_theta(3, DEV)
    theta[mlp.OFF["b1"][0]:mlp.OFF["b1"][0] + 256] = 0.1
    g = torch.Generator(device=DEV).manual_seed(2)
    x = torch.randn(rows, mlp.IN, device=DEV, generator=g).to(torch.bfloat16)
    p = mlp.forward(theta, x)
    torch.cuda.synchronize()
    ref = torch.sigmoid(_ref_forward(theta, x))
    assert (p - ref).abs().max().item() <= 1e-3


def test_first_adam_step_gradient_matches_autograd():
    theta = mlp.init_theta(5, DEV)
    g = torch.Generator(device=DEV).manual_seed(4)
    B = 256
    x = torch.randn(B, mlp.IN, device=DEV, generator=g).to(torch.bfloat16)
    y = (torch.rand(B, device=DEV, generator=g) < 0.3).float()
    th_ref = theta.clone().requires_grad_(True)
    logit = _ref_forward(th_ref, x)
    loss_ref = torch.nn.functional.binary_cross_entropy_with_logits(logit, y)
    loss_ref.backward()
    tr = mlp.Trainer(theta, batch=B, lr=1e-3)
    loss = tr.step(x, y)
    torch.cuda.synchronize()
    assert abs(loss.item() - loss_ref.item()) <= 1e-3 * abs(loss_ref.item())
    grad = tr.m / 0.1  # first moment after one step from zero: (1 - beta1) g
    for name, (o, n) in mlp.OFF.items():
        gr = th_ref.grad[o:o + n]
        gk = grad[o:o + n]
        rel = (gk - gr).norm().item() / max(gr.norm().item(), 1e-30)
        assert rel <= 2e-2, (name, rel)


def test_training_learns_a_disk():
    """Label = inside a disk of the first two features; a few hundred Adam steps
    reach 97 % accuracy on fresh points."""
    theta = mlp.init_theta(7, DEV)
    tr = mlp.Trainer(theta, batch=512, lr=2e-3)
    g = torch.Generator(device=DEV).manual_seed(6)

    def batch(n):
        x = torch.zeros(n, mlp.IN, device=DEV)
        x[:, :2] = torch.rand(n, 2, device=DEV, generator=g) * 2 - 1
        y = ((x[:, 0] ** 2 + x[:, 1] ** 2) < 0.4).float()
        return x.to(torch.bfloat16), y

    for _ in range(400):
        x, y = batch(512)
        tr.step(x, y)
    x, y = batch(8192)
    p = mlp.forward(theta, x)
    torch.cuda.synchronize()
    acc = ((p > 0.5).float() == y).float().mean().item()
    assert acc >= 0.97, acc


def test_no_gemm_tile_timed_out():
    # every GEMM of this module's tests completed its bounded waits, and the counter
    # reads back as zero after a check
    A = torch.randn(300, 128, device=DEV).to(torch.bfloat16)
    B = torch.randn(256, 128, device=DEV).to(torch.bfloat16)
    mlp.gemm_bf16(A, B)
    mlp.check_timeouts()
    mlp.check_timeouts()
