"""The paper's dual-path classifier (Sec. 3.2.2) on the tensor cores (psa_dual_*
through the C ABI) against a plain PyTorch FP32 reference that evaluates the two
pathways SEPARATELY, as the paper writes them (so the fused, block-structured
GEMMs of the kernels are checked against the architecture itself).

Bars as for the MLP: forward to 1e-3 in probability against a reference that
rounds every hidden activation to BF16 as the kernels do; the first Adam step's
gradient (from the first moment, m_1 = 0.1 g) to 2 % in norm per weight block;
structural zeros stay zero; a few hundred steps learn a separable problem.
"""
import numpy as np
import pytest
import torch

from paper_2605_04550_gb300 import mlp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _blocks(theta):
    """The paper's named weights as views of the fused parameter vector."""
    def blk(name):
        o, r, c = mlp.DUAL_BLOCKS[name]
        return theta[o:o + r * c].view(r, c)
    WA, bA, WB, bB = blk("WA"), blk("bA")[:, 0], blk("WB"), blk("bB")[:, 0]
    return {"Wc1": WA[0:64, 0:26], "bc1": bA[0:64], "Wm1": WA[64:192, 26:61], "bm1": bA[64:192],
            "Wc2": WB[0:64, 0:64], "bc2": bB[0:64], "Wm2": WB[64:128, 64:192], "bm2": bB[64:128],
            "W4": blk("W4"), "b4": blk("b4")[:, 0], "W5": blk("W5"), "b5": blk("b5")[:, 0],
            "W7": blk("W7")[0:64], "b7": blk("b7")[0:64, 0], "w8": blk("w8")[0:64, 0], "b8": blk("b8")[0, 0]}


def _ref_forward(theta, x):
    p = _blocks(theta.float())
    bf = lambda t: t.to(torch.bfloat16).float()
    silu = torch.nn.functional.silu
    lin = lambda h, W, b: h @ bf(W).T + b
    x = x.float()
    phi, f = x[:, 0:26], x[:, 26:61]
    hc = bf(silu(lin(bf(silu(lin(phi, p["Wc1"], p["bc1"]))), p["Wc2"], p["bc2"])))
    hm = bf(silu(lin(bf(silu(lin(f, p["Wm1"], p["bm1"]))), p["Wm2"], p["bm2"])))
    h3 = torch.cat([hc, hm], dim=1)
    h4 = bf(silu(lin(h3, p["W4"], p["b4"])))
    h6 = bf(silu(lin(h4, p["W5"], p["b5"])) + h4)
    h7 = bf(silu(lin(h6, p["W7"], p["b7"])))
    return h7 @ p["w8"] + p["b8"]


def _theta(seed):
    th = mlp.init_theta(seed, DEV, "dual")
    mask = torch.as_tensor(mlp.dual_param_mask(), device=DEV)
    g = torch.Generator(device=DEV).manual_seed(seed + 100)
    # nonzero biases, so that every bias enters the check
    th += 0.05 * torch.randn(th.numel(), device=DEV, generator=g) * mask * (th == 0)
    return th, mask


def test_parameter_count_matches_the_architecture():
    m = mlp.dual_param_mask()
    # 26*64+64 + 64*64+64 + 35*128+128 + 128*64+64 + 2*(128*128+128) + 128*64+64 + 64+1
    assert int(m.sum()) == mlp._native.DUAL_TRAINABLE == 60097


@pytest.mark.parametrize("rows", [1, 130, 1000])
def test_forward_matches_two_pathway_reference(rows):
    theta, _ = _theta(3)
    g = torch.Generator(device=DEV).manual_seed(2)
    x = torch.randn(rows, mlp.IN, device=DEV, generator=g).to(torch.bfloat16)
    p = mlp.forward(theta, x, net="dual")
    torch.cuda.synchronize()
    ref = torch.sigmoid(_ref_forward(theta, x))
    assert (p - ref).abs().max().item() <= 1e-3


def test_columns_past_the_features_are_ignored():
    theta, _ = _theta(4)
    g = torch.Generator(device=DEV).manual_seed(3)
    x = torch.randn(300, mlp.IN, device=DEV, generator=g)
    x2 = x.clone()
    x2[:, 61:] = 7.0
    p1 = mlp.forward(theta, x.to(torch.bfloat16), net="dual")
    p2 = mlp.forward(theta, x2.to(torch.bfloat16), net="dual")
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)


def test_first_adam_step_gradient_matches_autograd():
    theta, mask = _theta(5)
    g = torch.Generator(device=DEV).manual_seed(4)
    B = 256
    x = torch.randn(B, mlp.IN, device=DEV, generator=g).to(torch.bfloat16)
    y = (torch.rand(B, device=DEV, generator=g) < 0.3).float()
    th_ref = theta.clone().requires_grad_(True)
    loss_ref = torch.nn.functional.binary_cross_entropy_with_logits(_ref_forward(th_ref, x), y)
    loss_ref.backward()
    tr = mlp.Trainer(theta, batch=B, lr=1e-3, net="dual")
    loss = tr.step(x, y)
    torch.cuda.synchronize()
    assert abs(loss.item() - loss_ref.item()) <= 1e-3 * abs(loss_ref.item())
    grad = tr.m / 0.1  # first moment after one step from zero: (1 - beta1) g
    gk, gr = _blocks(grad), _blocks(th_ref.grad)
    for name in gk:
        rel = (gk[name] - gr[name]).norm().item() / max(gr[name].norm().item(), 1e-30)
        assert rel <= 2e-2, (name, rel)
    # structural zeros: no gradient, no moment, no update
    assert torch.all(tr.m[mask == 0] == 0) and torch.all(theta[mask == 0] == 0)


def test_training_learns_a_disk_through_the_coordinate_pathway():
    """Label = inside a disk of the first two feature columns (the coordinate pathway's
    inputs); a few hundred Adam steps reach 97 % accuracy on fresh points."""
    theta, mask = _theta(7)
    tr = mlp.Trainer(theta, batch=512, lr=2e-3, net="dual")
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
    p = mlp.forward(theta, x, net="dual")
    torch.cuda.synchronize()
    acc = ((p > 0.5).float() == y).float().mean().item()
    assert acc >= 0.97, acc
    assert torch.all(theta[mask == 0] == 0)
    mlp.check_timeouts()
