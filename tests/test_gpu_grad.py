"""GPU adjoint gradients (psa_sigma_min_grad through the C ABI) against the oracle.

Bars: d sigma / dz and the weighted band gradient match the oracle's dense-SVD
gradient (first-order perturbation of a simple singular value) to 1e-7 relative;
at the differentiation workload's size (Grcar-type n = 4000) d sigma / dz matches
central finite differences (h = 1e-6) of the GPU's own sigma to 1e-7 relative; the
autograd wrapper follows PyTorch's complex-gradient convention; Newton refinement
puts every eps-contour crossing on the level set.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2605_04550_gb300 as psa
from paper_2605_04550_gb300 import contour, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TIGHT = psa.LanczosOpts(tol=1e-15, k_max=4000)


def _t(a, dtype=torch.complex128):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _cases():
    b1, kl1, ku1 = inputs.grcar(100)
    b2, kl2, ku2, _ = inputs.random_toeplitz(120, 2, 5, seed=3)
    b3, kl3, ku3, _ = inputs.paper_class(4)
    rng = np.random.default_rng(0)
    return [(b1, kl1, ku1, rng.uniform(-1, 3, 24) + 1j * rng.uniform(-3.5, 3.5, 24)),
            (b2, kl2, ku2, rng.uniform(-12, 12, 24) + 1j * rng.uniform(-12, 12, 24)),
            (b3, kl3, ku3, rng.uniform(-4, 4, 24) + 1j * rng.uniform(-4, 4, 24))]


@pytest.mark.parametrize("ci", [0, 1, 2])
def test_grad_z_and_sigma_match_dense_oracle(ci):
    b, kl, ku, z = _cases()[ci]
    A = oracle.band_to_dense(b, kl, ku)
    r = psa.sigma_min_grad(_t(b), kl, ku, _t(z), opts=TIGHT)
    torch.cuda.synchronize()
    sig = r.sigma.cpu().numpy()
    gz = r.grad_z.cpu().numpy()
    st = r.status.cpu().numpy()
    for p, zz in enumerate(z):
        s_ref, g_ref, _ = oracle.sigma_min_grad_dense(A, zz)
        if s_ref < 1e-8 * np.abs(A).sum(0).max():
            continue  # below the roundoff floor the singular vectors are not determined
        assert st[p] == psa.PT_OK
        assert abs(sig[p] - s_ref) <= 1e-10 * s_ref, (p, sig[p], s_ref)
        assert abs(gz[p] - g_ref) <= 1e-7 * abs(g_ref) + 1e-12, (p, gz[p], g_ref)


def test_weighted_band_gradient_matches_dense_oracle():
    b, kl, ku, _ = inputs.random_toeplitz(60, 2, 5, seed=9)
    A = oracle.band_to_dense(b, kl, ku)
    rng = np.random.default_rng(1)
    cand = rng.uniform(-14, 14, 200) + 1j * rng.uniform(-14, 14, 200)
    # points whose smallest singular value is resolvable and simple (its singular
    # vectors are then determined up to a common phase)
    keep = []
    for zz in cand:
        sv = np.linalg.svd(zz * np.eye(60) - A, compute_uv=False)
        if sv[-1] > 1e-2 and (sv[-2] - sv[-1]) > 1e-3 * sv[-1]:
            keep.append(zz)
    z = np.array(keep[:40])
    assert z.size >= 20
    w = rng.standard_normal(z.size)
    r = psa.sigma_min_grad(_t(b), kl, ku, _t(z), weight=_t(w, torch.float64), opts=TIGHT)
    torch.cuda.synchronize()
    ref = np.zeros_like(b)
    for p, zz in enumerate(z):
        _, _, gA = oracle.sigma_min_grad_dense(A, zz)
        ref += w[p] * oracle.dense_grad_to_bands(gA, kl, ku)
    got = r.grad_bands.cpu().numpy()
    scale = np.abs(ref).max()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-7 * scale)


def test_grad_z_matches_central_differences_at_full_size():
    """Differentiation workload size: Grcar-type n = 4000 with N(0, 1e-2) band noise."""
    b, kl, ku = inputs.grcar_perturbed(4000, seed=0)
    bt = _t(b)
    rng = np.random.default_rng(2)
    # outside the curve, where sigma_min of the n = 4000 matrix is resolvable
    z = np.concatenate([rng.uniform(-1.0, 3.0, 4) + 1j * rng.uniform(3.3, 4.0, 4),
                        rng.uniform(3.1, 3.8, 4) + 1j * rng.uniform(-2.0, 2.0, 4)])
    h = 1e-6
    zs = np.concatenate([z, z + h, z - h, z + 1j * h, z - 1j * h])
    r = psa.sigma_min_grad(bt, kl, ku, _t(zs), opts=TIGHT)
    torch.cuda.synchronize()
    s = r.sigma.cpu().numpy().reshape(5, -1)
    gz = r.grad_z.cpu().numpy()[:8]
    fd = (s[1] - s[2]) / (2 * h) + 1j * (s[3] - s[4]) / (2 * h)
    ok = s[0] > 1e-6  # well above the floor: a simple, resolvable sigma_min
    assert ok.sum() >= 4
    err = np.abs(gz - fd)[ok] / np.abs(fd)[ok]
    assert err.max() <= 1e-7, (err, s[0])


def test_grad_matches_dense_oracle_at_full_size():
    """Differentiation workload size (Grcar-type n = 4000 with N(0, 1e-2) band noise):
    sigma, d sigma / dz and the whole band gradient of one point against the singular
    pair of the oracle's dense SVD, at 4 resolvable points outside the curve."""
    b, kl, ku = inputs.grcar_perturbed(4000, seed=0)
    A = oracle.band_to_dense(b, kl, ku)
    rng = np.random.default_rng(3)
    z = np.concatenate([rng.uniform(-0.5, 2.5, 2) + 1j * rng.uniform(3.4, 3.9, 2),
                        rng.uniform(3.2, 3.7, 2) + 1j * rng.uniform(-1.5, 1.5, 2)])
    w = np.zeros(z.size)
    w[0] = 1.0  # the band gradient of the first point alone
    r = psa.sigma_min_grad(_t(b), kl, ku, _t(z), weight=_t(w, torch.float64), opts=TIGHT)
    torch.cuda.synchronize()
    sig, gz, st = r.sigma.cpu().numpy(), r.grad_z.cpu().numpy(), r.status.cpu().numpy()
    assert np.all(st == psa.PT_OK)
    for p, zz in enumerate(z):
        s_ref, g_ref, gA = oracle.sigma_min_grad_dense(A, zz)
        assert s_ref > 1e-6, s_ref  # resolvable: far above the roundoff floor
        assert abs(sig[p] - s_ref) <= 1e-10 * s_ref, (p, sig[p], s_ref)
        assert abs(gz[p] - g_ref) <= 1e-7 * abs(g_ref), (p, gz[p], g_ref)
        if p == 0:
            ref = oracle.dense_grad_to_bands(gA, kl, ku)
            np.testing.assert_allclose(r.grad_bands.cpu().numpy(), ref, rtol=0, atol=1e-7 * np.abs(ref).max())


def test_sigma_of_grad_kernel_equals_grid_kernel():
    b, kl, ku = inputs.grcar(100)
    grid = inputs.Grid(-1.0, 3.0, -3.5, 3.5, 20, 12)
    out = psa.sigma_min(_t(b), kl, ku, grid)
    z = oracle.grid_points(grid).ravel()
    r = psa.sigma_min_grad(_t(b), kl, ku, _t(z))
    torch.cuda.synchronize()
    # same factorisation and Lanczos arithmetic per point
    np.testing.assert_array_equal(r.sigma.cpu().numpy(), out.sigma.cpu().numpy().ravel())


def test_autograd_function_complex_convention():
    b, kl, ku, _ = inputs.random_toeplitz(50, 1, 3, seed=4)
    A = oracle.band_to_dense(b, kl, ku)
    rng = np.random.default_rng(5)
    z = rng.uniform(-6, 6, 10) + 1j * rng.uniform(-6, 6, 10)
    w = rng.standard_normal(10)
    bt = _t(b).requires_grad_(True)
    zt = _t(z).requires_grad_(True)
    sig = psa.sigma_min_autograd(bt, zt, kl, ku, TIGHT)
    (sig * _t(w, torch.float64)).sum().backward()
    gb_ref = np.zeros_like(b)
    gz_ref = np.zeros(10, dtype=np.complex128)
    for p, zz in enumerate(z):
        _, gz, gA = oracle.sigma_min_grad_dense(A, zz)
        gb_ref += w[p] * oracle.dense_grad_to_bands(gA, kl, ku)
        gz_ref[p] = w[p] * gz
    np.testing.assert_allclose(bt.grad.cpu().numpy(), gb_ref, rtol=0, atol=1e-7 * np.abs(gb_ref).max())
    np.testing.assert_allclose(zt.grad.cpu().numpy(), gz_ref, rtol=0, atol=1e-7 * np.abs(gz_ref).max())


def test_newton_refinement_lands_on_the_contour():
    b, kl, ku = inputs.grcar(100)
    bt = _t(b)
    grid = inputs.Grid(-1.0, 3.0, -3.5, 3.5, 64, 48)
    eps = 1e-4
    out = psa.sigma_min(bt, kl, ku, grid, eps=(eps,))
    torch.cuda.synchronize()
    sig = out.sigma.cpu().numpy()
    ref = contour.refine_rows(bt, kl, ku, grid, sig, eps)
    assert ref.x.size > 10
    assert ref.converged.all(), ref.residual.max()
    # each refined point lies in its bracket and on the level set (checked by the oracle)
    hx = (grid.re_max - grid.re_min) / (grid.nx - 1)
    assert np.all(ref.x >= grid.re_min + ref.col * hx - 1e-12)
    assert np.all(ref.x <= grid.re_min + (ref.col + 1) * hx + 1e-12)
    s_or, _, _ = oracle.sigma_min_banded(b, kl, ku, ref.x[:12] + 1j * ref.y[:12])
    assert np.all(np.abs(s_or - eps) <= 1e-9 * eps)


def test_singular_pairs_and_band_gradient_from_them():
    """psa_sigma_min_pairs writes a singular pair (B v = sigma u, unit vectors, the phases
    of grad_z = conj(u^* v)); the band gradient contracted from stored pairs equals the
    adjoint kernel's weighted band gradient; a reusable workspace gives the same bits."""
    b, kl, ku, _ = inputs.random_toeplitz(70, 2, 4, seed=6)
    A = oracle.band_to_dense(b, kl, ku)
    rng = np.random.default_rng(8)
    z = rng.uniform(-12, 12, 40) + 1j * rng.uniform(-12, 12, 40)
    w = rng.standard_normal(40)
    bt, zt, wt = _t(b), _t(z), _t(w, torch.float64)
    ws = psa.GradWorkspace(70, kl, ku, 64, TIGHT, device=DEV)
    r = psa.sigma_min_grad(bt, kl, ku, zt, opts=TIGHT, pairs=True, workspace=ws)
    g1 = psa.sigma_min_grad(bt, kl, ku, zt, weight=wt, opts=TIGHT, workspace=ws)
    g2 = psa.sigma_min_grad(bt, kl, ku, zt, weight=wt, opts=TIGHT)
    gb = psa.band_grad_from_pairs(70, kl, ku, r.u, r.v, wt)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(g1.sigma.cpu().numpy(), g2.sigma.cpu().numpy())
    np.testing.assert_array_equal(r.sigma.cpu().numpy(), g1.sigma.cpu().numpy())
    u, v, s = r.u.cpu().numpy(), r.v.cpu().numpy(), r.sigma.cpu().numpy()
    for p in range(40):
        B = z[p] * np.eye(70) - A
        assert abs(np.linalg.norm(u[:, p]) - 1) < 1e-12 and abs(np.linalg.norm(v[:, p]) - 1) < 1e-12
        assert np.linalg.norm(B @ v[:, p] - s[p] * u[:, p]) <= 1e-9 * np.abs(B).sum(0).max()
        assert abs(np.conj(np.vdot(u[:, p], v[:, p])) - r.grad_z.cpu().numpy()[p]) <= 1e-12
    ref = g1.grad_bands.cpu().numpy()
    np.testing.assert_allclose(gb.cpu().numpy(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_autograd_falls_back_to_the_adjoint_kernel_without_room_for_pairs(monkeypatch):
    b, kl, ku, _ = inputs.random_toeplitz(50, 1, 3, seed=4)
    rng = np.random.default_rng(5)
    z = rng.uniform(-6, 6, 10) + 1j * rng.uniform(-6, 6, 10)
    w = rng.standard_normal(10)
    grads = []
    for budget in (psa.PAIR_BUDGET, 0):
        monkeypatch.setattr(psa, "PAIR_BUDGET", budget)
        bt = _t(b).requires_grad_(True)
        zt = _t(z).requires_grad_(True)
        (psa.sigma_min_autograd(bt, zt, kl, ku, TIGHT) * _t(w, torch.float64)).sum().backward()
        grads.append((bt.grad.cpu().numpy(), zt.grad.cpu().numpy()))
    np.testing.assert_array_equal(grads[0][1], grads[1][1])
    np.testing.assert_allclose(grads[0][0], grads[1][0], rtol=0, atol=1e-12 * np.abs(grads[1][0]).max())


def test_contour_kernels_match_the_bracketed_newton_rule():
    """psa_contour_init / psa_contour_step against the rule written out in NumPy: the
    first iterate interpolates log sigma within [0.05, 0.95] of the bracket; a step keeps
    the end whose sign f has, takes the Newton step when it stays inside, else bisects."""
    import ctypes
    from paper_2605_04550_gb300 import _native
    lib = _native.load()
    rng = np.random.default_rng(3)
    grid = inputs.Grid(-1.0, 3.0, -3.5, 3.5, 50, 40)
    m = 300
    rows = rng.integers(0, grid.ny, m).astype(np.int32)
    cols = rng.integers(0, grid.nx - 1, m).astype(np.int32)
    eps = 1e-4
    s_lo = 10.0 ** rng.uniform(-6, -2, m)
    s_hi = np.where(s_lo <= eps, 10.0 ** rng.uniform(-4, -2, m), 10.0 ** rng.uniform(-7, -4, m))
    s_lo[:5] = 0.0  # log of zero: the midpoint
    T = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=DEV)
    x, lo, hi, y, resid = (torch.empty(m, dtype=torch.float64, device=DEV) for _ in range(5))
    flo, done = (torch.empty(m, dtype=torch.uint8, device=DEV) for _ in range(2))
    z = torch.empty(m, dtype=torch.complex128, device=DEV)
    g = _native.PsaGrid(grid.re_min, grid.re_max, grid.im_min, grid.im_max, grid.nx, grid.ny)
    ptrs = [t.data_ptr() for t in (x, lo, hi, y, flo, done, resid, z)]
    r_t, c_t, sl_t, sh_t = T(rows, torch.int32), T(cols, torch.int32), T(s_lo), T(s_hi)
    assert lib.psa_contour_init(m, r_t.data_ptr(), c_t.data_ptr(), ctypes.byref(g), sl_t.data_ptr(),
                                sh_t.data_ptr(), eps, *ptrs, None) == 0
    hx, hy = 4.0 / 49, 7.0 / 39
    a, b = grid.re_min + cols * hx, grid.re_min + (cols + 1) * hx
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (np.log(eps) - np.log(np.maximum(s_lo, 1e-300))) / (np.log(np.maximum(s_hi, 1e-300)) -
                                                                np.log(np.maximum(s_lo, 1e-300)))
    t = np.where(np.isfinite(t), np.clip(t, 0.05, 0.95), 0.5)
    torch.cuda.synchronize()
    np.testing.assert_allclose(lo.cpu().numpy(), a, rtol=0, atol=1e-15)
    np.testing.assert_allclose(y.cpu().numpy(), grid.im_min + rows * hy, rtol=0, atol=1e-15)
    np.testing.assert_allclose(x.cpu().numpy(), a + t * (b - a), rtol=0, atol=1e-13)
    np.testing.assert_array_equal(flo.cpu().numpy(), (s_lo <= eps).astype(np.uint8))
    # one step for every other crossing
    act = np.arange(0, m, 2, dtype=np.int32)
    x0, lo0, hi0 = x.cpu().numpy(), lo.cpu().numpy(), hi.cpu().numpy()
    sig = eps * (1 + rng.uniform(-0.5, 0.5, act.size))
    sig[:3] = eps * (1 + 1e-14)  # converged
    slope = rng.uniform(-2e-3, 2e-3, act.size) + 1j * rng.standard_normal(act.size)
    a_t, s_t, g_t = T(act, torch.int32), T(sig), T(slope, torch.complex128)
    assert lib.psa_contour_step(act.size, a_t.data_ptr(), s_t.data_ptr(), g_t.data_ptr(), eps, 1e-12,
                                *ptrs, None) == 0
    torch.cuda.synchronize()
    f = sig - eps
    same = (f <= 0) == (s_lo[act] <= eps)
    l = np.where(same, x0[act], lo0[act])
    h = np.where(same, hi0[act], x0[act])
    with np.errstate(divide="ignore", invalid="ignore"):
        xn = x0[act] - f / slope.real
    xn = np.where(np.isfinite(xn) & (xn > l) & (xn < h), xn, 0.5 * (l + h))
    conv = np.abs(f) / eps <= 1e-12
    np.testing.assert_array_equal(lo.cpu().numpy()[act], l)
    np.testing.assert_array_equal(hi.cpu().numpy()[act], h)
    np.testing.assert_array_equal(x.cpu().numpy()[act], np.where(conv, x0[act], xn))
    np.testing.assert_array_equal(done.cpu().numpy()[act], (conv | (h - l <= 4e-16 * np.maximum(np.abs(l), 1))))
    np.testing.assert_array_equal(x.cpu().numpy()[1::2], x0[1::2])  # crossings not in the list keep their state
    np.testing.assert_array_equal(z.cpu().numpy()[act].real, x.cpu().numpy()[act])
