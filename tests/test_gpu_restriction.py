"""GPU learned restriction: feature kernels against NumPy references of the same
formulas, region and point-list kernels against NumPy, the hierarchical map
against the masked full map, and a small end-to-end run (train, calibrate,
restricted sigma_min equal bitwise to the full grid on the region)."""
import numpy as np
import pytest
import torch

import paper_2605_04550_gb300 as psa
from paper_2605_04550_gb300 import _native, inputs, mlp, restriction
import oracle
from oracle import features as FO

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.complex128, device=DEV)


def _dense(b, kl, ku):
    n = b.shape[1]
    A = np.zeros((n, n), dtype=np.complex128)
    for d in range(-kl, ku + 1):
        for i in range(n):
            if 0 <= i + d < n:
                A[i, i + d] = b[d + kl, i]
    return A


def test_matrix_stats_match_the_feature_oracle():
    b, kl, ku, a = inputs.random_toeplitz(150, 2, 5, seed=11)
    b = b + 0.01 * np.random.default_rng(0).standard_normal(b.shape)
    b = inputs._zero_outside(b.astype(np.complex128), 150, kl, ku)
    ctx = restriction.matrix_contexts([(_t(b), kl, ku)])[0]
    st = ctx.stats.cpu().numpy()
    ref, f = FO.matrix_stats(b, kl, ku)
    np.testing.assert_allclose(st, ref, rtol=1e-10, atol=1e-13 * np.abs(ref).max())
    np.testing.assert_allclose(ctx.symbol.cpu().numpy(), f, rtol=0, atol=1e-12 * np.abs(f).max())
    # global features from the library's statistics and the oracle's sigma_min probes
    cen = complex(ref[0], ref[1])
    s4, _, _ = oracle.sigma_min_banded(b, kl, ku, np.array([0.0, cen + 0.5, cen + 1.0, cen + 2.0]),
                                       k_max=300, tol=1e-6)
    g = ctx.glob.cpu().numpy()
    np.testing.assert_allclose(g, FO.global_features(ref, s4, restriction.EPS), rtol=2e-5, atol=2e-5)


def test_resolvent_probe_features_closed_form():
    """Hermitian tridiagonal Toeplitz A + shift: sigma_min(zI - A) = min_k |z - lambda_k|,
    lambda_k = a + 2|b| cos(k pi / (n + 1)); the global features take log10 of the
    probes at z = 0 and the centroid + 0.5, 1, 2."""
    n, a, bb = 90, 3.0 + 0.5j, 0.8 - 0.6j
    bands, kl, ku = inputs.hermitian_toeplitz_tridiag(n, 3.0, bb)
    bands = bands.copy()
    bands[kl] += 0.5j  # normal: a Hermitian matrix plus a multiple of I
    ctx = restriction.matrix_contexts([(_t(bands), kl, ku)])[0]
    st = ctx.stats.cpu().numpy()
    g = ctx.glob.cpu().numpy()
    lam = a + 2 * abs(bb) * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    s0 = np.abs(lam).min()
    A = _dense(bands, kl, ku)
    s1 = np.sqrt(np.abs(A).sum(0).max() * np.abs(A).sum(1).max())
    assert abs(g[11] - np.log10(s1 / s0 + 1e-12)) < 2e-5
    for k, dl in enumerate((0.5, 1.0, 2.0)):
        sk = np.abs(a + dl - lam).min()
        assert abs(g[20 + k] - np.log10(st[2] / sk)) < 2e-5


def test_point_features_match_the_feature_oracle():
    b, kl, ku = inputs.grcar(120)
    ctx = restriction.matrix_contexts([(_t(b), kl, ku)])[0]
    grid = inputs.Grid(-1.0, 3.0, -3.5, 3.5, 23, 17)
    x = restriction.point_features(ctx, grid).float().cpu().numpy()
    idx = torch.as_tensor(np.array([5, 77, 390], dtype=np.int32), device=DEV)
    xi = restriction.point_features(ctx, grid, idx).float().cpu().numpy()
    np.testing.assert_array_equal(xi, x[[5, 77, 390]])
    st = ctx.stats.cpu().numpy()
    sym = ctx.symbol.cpu().numpy()
    gl = ctx.glob.cpu().numpy().astype(np.float64)
    pts = np.arange(grid.npoints)
    ref = FO.point_features(grid, st, sym, gl, pts)
    # BF16 rows: 8 significant bits
    np.testing.assert_allclose(x, ref, rtol=1e-2, atol=2e-2)
    assert np.all(x[:, 33 + _native.GLOBAL_FEATURES:] == 0)


def test_region_and_tile_list_match_numpy():
    rng = np.random.default_rng(3)
    grid = inputs.Grid(0.0, 1.0, 0.0, 1.0, 37, 29)
    prob = rng.random((29, 37)).astype(np.float32) ** 6
    pt = torch.as_tensor(prob.ravel(), device=DEV)
    for tau, r in ((0.5, 2), (0.9, 1), (0.99, 0)):
        m = restriction.region_mask(pt, grid, tau, r).cpu().numpy().astype(bool)
        np.testing.assert_array_equal(m, restriction.dilate_np(prob >= tau, r))
        lst = restriction.region_list(torch.as_tensor(m.astype(np.uint8), device=DEV), grid).cpu().numpy()
        np.testing.assert_array_equal(lst, psa.tile_order(np.flatnonzero(m.ravel()), grid.nx))


def test_hierarchical_map_is_masked_full_map():
    b, kl, ku = inputs.grcar(100)
    ctx = restriction.matrix_contexts([(_t(b), kl, ku)])[0]
    r = restriction.Restriction(DEV, seed=1)
    grid = inputs.Grid(-1.0, 3.0, -3.5, 3.5, 42, 30)
    full = r.predict(ctx, grid, hierarchical=False)
    nc = r.coarse_near(ctx, grid)
    assert nc.any()  # the Grcar symbol curve crosses this grid
    for tau in (0.2, 0.5, 0.8):
        h = r.predict(ctx, grid, hierarchical=True, tau=tau)
        torch.testing.assert_close(h, restriction.Restriction.hierarchical_mask(full, tau, nc), rtol=0, atol=0)


def test_points_near_the_symbol_curve_enter_the_region():
    """A nearly normal band (kl = ku Grcar-type: A - I is skew-symmetric, plus 1e-3 noise)
    has a sensitive zone of width about 2 eps along its spectrum, the symbol segment:
    every sensitive point gets probability 1 from the near-curve rule, whatever the
    network says (an untrained network here)."""
    rng = np.random.default_rng(4)
    b = inputs.grcar_type(3000, 1, 1)
    b = b + 1e-3 * (rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape))
    grid = inputs.toeplitz_symbol_grid(np.array([-1.0, 1.0, 1.0], dtype=np.complex128), 1, 1, 97, 96, min_aspect=0.5)
    bt = _t(b)
    ctx = restriction.matrix_contexts([(bt, 1, 1)])[0]
    r = restriction.Restriction(DEV, seed=3)
    p = r.predict(ctx, grid, hierarchical=True, tau=0.5).cpu().numpy()
    sig = psa.sigma_min(bt, 1, 1, grid).sigma.cpu().numpy()
    sens = sig <= restriction.EPS
    assert sens.sum() >= 20 and np.all(p[sens] == 1.0)


def test_small_end_to_end_pipeline():
    rng = np.random.default_rng(0)
    tr = inputs.restriction_matrices(48, seed=5, n_min=150, n_max=400, nx=16, ny=16)
    va = inputs.restriction_matrices(6, seed=6, n_min=150, n_max=400, nx=48, ny=48)
    r = restriction.Restriction(DEV, seed=2)
    mats = [(_t(b), kl, ku) for b, kl, ku, _, _ in tr]
    x, y, _ = r.build_training_set(mats, [g for *_, g, _ in tr], rng)
    hist = r.train(x, y, rng, epochs=6, patience=3)
    assert hist[-1]["val_loss"] < hist[0]["val_loss"] * 1.5 and min(h["val_acc"] for h in hist) > 0.5
    vm = [(_t(b), kl, ku) for b, kl, ku, _, _ in va]
    vctx = restriction.matrix_contexts(vm)
    vg = [g for *_, g, _ in va]
    truth = []
    for (b, kl, ku), g in zip(vm, vg):
        truth.append(psa.sigma_min(b, kl, ku, g).sigma.cpu().numpy())
    cal = r.calibrate(vctx, vg, truth)
    assert 0.0 < cal["tau"] < 1.0
    # restricted run on a fresh matrix: sigma on R equals the full grid bitwise
    b, kl, ku, g = inputs.restriction_test_matrix(n=600, kl=2, ku=4, nx=64, ny=48, seed=9)
    bt = _t(b)
    ctx = restriction.matrix_contexts([(bt, kl, ku)])[0]
    full = psa.sigma_min(bt, kl, ku, g, eps=(restriction.EPS,))
    out, mask, idx, tm = r.restricted(ctx, g, (restriction.EPS,))
    m = mask.cpu().numpy().astype(bool).ravel()
    np.testing.assert_array_equal(out.sigma.cpu().numpy().ravel()[m], full.sigma.cpu().numpy().ravel()[m])
    assert np.all(out.status.cpu().numpy().ravel()[~m] == psa.PT_NOT_EVALUATED)
    # a network trained on 48 small matrices for a few epochs (the weights depend on the
    # order of atomic gradient sums) is only checked for doing better than chance here;
    # the recall bar is on the shipped classifier below
    met = restriction.recall_metrics(full.sigma.cpu().numpy() <= restriction.EPS, m.reshape(g.ny, g.nx))
    assert met["recall"] >= 0.5, met


@pytest.mark.parametrize("net", ["mlp", "dual"])
def test_shipped_classifier_reaches_recall_on_a_fresh_matrix(net):
    """The classifiers shipped with the package (the MLP and the paper's dual-path net,
    trained on the same labels of 2000 seeded matrices, thresholds calibrated above the
    grid minimum) on matrices outside their training set: recall against the
    3x3-dilated truth >= 0.99, sigma on the region bitwise equal to the full grid."""
    import os
    path = os.path.join(os.path.dirname(restriction.__file__), "data", f"restriction_{net}.npz")
    r = restriction.Restriction.load(path, DEV)
    assert r.net == net and r.tau > 0.01 and r.calibration["row"]["min_recall"] >= 0.99
    for n, kl, ku, nx, ny, seed in ((600, 2, 4, 64, 48, 9), (1500, 3, 6, 96, 80, 31)):
        b, kl, ku, g = inputs.restriction_test_matrix(n=n, kl=kl, ku=ku, nx=nx, ny=ny, seed=seed)
        bt = _t(b)
        ctx = restriction.matrix_contexts([(bt, kl, ku)])[0]
        full = psa.sigma_min(bt, kl, ku, g, eps=(restriction.EPS,))
        out, mask, idx, tm = r.restricted(ctx, g, (restriction.EPS,))
        m = mask.cpu().numpy().astype(bool)
        np.testing.assert_array_equal(out.sigma.cpu().numpy()[m], full.sigma.cpu().numpy()[m])
        met = restriction.recall_metrics(full.sigma.cpu().numpy() <= restriction.EPS, m)
        assert met["recall"] >= 0.99, (n, met)


def test_eigenvalue_features_match_the_feature_oracle():
    """The paper's own spectrum features (Sec. 3.1, Table "matrix"; Eq. (dist)) over the
    eigenvalues: statistics, global features and point rows against the oracle."""
    b, kl, ku, a = inputs.random_toeplitz(150, 2, 5, seed=11)
    b = b + 0.01 * np.random.default_rng(0).standard_normal(b.shape)
    b = inputs._zero_outside(b.astype(np.complex128), 150, kl, ku)
    lam = np.linalg.eigvals(_dense(b, kl, ku))
    ctx = restriction.matrix_contexts([(_t(b), kl, ku)], spectra=[lam])[0]
    st0, _ = FO.matrix_stats(b, kl, ku)
    ref = FO.point_set_stats(st0, lam)
    st = ctx.stats.cpu().numpy()
    np.testing.assert_allclose(st, ref, rtol=1e-10, atol=1e-13 * np.abs(ref).max())
    cen = complex(ref[0], ref[1])
    s4, _, _ = oracle.sigma_min_banded(b, kl, ku, np.array([0.0, cen + 0.5, cen + 1.0, cen + 2.0]),
                                       k_max=300, tol=1e-6)
    gl = ctx.glob.cpu().numpy()
    np.testing.assert_allclose(gl, FO.global_features(ref, s4, restriction.EPS), rtol=2e-5, atol=2e-5)
    grid = inputs.toeplitz_symbol_grid(a, kl, ku, 23, 17)
    x = restriction.point_features(ctx, grid).float().cpu().numpy()
    xr = FO.point_features(grid, st, lam, gl.astype(np.float64), np.arange(grid.npoints), closed=False)
    np.testing.assert_allclose(x, xr, rtol=1e-2, atol=2e-2)
    assert np.all(x[:, 31] == 0)


@pytest.mark.parametrize("closed", [0, 1])
def test_point_features_over_a_set_of_several_chunks(closed):
    """A set of 5000 points passes through shared memory in chunks of 2048 (two full
    chunks and a ragged one); the closed polyline joins the chunks and wraps around."""
    import ctypes
    lib = _native.load()
    rng = np.random.default_rng(8)
    b, kl, ku = inputs.grcar(120)
    ctx = restriction.matrix_contexts([(_t(b), kl, ku)])[0]
    pts = np.exp(2j * np.pi * np.sort(rng.random(5000))) * (1.0 + 0.3 * rng.random(5000)) + 1.0
    grid = inputs.Grid(-1.0, 3.0, -2.0, 2.0, 31, 29)
    sel = np.sort(rng.choice(grid.npoints, 60, replace=False)).astype(np.int32)
    idx = torch.as_tensor(sel, device=DEV)
    dp = _t(pts)
    x = torch.empty((sel.size, mlp.IN), dtype=torch.bfloat16, device=DEV)
    g = restriction._grid_c(grid)
    _native.check(lib.psa_point_features_set(ctypes.byref(g), idx.data_ptr(), sel.size, ctx.stats.data_ptr(),
                                             dp.data_ptr(), pts.size, closed, ctx.glob.data_ptr(), x.data_ptr(),
                                             torch.cuda.current_stream().cuda_stream), "psa_point_features_set")
    xr = FO.point_features(grid, ctx.stats.cpu().numpy(), pts, ctx.glob.cpu().numpy().astype(np.float64), sel,
                           closed=bool(closed))
    np.testing.assert_allclose(x.float().cpu().numpy(), xr, rtol=1e-2, atol=2e-2)
    if closed:
        np.testing.assert_array_equal(x.float().cpu().numpy()[:, 31], xr[:, 31])


def test_classifier_on_eigenvalue_features_trains_and_predicts():
    rng = np.random.default_rng(0)
    tr = inputs.restriction_matrices(24, seed=5, n_min=150, n_max=300, nx=16, ny=16)
    mats = [(_t(b), kl, ku) for b, kl, ku, _, _ in tr]
    spectra = [np.linalg.eigvals(_dense(b, kl, ku)) for b, kl, ku, _, _ in tr]
    grids = [g for *_, g, _ in tr]
    sym = restriction.Restriction(DEV, seed=2, net="dual")
    x0, y0, _ = sym.build_training_set(mats, grids, np.random.default_rng(1))
    eig = restriction.Restriction(DEV, seed=2, net="dual", features="eigen")
    x1, y1, ctxs = eig.build_training_set(mats, grids, np.random.default_rng(1), spectra=spectra,
                                          labels=sym.last_labels)
    # the same labels and the same drawn points; the Fourier columns agree, the spectrum ones not
    assert torch.equal(y0, y1)
    assert torch.equal(x0[:, :26], x1[:, :26]) and not torch.equal(x0[:, 26:61], x1[:, 26:61])
    hist = eig.train(x1, y1, rng, epochs=4, patience=2)
    assert np.isfinite(hist[-1]["val_loss"])
    p = eig.predict(ctxs[0], grids[0]).cpu().numpy()
    assert p.shape == (grids[0].ny, grids[0].nx) and np.all((p >= 0) & (p <= 1))
    with pytest.raises(ValueError):
        sym.predict(ctxs[0], grids[0])  # a symbol-feature classifier refuses eigenvalue contexts
