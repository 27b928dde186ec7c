"""GPU batches (psa_sigma_min_batched through the C ABI).

Bars: every output of a batched call is bit-identical to one psa_sigma_min call per
matrix (same arithmetic per point, same start vector); so are the three work orders,
a small points-in-flight cap, a workspace that holds one warp only, and CUDA-graph
replays (which re-read the bands each time). Sampled points of the batch workload
at its full sizes meet the oracle parity rule.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2605_04550_gb300 as psa
from paper_2605_04550_gb300 import batch, inputs
from tests.parity import ABS, band_norm1, check_masks, check_sigma

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
EPS = (1e-1, 1e-3, 1e-6)


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.complex128, device=DEV)


def _small_batch():
    """Mixed shapes and sizes: several matrices per class, ragged and one-point grids."""
    mats = []
    b, kl, ku = inputs.grcar(60)
    mats.append((b, kl, ku, inputs.Grid(-1.0, 3.0, -3.5, 3.5, 13, 9)))
    for k, (n, kl, ku, nx, ny) in enumerate([(75, 2, 5, 30, 17), (130, 2, 5, 8, 4), (45, 2, 5, 1, 1),
                                              (90, 1, 1, 21, 11), (50, 0, 2, 16, 8), (64, 4, 8, 19, 23),
                                              (120, 3, 6, 40, 6), (33, 1, 3, 9, 33), (200, 2, 5, 24, 24)]):
        b, _, _, a = inputs.random_toeplitz(n, kl, ku, seed=100 + k, super_scale=3.0)
        mats.append((b, kl, ku, inputs.toeplitz_symbol_grid(a, kl, ku, nx, ny)))
    return mats


def _individual(mats, eps, opts=None):
    outs = []
    for b, kl, ku, g in mats:
        r = psa.sigma_min(_t(b), kl, ku, g, eps=eps, opts=opts)
        outs.append([x.cpu().numpy().ravel() for x in (r.sigma, r.mask, r.status, r.steps)])
    return outs


def _batched(plan, eps, **kw):
    r = batch.sigma_min_batched(plan, eps, **kw)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in (r.sigma, r.mask, r.status, r.steps)]


def _assert_bitwise(plan, flat, ref):
    for m, o in enumerate(plan.offsets):
        ny, nx = plan.shapes[m]
        for f, r in zip(flat, ref[m]):
            np.testing.assert_array_equal(f[o:o + ny * nx], r, err_msg=f"matrix {m}")


@pytest.fixture(scope="module")
def small():
    mats = _small_batch()
    plan = batch.BatchPlan([(_t(b), kl, ku, g) for b, kl, ku, g in mats])
    return mats, plan, _individual(mats, EPS)


def test_batched_is_bitwise_individual_calls(small):
    mats, plan, ref = small
    assert len(plan.classes()) == 6
    _assert_bitwise(plan, _batched(plan, EPS), ref)


@pytest.mark.parametrize("cfg", [batch.BatchConfig(0, batch.ORDER_PLAN), batch.BatchConfig(0, batch.ORDER_ESTIMATE),
                                 batch.BatchConfig(32, batch.ORDER_AUTO), batch.BatchConfig(96, batch.ORDER_ESTIMATE),
                                 batch.BatchConfig(0, batch.ORDER_AUTO, 1), batch.BatchConfig(64, batch.ORDER_PLAN, 1),
                                 batch.BatchConfig(0, batch.ORDER_AUTO, 2), batch.BatchConfig(0, batch.ORDER_AUTO, 8)])
def test_launch_controls_do_not_change_results(small, cfg):
    mats, plan, ref = small
    _assert_bitwise(plan, _batched(plan, EPS, config=cfg), ref)


def test_one_warp_workspace(small):
    mats, plan, ref = small
    # room for exactly one warp of the largest class: every class runs with one warp
    one = batch.batch_workspace_bytes(plan, 32)
    ws = batch.BatchWorkspace(plan, max_bytes=one)
    _assert_bitwise(plan, _batched(plan, EPS, workspace=ws), ref)


@pytest.mark.parametrize("streams", [1, 4, 8])
def test_graph_replay_rereads_the_bands(small, streams):
    mats, plan, ref = small
    g = batch.BatchGraph(plan, EPS, config=batch.BatchConfig(streams=streams))
    for _ in range(2):
        out = g.replay()
        torch.cuda.synchronize()
        _assert_bitwise(plan, [x.cpu().numpy() for x in (out.sigma, out.mask, out.status, out.steps)], ref)
    # change matrix 1's bands in place: the replay sees the new values
    b1 = plan.bands[1]
    saved = b1.clone()
    b1.mul_(0.5)
    out = g.replay()
    torch.cuda.synchronize()
    b, kl, ku, grid = mats[1]
    r = psa.sigma_min(b1, kl, ku, grid, eps=EPS)
    torch.cuda.synchronize()
    o = plan.offsets[1]
    np.testing.assert_array_equal(out.sigma.cpu().numpy()[o:o + grid.npoints], r.sigma.cpu().numpy().ravel())
    b1.copy_(saved)


def test_nonfinite_matrix_is_flagged_alone():
    mats = _small_batch()[:4]
    bad = mats[2][0].copy()
    bad[1, 7] = np.nan
    mats[2] = (bad, *mats[2][1:])
    plan = batch.BatchPlan([(_t(b), kl, ku, g) for b, kl, ku, g in mats])
    sig, mask, st, steps = _batched(plan, EPS)
    ref = _individual(mats, EPS)
    for m, o in enumerate(plan.offsets):
        npts = mats[m][3].npoints
        if m == 2:
            assert np.all(st[o:o + npts] == psa.PT_NONFINITE) and np.all(sig[o:o + npts] == 0.0)
        np.testing.assert_array_equal(sig[o:o + npts], ref[m][0])
        np.testing.assert_array_equal(st[o:o + npts], ref[m][2])


def test_batched_matches_oracle_on_small_batch(small):
    mats, plan, _ = small
    sig, mask, st, _ = _batched(plan, EPS)
    for m, (b, kl, ku, g) in enumerate(mats):
        o = plan.offsets[m]
        z = oracle.grid_points(g).ravel()
        ref, st_ref, _ = oracle.sigma_min_banded(b, kl, ku, z)
        nrm = band_norm1(b, kl, ku, z)
        s = sig[o:o + z.size]
        bad, info = check_sigma(s, ref, nrm)
        assert not bad.any(), (m, info)
        bad_m, _ = check_masks(mask[o:o + z.size].view(np.uint32), oracle.masks(ref, EPS), ref, nrm, EPS)
        assert not bad_m.any(), m


def test_batch_workload_full_size_sampled():
    """The first 24 matrices of the 256-matrix batch workload (n log-uniform in
    [200, 8000], kl 1..4, ku 1..8, 128 x 128 grids) in the benchmark's launch
    configuration: 6 random points per matrix and up to 4 of its points of each of
    the statuses NOT_CONVERGED and SINGULAR against the oracle."""
    w = inputs.batch_workload()[:24]
    plan = batch.BatchPlan([(_t(b), kl, ku, g) for b, kl, ku, g, _ in w])
    sig, mask, st, _ = _batched(plan, inputs.EPS_LEVELS_8)
    rng = np.random.default_rng(7)
    for m, (b, kl, ku, g, kind) in enumerate(w):
        o = plan.offsets[m]
        stm = st[o:o + g.npoints]
        # SINGULAR: a pivot column that is exactly zero (deep inside the spectrum of a
        # large matrix the eliminated entries underflow)
        assert np.all(np.isin(stm, (psa.PT_OK, psa.PT_UNDERFLOW, psa.PT_NOT_CONVERGED, psa.PT_SINGULAR))), \
            (m, np.unique(stm))
        odd = [np.flatnonzero(stm == c)[:4] for c in (psa.PT_NOT_CONVERGED, psa.PT_SINGULAR)]
        smp = np.unique(np.concatenate([rng.choice(g.npoints, 6, replace=False), *odd]))
        z = oracle.grid_points(g).ravel()[smp]
        ref, st_ref, _ = oracle.sigma_min_banded(b, kl, ku, z)
        nrm = band_norm1(b, kl, ku, z)
        bad, info = check_sigma(sig[o + smp], ref, nrm)
        assert not bad.any(), (m, kind, b.shape, info)
        # an exact zero pivot that comes from underflow is decided by the rounding of
        # values far below the floor: where either side reports SINGULAR, both sigma
        # lie below the floor (the sigma rule above then holds with sigma = 0)
        sing = (stm[smp] == psa.PT_SINGULAR) | (st_ref == psa.PT_SINGULAR)
        assert np.all(np.maximum(sig[o + smp], ref)[sing] <= ABS * nrm[sing]), m
        bad_m, _ = check_masks(mask[o + smp].view(np.uint32), oracle.masks(ref, inputs.EPS_LEVELS_8), ref, nrm,
                               inputs.EPS_LEVELS_8)
        assert not bad_m.any(), m


def test_autotune_returns_a_timed_candidate(small):
    mats, plan, ref = small
    cands = [batch.BatchConfig(0, batch.ORDER_AUTO), batch.BatchConfig(64, batch.ORDER_PLAN)]
    best, times = batch.autotune(plan, EPS, candidates=cands)
    assert best in cands and set(times) == set(cands) and all(t > 0 for t in times.values())
