"""Pins of the feature oracle (oracle/features.py) against closed forms, invariances
and independent library routines, CPU only. Each is chosen so that a slip in a
definition (a wrong diagonal in the symbol, a transposed norm, a sign in the winding
sum, a missing scale) fails one of them."""
import numpy as np
import pytest

import oracle
from oracle import features as F
from paper_2605_04550_gb300 import inputs


def _toeplitz(n, coef, kl, ku):
    b = np.zeros((kl + ku + 1, n), dtype=np.complex128)
    for d in range(-kl, ku + 1):
        b[d + kl] = coef[d + kl]
    return inputs._zero_outside(b, n, kl, ku)


def test_symbol_of_a_tridiagonal_toeplitz_is_its_ellipse():
    # f(t) = a + b e^{-it} + c e^{it} = a + (b + c) cos t + i (c - b) sin t for real b, c
    a, b, c = 0.3, 0.5, 2.0
    f = F.symbol_samples(_toeplitz(40, [b, a, c], 1, 1), 1, 1)
    t = 2 * np.pi * np.arange(256) / 256
    np.testing.assert_allclose(f.real, a + (b + c) * np.cos(t), atol=1e-14)
    np.testing.assert_allclose(f.imag, (c - b) * np.sin(t), atol=1e-14)


def test_stats_against_eigenvalues_and_library_norms():
    b, kl, ku, _ = inputs.random_toeplitz(60, 2, 3, seed=4)
    b = inputs._zero_outside(b + 0.1 * np.random.default_rng(1).standard_normal(b.shape), 60, kl, ku)
    st, f = F.matrix_stats(b, kl, ku)
    A = F.dense(b, kl, ku)
    lam = np.linalg.eigvals(A)
    assert abs(complex(st[0], st[1]) - lam.mean()) <= 1e-12 * np.abs(lam).max()  # centroid = eigenvalue mean
    assert np.isclose(st[3], np.sqrt(np.sum(np.linalg.svd(A, compute_uv=False) ** 2)))
    assert np.isclose(st[4], np.linalg.norm(A, 1)) and np.isclose(st[5], np.linalg.norm(A, np.inf))
    assert st[12] == np.count_nonzero(np.abs(A) > 1e-10)
    assert st[22] == 60 and st[23] == 16 * 2 + 3
    # symmetric and Hermitian bands have no departure
    bs, kls, kus = inputs.hermitian_toeplitz_tridiag(30, 1.0, 0.7)
    sts, _ = F.matrix_stats(bs, kls, kus)
    assert sts[6] < 1e-14 and sts[7] < 1e-14
    bh, klh, kuh = inputs.hermitian_toeplitz_tridiag(30, 1.0, 0.7 - 0.2j)
    sth, _ = F.matrix_stats(bh, klh, kuh)
    assert sth[7] < 1e-14 and sth[6] > 0.1


def test_polyline_distance_and_winding_on_the_unit_circle():
    # A = the shift (a_1 = 1): symbol e^{it}, the unit circle (a regular 256-gon)
    f = F.symbol_samples(_toeplitz(30, [0.0, 1.0], 0, 1), 0, 1)
    st, _ = F.matrix_stats(_toeplitz(30, [0.0, 1.0], 0, 1), 0, 1)
    assert np.isclose(st[2], 1.0) and abs(st[0]) < 1e-15 and abs(st[1]) < 1e-15
    chord = np.cos(np.pi / 256)  # distance from the centre to each edge of the 256-gon
    assert np.isclose(F.polyline_distance(f, 0.0), chord, rtol=1e-12)
    for z in (1.5, -2.0j, 0.3 + 0.4j, 1.0):
        assert abs(F.polyline_distance(f, z) - abs(abs(z) - 1.0)) <= 1.0 - chord + 1e-12
    assert F.winding_number(f, 0.2 - 0.1j) == 1 and F.winding_number(f, 1.4) == 0
    # the same circle traversed backwards (a_{-1} = 1: symbol e^{-it}) winds -1
    g = F.symbol_samples(_toeplitz(30, [1.0, 0.0], 1, 0), 1, 0)
    assert F.winding_number(g, 0.0) == -1


def test_global_features_are_scale_free():
    b, kl, ku, _ = inputs.random_toeplitz(50, 1, 4, seed=7)
    st, _ = F.matrix_stats(b, kl, ku)
    st2, _ = F.matrix_stats(4.0 * b, kl, ku)
    s4 = np.array([0.3, 0.5, 0.7, 0.9])
    g1 = F.global_features(st, s4, 0.01)
    g2 = F.global_features(st2, 4.0 * s4, 0.04)  # sigma and eps scale with A
    np.testing.assert_allclose(np.delete(g1, 23), np.delete(g2, 23), atol=1e-12)
    assert np.isclose(g2[23] - g1[23], np.log10(4.0))  # log R is the one scale


def test_point_feature_identities():
    b, kl, ku = inputs.grcar(40)
    st, f = F.matrix_stats(b, kl, ku)
    g = F.global_features(st, np.array([0.1, 0.2, 0.3, 0.4]), 0.01)
    grid = inputs.Grid(-1.0, 3.0, -3.5, 3.5, 9, 7)
    x = F.point_features(grid, st, f, g, np.arange(grid.npoints))
    np.testing.assert_allclose(x[[0, 8, 54, 62], :2], [[-1, -1], [1, -1], [-1, 1], [1, 1]], atol=1e-15)
    for k in range(6):
        s, c = x[:, 2 + 4 * k:4 + 4 * k], x[:, 4 + 4 * k:6 + 4 * k]
        np.testing.assert_allclose(s ** 2 + c ** 2, 1.0, atol=1e-14)
    np.testing.assert_allclose(x[:, 60] - x[:, 29], -g[24], atol=1e-12)
    # the polyline passes through the samples: never farther than the nearest sample
    z = oracle.grid_points(grid).ravel()
    assert np.all(x[:, 26] <= np.abs(f[None, :] - z[:, None]).min(axis=1) / st[2] + 1e-15)
    assert np.all(x[:, 61:] == 0)


def test_point_set_stats_of_a_symmetric_cross():
    # four points c +- a, c +- i b about the centroid c: means 0, extremes +-a and +-b
    st, _ = F.matrix_stats(_toeplitz(20, [0.5, 1.0 + 2.0j, 0.0], 1, 1), 1, 1)
    c = complex(st[0], st[1])
    assert np.isclose(c, 1.0 + 2.0j)
    a, b = 0.7, 0.3
    out = F.point_set_stats(st, [c + a, c - a, c + 1j * b, c - 1j * b])
    assert np.isclose(out[2], a) and np.isclose(out[21], b)
    np.testing.assert_allclose(out[[13, 17]], 0.0, atol=1e-15)
    np.testing.assert_allclose(out[[15, 16, 19, 20]], [-a, a, -b, b], atol=1e-15)
    assert np.isclose(out[14], np.sqrt(a * a / 2)) and np.isclose(out[18], np.sqrt(b * b / 2))
    # every entry that does not describe the spectrum is kept
    keep = [k for k in range(24) if k != 2 and not 13 <= k <= 21]
    np.testing.assert_array_equal(out[keep], st[keep])
    # the symbol samples as the set give back the symbol statistics
    st2, f2 = F.matrix_stats(_toeplitz(20, [0.5, 1.0, 2.0], 1, 1), 1, 1)
    np.testing.assert_allclose(F.point_set_stats(st2, f2), st2, rtol=1e-13, atol=1e-15)


def test_point_set_features_of_a_ring_and_a_single_point():
    grid = inputs.Grid(-1.0, 1.0, -1.0, 1.0, 5, 5)  # grid point 12 is z = 0
    b = _toeplitz(30, [0.0, 1.0], 0, 1)  # centroid 0
    st, _ = F.matrix_stats(b, 0, 1)
    r = 0.4
    ring = r * np.exp(2j * np.pi * np.arange(64) / 64)
    sst = F.point_set_stats(st, ring)
    g = F.global_features(sst, np.array([0.1, 0.2, 0.3, 0.4]), 0.01)
    x = F.point_features(grid, sst, ring, g, [12], closed=False)[0]
    # every point of the ring is r from its centre, and R = r: g1 = g3 = 1
    assert np.isclose(x[26], 1.0) and np.isclose(x[28], 1.0) and x[31] == 0
    # the polyline through the same points is closer (its chords cut inside) and winds once
    xc = F.point_features(grid, sst, ring, g, [12], closed=True)[0]
    assert xc[26] < x[26] and xc[31] == 1
    # a single eigenvalue: g1 = g3 = |z - lambda| / R at every point
    lam = 0.25 - 0.5j
    s1 = F.point_set_stats(st, [lam])
    g1 = F.global_features(s1, np.array([0.1, 0.2, 0.3, 0.4]), 0.01)
    xs = F.point_features(grid, s1, np.array([lam]), g1, np.arange(25), closed=False)
    z = oracle.grid_points(grid).ravel()
    np.testing.assert_allclose(xs[:, 26], np.abs(z - lam) / abs(lam), rtol=1e-14)
    np.testing.assert_allclose(xs[:, 28], xs[:, 26], rtol=0, atol=0)
