"""Pins of the CPU oracle against what the mathematics and independent libraries fix.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a conjugate missed, a transposed index, a different pivot rule)
fails at least one of them:

* closed forms for normal A: sigma_min(zI - A) = min_k |z - lambda_k|
  (paper Sec. 2, Definition "Resolvent Norm"), three families;
* LAPACK zgbtrf (an independent banded LU with the same |Re|+|Im| pivot rule)
  for the pivot sequence and the factor;
* dense linear solves for B x = b and B^* y = b;
* SciPy's tridiagonal eigensolver for theta_max(T_j) and the eigenvector's
  last component;
* dense SVD (the paper's own method, Sec. 2.1) on n <= 64;
* exact Lanczos sanity: the eigenvalues of T_n equal those of H for n steps;
* invariances of sigma_min (unitary diagonal similarity, transpose,
  conjugation, shift; power-of-two scaling bitwise);
* the published SplitMix64 output sequence; the grid against numpy.linspace.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2605_04550_gb300 import inputs
from tests.parity import band_norm1, check_sigma, ABS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_points(rng, k, box=(-3, 3, -3, 3)):
    return rng.uniform(box[0], box[1], k) + 1j * rng.uniform(box[2], box[3], k)


# ------------------------------------------------------------ generators
def test_splitmix64_published_sequence():
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) as f:
        want = [int(l) for l in f if l.strip() and not l.startswith("#")]
    got = [oracle.splitmix64(1234567, c) for c in range(len(want))]
    assert got == want


def test_start_vector_unit_and_seeded():
    q = oracle.start_vector(257, 0)
    assert abs(np.linalg.norm(q) - 1.0) < 1e-15
    assert not np.allclose(q, oracle.start_vector(257, 1))
    # components come from disjoint counters 2i, 2i+1
    raw0 = (oracle.splitmix64(0, 0) >> 11) * 2.0**-52 - 1.0
    raw1 = (oracle.splitmix64(0, 1) >> 11) * 2.0**-52 - 1.0
    h = np.array([(oracle.splitmix64(0, 2 * i) >> 11) * 2.0**-52 - 1.0 +
                  1j * ((oracle.splitmix64(0, 2 * i + 1) >> 11) * 2.0**-52 - 1.0) for i in range(257)])
    assert q[0] == pytest.approx((raw0 + 1j * raw1) / np.linalg.norm(h), rel=1e-15)


def test_grid_matches_linspace_and_orientation():
    g = inputs.Grid(-1.0, 3.0, -3.5, 3.5, 100, 77)
    z = oracle.grid_points(g)
    assert z.shape == (77, 100)
    np.testing.assert_allclose(z[0].real, np.linspace(-1, 3, 100), rtol=0, atol=4e-16 * 3)
    np.testing.assert_allclose(z[:, 0].imag, np.linspace(-3.5, 3.5, 77), rtol=0, atol=4e-16 * 3.5)
    assert z[0, 0] == complex(-1.0, -3.5)          # row 0 = Im min, column 0 = Re min
    assert np.all(np.diff(z[:, 5].imag) > 0) and np.all(np.diff(z[5].real) > 0)
    g1 = inputs.Grid(0.5, 0.5, 2.0, 2.0, 1, 1)
    assert oracle.grid_points(g1)[0, 0] == complex(0.5, 2.0)


# ------------------------------------------------------ normal matrices
def test_closed_form_diagonal():
    b, kl, ku, lam = inputs.diagonal_normal(40, seed=3)
    rng = np.random.default_rng(0)
    z = _rand_points(rng, 60)
    s, st, _ = oracle.sigma_min_banded(b, kl, ku, z)
    exact = np.array([np.min(np.abs(zz - lam)) for zz in z])
    bad, info = check_sigma(s, exact, band_norm1(b, kl, ku, z), rel=1e-12)
    assert not bad.any(), info
    assert np.all(st == oracle.OK)


@pytest.mark.parametrize("n,a,bb", [(50, 0.3, 0.7 - 0.4j), (7, -1.0, 2.0j), (1, 0.25, 0.0)])
def test_closed_form_hermitian_toeplitz_tridiagonal(n, a, bb):
    b, kl, ku = inputs.hermitian_toeplitz_tridiag(n, a, bb)
    k = np.arange(1, n + 1)
    lam = a + 2 * abs(bb) * np.cos(k * np.pi / (n + 1))
    rng = np.random.default_rng(1)
    z = _rand_points(rng, 40)
    s, st, _ = oracle.sigma_min_banded(b, kl, ku, z)
    exact = np.array([np.min(np.abs(zz - lam)) for zz in z])
    bad, info = check_sigma(s, exact, band_norm1(b, kl, ku, z), rel=1e-12)
    assert not bad.any(), info


@pytest.mark.parametrize("k", [1, 2, 4])
def test_closed_form_scaled_shifted_hermitian(k):
    alpha, shift = 0.8 * np.exp(0.7j), 0.3 - 0.2j
    b, kl, ku, H = inputs.shifted_hermitian_band(45, k, alpha, shift, seed=k)
    lam = alpha * np.linalg.eigvalsh(H) + shift
    rng = np.random.default_rng(2)
    z = _rand_points(rng, 40, box=(-4, 4, -4, 4))
    s, _, _ = oracle.sigma_min_banded(b, kl, ku, z)
    exact = np.array([np.min(np.abs(zz - lam)) for zz in z])
    bad, info = check_sigma(s, exact, band_norm1(b, kl, ku, z), rel=1e-12)
    assert not bad.any(), info


# -------------------------------------------------------- banded LU step
def _lapack_band(bands, kl, ku, z):
    """zI - A in LAPACK's gbtrf band layout (2kl+ku+1 rows)."""
    n = bands.shape[1]
    ab = np.zeros((2 * kl + ku + 1, n), dtype=np.complex128)
    A = oracle.band_to_dense(bands, kl, ku)
    B = z * np.eye(n) - A
    for j in range(n):
        for i in range(max(0, j - ku), min(n, j + kl + 1)):
            ab[kl + ku + i - j, j] = B[i, j]
    return ab, B


@pytest.mark.parametrize("case", ["grcar", "toeplitz", "paper"])
def test_lu_pivots_match_lapack_zgbtrf(case):
    if case == "grcar":
        b, kl, ku = inputs.grcar(60)
    elif case == "toeplitz":
        b, kl, ku, _ = inputs.random_toeplitz(70, 2, 5, seed=4)
    else:
        b, kl, ku, _ = inputs.paper_class(5)
    rng = np.random.default_rng(5)
    for z in _rand_points(rng, 6):
        factor, piv, rc = oracle.band_lu(b, kl, ku, z)
        assert rc == 0
        ab, B = _lapack_band(b, kl, ku, z)
        lu, ipiv, info = sla.lapack.zgbtrf(ab, kl, ku)
        assert info == 0
        np.testing.assert_array_equal(piv, ipiv)          # same rows chosen, 0-based
        n = B.shape[0]
        # U from LAPACK: lu[kl+ku+i-j, j] = U[i, j]; ours: factor[i, j-i+kl]
        for i in range(n):
            for j in range(i, min(n, i + kl + ku + 1)):
                np.testing.assert_allclose(factor[i, j - i + kl], lu[kl + ku + i - j, j],
                                           rtol=1e-13, atol=1e-13 * np.abs(B).max())


def test_lu_reconstructs_B():
    b, kl, ku, _ = inputs.random_toeplitz(50, 3, 2, seed=8)
    z = 0.3 + 1.1j
    factor, piv, rc = oracle.band_lu(b, kl, ku, z)
    n = 50
    B = z * np.eye(n) - oracle.band_to_dense(b, kl, ku)
    # apply the recorded eliminations to B and compare with U
    M = B.copy()
    for j in range(n):
        M[[j, piv[j]]] = M[[piv[j], j]]
        for i in range(j + 1, min(n, j + kl + 1)):
            M[i] -= factor[i, j - i + kl] * M[j]
    Uo = np.zeros_like(M)
    for i in range(n):
        for j in range(i, min(n, i + kl + ku + 1)):
            Uo[i, j] = factor[i, j - i + kl]
    np.testing.assert_allclose(np.triu(M), Uo, atol=1e-13 * np.abs(B).max())
    assert np.abs(np.tril(M, -1)).max() < 1e-13 * np.abs(B).max()


def test_singular_zero_pivot():
    b, kl, ku, lam = inputs.diagonal_normal(10, seed=1)
    s, st, _ = oracle.sigma_min_banded(b, kl, ku, [lam[3]])
    assert st[0] == oracle.SINGULAR and s[0] == 0.0
    jb, jkl, jku = inputs.jordan_block(32)
    s, st, _ = oracle.sigma_min_banded(jb, jkl, jku, [0.0])
    assert st[0] == oracle.SINGULAR and s[0] == 0.0


def test_nonfinite_input():
    b, kl, ku = inputs.grcar(20)
    b = b.copy()
    b[2, 5] = np.nan
    s, st, _ = oracle.sigma_min_banded(b, kl, ku, [0.5 + 0.5j])
    assert st[0] == oracle.NONFINITE


# ------------------------------------------------------------ solve step
@pytest.mark.parametrize("adjoint", [False, True])
def test_band_solves_match_dense(adjoint):
    b, kl, ku, _ = inputs.random_toeplitz(64, 2, 5, seed=11)
    z = -0.7 + 2.2j
    factor, piv, _ = oracle.band_lu(b, kl, ku, z)
    B = z * np.eye(64) - oracle.band_to_dense(b, kl, ku)
    rng = np.random.default_rng(3)
    rhs = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    x = oracle.band_solve(factor, piv, kl, ku, rhs, adjoint=adjoint)
    ref = np.linalg.solve(B.conj().T if adjoint else B, rhs)
    np.testing.assert_allclose(x, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


# ----------------------------------------------------- tridiagonal step
@pytest.mark.parametrize("m", [1, 2, 3, 10, 57])
def test_tridiag_top_matches_scipy(m):
    rng = np.random.default_rng(m)
    a = rng.uniform(0, 5, m)
    bo = rng.uniform(0.01, 2, max(m - 1, 0))
    th, s = oracle.tridiag_top(a, bo)
    if m == 1:
        assert th == a[0] and s == 1.0
        return
    w, v = sla.eigh_tridiagonal(a, bo)
    assert th == pytest.approx(w[-1], rel=4e-16 * m, abs=1e-15)
    assert abs(s - abs(v[-1, -1])) <= 1e-9 * abs(v[-1, -1]) + 1e-13


# ------------------------------------------------------ Lanczos recurrence
@pytest.mark.parametrize("z,full", [(9.0 + 7.0j, True), (0.4 - 0.3j, False)])
def test_lanczos_tridiagonal_spectrum_equals_H_after_n_steps(z, full):
    """After n steps T_n is similar to H / 2^(2 e1) (exact arithmetic). With a
    well-conditioned H (z far from the spectrum) orthogonality survives and all
    n eigenvalues match; with an ill-conditioned H only the top one is kept."""
    n = 6
    b, kl, ku, _ = inputs.random_toeplitz(n, 1, 2, seed=2)
    alpha, beta, e1 = oracle.lanczos_coeffs(b, kl, ku, z, k=n)
    assert len(alpha) == n
    T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    B = z * np.eye(n) - oracle.band_to_dense(b, kl, ku)
    sv = np.linalg.svd(B, compute_uv=False)
    eig_H_scaled = np.sort(1.0 / sv**2) / 2.0**(2 * e1)
    got = np.sort(np.linalg.eigvalsh(T))
    assert got[-1] == pytest.approx(eig_H_scaled[-1], rel=1e-12)
    if full:
        np.testing.assert_allclose(got, eig_H_scaled, rtol=1e-12)
        assert beta[-1] < 1e-10 * eig_H_scaled.max()      # breakdown after n steps


def test_lanczos_first_coefficient_is_rayleigh_quotient():
    b, kl, ku = inputs.grcar(30)
    z = 2.5 + 3.0j                      # moderately conditioned point
    alpha, beta, e1 = oracle.lanczos_coeffs(b, kl, ku, z, k=2)
    B = z * np.eye(30) - oracle.band_to_dense(b, kl, ku)
    q = oracle.start_vector(30, 0)
    Hq = np.linalg.solve(B.conj().T, np.linalg.solve(B, q)) / 2.0**(2 * e1)
    assert alpha[0] == pytest.approx(np.real(q.conj() @ Hq), rel=1e-12)
    w = Hq - alpha[0] * q
    assert beta[0] == pytest.approx(np.linalg.norm(w), rel=1e-10)


# ------------------------------------------------------- dense SVD (paper)
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_paper_class_matches_dense_svd(seed):
    b, kl, ku, A = inputs.paper_class(seed)
    z = oracle.grid_points(inputs.paper_grid_100()).ravel()[::53]
    s, st, _ = oracle.sigma_min_banded(b, kl, ku, z)
    ref = oracle.sigma_min_dense(A, z)
    bad, info = check_sigma(s, ref, band_norm1(b, kl, ku, z))
    assert not bad.any(), info
    assert np.all(st == oracle.OK)


def test_jordan_block_matches_dense_svd():
    jb, kl, ku = inputs.jordan_block(32)
    A = oracle.band_to_dense(jb, kl, ku)
    z = np.array([0.5, 0.9j, -1.2 + 0.3j, 0.99, 0.2 - 0.2j, 2.0])
    s, _, _ = oracle.sigma_min_banded(jb, kl, ku, z)
    ref = oracle.sigma_min_dense(A, z)
    bad, info = check_sigma(s, ref, band_norm1(jb, kl, ku, z))
    assert not bad.any(), info


def test_grcar_and_toeplitz_match_dense_svd():
    for b, kl, ku, box in [(*inputs.grcar(64), (-1, 3, -3.5, 3.5)),
                           (*inputs.random_toeplitz(64, 2, 5, seed=0)[:3], (-15, 15, -15, 15))]:
        A = oracle.band_to_dense(b, kl, ku)
        rng = np.random.default_rng(7)
        z = _rand_points(rng, 40, box)
        s, _, _ = oracle.sigma_min_banded(b, kl, ku, z)
        ref = oracle.sigma_min_dense(A, z)
        bad, info = check_sigma(s, ref, band_norm1(b, kl, ku, z))
        assert not bad.any(), info


# ------------------------------------------------------------ invariances
def _field(b, kl, ku, z):
    return oracle.sigma_min_banded(b, kl, ku, z)[0]


def test_invariance_unitary_diagonal_similarity():
    b, kl, ku, _ = inputs.random_toeplitz(80, 2, 3, seed=5)
    rng = np.random.default_rng(9)
    phi = rng.uniform(0, 2 * np.pi, 80)
    b2 = b.copy()
    for d in range(-kl, ku + 1):
        i = np.arange(80)
        j = np.clip(i + d, 0, 79)
        b2[d + kl] = b[d + kl] * np.exp(1j * (phi[i] - phi[j]))
    z = _rand_points(rng, 30, (-12, 12, -12, 12))
    bad, info = check_sigma(_field(b2, kl, ku, z), _field(b, kl, ku, z), band_norm1(b, kl, ku, z))
    assert not bad.any(), info


def test_invariance_transpose_conjugate_shift():
    b, kl, ku, _ = inputs.random_toeplitz(90, 1, 4, seed=6)
    n = 90
    rng = np.random.default_rng(10)
    z = _rand_points(rng, 30, (-12, 12, -12, 12))
    ref = _field(b, kl, ku, z)
    nrm = band_norm1(b, kl, ku, z)
    # transpose: A^T[i, i+d] = A[i+d, i] -> kl and ku swap
    bt = np.zeros((kl + ku + 1, n), dtype=np.complex128)
    for d in range(-ku, kl + 1):
        for i in range(n):
            if 0 <= i + d < n:
                bt[d + ku, i] = b[-d + kl, i + d]
    bad, info = check_sigma(_field(bt, ku, kl, z), ref, nrm)
    assert not bad.any(), ("transpose", info)
    bad, info = check_sigma(_field(np.conj(b), kl, ku, np.conj(z)), ref, nrm)
    assert not bad.any(), ("conjugate", info)
    s = 0.75 - 1.25j
    bs = b.copy()
    bs[kl] += s
    bad, info = check_sigma(_field(bs, kl, ku, z + s), ref, nrm)
    assert not bad.any(), ("shift", info)


def test_invariance_power_of_two_scaling_is_bitwise():
    b, kl, ku = inputs.grcar(100)
    z = oracle.grid_points(inputs.grcar_grid_100()).ravel()[::37]
    ref = _field(b, kl, ku, z)
    for m in (-7, 3, 40):
        got = _field(b * 2.0**m, kl, ku, z * 2.0**m)
        np.testing.assert_array_equal(got, ref * 2.0**m)


def test_real_matrix_field_is_mirror_symmetric():
    b, kl, ku = inputs.grcar(100)
    z = oracle.grid_points(inputs.grcar_grid_100())
    top = _field(b, kl, ku, z[:5].ravel())
    bottom = _field(b, kl, ku, np.conj(z[:5]).ravel())
    bad, info = check_sigma(bottom, top, band_norm1(b, kl, ku, z[:5].ravel()))
    assert not bad.any(), info


# ------------------------------------------------------------------- masks
def test_masks_inclusive_and_monotone():
    eps = inputs.EPS_LEVELS_8
    sig = np.array([1.0, 0.1, 0.05, 1e-8, 0.0, 2e-8, np.nextafter(0.1, 1)])
    m = oracle.masks(sig, eps)
    assert m[0] == 0
    assert m[1] & 1                          # sigma == eps_0 is sensitive (<=)
    assert m[6] == 0
    assert m[3] == 0xFF and m[4] == 0xFF
    for v in m:                              # bit l set => all larger levels set
        bits = [(int(v) >> l) & 1 for l in range(len(eps))]
        for l in range(1, len(eps)):
            assert bits[l] <= bits[l - 1]


def test_fixed_step_mode_runs_exactly_k_steps():
    b, kl, ku = inputs.grcar(100)
    z = oracle.grid_points(inputs.grcar_grid_100()).ravel()[::101]
    _, st, k = oracle.sigma_min_banded(b, kl, ku, z, k_min=20, k_max=20)
    assert np.all(k == 20)
    assert np.all((st == oracle.OK) | (st == oracle.NOT_CONVERGED))


# --------------------------------------------------------- gradient oracle
def _fd_sigma(A, z, h=1e-6):
    s = lambda zz: oracle.sigma_min_dense(A, [zz])[0]
    return complex((s(z + h) - s(z - h)) / (2 * h), (s(z + 1j * h) - s(z - 1j * h)) / (2 * h))


@pytest.mark.parametrize("case", ["grcar", "toeplitz", "paper"])
def test_gradient_formula_matches_finite_differences(case):
    if case == "grcar":
        b, kl, ku = inputs.grcar(40)
        zs = [1.5 + 2.5j, 0.3 - 1.7j]
    elif case == "toeplitz":
        b, kl, ku, _ = inputs.random_toeplitz(30, 2, 5, seed=1)
        zs = [6.0 + 4.0j, -3.0 + 1.0j]
    else:
        b, kl, ku, _ = inputs.paper_class(2)
        zs = [2.5 + 1.5j, -3.0 - 2.0j]
    A = oracle.band_to_dense(b, kl, ku)
    for z in zs:
        s, gz, gA = oracle.sigma_min_grad_dense(A, z)
        fd = _fd_sigma(A, z)
        assert abs(gz - fd) <= 1e-6 * abs(fd) + 1e-9, (z, gz, fd)
        # one band entry, real and imaginary directions
        i, d = 7, 1
        E = np.zeros_like(A)
        E[i, i + d] = 1.0
        h = 1e-6
        sp = oracle.sigma_min_dense(A + h * E, [z])[0]
        sm = oracle.sigma_min_dense(A - h * E, [z])[0]
        spi = oracle.sigma_min_dense(A + 1j * h * E, [z])[0]
        smi = oracle.sigma_min_dense(A - 1j * h * E, [z])[0]
        fda = complex((sp - sm) / (2 * h), (spi - smi) / (2 * h))
        gb = oracle.dense_grad_to_bands(gA, kl, ku)
        assert abs(gb[d + kl, i] - fda) <= 1e-6 * abs(fda) + 1e-9, (gb[d + kl, i], fda)


def _hard_points_n2000():
    """Points of the n = 2000 Toeplitz grid (kl = 2, ku = 5, 512 x 512 over the symbol
    box +20 %) where the stopping rule can fail: the 14 that need the most Lanczos
    steps among 384 random grid points (outside the symbol curve, 40-300 steps), 4
    on the edge of the curve (sigma / |zI - A|_1 in [1e-8, 1e-6), [1e-5, 1e-4),
    [1e-4, 1e-3) and [1e-3, 1e-2)) and 2 inside (far below the roundoff floor)."""
    bands, kl, ku, a = inputs.random_toeplitz(2000, 2, 5, seed=0)
    grid = inputs.toeplitz_symbol_grid(a, kl, ku, 512, 512)
    rng = np.random.default_rng(11)
    z = oracle.grid_points(grid).ravel()[rng.choice(grid.npoints, 384, replace=False)]
    s, st, k = oracle.sigma_min_banded(bands, kl, ku, z, k_max=1000, tol=1e-13)
    rel = s / band_norm1(bands, kl, ku, z)
    hard = np.argsort(-k, kind="stable")[:14]
    edge = np.array([np.flatnonzero((rel >= lo) & (rel < 10 * lo) if lo != 1e-8 else (rel >= lo) & (rel < 1e-6))[0]
                     for lo in (1e-8, 1e-5, 1e-4, 1e-3)])
    inside = np.flatnonzero(rel < 1e-20)[:2]
    return bands, kl, ku, z[np.concatenate([hard, edge, inside])], k[hard]


def test_oracle_n2000_matches_dense_svd_where_lanczos_is_slow():
    """The stopping rule at the benchmark's order: the oracle in both its exact tier
    (tol 1e-15) and the library's settings (tol 1e-13, k_max 1000) against the dense
    SVD (paper Sec. 2.1) at points that need tens to hundreds of Lanczos steps."""
    bands, kl, ku, z, k_hard = _hard_points_n2000()
    assert k_hard.min() >= 40, k_hard  # the points really are slow to converge
    ref = oracle.sigma_min_dense(oracle.band_to_dense(bands, kl, ku), z)
    nrm = band_norm1(bands, kl, ku, z)
    for kw in ({}, {"k_max": 1000, "tol": 1e-13}):
        s, st, _ = oracle.sigma_min_banded(bands, kl, ku, z, **kw)
        bad, info = check_sigma(s, ref, nrm)
        assert not bad.any(), (kw, info, s[bad], ref[bad])
        assert info["max_rel_well"] <= 1e-10, (kw, info)
