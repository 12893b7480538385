"""Pins of the oracle's randomized resolvent analysis (Algorithm 1) and of its
Gaussian test matrix, against brute force, closed forms, inequalities and
probabilistic bounds that the mathematics fixes."""
import math

import numpy as np
import pytest
import scipy.stats as st

import workloads as W
from oracle import operator as op
from oracle import philox
from oracle import resolvent as rs


# ---------------------------------------------------------------- generator
def test_gaussian_entries_are_standard_normal():
    g = philox.gaussian(1234, 20000, 8).ravel()
    assert abs(g.mean()) < 4 / math.sqrt(g.size)
    assert abs(g.var() - 1) < 0.02
    assert st.kstest(g, "norm").pvalue > 1e-3
    # fourth moment of N(0,1) is 3
    assert abs(np.mean(g ** 4) - 3) < 0.1


def test_gaussian_columns_and_seeds_independent():
    a = philox.gaussian(5, 40000, 4)
    b = philox.gaussian(6, 40000, 4)
    c = np.corrcoef(np.concatenate([a, b], axis=1).T)
    off = c - np.eye(8)
    assert np.max(np.abs(off)) < 0.03
    # counter-based: a block of rows is a prefix of a longer draw
    np.testing.assert_array_equal(philox.gaussian(5, 100, 4), a[:100])


def test_philox_uniforms_in_range():
    w = philox.raw_words(99, 5000, 3)
    assert all(x.dtype == np.uint32 for x in w)
    words = np.stack(w).ravel().astype(np.float64)
    # uniform 32-bit words: mean 2^31, KS against U(0, 2^32)
    assert st.kstest(words / 2 ** 32, "uniform").pvalue > 1e-3
    # the 53-bit integers and u1 in (0, 1]
    g = philox.gaussian(99, 5000, 3)
    assert np.all(np.isfinite(g))


def test_physics_weighted_test_matrix():
    phi = np.linspace(0.0, 2.0, 50)
    om = philox.test_matrix(3, 50, 5, phi)
    np.testing.assert_array_equal(om.imag, 0.0)
    np.testing.assert_allclose(om.real, phi[:, None] * philox.gaussian(3, 50, 5))


# -------------------------------------------------------------- brute force
@pytest.mark.parametrize("case", ["advdiff", "ns"])
def test_full_width_sketch_equals_exact_svd(case):
    """With k = N the sketch spans C^N: Algorithm 1 returns the exact SVD."""
    if case == "advdiff":
        g = W.Grid(kind=W.KIND_ADVDIFF, nx=8, ny=6, x0=0, x1=10, y0=-5, y1=5,
                   re=100.0)
        flow = W.tanh_shear_flow(g)
    else:
        g = W.ns_grid(6, 5)
        flow = W.smooth_random_flow(g, 11)
    L = op.assemble(g, flow)
    n = L.shape[0]
    s = 0.8j
    S, U, V = rs.exact_svd(L, s)
    r = rs.randomized(L, s, n, seed=17)
    np.testing.assert_allclose(r.sigma, S, rtol=1e-9)
    np.testing.assert_allclose(r.sigma_halko, S, rtol=1e-9)
    for j in range(3):
        assert rs.cosine_similarity(r.U[:, j], U[:, j]) > 1 - 1e-10
        assert rs.cosine_similarity(r.V[:, j], V[:, j]) > 1 - 1e-10


def test_low_rank_operator_recovered_exactly():
    """If R has exact rank <= k, the sketch captures it: sigma_1..k exact."""
    rng = np.random.default_rng(0)
    n, r = 60, 4
    A = ((rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r)))
         @ (rng.standard_normal((r, n)) + 1j * rng.standard_normal((r, n))))
    # R = (sI - L)^{-1} with rank deficiency is impossible for an inverse, so
    # the statement is checked on the projection itself: Q Q^H A = A
    om = philox.test_matrix(3, n, 6)
    Q, _ = np.linalg.qr(A @ om)
    assert np.linalg.norm(A - Q @ (Q.conj().T @ A)) < 1e-10 * np.linalg.norm(A)


def test_halko_and_present_recovery_inequalities():
    """sigma_j(B) <= sigma_j(R) (B = Q^H R is a projection), and for the
    leading triplet sigma_1^Halko = ||B v_1|| <= ||R v_1|| = sigma_1^present
    <= sigma_1 (the accuracy claim of Eq. 8 as an inequality)."""
    wl = W.config_small_ns(10, 8)
    L = op.assemble(wl.grid, wl.flow)
    for om in (0.4, 1.3, 3.0):
        S, _, _ = rs.exact_svd(L, 1j * om)
        for seed in range(5):
            r = rs.randomized(L, 1j * om, 6, seed)
            assert np.all(r.sigma_halko <= S[:6] * (1 + 1e-12))
            assert r.sigma_halko[0] <= r.sigma[0] * (1 + 1e-12)
            assert r.sigma[0] <= S[0] * (1 + 1e-12)


def test_present_recovery_more_accurate_than_halko():
    """Sec. II.B / Fig. 3: the third solve recovers sigma_1 better."""
    wl = W.config_tiny()
    L = op.assemble(wl.grid, wl.flow)
    S, _, _ = rs.exact_svd(L, 0.5j)
    for seed in range(3):
        r = rs.randomized(L, 0.5j, 10, 1000 + seed)
        assert abs(r.sigma[0] - S[0]) <= abs(r.sigma_halko[0] - S[0])


# -------------------------------------------------------------------- bounds
def test_error_bounds_over_seeds():
    """Sec. II.B bound ||R - QQ^H R|| <= (1 + 9 sqrt(k+p) sqrt(m)) sigma_{k+1}
    for every one of 100 seeds (p = 2), and the Halko-Martinsson-Tropp
    (SIAM Rev. 2011, Thm. 10.6) expected-error bound on the seed average:
    E||.|| <= (1 + sqrt(k/(p-1))) sigma_{k+1}
              + e sqrt(k+p)/p (sum_{j>k} sigma_j^2)^{1/2}."""
    g = W.Grid(kind=W.KIND_ADVDIFF, nx=16, ny=12, x0=0, x1=10, y0=-5, y1=5,
               re=100.0)
    L = op.assemble(g, W.tanh_shear_flow(g))
    s = 0.5j
    S, _, _ = rs.exact_svd(L, s)
    m = L.shape[0]
    k, p = 6, 2
    errs = []
    for seed in range(100):
        r = rs.randomized(L, s, k + p, seed)
        errs.append(rs.projection_error(L, s, r.Q))
    errs = np.array(errs)
    paper = (1 + 9 * math.sqrt(k + p) * math.sqrt(m)) * S[k]
    assert np.all(errs <= paper)
    hmt = ((1 + math.sqrt(k / (p - 1))) * S[k]
           + math.e * math.sqrt(k + p) / p * math.sqrt(np.sum(S[k:] ** 2)))
    assert errs.mean() <= hmt
    # and the error is never below the optimal rank-(k+p) error
    assert np.all(errs >= S[k + p] * (1 - 1e-9))


# ------------------------------------------------------------- solver pins
@pytest.mark.parametrize("method", ["dense", "banded"])
def test_solves_satisfy_the_operator(method):
    """||(sI-L) Y - Omega|| small, checked with the sparse operator only."""
    wl = W.config_small_ns(16, 12)
    L = op.assemble(wl.grid, wl.flow)
    s = 0.3 + 1.7j
    A = op.shifted(L, s)
    lu = rs.factor(A, method)
    om = philox.test_matrix(5, L.shape[0], 4)
    y = lu.solve(om)
    assert np.linalg.norm(A @ y - om) <= 1e-12 * np.linalg.norm(om)
    z = lu.solve_adjoint(om)
    assert np.linalg.norm(A.conj().T @ z - om) <= 1e-12 * np.linalg.norm(om)


def test_orthonormal_basis_and_weights():
    wl = W.config_small_ns(12, 10)
    L = op.assemble(wl.grid, wl.flow)
    n = L.shape[0]
    rng = np.random.default_rng(1)
    w = rng.uniform(0.5, 2.0, n)
    r = rs.randomized(L, 1.0j, 8, 3, weights=w)
    assert np.linalg.norm(r.Q.conj().T @ r.Q - np.eye(8)) < 1e-13
    # weighted resolvent = similarity transform of the unweighted one
    S, _, _ = rs.exact_svd(L, 1.0j, weights=w)
    Rw = np.diag(np.sqrt(w)) @ np.linalg.inv(op.shifted(L, 1.0j).toarray()) \
        @ np.diag(1 / np.sqrt(w))
    np.testing.assert_allclose(S, np.linalg.svd(Rw, compute_uv=False),
                               rtol=1e-10)
    # identity weights = no weights
    r1 = rs.randomized(L, 1.0j, 8, 3)
    r2 = rs.randomized(L, 1.0j, 8, 3, weights=np.ones(n))
    np.testing.assert_allclose(r1.sigma, r2.sigma, rtol=1e-13)


def test_column_phase_invariance():
    """Omega -> Omega D (|D_jj| = 1) leaves sigma and the phase-normalised
    modes unchanged (catches conjugation slips)."""
    wl = W.config_small_ns(10, 8)
    L = op.assemble(wl.grid, wl.flow)
    n = L.shape[0]
    om = philox.test_matrix(8, n, 6)
    d = np.exp(1j * np.linspace(0.3, 2.9, 6))
    r1 = rs.randomized(L, 0.7j, 6, 0, omega=om)
    r2 = rs.randomized(L, 0.7j, 6, 0, omega=om * d[None, :])
    np.testing.assert_allclose(r1.sigma, r2.sigma, rtol=1e-10)
    np.testing.assert_allclose(r1.V, r2.V, atol=1e-8)
    np.testing.assert_allclose(r1.U, r2.U, atol=1e-8)


def test_orthogonalized_output():
    """Optional last steps of Algorithm 1: U orthonormal and sigma = svd(U Sigma)."""
    wl = W.config_small_ns(10, 8)
    L = op.assemble(wl.grid, wl.flow)
    r0 = rs.randomized(L, 0.7j, 6, 2)
    r = rs.randomized(L, 0.7j, 6, 2, orthogonalize=True)
    assert np.linalg.norm(r.U.conj().T @ r.U - np.eye(6)) < 1e-12
    assert np.linalg.norm(r.V.conj().T @ r.V - np.eye(6)) < 1e-12
    US = r0.U * r0.sigma
    np.testing.assert_allclose(r.sigma, np.linalg.svd(US, compute_uv=False),
                               rtol=1e-10)
    # R V = U Sigma for the rotated V as well
    A = op.shifted(L, 0.7j).toarray()
    np.testing.assert_allclose(np.linalg.solve(A, r.V), r.U * r.sigma,
                               atol=1e-9 * r.sigma[0])


def test_spectral_gap_controls_mode_error():
    """Sec. III.B: a large sigma_1/sigma_2 gap gives accurate leading modes;
    the response mode is more accurate than the forcing mode."""
    wl = W.config_small_ns(16, 12)
    L = op.assemble(wl.grid, wl.flow)
    best = None
    for om in (0.2, 0.6, 1.5, 3.0):
        S, U, V = rs.exact_svd(L, 1j * om)
        r = rs.randomized(L, 1j * om, 10, 1000)
        gap = S[0] / S[1]
        ev = 1 - rs.cosine_similarity(r.V[:, 0], V[:, 0])
        eu = 1 - rs.cosine_similarity(r.U[:, 0], U[:, 0])
        if best is None or gap > best[0]:
            best = (gap, ev, eu)
    gap, ev, eu = best
    assert gap > 3
    assert eu <= ev + 1e-15
    assert ev < 1e-3


def test_philox_matches_published_known_answers():
    """The oracle's Philox-4x32-10 reproduces the generator's published
    known-answer vectors (tests/golden/philox4x32_10_kat.txt), so Omega rests
    on the published definition, not on the oracle's reading of it."""
    import os
    from oracle import philox
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(*[[c] for c in v[:4]], v[4], v[5])
        assert [int(o[0]) for o in out] == v[6:]
