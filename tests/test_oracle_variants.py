"""Pins of the oracle's test-matrix variants (Rademacher, sparse Rademacher,
orthonormalised Gaussian; Sec. II.B.2) and of its subspace (power) iterations
(Sec. II.B.1), against what probability and linear algebra fix: exact value
sets, binomial counts, range identities, the dense matrix-power definition of
the iteration and the Halko-Martinsson-Tropp bound with power iterations."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import operator as op
from oracle import philox
from oracle import resolvent as rs


def _advdiff(nx, ny):
    g = W.Grid(kind=W.KIND_ADVDIFF, nx=nx, ny=ny, x0=0, x1=10, y0=-5, y1=5, re=100.0)
    return op.assemble(g, W.tanh_shear_flow(g))


def _dense_r(L, s):
    lu = rs.DenseLU(op.shifted(L, s))
    return lu.solve(np.eye(L.shape[0], dtype=np.complex128))


# ---------------------------------------------------------------- Rademacher
def test_rademacher_values_and_balance():
    r = philox.rademacher(7, 50000, 4)
    assert set(np.unique(r)) == {-1.0, 1.0}
    n = r.size
    plus = int(np.sum(r > 0))
    # binomial(n, 1/2): 5 standard deviations
    assert abs(plus - n / 2) < 5 * math.sqrt(n / 4)
    # per column too, and columns / seeds uncorrelated
    both = np.concatenate([r, philox.rademacher(8, 50000, 4)], axis=1)
    c = np.corrcoef(both.T) - np.eye(8)
    assert np.max(np.abs(c)) < 5 / math.sqrt(50000)


def test_rademacher_is_independent_of_the_gaussian_draw():
    """Both come from one Philox block; the sign bit must not track the normal."""
    r = philox.rademacher(11, 40000, 2).ravel()
    g = philox.gaussian(11, 40000, 2).ravel()
    assert abs(np.corrcoef(r, g)[0, 1]) < 5 / math.sqrt(r.size)


@pytest.mark.parametrize("density", [1.0 / 3.0, 0.05, 0.5])
def test_sparse_rademacher_values_density_and_variance(density):
    x = philox.sparse_rademacher(21, 40000, 4, density)
    mag = 1.0 / math.sqrt(density)
    vals = set(np.unique(x))
    assert vals <= {-mag, 0.0, mag} and 0.0 in vals
    n = x.size
    nz = int(np.count_nonzero(x))
    assert abs(nz - density * n) < 5 * math.sqrt(n * density * (1 - density))
    # mean 0, E[x^2] = 1 (exact per-entry variance; sample within 5 sigma)
    assert abs(x.mean()) < 5 * math.sqrt(1.0 / n)
    var4 = 1.0 / density - 1.0  # Var(x^2) = E x^4 - 1
    assert abs(np.mean(x ** 2) - 1.0) < 5 * math.sqrt(var4 / n)
    # signs of the kept entries are the Rademacher signs
    r = philox.rademacher(21, 40000, 4)
    keep = x != 0
    np.testing.assert_array_equal(np.sign(x[keep]), r[keep])


def test_sparse_rademacher_density_one_is_rademacher():
    np.testing.assert_array_equal(philox.sparse_rademacher(3, 500, 6, 1.0),
                                  philox.rademacher(3, 500, 6))
    with pytest.raises(ValueError):
        philox.sparse_threshold(0.0)
    with pytest.raises(ValueError):
        philox.sparse_threshold(1.5)
    assert philox.sparse_threshold(1.0) == 2 ** 32
    assert philox.sparse_threshold(0.25) == 2 ** 30


def test_test_matrix_kinds_and_phi():
    phi = np.linspace(0.5, 2.0, 300)
    for kind in ("rademacher", "sparse_rademacher"):
        om = philox.test_matrix(4, 300, 3, phi, kind=kind, density=0.25)
        assert om.dtype == np.complex128
        np.testing.assert_array_equal(om.imag, 0.0)
        base = (philox.rademacher(4, 300, 3) if kind == "rademacher"
                else philox.sparse_rademacher(4, 300, 3, 0.25))
        np.testing.assert_array_equal(om.real, phi[:, None] * base)
    with pytest.raises(ValueError):
        philox.test_matrix(4, 10, 2, kind="cauchy")


# --------------------------------------------------- orthonormal test matrix
def test_orthonormal_test_matrix_is_the_q_of_the_gaussian():
    phi = np.linspace(0.1, 3.0, 200)
    G = phi[:, None] * philox.gaussian(9, 200, 7)
    Q = rs._householder_q(G.astype(np.complex128))
    np.testing.assert_allclose(Q.conj().T @ Q, np.eye(7), atol=1e-14)
    Rm = Q.conj().T @ G                       # must be the R factor
    np.testing.assert_allclose(np.tril(Rm, -1), 0.0, atol=1e-12)
    assert np.all(np.diag(Rm).real > 0)
    np.testing.assert_allclose(np.diag(Rm).imag, 0.0, atol=1e-12)
    np.testing.assert_allclose(Q @ Rm, G, atol=1e-12)


def test_range_of_omega_decides_the_result():
    """Y = R Omega is orthonormalised, so Omega and its Q factor (same range)
    give the same gains and modes up to rounding."""
    L = _advdiff(12, 10)
    a = rs.randomized(L, 0.5j, 8, 1003)
    b = rs.randomized(L, 0.5j, 8, 1003, kind="orthonormal")
    np.testing.assert_allclose(b.sigma, a.sigma, rtol=1e-10)
    np.testing.assert_allclose(b.sigma_halko, a.sigma_halko, rtol=1e-10)
    assert rs.principal_angle(a.V, b.V) < 1e-8


@pytest.mark.parametrize("kind", ["rademacher", "sparse_rademacher", "orthonormal"])
def test_full_width_sketch_exact_for_every_kind(kind):
    """k = N: any full-rank test matrix spans C^N and Algorithm 1 is exact."""
    L = _advdiff(6, 5)
    n = L.shape[0]
    S, _, _ = rs.exact_svd(L, 0.7j)
    for seed in range(20):  # the first seed whose N x N matrix has full rank
        om = philox.test_matrix(seed, n, n, kind=kind, density=0.5)
        if np.linalg.matrix_rank(om) == n:
            break
    r = rs.randomized(L, 0.7j, n, seed, kind=kind, density=0.5)
    np.testing.assert_allclose(r.sigma, S, rtol=1e-9)


# --------------------------------------------------------- power iterations
@pytest.mark.parametrize("q", [1, 2])
def test_power_iterations_span_the_matrix_power(q):
    """After q subspace iterations, range(Q) = range((R R^H)^q R Omega)."""
    L = _advdiff(8, 6)
    s = 0.5j
    R = _dense_r(L, s)
    k = 4
    om = philox.test_matrix(77, L.shape[0], k)
    M = R @ om
    for _ in range(q):
        M = R @ (R.conj().T @ M)
    r = rs.randomized(L, s, k, 77, power_iters=q)
    assert rs.principal_angle(M, r.Q) < 1e-8


def test_power_iterations_with_weights_follow_the_weighted_operator():
    L = _advdiff(8, 6)
    s = 0.9j
    n = L.shape[0]
    w = np.linspace(0.5, 2.0, n)
    wh = np.sqrt(w)
    R = wh[:, None] * _dense_r(L, s) / wh[None, :]
    om = philox.test_matrix(5, n, 3)
    M = R @ (R.conj().T @ (R @ om))
    r = rs.randomized(L, s, 3, 5, weights=w, power_iters=1)
    assert rs.principal_angle(M, r.Q) < 1e-8


def test_power_iteration_error_bound_and_improvement():
    """Halko, Martinsson & Tropp (SIAM Rev. 2011), Cor. 10.10: with q power
    iterations E||(I - QQ^H) R|| <= [(1 + sqrt(k/(p-1))) s_{k+1}^{2q+1}
    + e sqrt(k+p)/p (sum_{j>k} s_j^{2(2q+1)})^{1/2}]^{1/(2q+1)}; and the seed
    average of the error and of the leading-gain error fall as q grows."""
    L = _advdiff(16, 12)
    s = 0.5j
    S, _, _ = rs.exact_svd(L, s)
    k, p = 6, 2
    means, gain = [], []
    for q in (0, 1, 2):
        e, ge = [], []
        for seed in range(30):
            r = rs.randomized(L, s, k + p, seed, power_iters=q)
            e.append(rs.projection_error(L, s, r.Q))
            ge.append(np.max(np.abs(r.sigma_halko[:k] - S[:k]) / S[:k]))
        e = np.array(e)
        t = 2 * q + 1
        bound = ((1 + math.sqrt(k / (p - 1))) * S[k] ** t
                 + math.e * math.sqrt(k + p) / p * math.sqrt(np.sum(S[k:] ** (2 * t)))) ** (1 / t)
        assert e.mean() <= bound
        assert np.all(e >= S[k + p] * (1 - 1e-9))
        means.append(e.mean())
        gain.append(np.mean(ge))
    assert means[0] > means[1] > means[2]
    assert gain[0] > gain[1] > gain[2]


def test_power_iterations_keep_full_width_exact():
    L = _advdiff(5, 5)
    n = L.shape[0]
    S, _, _ = rs.exact_svd(L, 1.3j)
    r = rs.randomized(L, 1.3j, n, 2, power_iters=1)
    np.testing.assert_allclose(r.sigma, S, rtol=1e-9)
