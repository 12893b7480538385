"""Pins of the oracle's operator assembly (Sec. II.A, Eq. 1) and of Phi (Eq. 9).

Each pin is fixed by something other than the oracle itself:
  * the closed-form spectrum of Dirichlet diffusion (normal, symmetric) and of
    periodic advection-diffusion (normal, complex eigenvalues): sigma_j of the
    resolvent is exactly 1/|s - lambda_j|;
  * second-order consistency of the discrete operator with the linearisation
    of the full nonlinear isothermal Navier-Stokes equations, derived here by
    symbolic differentiation (sympy), so a dropped term, a wrong sign or a
    transposed coupling gives an O(1) error instead of O(h^2);
  * the sponge profile at chosen depths, and Phi against the analytic
    velocity-gradient norm.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import operator as op
from oracle import resolvent as rs

sy = pytest.importorskip("sympy")


def _diffusion_eigs(g, nu):
    p = np.arange(1, g.nx + 1)[:, None]
    q = np.arange(1, g.ny + 1)[None, :]
    return -nu * ((4 / g.dx ** 2) * np.sin(p * np.pi / (2 * (g.nx + 1))) ** 2
                  + (4 / g.dy ** 2) * np.sin(q * np.pi / (2 * (g.ny + 1))) ** 2)


def test_dirichlet_diffusion_closed_form():
    g = W.Grid(kind=W.KIND_ADVDIFF, nx=12, ny=9, x0=0, x1=3, y0=-1, y1=1,
               re=2.0)
    L = op.assemble(g, W.zero_flow(g))
    lam = _diffusion_eigs(g, 0.5).ravel()
    for s in (0.7j, 0.3 + 2.0j, -1.5j):
        sig = np.sort(1.0 / np.abs(s - lam))[::-1]
        S, U, V = rs.exact_svd(L, s)
        np.testing.assert_allclose(S, sig, rtol=1e-12)
        # leading mode = product of first sines (simple eigenvalue)
        x = np.sin(np.pi * np.arange(1, g.nx + 1) / (g.nx + 1))
        y = np.sin(np.pi * np.arange(1, g.ny + 1) / (g.ny + 1))
        e = np.outer(x, y).ravel()
        assert rs.cosine_similarity(V[:, 0], e) > 1 - 1e-12
        assert rs.cosine_similarity(U[:, 0], e) > 1 - 1e-12


def test_periodic_advection_diffusion_closed_form():
    vconst, re = 0.8, 5.0
    nu = 1.0 / re
    g = W.Grid(kind=W.KIND_ADVDIFF, nx=7, ny=10, x0=0, x1=2, y0=0, y1=3,
               re=re, periodic_y=True)
    L = op.assemble(g, W.zero_flow(g, v_const=vconst))
    p = np.arange(1, g.nx + 1)[:, None]
    q = np.arange(g.ny)[None, :]
    mu = -nu * (4 / g.dx ** 2) * np.sin(p * np.pi / (2 * (g.nx + 1))) ** 2
    kap = (-1j * vconst * np.sin(2 * np.pi * q / g.ny) / g.dy
           - nu * (4 / g.dy ** 2) * np.sin(np.pi * q / g.ny) ** 2)
    lam = (mu + kap).ravel()
    # L is normal: the eigenvalues match and sigma = 1/|s - lambda|
    ev = np.linalg.eigvals(L.toarray())
    from scipy.optimize import linear_sum_assignment
    r, c = linear_sum_assignment(np.abs(ev[:, None] - lam[None, :]))
    assert np.max(np.abs(ev[r] - lam[c])) < 1e-10
    s = 1.1j
    S, _, _ = rs.exact_svd(L, s)
    np.testing.assert_allclose(S, np.sort(1 / np.abs(s - lam))[::-1],
                               rtol=1e-11)


def _sym_ns_linearised(g, R0, U0, V0, r1, u1, v1, x, y):
    """Gateaux derivative of the nonlinear isothermal NS right-hand side."""
    eps = sy.Symbol("eps")
    c2 = 1 / sy.Float(g.mach) ** 2
    re = sy.Float(g.re)
    rho, u, v = R0 + eps * r1, U0 + eps * u1, V0 + eps * v1
    div = sy.diff(u, x) + sy.diff(v, y)
    cont = -sy.diff(rho * u, x) - sy.diff(rho * v, y)
    mx = (-(u * sy.diff(u, x) + v * sy.diff(u, y)) - c2 / rho * sy.diff(rho, x)
          + (sy.diff(u, x, 2) + sy.diff(u, y, 2) + sy.diff(div, x) / 3)
          / (rho * re))
    my = (-(u * sy.diff(v, x) + v * sy.diff(v, y)) - c2 / rho * sy.diff(rho, y)
          + (sy.diff(v, x, 2) + sy.diff(v, y, 2) + sy.diff(div, y) / 3)
          / (rho * re))
    return [sy.diff(f, eps).subs(eps, 0) for f in (cont, mx, my)]


def _ns_consistency_error(nx, ny):
    g = W.Grid(kind=W.KIND_NS2D, nx=nx, ny=ny, x0=0.0, x1=4.0, y0=-1.5,
               y1=1.5, re=50.0, mach=0.5)
    x, y = sy.symbols("x y", real=True)
    R0 = 1 + sy.Rational(1, 5) * sy.sin(x / 2) * sy.cos(3 * y / 5)
    U0 = sy.tanh(2 * y) + sy.Rational(1, 10) * sy.cos(x / 3)
    V0 = sy.Rational(1, 10) * sy.sin(2 * x / 5) * sy.sin(y)
    bump = sy.sin(sy.pi * x / 4) * sy.sin(sy.pi * (y + sy.Rational(3, 2)) / 3)
    r1 = bump * sy.cos(4 * x / 5)
    u1 = bump * sy.sin(y / 2 + sy.Rational(3, 10))
    v1 = bump * sy.cos(2 * x / 5 + y / 5)
    lin = _sym_ns_linearised(g, R0, U0, V0, r1, u1, v1, x, y)
    X, Y = g.mesh()
    f = lambda e: np.broadcast_to(sy.lambdify((x, y), e, "numpy")(X, Y),
                                  X.shape).astype(float)
    flow = W.BaseFlow(rho=f(R0), u=f(U0), v=f(V0))
    qp = np.stack([f(r1), f(u1), f(v1)], axis=-1).ravel()
    L = op.assemble(g, flow)
    got = (L @ qp).reshape(nx, ny, 3)
    want = np.stack([f(e) for e in lin], axis=-1)
    inner = (slice(2, nx - 2), slice(2, ny - 2))
    return np.max(np.abs(got[inner] - want[inner])), np.max(np.abs(want))


def test_ns_operator_is_second_order_consistent():
    e1, scale = _ns_consistency_error(24, 20)
    e2, _ = _ns_consistency_error(48, 40)
    assert e1 < 0.05 * scale
    ratio = e1 / e2
    assert 3.2 < ratio < 5.0, (e1, e2, ratio)


def _ns_boundary_consistency_error(nx, ny):
    """Consistency on every row, boundary rows included.  A bilinear base
    flow makes the base-flow differences exact at every node (one-sided first
    differences at the ends are exact on linear fields, the re-centred second
    differences on quadratics), and perturbations that vanish at the ghost
    nodes make the Dirichlet closure exact, so the first and last rows must
    converge at second order like the interior ones."""
    g = W.Grid(kind=W.KIND_NS2D, nx=nx, ny=ny, x0=0.0, x1=4.0, y0=-1.5,
               y1=1.5, re=50.0, mach=0.5)
    x, y = sy.symbols("x y", real=True)
    R0 = 1 + 3 * x / 10 + y / 10 + x * y / 20
    U0 = sy.Rational(1, 2) + 2 * x / 5 - 3 * y / 10 - x * y / 10
    V0 = sy.Rational(1, 5) - 3 * x / 10 + y / 5 + x * y / 10
    bump = sy.sin(sy.pi * x / 4) * sy.sin(sy.pi * (y + sy.Rational(3, 2)) / 3)
    r1 = bump * sy.cos(4 * x / 5)
    u1 = bump * sy.sin(y / 2 + sy.Rational(3, 10))
    v1 = bump * sy.cos(2 * x / 5 + y / 5)
    lin = _sym_ns_linearised(g, R0, U0, V0, r1, u1, v1, x, y)
    X, Y = g.mesh()
    f = lambda e: np.broadcast_to(sy.lambdify((x, y), e, "numpy")(X, Y),
                                  X.shape).astype(float)
    flow = W.BaseFlow(rho=f(R0), u=f(U0), v=f(V0))
    qp = np.stack([f(r1), f(u1), f(v1)], axis=-1).ravel()
    got = (op.assemble(g, flow) @ qp).reshape(nx, ny, 3)
    want = np.stack([f(e) for e in lin], axis=-1)
    err = np.abs(got - want)
    edge = np.zeros((nx, ny), dtype=bool)
    edge[[0, -1], :] = True
    edge[:, [0, -1]] = True
    return np.max(err[edge]), np.max(err), np.max(np.abs(want))


def test_ns_boundary_rows_are_second_order_consistent():
    e1, a1, scale = _ns_boundary_consistency_error(24, 20)
    e2, a2, _ = _ns_boundary_consistency_error(48, 40)
    assert a1 < 0.05 * scale
    assert 3.2 < e1 / e2 < 5.0, (e1, e2)
    assert 3.2 < a1 / a2 < 5.0, (a1, a2)


def test_field_differences_exact_on_polynomials_at_every_node():
    """The base-flow differences, end nodes included: the one-sided first
    difference is exact on linear fields, the re-centred second difference on
    quadratics, the cross difference on bilinear fields."""
    g = W.ns_grid(9, 7)
    X, Y = g.mesh()
    lin = 0.3 + 1.7 * X - 0.9 * Y
    d = op.field_derivatives(g, lin)
    np.testing.assert_allclose(d["x"], 1.7, rtol=1e-12)
    np.testing.assert_allclose(d["y"], -0.9, rtol=1e-12)
    quad = 0.5 - 0.4 * X + 2.5 * X ** 2 + 0.7 * Y - 1.3 * Y ** 2
    d = op.field_derivatives(g, quad)
    np.testing.assert_allclose(d["xx"], 5.0, rtol=1e-10)
    np.testing.assert_allclose(d["yy"], -2.6, rtol=1e-10)
    bil = 0.2 + X - 0.5 * Y + 0.25 * X * Y
    d = op.field_derivatives(g, bil)
    np.testing.assert_allclose(d["xy"], 0.25, rtol=1e-12)
    np.testing.assert_allclose(d["x"], 1 + 0.25 * Y, rtol=1e-12)
    # a periodic direction: central differences wrap around
    gp = W.Grid(kind=W.KIND_ADVDIFF, nx=5, ny=16, x0=0, x1=1, y0=0, y1=2 * np.pi,
                re=1.0, periodic_y=True)
    _, Yp = gp.mesh()
    dp = op.field_derivatives(gp, np.sin(Yp))
    h = gp.dy
    np.testing.assert_allclose(dp["y"], np.cos(Yp) * np.sin(h) / h, rtol=1e-12, atol=1e-14)


def _advdiff_consistency_error(nx, ny):
    g = W.Grid(kind=W.KIND_ADVDIFF, nx=nx, ny=ny, x0=0.0, x1=10.0, y0=-5.0,
               y1=5.0, re=100.0)
    x, y = sy.symbols("x y", real=True)
    U0 = sy.tanh(y)
    V0 = sy.Rational(1, 5) * sy.sin(x / 3)
    ph = sy.sin(sy.pi * x / 10) * sy.sin(sy.pi * (y + 5) / 10) * sy.cos(x / 2)
    want_e = (-U0 * sy.diff(ph, x) - V0 * sy.diff(ph, y)
              + (sy.diff(ph, x, 2) + sy.diff(ph, y, 2)) / 100)
    X, Y = g.mesh()
    f = lambda e: np.broadcast_to(sy.lambdify((x, y), e, "numpy")(X, Y),
                                  X.shape).astype(float)
    L = op.assemble(g, W.BaseFlow(rho=np.ones_like(X), u=f(U0), v=f(V0)))
    got = (L @ f(ph).ravel()).reshape(nx, ny)
    return np.max(np.abs(got - f(want_e)))


def test_advdiff_operator_is_second_order_consistent():
    e1 = _advdiff_consistency_error(32, 32)
    e2 = _advdiff_consistency_error(64, 64)
    assert 3.2 < e1 / e2 < 5.0


def test_sponge_profile():
    g = W.Grid(kind=W.KIND_ADVDIFF, nx=99, ny=49, x0=0.0, x1=20.0, y0=-5.0,
               y1=5.0, re=1e30, sponge_max=1.0, sponge_frac=0.1)
    s = op.sponge(g)
    X, Y = g.mesh()
    # node at x = 0.2 * 5 = 1.0: depth (2 - 1)/2 = 0.5 -> 0.25 (y in the core)
    i = int(np.argmin(np.abs(X[:, 0] - 1.0)))
    j = int(np.argmin(np.abs(Y[0, :] - 0.0)))
    assert math.isclose(X[i, 0], 1.0) and math.isclose(Y[0, j], 0.0, abs_tol=1e-12)
    assert math.isclose(s[i, j], 0.25, rel_tol=1e-12)
    # core of the domain: no sponge; corners take the larger of the two layers
    assert s[49, 24] == 0.0
    assert s[0, 0] == pytest.approx(max(((2 - X[0, 0]) / 2) ** 2,
                                        ((Y[0, 0] + 4) / 1) ** 2))
    # the assembled diagonal carries -s_s (advection/diffusion vanish here)
    L = op.assemble(g, W.zero_flow(g))
    np.testing.assert_allclose(-L.diagonal().reshape(99, 49) - s,
                               2 / 1e30 * (1 / g.dx ** 2 + 1 / g.dy ** 2),
                               atol=1e-14)


def _phi_error(nx, ny):
    g = W.ns_grid(nx, ny)
    X, Y = g.mesh()
    u = np.tanh(Y) + 0.1 * np.sin(0.3 * X)
    v = 0.2 * np.cos(0.5 * X) * np.sin(0.4 * Y)
    want = np.sqrt((0.03 * np.cos(0.3 * X)) ** 2 + (1 - np.tanh(Y) ** 2) ** 2
                   + (-0.1 * np.sin(0.5 * X) * np.sin(0.4 * Y)) ** 2
                   + (0.08 * np.cos(0.5 * X) * np.cos(0.4 * Y)) ** 2)
    ph = op.phi(g, W.BaseFlow(rho=np.ones_like(X), u=u, v=v))
    ph = ph.reshape(nx, ny, 3)
    assert np.all(ph[..., 0] == ph[..., 1]) and np.all(ph[..., 0] == ph[..., 2])
    return np.max(np.abs(ph[1:-1, 1:-1, 0] - want[1:-1, 1:-1]))


def test_phi_is_velocity_gradient_norm():
    """Eq. (9): Phi converges to the analytic ||grad v|| at second order."""
    e1 = _phi_error(80, 60)
    e2 = _phi_error(160, 120)
    assert e1 < 2e-2
    assert 3.2 < e1 / e2 < 5.0


def test_shift_conjugation_gives_equal_gains():
    """For real L, (conj(s) I - L) = conj(s I - L): equal sigma (reading of the
    paper's -i omega convention vs i omega)."""
    wl = W.config_small_ns(10, 8)
    L = op.assemble(wl.grid, wl.flow)
    S1, _, _ = rs.exact_svd(L, 0.9j)
    S2, _, _ = rs.exact_svd(L, -0.9j)
    np.testing.assert_allclose(S1, S2, rtol=1e-10)


def test_ns_block_structure():
    """Couplings reach only the neighbouring streamwise column: block-tridiagonal."""
    wl = W.config_small_ns(9, 7)
    g = wl.grid
    L = op.assemble(g, W.smooth_random_flow(g, 3)).tocoo()
    col_r = L.row // g.b
    col_c = L.col // g.b
    assert np.max(np.abs(col_r - col_c)) == 1
    assert np.max(np.bincount(L.row)) <= 27
