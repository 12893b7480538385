"""Pins of the oracle's bi-global operator (Sec. III.A/B: perturbations
(rho', u', v', w') exp(i kz z) about a flow that does not vary in z, W = 0).

* At kz = 0 it is the (rho, u, v) operator plus a decoupled w' equation, and
  w' is then plain advection-diffusion (the pins of that operator carry over).
* Second-order consistency, on the interior rows, with the linearisation of the full
  nonlinear three-dimensional isothermal Navier-Stokes equations derived here
  by symbolic differentiation (sympy): a dropped i kz term, a wrong sign or a
  transposed coupling gives an O(1) error instead of O(h^2).
* The invariants the GPU path relies on: with D = diag(1, 1, 1, i) per point,
  D^{-1} L(kz) D is real, and L(-kz) = conj(L(kz)), so kz and -kz give equal
  gains.
"""
import numpy as np
import pytest

import workloads as W
from oracle import operator as op
from oracle import resolvent as rs

sy = pytest.importorskip("sympy")


def test_kz_zero_reduces_to_the_2d_operator():
    g4 = W.kz_grid(9, 7, 0.0)
    g3 = W.ns_grid(9, 7)
    L4 = op.assemble(g4, W.smooth_random_flow(g4, 3)).toarray()
    L3 = op.assemble(g3, W.smooth_random_flow(g3, 3)).toarray()
    n = L4.shape[0]
    uvw = np.array([i for i in range(n) if i % 4 < 3])
    w = np.array([i for i in range(n) if i % 4 == 3])
    np.testing.assert_array_equal(L4[np.ix_(uvw, uvw)], L3)
    assert np.all(L4[np.ix_(uvw, w)] == 0) and np.all(L4[np.ix_(w, uvw)] == 0)
    # the w' equation is the advection-diffusion operator with its viscous
    # part divided by rho (coefficient 1/(rho Re) instead of 1/Re)
    flow = W.smooth_random_flow(g4, 3)
    bf = W.BaseFlow(rho=flow.rho, u=flow.u, v=flow.v)

    def advdiff(re):
        return op.assemble(W.Grid(kind=W.KIND_ADVDIFF, nx=9, ny=7, x0=0.0, x1=20.0, y0=-5.0,
                                  y1=5.0, re=re, sponge_max=1.0, sponge_frac=0.1), bf).toarray()
    A0 = advdiff(1e300)                    # advection and sponge only
    visc = advdiff(500.0) - A0             # (1/Re) lap
    np.testing.assert_allclose(L4[np.ix_(w, w)], A0 + visc / flow.rho.ravel()[:, None],
                               rtol=1e-12, atol=1e-12)


def _sym_ns3d_linearised(g, R0, U0, V0, r1, u1, v1, w1, x, y, z):
    """Gateaux derivative of the nonlinear 3-D isothermal NS right-hand side at
    (R0, U0, V0, W = 0) in the direction (r1, u1, v1, w1), all symbolic."""
    eps = sy.Symbol("eps")
    c2 = 1 / sy.Float(g.mach) ** 2
    re = sy.Float(g.re)
    rho, u, v, w = R0 + eps * r1, U0 + eps * u1, V0 + eps * v1, eps * w1
    X = (x, y, z)
    vel = (u, v, w)
    div = sum(sy.diff(vel[a], X[a]) for a in range(3))

    def lap(f):
        return sum(sy.diff(f, X[a], 2) for a in range(3))

    cont = -sum(sy.diff(rho * vel[a], X[a]) for a in range(3))
    mom = []
    for a in range(3):
        conv = -sum(vel[bb] * sy.diff(vel[a], X[bb]) for bb in range(3))
        mom.append(conv - c2 / rho * sy.diff(rho, X[a])
                   + (lap(vel[a]) + sy.diff(div, X[a]) / 3) / (rho * re))
    return [sy.diff(f, eps).subs(eps, 0) for f in [cont] + mom]


def _kz_consistency_error(nx, ny, kz):
    # a low Reynolds number keeps the viscous kz terms as large as the others
    g = W.Grid(kind=W.KIND_NS2D_KZ, nx=nx, ny=ny, x0=0.0, x1=4.0, y0=-1.5, y1=1.5,
               re=2.0, mach=0.5, kz=kz)
    x, y, z = sy.symbols("x y z", real=True)
    R0 = 1 + sy.Rational(1, 5) * sy.sin(x / 2) * sy.cos(3 * y / 5)
    U0 = sy.tanh(2 * y) + sy.Rational(1, 10) * sy.cos(x / 3)
    V0 = sy.Rational(1, 10) * sy.sin(2 * x / 5) * sy.sin(y)
    bump = sy.sin(sy.pi * x / 4) * sy.sin(sy.pi * (y + sy.Rational(3, 2)) / 3)
    ez = sy.exp(sy.I * sy.Float(kz) * z)
    hats = [bump * sy.cos(4 * x / 5), bump * sy.sin(y / 2 + sy.Rational(3, 10)),
            bump * sy.cos(2 * x / 5 + y / 5), bump * sy.sin(3 * x / 7 - y / 3)]
    lin = _sym_ns3d_linearised(g, R0, U0, V0, *[h * ez for h in hats], x, y, z)
    # every term carries exp(i kz z): its coefficient is the value at z = 0
    lin = [e.subs(z, 0) for e in lin]
    X, Y = g.mesh()

    def f(e):
        val = sy.lambdify((x, y), e, "numpy")(X, Y)
        return np.broadcast_to(val, X.shape).astype(np.complex128)
    flow = W.BaseFlow(rho=f(R0).real, u=f(U0).real, v=f(V0).real)
    qp = np.stack([f(h) for h in hats], axis=-1).ravel()
    got = (op.assemble(g, flow) @ qp).reshape(nx, ny, 4)
    want = np.stack([f(e) for e in lin], axis=-1)
    inner = (slice(2, nx - 2), slice(2, ny - 2))
    return np.max(np.abs(got[inner] - want[inner])), np.max(np.abs(want))


@pytest.mark.parametrize("kz", [0.7, 3.0])
def test_kz_operator_is_second_order_consistent(kz):
    e1, scale = _kz_consistency_error(24, 20, kz)
    e2, _ = _kz_consistency_error(48, 40, kz)
    assert e1 < 0.05 * scale
    assert 3.2 < e1 / e2 < 5.0, (e1, e2)


def test_kz_similarity_to_a_real_operator_and_conjugation():
    g = W.kz_grid(7, 6, 1.3, neumann=(1, 15, 9, 9))
    flow = W.smooth_random_flow(g, 4)
    L = op.assemble(g, flow).toarray()
    d = np.tile([1, 1, 1, 1j], g.npts)
    Lt = (L * d[None, :]) / d[:, None]
    assert np.abs(Lt.imag).max() == 0.0
    assert np.abs(Lt.real).max() > 0
    gm = W.kz_grid(7, 6, -1.3, neumann=(1, 15, 9, 9))
    Lm = op.assemble(gm, flow).toarray()
    np.testing.assert_array_equal(Lm, np.conj(L))
    S1, _, _ = rs.exact_svd(op.assemble(g, flow), 0.8j)
    S2, _, _ = rs.exact_svd(op.assemble(gm, flow), 0.8j)
    np.testing.assert_allclose(S1, S2, rtol=1e-10)
