"""Pins of the oracle's gain gradient (d sum sigma_j^2 / d base flow) against
central finite differences of the exact-SVD objective and against the
closed form of a normal operator."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import gradient as gr
from oracle import operator as op
from oracle import resolvent as rs


def _fd(grid, flow, shifts, J, d, h, weights=None):
    """Central difference, Richardson-extrapolated from steps h and h/2
    (error O(h^4)); the objective is strongly curved near resonances."""
    def shifted(t):
        f = dataclasses.replace(flow, rho=flow.rho + t * d[0], u=flow.u + t * d[1],
                                v=flow.v + t * d[2])
        return gr.objective(grid, f, shifts, J, weights)

    def central(t):
        return (shifted(t) - shifted(-t)) / (2 * t)
    return (4.0 * central(h / 2) - central(h)) / 3.0


def _ns_tiny():
    g = W.ns_grid(6, 5)
    g = dataclasses.replace(g, re=50.0)
    return g, W.smooth_random_flow(g, 3, amp=0.2)


@pytest.mark.parametrize("case", ["advdiff", "ns"])
def test_gradient_matches_central_differences(case):
    if case == "advdiff":
        g = W.Grid(kind=W.KIND_ADVDIFF, nx=7, ny=6, x0=0, x1=10, y0=-5, y1=5, re=20.0)
        flow = W.smooth_random_flow(g, 4, amp=0.3)
    else:
        g, flow = _ns_tiny()
    shifts = [0.4j, 1.3j]
    J = 2
    grad = gr.gain_grad(g, flow, shifts, J)
    if case == "advdiff":
        np.testing.assert_array_equal(grad[0], 0.0)
    rng = np.random.default_rng(11)
    for _ in range(3):
        d = rng.standard_normal((3, g.nx, g.ny))
        if case == "advdiff":
            d[0] = 0.0
        fd = _fd(g, flow, shifts, J, d, 1e-4)
        an = float(np.sum(grad * d))
        assert abs(an - fd) <= 1e-6 * abs(fd)
    # single entries: a rho node and a V node
    for fi, p in ((0, 7), (2, 12)):
        if case == "advdiff" and fi == 0:
            continue
        d = np.zeros((3, g.nx, g.ny))
        d[fi].reshape(-1)[p] = 1.0
        fd = _fd(g, flow, shifts, J, d, 1e-4)
        assert abs(grad[fi].reshape(-1)[p] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(grad).max())


def test_gradient_with_weights_matches_central_differences():
    g, flow = _ns_tiny()
    w = np.linspace(0.5, 2.0, g.n)
    shifts = [0.8j]
    grad = gr.gain_grad(g, flow, shifts, 3, weights=w)
    d = np.random.default_rng(2).standard_normal((3, g.nx, g.ny))
    fd = _fd(g, flow, shifts, 3, d, 1e-4, weights=w)
    assert abs(float(np.sum(grad * d)) - fd) <= 1e-6 * abs(fd)


def test_uniform_v_derivative_closed_form():
    """Periodic-y advection-diffusion with U = 0 and constant V is normal:
    lambda_pq = nu mu_p + nu m_q - i V kappa_q and sigma = 1/|s - lambda|, so
    d sigma^2/dV = -2 (omega + V kappa_q) kappa_q / |s - lambda|^4.  A uniform
    change of V is the sum of the V-gradient over all nodes."""
    vconst, re = 0.8, 5.0
    nu = 1.0 / re
    g = W.Grid(kind=W.KIND_ADVDIFF, nx=5, ny=8, x0=0, x1=2, y0=0, y1=3, re=re,
               periodic_y=True)
    flow = W.zero_flow(g, v_const=vconst)
    om = 1.1
    p = np.arange(1, g.nx + 1)[:, None]
    q = np.arange(g.ny)[None, :]
    mu = -(4 / g.dx ** 2) * np.sin(p * np.pi / (2 * (g.nx + 1))) ** 2
    m = -(4 / g.dy ** 2) * np.sin(np.pi * q / g.ny) ** 2
    kap = np.sin(2 * np.pi * q / g.ny) / g.dy + 0 * p
    re_part = (nu * (mu + m)).ravel()
    kap = kap.ravel()
    mod2 = re_part ** 2 + (om + vconst * kap) ** 2
    sig2 = 1.0 / mod2
    order = np.argsort(-sig2)
    J = 3
    assert sig2[order[J - 1]] > sig2[order[J]] * (1 + 1e-6)  # simple top-J set
    want = float(np.sum((-2 * (om + vconst * kap) * kap / mod2 ** 2)[order[:J]]))
    grad = gr.gain_grad(g, flow, [1j * om], J, fields=("v",))
    assert abs(grad[2].sum() - want) <= 1e-8 * abs(want)
    # and the oracle's objective agrees with the closed form
    assert abs(gr.objective(g, flow, [1j * om], J) - sig2[order[:J]].sum()) < 1e-12 * sig2.sum()


def test_gradient_from_given_triplets_is_phase_invariant():
    g, flow = _ns_tiny()
    L = op.assemble(g, flow)
    s = 0.6j
    S, U, V = rs.exact_svd(L, s)
    ph = np.exp(1j * np.array([0.3, -1.2]))
    a = gr.gain_grad_triplets(g, flow, [s], [(S[:2], U[:, :2], V[:, :2])], 2, fields=("rho",))
    b = gr.gain_grad_triplets(g, flow, [s], [(S[:2], U[:, :2] * ph, V[:, :2] * ph)], 2,
                              fields=("rho",))
    np.testing.assert_allclose(b, a, rtol=1e-10, atol=1e-14 * np.abs(a).max())


def test_gradient_with_neumann_closure_matches_central_differences():
    """Sec. III.A's closure (Neumann rho' at the far field, every variable at
    the outlet): the ghost coefficients fold onto boundary nodes, so the
    gradient's boundary entries change; central differences of the exact
    objective pin them."""
    g, flow = _ns_tiny()
    g = dataclasses.replace(g, neumann=W.PAPER_NEUMANN)
    shifts = [0.6j]
    J = 2
    grad = gr.gain_grad(g, flow, shifts, J)
    rng = np.random.default_rng(17)
    for _ in range(2):
        d = rng.standard_normal((3, g.nx, g.ny))
        fd = _fd(g, flow, shifts, J, d, 1e-4)
        assert abs(float(np.sum(grad * d)) - fd) <= 1e-6 * abs(fd)
    # an outlet node of each field
    for fi in range(3):
        d = np.zeros((3, g.nx, g.ny))
        d[fi, g.nx - 1, 2] = 1.0
        fd = _fd(g, flow, shifts, J, d, 1e-4)
        assert abs(grad[fi, g.nx - 1, 2] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(grad).max())
