"""GPU parity of the gain gradient rr_gain_grad and of its autograd wrapper.

1. Kernel parity: the oracle's exact singular triplets are fed to the CUDA
   path, so both sides evaluate sum 2 sigma_j Re(a_j^H dL b_j) for the same
   (u_j, sigma_j, v_j); the CUDA path differentiates the stencil formulas by
   hand, the oracle differentiates the assembled matrix numerically (five-
   point, error ~1e-10 relative).  Bar: 1e-8 of the largest entry.
2. End to end: the CUDA path's own randomized triplets (with subspace
   iterations) against the oracle's exact-triplet gradient (1e-5), and the
   autograd gradient against central finite differences (h = 1e-6) of the
   CUDA objective on random base-flow directions (1e-5 relative), the check
   the gradient workload asks for.
"""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import gradient as gr
from oracle import operator as op
from oracle import resolvent as rs
from tests.gpu_util import lib, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    return torch, lib()


def _cases():
    ns = dataclasses.replace(W.ns_grid(7, 6), re=50.0)
    ad = W.Grid(kind=W.KIND_ADVDIFF, nx=8, ny=7, x0=0, x1=10, y0=-5, y1=5, re=20.0)
    per = W.Grid(kind=W.KIND_ADVDIFF, nx=6, ny=5, x0=0, x1=2, y0=0, y1=3, re=5.0,
                 periodic_y=True)
    nsp = dataclasses.replace(W.ns_grid(6, 4), re=80.0, periodic_y=True, sponge_max=0.0)
    nsn = dataclasses.replace(W.ns_grid(7, 6, neumann=W.PAPER_NEUMANN), re=50.0)
    adn = dataclasses.replace(ad, neumann=(1, 1, 0, 1))
    return [("ns", ns, W.smooth_random_flow(ns, 3, amp=0.2), None),
            ("ns-neumann", nsn, W.smooth_random_flow(nsn, 8, amp=0.2), None),
            ("advdiff-neumann", adn, W.smooth_random_flow(adn, 9, amp=0.3), None),
            ("ns-weighted", ns, W.smooth_random_flow(ns, 4, amp=0.2), "w"),
            ("ns-periodic", nsp, W.smooth_random_flow(nsp, 6, amp=0.2), None),
            ("advdiff", ad, W.smooth_random_flow(ad, 5, amp=0.3), None),
            ("advdiff-periodic", per, W.smooth_random_flow(per, 7, amp=0.3), None)]


@pytest.mark.parametrize("name,g,flow,wkind", _cases())
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gradient_kernel_matches_oracle_on_exact_triplets(env, name, g, flow, wkind,
                                                           precision):
    torch, rr = env
    L = op.assemble(g, flow)
    w = np.linspace(0.5, 2.0, L.shape[0]) if wkind else None
    shifts = [0.5j, 1.7j]
    J = 3
    trip = []
    for s in shifts:
        S, U, V = rs.exact_svd(L, s, w)
        trip.append((S[:J], U[:, :J], V[:, :J]))
    want = gr.gain_grad_triplets(g, flow, shifts, trip, J, w)
    o = rr.Operator(g, flow, weights=w)
    fa = o.factor(shifts, precision)
    Ud = to_dev(np.stack([t[1] for t in trip]), torch)
    Vd = to_dev(np.stack([t[2] for t in trip]), torch)
    sd = to_dev(np.stack([t[0] for t in trip]), torch)
    grad, info = fa.gain_grad(J, Ud, Vd, sd)
    got = grad.cpu().numpy()
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-8 * scale, name
    if g.kind == W.KIND_ADVDIFF:
        np.testing.assert_array_equal(got[0], 0.0)
    # accumulation: a second call adds the same amount
    fa.gain_grad(J, Ud, Vd, sd, grad)
    assert np.abs(grad.cpu().numpy() - 2 * got).max() <= 1e-12 * scale


def test_gradient_from_gpu_triplets_matches_exact_gradient(env):
    """Randomized triplets with subspace iterations carry the exact gradient."""
    torch, rr = env
    g = dataclasses.replace(W.ns_grid(12, 10), re=100.0)
    flow = W.smooth_random_flow(g, 8, amp=0.1)
    shifts = [0.6j, 1.4j]
    J = 3
    want = gr.gain_grad(g, flow, shifts, J)
    o = rr.Operator(g, flow)
    fa = o.factor(shifts, "fp64")
    res = fa.randomized_resolvent(16, [11, 12], power_iters=2)
    grad, _ = fa.gain_grad(J, res.U, res.V, res.sigma)
    got = grad.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()


def test_gain_grad_argument_errors(env):
    torch, rr = env
    g = W.ns_grid(6, 5)
    flow = W.shear_bubble_flow(g)
    o = rr.Operator(g, flow)
    fa = o.factor([0.5j], "fp64")
    U = torch.zeros(1, o.n, 4, dtype=torch.complex128, device="cuda:0")
    s = torch.ones(1, 4, dtype=torch.float64, device="cuda:0")
    for J in (0, 5):
        with pytest.raises(rr.RRError) as e:
            fa.gain_grad(J, U, U.clone(), s)
        assert e.value.status == 1


def test_autograd_matches_finite_differences(env):
    """The gradient workload's check at a reduced grid: 64 random base-flow
    directions, central differences with h = 1e-6 of the CUDA objective
    (Algorithm 1 with two subspace iterations, FP64 factors), factors
    recomputed per chunk of 4 frequencies in the backward pass."""
    torch, rr = env
    from paper_1902_01458_gb300.autograd import gain_objective
    g = dataclasses.replace(W.ns_grid(16, 12), re=100.0)
    base = W.smooth_random_flow(g, 2, amp=0.1)
    omegas = W.log_omegas(6, 0.3, 3.0)
    seeds = [1000 + i for i in range(6)]
    kw = dict(grid=g, omegas=omegas, k=16, J=3, seeds=seeds, chunk=4, precision="fp64",
              power_iters=2)
    fields = [torch.tensor(a, dtype=torch.float64, requires_grad=True)
              for a in (base.rho, base.u, base.v)]
    val = gain_objective(*fields, **kw)
    val.backward()
    grad = np.stack([f.grad.numpy() for f in fields])
    want = gr.gain_grad(g, base, 1j * omegas, 3)
    assert np.abs(grad - want).max() <= 1e-5 * np.abs(want).max()
    rng = np.random.default_rng(5)
    h = 1e-6
    an, fd = [], []
    for _ in range(64):
        d = rng.standard_normal((3, g.nx, g.ny))

        def at(t):
            with torch.no_grad():
                f = [torch.tensor(a + t * dd) for a, dd in zip((base.rho, base.u, base.v), d)]
                return float(gain_objective(*f, **kw))
        fd.append((at(h) - at(-h)) / (2 * h))
        an.append(float(np.sum(grad * d)))
    an, fd = np.array(an), np.array(fd)
    # a random direction can be nearly orthogonal to the gradient, so the
    # error is measured against the rms directional derivative
    scale = np.sqrt(np.mean(fd ** 2))
    assert np.max(np.abs(an - fd)) <= 1e-5 * scale
    assert np.median(np.abs(an - fd) / np.abs(fd)) <= 1e-6
