"""GPU parity of the wide FP32 factorisation (two-level Gauss-Jordan with
implicit pivoting: 16-column register-resident panels, rank-16 updates of the
128-column slab, rank-128 tensor-core updates of the rest) in its three
operand splits (TF32 x3, BF16 x3, BF16 x6), through the solves it serves.

Checked against the oracle's dense LU solve of s I - L on the same inputs:
* after FP64 refinement the solution to 1e-9 relative (the FP32 factors'
  bar), normal and adjoint;
* the first, unrefined solve to the accuracy its split allows (the factors
  are a correct inverse, not merely a usable preconditioner): 1e-4 relative
  for TF32 x3 and BF16 x6 (FP32-level products), 5e-2 for BF16 x3;
* Algorithm 1 end to end on one case per split (sigma 1e-6, subspaces 1e-5).
Block sizes cover one slab with a ragged row tile (b = 72, 144), several
slabs with a ragged last slab and column tile (b = 264), and exact tiles
(b = 384).
"""
import numpy as np
import pytest

import workloads as W
from oracle import operator as op
from oracle import resolvent as rs
from tests.gpu_util import lib, rel_err, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

SPLITS = [("fp32", 1e-4), ("fp32_bf16x6", 1e-4), ("fp32_bf16x3", 5e-2)]
SHAPES = [(4, 24), (3, 48), (3, 88), (3, 128)]


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    return torch, lib()


@pytest.mark.parametrize("nx,ny", SHAPES)
@pytest.mark.parametrize("precision,first_tol", SPLITS)
@pytest.mark.parametrize("adjoint", [False, True])
def test_wide_factor_solves_match_oracle(env, nx, ny, precision, first_tol, adjoint):
    torch, rr = env
    g = W.ns_grid(nx, ny)
    flow = W.smooth_random_flow(g, 11)
    L = op.assemble(g, flow)
    o = rr.Operator(g, flow)
    shifts = np.array([0.4j, 0.05 + 2.3j])
    fa = o.factor(shifts, precision)
    rng = np.random.default_rng(nx * 1000 + ny)
    k = 6
    b = rng.standard_normal((2, o.n, k)) + 1j * rng.standard_normal((2, o.n, k))
    bd = to_dev(b, torch)
    x0, _ = fa.solve(bd, adjoint, refine_tol=0.0, max_refine=0, check=False)
    x, info = fa.solve(bd, adjoint)
    x0, x = x0.cpu().numpy(), x.cpu().numpy()
    for f, s in enumerate(shifts):
        A = op.shifted(L, s).toarray()
        want = np.linalg.solve(A.conj().T if adjoint else A, b[f])
        assert rel_err(x0[f], want) < first_tol, (f, rel_err(x0[f], want))
        assert rel_err(x[f], want) < 1e-9, (f, rel_err(x[f], want))
    fa.close()


@pytest.mark.parametrize("precision", [p for p, _ in SPLITS])
def test_wide_factor_algorithm1_matches_oracle(env, precision):
    torch, rr = env
    wl = W.config_small_ns(6, 64, k=8, nfreq=2)
    g, flow = wl.grid, wl.flow
    L = op.assemble(g, flow)
    phi = op.phi(g, flow)
    o = rr.Operator(g, flow)
    shifts = 1j * wl.omegas
    seeds = [wl.seed0 + i for i in range(len(shifts))]
    fa = o.factor(shifts, precision)
    res = fa.randomized_resolvent(wl.k, seeds, phi=to_dev(phi, torch))
    for f, s in enumerate(shifts):
        ref = rs.randomized(L, s, wl.k, seeds[f], phi=phi)
        np.testing.assert_allclose(res.sigma.cpu().numpy()[f], ref.sigma, rtol=1e-6)
        np.testing.assert_allclose(res.sigma_halko.cpu().numpy()[f], ref.sigma_halko, rtol=1e-6)
        assert rs.principal_angle(res.V.cpu().numpy()[f], ref.V) < 1e-5
        assert rs.principal_angle(res.U.cpu().numpy()[f], ref.U) < 1e-5
    fa.close()


def test_refinement_runs_per_problem(env):
    """Refinement on the tensor-core sweep path runs each problem on its own: a
    problem whose right-hand side is zero is solved exactly by the first
    sweep and takes no correction, while the other problem's corrections run
    alone.  Block solves counted: 2 first solves + one per correction of
    problem 0 (all-problem refinement would count 2 per correction)."""
    torch, rr = env
    g = W.ns_grid(3, 64)  # block 192: wide factorisation, tensor-core sweeps
    flow = W.smooth_random_flow(g, 5)
    L = op.assemble(g, flow)
    o = rr.Operator(g, flow)
    shifts = np.array([0.3j, 1.1j])
    fa = o.factor(shifts, "fp32")
    rng = np.random.default_rng(17)
    b = rng.standard_normal((2, o.n, 8)) + 1j * rng.standard_normal((2, o.n, 8))
    b[1] = 0.0
    x, info = fa.solve(to_dev(b, torch), False)
    x = x.cpu().numpy()
    assert info["refine_iters"] >= 1
    assert info["problem_solves"] == 2 + info["refine_iters"], info
    want = np.linalg.solve(op.shifted(L, shifts[0]).toarray(), b[0])
    assert rel_err(x[0], want) < 1e-9
    assert np.all(x[1] == 0)
    fa.close()
