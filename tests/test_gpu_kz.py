"""GPU parity of the bi-global operator (Sec. III.A/B: perturbations
(rho', u', v', w') exp(i kz z) about a z-invariant flow with no spanwise
velocity), through the C ABI, against the oracle's complex L(kz).

The library factors and sweeps the real operator D^{-1} L D (D = diag(1, 1,
1, i) per point) and conjugates by D at its boundary, so every result must
match the oracle's complex operator directly: its application (1e-13), the
solves (FP64 1e-11; FP32 factors with refinement 1e-9), and Algorithm 1 end
to end (sigma and sigma_halko 1e-9 FP64, 1e-6 FP32; mode subspaces 1e-5 and
the phase convention), at the paper's spanwise wavenumber k_z L_c = 20 pi
scaled to the domain and at a small one.
"""
import numpy as np
import pytest

import workloads as W
from oracle import operator as op
from oracle import resolvent as rs
from tests.gpu_util import lib, rel_err, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

KZ = [0.8, 2.0 * np.pi]


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    return torch, lib()


@pytest.mark.parametrize("kz", KZ)
@pytest.mark.parametrize("adjoint", [False, True])
def test_kz_apply_matches_oracle(env, kz, adjoint):
    torch, rr = env
    g = W.kz_grid(11, 9, kz, neumann=(1, 15, 1, 1))
    flow = W.smooth_random_flow(g, 6)
    L = op.assemble(g, flow)
    o = rr.Operator(g, flow)
    assert (o.q, o.b) == (4, 36)
    rng = np.random.default_rng(8)
    shifts = np.array([0.6j, 0.1 + 1.7j])
    x = rng.standard_normal((2, o.n, 5)) + 1j * rng.standard_normal((2, o.n, 5))
    y = o.apply(shifts, to_dev(x, torch), adjoint).cpu().numpy()
    for f, s in enumerate(shifts):
        A = op.shifted(L, s)
        want = (A.conj().T if adjoint else A) @ x[f]
        assert rel_err(y[f], want) < 1e-13


@pytest.mark.parametrize("kz", KZ)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 1e-9)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_kz_solve_matches_oracle(env, kz, precision, tol, adjoint):
    torch, rr = env
    # block 4 * 40 = 160: the wide tensor-core factorisation and sweeps in FP32
    g = W.kz_grid(6, 40, kz)
    flow = W.smooth_random_flow(g, 2)
    L = op.assemble(g, flow)
    o = rr.Operator(g, flow)
    shifts = np.array([0.5j, 2.2j])
    fa = o.factor(shifts, precision)
    rng = np.random.default_rng(3)
    b = rng.standard_normal((2, o.n, 6)) + 1j * rng.standard_normal((2, o.n, 6))
    x, _ = fa.solve(to_dev(b, torch), adjoint)
    x = x.cpu().numpy()
    for f, s in enumerate(shifts):
        A = op.shifted(L, s).toarray()
        want = np.linalg.solve(A.conj().T if adjoint else A, b[f])
        assert rel_err(x[f], want) < tol
    fa.close()


@pytest.mark.parametrize("kz", KZ)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-6)])
def test_kz_algorithm1_matches_oracle(env, kz, precision, tol):
    torch, rr = env
    g = W.kz_grid(10, 32, kz)
    flow = W.shear_bubble_flow(g)
    L = op.assemble(g, flow)
    phi = op.phi(g, flow)
    o = rr.Operator(g, flow)
    shifts = 1j * np.array([0.4, 1.9])
    seeds = [1000, 1001]
    fa = o.factor(shifts, precision)
    res = fa.randomized_resolvent(8, seeds, phi=to_dev(phi, torch))
    for f, s in enumerate(shifts):
        ref = rs.randomized(L, s, 8, seeds[f], phi=phi)
        np.testing.assert_allclose(res.sigma.cpu().numpy()[f], ref.sigma, rtol=tol)
        np.testing.assert_allclose(res.sigma_halko.cpu().numpy()[f], ref.sigma_halko, rtol=tol)
        V, U = res.V.cpu().numpy()[f], res.U.cpu().numpy()[f]
        assert rs.principal_angle(V, ref.V) < 1e-5
        assert rs.principal_angle(U, ref.U) < 1e-5
        # phase convention on the vectors of L itself: the largest entry of
        # each v_j is real and positive
        for j in range(8):
            i = int(np.argmax(np.abs(V[:, j])))
            assert abs(V[i, j].imag) < 1e-12 * abs(V[i, j]) and V[i, j].real > 0
    fa.close()


def test_kz_unsupported_calls(env):
    torch, rr = env
    from paper_1902_01458_gb300 import _lib
    g = W.kz_grid(5, 6, 1.0)
    o = rr.Operator(g, W.shear_bubble_flow(g))
    x = torch.zeros(1, o.n, 1, dtype=torch.complex128, device="cuda:0")
    y = torch.zeros_like(x)
    with pytest.raises(rr.RRError) as e:
        _lib.rr_apply_static(o.handle, [1j], x, y)
    assert e.value.status == 8
    fa = o.factor([0.7j], "fp64")
    U = torch.zeros(1, o.n, 2, dtype=torch.complex128, device="cuda:0")
    s = torch.ones(1, 2, dtype=torch.float64, device="cuda:0")
    with pytest.raises(rr.RRError) as e:
        fa.gain_grad(1, U, U.clone(), s)
    assert e.value.status == 8
