"""GPU parity of the test-matrix variants (Sec. II.B.2) and of subspace
iterations (Sec. II.B.1) through the C ABI, against the oracle on the same seeds.

Rademacher and sparse Rademacher entries are integer decisions on Philox
words followed by one multiply by Phi: bit-exact.  Sketch results carry the
accuracy targets of the method: sigma within 1e-9 (FP64) / 1e-6 (FP32 with
refinement) relative, subspaces within 1e-5 rad."""
import numpy as np
import pytest

import workloads as W
from oracle import operator as op
from oracle import philox
from oracle import resolvent as rs
from tests.gpu_util import lib, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    return torch, lib()


@pytest.mark.parametrize("kind,density", [("rademacher", 1.0), ("sparse_rademacher", 1 / 3),
                                          ("sparse_rademacher", 0.02),
                                          ("sparse_rademacher", 1.0)])
def test_test_matrix_bit_exact(env, kind, density):
    torch, rr = env
    n, k = 4099, 9
    seeds = [12, 2 ** 37 + 5, 1000]
    phi = np.linspace(0.05, 3.0, n)
    om = torch.empty(len(seeds), n, k, dtype=torch.complex128, device="cuda:0")
    rr.rr_test_matrix(seeds, n, k, to_dev(phi, torch), om, kind=kind, density=density)
    got = om.cpu().numpy()
    for f, s in enumerate(seeds):
        want = philox.test_matrix(s, n, k, phi, kind=kind, density=density)
        np.testing.assert_array_equal(got[f], want)
    # without phi
    rr.rr_test_matrix(seeds[:1], n, k, None, om[:1], kind=kind, density=density)
    np.testing.assert_array_equal(om[0].cpu().numpy(),
                                  philox.test_matrix(seeds[0], n, k, kind=kind, density=density))


def test_test_matrix_argument_errors(env):
    torch, rr = env
    om = torch.empty(1, 10, 2, dtype=torch.complex128, device="cuda:0")
    for kind, dens in ((3, 1.0), (7, 1.0), (2, 0.0), (2, 1.5)):
        with pytest.raises(rr.RRError) as e:
            rr.rr_test_matrix([1], 10, 2, None, om, kind=kind, density=dens)
        assert e.value.status == 1


def _problem(nx=16, ny=14, nfreq=2, k=6):
    wl = W.config_small_ns(nx, ny, k=k, nfreq=nfreq)
    return wl, op.assemble(wl.grid, wl.flow), op.phi(wl.grid, wl.flow)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kind,power", [("gaussian", 1), ("gaussian", 2), ("rademacher", 0),
                                        ("sparse_rademacher", 1), ("orthonormal", 0)])
def test_sketch_variants_match_oracle(env, precision, kind, power):
    torch, rr = env
    wl, L, phi = _problem()
    o = rr.Operator(wl.grid, wl.flow)
    shifts = 1j * wl.omegas
    seeds = [wl.seed0 + i for i in range(len(shifts))]
    fa = o.factor(shifts, precision)
    res = fa.randomized_resolvent(wl.k, seeds, phi=to_dev(phi, torch), omega_kind=kind,
                                  density=0.3, power_iters=power)
    tol = 1e-9 if precision == "fp64" else 1e-6
    for f, s in enumerate(shifts):
        ref = rs.randomized(L, s, wl.k, seeds[f], phi=phi, kind=kind, density=0.3,
                            power_iters=power)
        np.testing.assert_allclose(res.sigma_halko.cpu().numpy()[f], ref.sigma_halko, rtol=tol)
        np.testing.assert_allclose(res.sigma.cpu().numpy()[f], ref.sigma, rtol=tol)
        assert rs.principal_angle(res.V.cpu().numpy()[f], ref.V) < 1e-5
        assert rs.principal_angle(res.U.cpu().numpy()[f], ref.U) < 1e-5


def test_power_iterations_with_weights(env):
    torch, rr = env
    wl, L, phi = _problem(12, 10, nfreq=1, k=5)
    w = np.linspace(0.5, 2.0, L.shape[0])
    o = rr.Operator(wl.grid, wl.flow, weights=w)
    s = 1j * wl.omegas[0]
    fa = o.factor([s], "fp64")
    res = fa.randomized_resolvent(5, [77], power_iters=2)
    ref = rs.randomized(L, s, 5, 77, weights=w, power_iters=2)
    np.testing.assert_allclose(res.sigma.cpu().numpy()[0], ref.sigma, rtol=1e-9)
    assert rs.principal_angle(res.V.cpu().numpy()[0], ref.V) < 1e-5


def test_orthonormal_omega_gives_the_gaussian_result(env):
    """Omega and its Q factor span the same range: same gains on the GPU."""
    torch, rr = env
    wl, L, phi = _problem(20, 12, nfreq=3, k=8)
    o = rr.Operator(wl.grid, wl.flow)
    fa = o.factor(1j * wl.omegas, "fp64")
    seeds = [3, 4, 5]
    a = fa.randomized_resolvent(8, seeds, phi=to_dev(phi, torch))
    b = fa.randomized_resolvent(8, seeds, phi=to_dev(phi, torch), omega_kind="orthonormal")
    np.testing.assert_allclose(b.sigma.cpu().numpy(), a.sigma.cpu().numpy(), rtol=1e-10)


def test_power_iterations_improve_leading_gains(env):
    """On the advection-diffusion workload the leading sigma approach the
    exact SVD as the number of subspace iterations grows."""
    torch, rr = env
    g = W.Grid(kind=W.KIND_ADVDIFF, nx=16, ny=12, x0=0, x1=10, y0=-5, y1=5, re=100.0)
    flow = W.tanh_shear_flow(g)
    L = op.assemble(g, flow)
    S, _, _ = rs.exact_svd(L, 0.5j)
    o = rr.Operator(g, flow)
    seeds = list(range(100, 116))
    fa = o.factor([0.5j] * len(seeds), "fp64")
    errs = []
    for q in (0, 1, 2):
        res = fa.randomized_resolvent(6, seeds, power_iters=q)
        sh = res.sigma_halko.cpu().numpy()
        errs.append(np.mean(np.abs(sh[:, :3] - S[:3]) / S[:3]))
    assert errs[0] > errs[1] > errs[2]


def test_sketch_option_errors(env):
    torch, rr = env
    wl, L, phi = _problem(8, 6, nfreq=1, k=3)
    o = rr.Operator(wl.grid, wl.flow)
    fa = o.factor([0.5j], "fp64")
    for kw in (dict(omega_kind=9), dict(omega_kind="sparse_rademacher", density=0.0),
               dict(power_iters=-1), dict(power_iters=65)):
        with pytest.raises(rr.RRError) as e:
            fa.sketch(3, [1], **kw)
        assert e.value.status == 1
