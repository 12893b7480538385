"""GPU parity: every step of the CUDA path, called through the C ABI, against
the FP64 CPU oracle on the same seeded inputs.

Tolerances (fixed by the method's accuracy targets): FP64 path sigma_j within
1e-9 relative of the oracle; FP32 factors + FP64 refinement within 1e-6; mode
subspaces within 1e-5 radians (largest principal angle).  Operator application
and Omega are compared at rounding level.
"""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle import operator as op
from oracle import philox
from oracle import resolvent as rs
from tests.gpu_util import lib, rel_err, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    return torch, lib()


def _cases():
    g1 = W.Grid(kind=W.KIND_ADVDIFF, nx=7, ny=10, x0=0, x1=2, y0=0, y1=3, re=5.0,
                periodic_y=True)
    return [
        ("ns-24x20", W.config_small_ns(24, 20).grid, None),
        ("ns-random-13x9", W.ns_grid(13, 9), "random"),
        ("advdiff-32x32", W.config_tiny().grid, None),
        ("advdiff-periodic", g1, "vconst"),
        # Sec. III.A's closure: Neumann rho' at the far field, all at the outlet
        ("ns-neumann-9x11", W.ns_grid(9, 11, neumann=W.PAPER_NEUMANN), "random"),
        ("advdiff-neumann-all", W.Grid(kind=W.KIND_ADVDIFF, nx=8, ny=9, x0=0, x1=2, y0=0,
                                       y1=3, re=5.0, neumann=(1, 1, 1, 1)), "random"),
        # NS with a periodic y direction and Neumann x sides: the widest ELL rows
        # (folded ghost coefficients, wrapped neighbours) against the oracle
        ("ns-periodic-neumann-x", dataclasses.replace(W.ns_grid(10, 8), periodic_y=True,
                                                      neumann=(1, 7, 0, 0)), "random"),
    ]


def _flow(g, how):
    if how == "random":
        return W.smooth_random_flow(g, 5)
    if how == "vconst":
        return W.zero_flow(g, 0.8)
    if g.kind == W.KIND_ADVDIFF:
        return W.tanh_shear_flow(g)
    return W.shear_bubble_flow(g)


@pytest.mark.parametrize("name,g,how", _cases())
@pytest.mark.parametrize("adjoint", [False, True])
def test_apply_matches_oracle(env, name, g, how, adjoint):
    torch, rr = env
    flow = _flow(g, how)
    L = op.assemble(g, flow)
    o = rr.Operator(g, flow)
    rng = np.random.default_rng(3)
    shifts = np.array([0.7j, 0.2 + 1.9j])
    x = rng.standard_normal((2, o.n, 5)) + 1j * rng.standard_normal((2, o.n, 5))
    y = o.apply(shifts, to_dev(x, torch), adjoint).cpu().numpy()
    for f, s in enumerate(shifts):
        A = op.shifted(L, s)
        want = (A.conj().T if adjoint else A) @ x[f]
        assert rel_err(y[f], want) < 1e-13


def test_phi_matches_oracle(env):
    torch, rr = env
    g = W.ns_grid(40, 30)
    flow = W.smooth_random_flow(g, 9)
    o = rr.Operator(g, flow)
    got = o.phi().cpu().numpy()
    assert rel_err(got, op.phi(g, flow)) < 1e-13


def test_gaussian_matches_oracle(env):
    torch, rr = env
    n, k = 3001, 7
    seeds = [5, 2 ** 40 + 17]
    phi = np.linspace(0.1, 2.0, n)
    om = torch.empty(2, n, k, dtype=torch.complex128, device="cuda:0")
    rr.rr_gaussian(seeds, n, k, to_dev(phi, torch), om)
    got = om.cpu().numpy()
    for f, s in enumerate(seeds):
        want = philox.test_matrix(s, n, k, phi)
        np.testing.assert_allclose(got[f], want, rtol=2e-14, atol=1e-15)


SOLVE_CASES = [
    ("ns-24x20", lambda: W.config_small_ns(24, 20).grid, None),
    ("ns-random-11x14", lambda: W.ns_grid(11, 14), "random"),
    ("ns-9x40-four-panels", lambda: W.ns_grid(9, 40), "random"),
    # b = 264: tensor-core update with ragged row and column tiles and a last
    # panel of 8 columns
    ("ns-5x88-ragged-tc-update", lambda: W.ns_grid(5, 88), "random"),
    ("advdiff-periodic", lambda: W.Grid(kind=W.KIND_ADVDIFF, nx=9, ny=12, x0=0, x1=2,
                                        y0=0, y1=3, re=5.0, periodic_y=True), "vconst"),
    # Neumann closure, b = 144 (tensor-core update and sweeps)
    ("ns-neumann-6x48", lambda: W.ns_grid(6, 48, neumann=W.PAPER_NEUMANN), "random"),
]


@pytest.mark.parametrize("name,gf,how", SOLVE_CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_simt"])
@pytest.mark.parametrize("adjoint", [False, True])
def test_solve_matches_oracle(env, name, gf, how, precision, adjoint):
    torch, rr = env
    g = gf()
    flow = _flow(g, how)
    L = op.assemble(g, flow)
    rng = np.random.default_rng(11)
    w = rng.uniform(0.5, 2.0, g.n)
    o = rr.Operator(g, flow, weights=w)
    shifts = np.array([0.4j, 1.3j, 0.1 + 2.8j])
    fa = o.factor(shifts, precision)
    k = 6
    b = rng.standard_normal((3, g.n, k)) + 1j * rng.standard_normal((3, g.n, k))
    x, info = fa.solve(to_dev(b, torch), adjoint=adjoint, refine_tol=1e-12, max_refine=20)
    x = x.cpu().numpy()
    wh = np.sqrt(w)
    for f, s in enumerate(shifts):
        A = op.shifted(L, s).toarray()
        if adjoint:
            want = np.linalg.solve(A.conj().T, wh[:, None] * b[f]) / wh[:, None]
        else:
            want = wh[:, None] * np.linalg.solve(A, b[f] / wh[:, None])
        assert rel_err(x[f], want) < (1e-11 if precision == "fp64" else 1e-9), f
    assert info["refine_residual"] <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_simt"])
@pytest.mark.parametrize("orthogonalize", [False, True])
def test_algorithm1_matches_oracle(env, precision, orthogonalize):
    """Sketch, QR, adjoint solve, small SVD, recovery: sigma, sigma_halko, U, V."""
    torch, rr = env
    wl = W.config_small_ns(24, 20, k=8, nfreq=3)
    g, flow = wl.grid, wl.flow
    L = op.assemble(g, flow)
    o = rr.Operator(g, flow)
    phi = op.phi(g, flow)
    shifts = 1j * wl.omegas
    seeds = [wl.seed0 + i for i in range(len(shifts))]
    fa = o.factor(shifts, precision)
    res = fa.randomized_resolvent(wl.k, seeds, phi=to_dev(phi, torch),
                                  orthogonalize=orthogonalize)
    sig = res.sigma.cpu().numpy()
    sh = res.sigma_halko.cpu().numpy()
    U = res.U.cpu().numpy()
    V = res.V.cpu().numpy()
    tol = 1e-9 if precision == "fp64" else 1e-6
    for f, s in enumerate(shifts):
        ref = rs.randomized(L, s, wl.k, seeds[f], phi=phi, orthogonalize=orthogonalize)
        np.testing.assert_allclose(sig[f], ref.sigma, rtol=tol)
        np.testing.assert_allclose(sh[f], ref.sigma_halko, rtol=tol)
        assert rs.principal_angle(V[f], ref.V) < 1e-5
        assert rs.principal_angle(U[f], ref.U) < 1e-5
        for j in range(3):
            assert rs.cosine_similarity(U[f][:, j], ref.U[:, j]) > 1 - 1e-8
            assert rs.cosine_similarity(V[f][:, j], ref.V[:, j]) > 1 - 1e-8
        # phase convention: the largest |v_j| entry is real positive
        for j in range(wl.k):
            i = int(np.argmax(np.abs(V[f][:, j])))
            assert abs(V[f][i, j].imag) < 1e-12 * abs(V[f][i, j]) and V[f][i, j].real > 0


def test_tiny_advdiff_workload(env):
    """Scalar advection-diffusion 32x32, omega = 0.5, k = 10, identity weights."""
    torch, rr = env
    wl = W.config_tiny()
    L = op.assemble(wl.grid, wl.flow)
    o = rr.Operator(wl.grid, wl.flow)
    fa = o.factor([0.5j], "fp64")
    res = fa.randomized_resolvent(10, [1000])
    ref = rs.randomized(L, 0.5j, 10, 1000)
    np.testing.assert_allclose(res.sigma.cpu().numpy()[0], ref.sigma, rtol=1e-9)
    np.testing.assert_allclose(res.sigma_halko.cpu().numpy()[0], ref.sigma_halko, rtol=1e-9)
    assert rs.principal_angle(res.V.cpu().numpy()[0], ref.V) < 1e-5
    assert rs.principal_angle(res.U.cpu().numpy()[0], ref.U) < 1e-5


def test_full_width_sketch_is_exact(env):
    """k = N on a tiny grid: the GPU path returns the exact SVD (closed form)."""
    torch, rr = env
    g = W.Grid(kind=W.KIND_ADVDIFF, nx=8, ny=6, x0=0, x1=3, y0=-1, y1=1, re=2.0)
    L = op.assemble(g, W.zero_flow(g))
    p = np.arange(1, 9)[:, None]
    q = np.arange(1, 7)[None, :]
    lam = -0.5 * ((4 / g.dx ** 2) * np.sin(p * np.pi / 18) ** 2
                  + (4 / g.dy ** 2) * np.sin(q * np.pi / 14) ** 2)
    s = 0.7j
    sig_exact = np.sort(1 / np.abs(s - lam.ravel()))[::-1]
    o = rr.Operator(g, W.zero_flow(g))
    fa = o.factor([s], "fp64")
    res = fa.randomized_resolvent(48, [3])
    np.testing.assert_allclose(res.sigma.cpu().numpy()[0], sig_exact, rtol=1e-10)
    np.testing.assert_allclose(res.sigma_halko.cpu().numpy()[0], sig_exact, rtol=1e-10)


@pytest.mark.parametrize("k", [1, 3, 64])
def test_k_edges(env, k):
    torch, rr = env
    g = W.ns_grid(9, 11)
    flow = W.shear_bubble_flow(g)
    L = op.assemble(g, flow)
    o = rr.Operator(g, flow)
    fa = o.factor([0.9j], "fp64")
    res = fa.randomized_resolvent(k, [7])
    ref = rs.randomized(L, 0.9j, k, 7)
    np.testing.assert_allclose(res.sigma.cpu().numpy()[0], ref.sigma, rtol=1e-9)


def test_singular_shift_is_reported(env):
    """L = 0 (no flow, no diffusion, no sponge) and s = 0: exact zero pivot."""
    torch, rr = env
    g = W.Grid(kind=W.KIND_ADVDIFF, nx=4, ny=5, x0=0, x1=1, y0=0, y1=1, re=1e308)
    o = rr.Operator(g, W.zero_flow(g))
    with pytest.raises(rr.RRError) as e:
        o.factor([0.0], "fp64")
    assert e.value.status == 3


def test_argument_errors(env):
    torch, rr = env
    g = W.ns_grid(5, 4)
    o = rr.Operator(g, W.shear_bubble_flow(g))
    fa = o.factor([1j], "fp64")
    with pytest.raises(rr.RRError) as e:
        fa.sketch(65, [1])
    assert e.value.status == 1
    with pytest.raises(rr.RRError) as e:
        fa.sketch(0, [1])
    assert e.value.status == 1
    with pytest.raises(rr.RRError):
        rr.Operator(W.ns_grid(2, 4), W.shear_bubble_flow(W.ns_grid(2, 4)))


def test_refinement_reports_non_convergence(env):
    torch, rr = env
    g = W.ns_grid(10, 8)
    o = rr.Operator(g, W.shear_bubble_flow(g))
    fa = o.factor([1j], "fp32")
    b = torch.ones(1, g.n, 2, dtype=torch.complex128, device="cuda:0")
    x, info = fa.solve(b, refine_tol=1e-30, max_refine=1, check=False)
    from paper_1902_01458_gb300._lib import rr_solve
    st, _ = rr_solve(fa.handle, b, x, False, 1e-30, 1)
    assert st == 4


@pytest.mark.parametrize("grid_shape", [(24, 20), (9, 40), (8, 50), (5, 88), (4, 128)])
@pytest.mark.parametrize("k", [3, 16, 32, 48, 64])
@pytest.mark.parametrize("adjoint", [False, True])
def test_tensor_core_sweeps_match_cuda_core_sweeps(env, grid_shape, k, adjoint):
    """One unrefined FP32 solve: the tensor-core path (tcgen05 3xTF32 trailing
    update when b % 8 == 0, tcgen05 sweeps) against the FP32 CUDA-core path,
    and both against the FP64 oracle."""
    torch, rr = env
    g = W.ns_grid(*grid_shape)
    flow = W.smooth_random_flow(g, 2)
    L = op.assemble(g, flow)
    o = rr.Operator(g, flow)
    shifts = np.array([0.6j, 2.2j])
    rng = np.random.default_rng(5)
    b = rng.standard_normal((2, g.n, k)) + 1j * rng.standard_normal((2, g.n, k))
    bd = to_dev(b, torch)
    xs = {}
    for prec in ("fp32", "fp32_simt"):
        fa = o.factor(shifts, prec)
        x, _ = fa.solve(bd, adjoint=adjoint, refine_tol=0.0, max_refine=0)
        xs[prec] = x.cpu().numpy()
        fa.close()
    assert rel_err(xs["fp32"], xs["fp32_simt"]) < 1e-4
    for f, s in enumerate(shifts):
        A = op.shifted(L, s).toarray()
        want = np.linalg.solve(A.conj().T if adjoint else A, b[f])
        assert rel_err(xs["fp32"][f], want) < 1e-4


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_algorithm1_with_neumann_closure_matches_oracle(env, precision):
    """Sec. III.A's boundary closure (Neumann rho' at the far field, every
    variable at the outlet) end to end."""
    torch, rr = env
    g = W.ns_grid(16, 44, neumann=W.PAPER_NEUMANN)
    flow = W.shear_bubble_flow(g)
    L = op.assemble(g, flow)
    phi = op.phi(g, flow)
    o = rr.Operator(g, flow)
    shifts = 1j * np.array([0.35, 2.2])
    seeds = [77, 78]
    fa = o.factor(shifts, precision)
    res = fa.randomized_resolvent(6, seeds, phi=to_dev(phi, torch))
    tol = 1e-9 if precision == "fp64" else 1e-6
    for f, s in enumerate(shifts):
        ref = rs.randomized(L, s, 6, seeds[f], phi=phi)
        np.testing.assert_allclose(res.sigma.cpu().numpy()[f], ref.sigma, rtol=tol)
        np.testing.assert_allclose(res.sigma_halko.cpu().numpy()[f], ref.sigma_halko, rtol=tol)
        assert rs.principal_angle(res.V.cpu().numpy()[f], ref.V) < 1e-5
        assert rs.principal_angle(res.U.cpu().numpy()[f], ref.U) < 1e-5


def test_operator_rejects_bad_closure_masks(env):
    torch, rr = env
    import dataclasses
    g = W.ns_grid(6, 5)
    for bad in [dataclasses.replace(g, neumann=(8, 0, 0, 0)),
                dataclasses.replace(g, neumann=(0, 0, 1, 0), periodic_y=True)]:
        with pytest.raises(rr.RRError) as e:
            rr.Operator(bad, W.shear_bubble_flow(g))
        assert e.value.status == 1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("adjoint", [False, True])
def test_solve_at_the_largest_block(env, precision, adjoint):
    """b = 1020, next to the 1024 maximum: the narrowest panels (16 columns in
    FP32, 8 in FP64, set by shared memory) and the largest sweep tiles."""
    torch, rr = env
    g = W.ns_grid(4, 340)
    flow = W.smooth_random_flow(g, 5)
    L = op.assemble(g, flow)
    o = rr.Operator(g, flow)
    shifts = np.array([0.4j, 2.1j])
    fa = o.factor(shifts, precision)
    rng = np.random.default_rng(13)
    k = 4
    b = rng.standard_normal((2, g.n, k)) + 1j * rng.standard_normal((2, g.n, k))
    x, info = fa.solve(to_dev(b, torch), adjoint=adjoint, refine_tol=1e-12, max_refine=20)
    x = x.cpu().numpy()
    for f, s in enumerate(shifts):
        A = op.shifted(L, s).toarray()
        want = np.linalg.solve(A.conj().T if adjoint else A, b[f])
        assert rel_err(x[f], want) < (1e-11 if precision == "fp64" else 1e-9), f
