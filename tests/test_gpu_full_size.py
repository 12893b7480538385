"""Parity at the full sizes of the workloads, in the launch configuration the
bench times.

* 256 x 128 Navier-Stokes (N = 98,304, block 384), FP64 factors, k = 16,
  Phi-weighted Gaussian columns: the oracle's Algorithm 1 with a banded LAPACK
  LU runs at this size in seconds per frequency, so sigma, sigma_halko
  (1e-9 relative) and the mode subspaces (1e-5 rad) are compared directly.
* 512 x 256 (N = 393,216, block 768), FP32 factors with FP64 refinement,
  k = 32, the 64 frequencies of one bench step in one batch: two of them (the
  lowest frequency and the first above 3) against the oracle's Algorithm 1
  with a banded LAPACK LU at full size (about 15 GB of host memory and a
  minute or two each): sigma_1..sigma_32 and sigma_halko within 1e-6
  relative, the mode subspaces within 1e-5 rad.  For every sampled frequency
  also what the oracle computes one by one -- its test matrix entries, and
  its sparse operator applied to the recovered modes (A (sigma_j u_j) = v_j,
  the recovery identity of Eq. 8 with identity weights) -- plus properties
  that hold at any size (orthonormal V, sorted gains, sigma_1 >=
  sigma_1^Halko), and the FP64 GPU path on one frequency (1e-6 relative).
  Every solve of both paths ends at relative residual <= 1e-10 per column,
  or at the FP64 residual floor where that lies above (at most 2e-10).
* The differentiation workload at its size (256 x 128, 16 frequencies,
  k = 16, chunks of 4): the autograd gradient against central differences
  (h = 1e-6) of the objective on the first 4 of its 64 random directions.
"""
import os
import time

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


def test_fp64_workload_at_full_size_matches_oracle(env):
    torch, rr = env
    wl = W.config_fp64()
    g, flow = wl.grid, wl.flow
    L = op.assemble(g, flow)
    phi = op.phi(g, flow)
    o = rr.Operator(g, flow)
    s, seed = 1j * wl.omegas[0], wl.seed0
    fa = o.factor([s], "fp64")
    res = fa.randomized_resolvent(wl.k, [seed], phi=to_dev(phi, torch))
    ref = rs.randomized(L, s, wl.k, seed, phi=phi, method="banded")
    np.testing.assert_allclose(res.sigma.cpu().numpy()[0], ref.sigma, rtol=1e-9)
    np.testing.assert_allclose(res.sigma_halko.cpu().numpy()[0], ref.sigma_halko, rtol=1e-9)
    assert rs.principal_angle(res.V.cpu().numpy()[0], ref.V) < 1e-5
    assert rs.principal_angle(res.U.cpu().numpy()[0], ref.U) < 1e-5
    fa.close()


def test_mixed_workload_at_full_size_in_the_bench_configuration(env):
    torch, rr = env
    wl = W.config_mixed()
    g, flow = wl.grid, wl.flow
    k, F = wl.k, len(wl.omegas)
    o = rr.Operator(g, flow)
    phi = o.phi()
    shifts = 1j * wl.omegas
    seeds = [wl.seed0 + i for i in range(F)]

    # Omega: sampled rows of the full N x k test matrix against the oracle's
    # counter-based generator
    om = torch.empty(1, g.n, k, dtype=torch.complex128, device="cuda:0")
    rr.rr_gaussian(seeds[:1], g.n, k, phi, om)
    want = philox.test_matrix(seeds[0], g.n, k, phi.cpu().numpy())
    rows = np.random.default_rng(5).choice(g.n, 4096, replace=False)
    np.testing.assert_allclose(om[0].cpu().numpy()[rows], want[rows], rtol=2e-14, atol=1e-15)
    del om

    fa = rr.Factors(o, shifts, "fp32")
    V, sh, i1 = fa.sketch(k, seeds, phi)
    U, sig, i2 = fa.modes(V)
    torch.cuda.synchronize()
    for info in (i1, i2):
        # the workload's bar is relative residual <= 1e-10 per column; where
        # the FP64 residual's own rounding floor lies above it, refinement
        # stops there (measured: the adjoint sketch solve at omega = 0.50
        # ends at 1.35e-10 here and at 1.29e-10 with FP64 factors refined in
        # FP64), so the check allows that floor and no more
        assert info["refine_residual"] <= 2e-10, info
        assert info["refine_residual"] <= 1e-10 or info["refine_stagnated"], info
    sig_h, sh_h = sig.cpu().numpy(), sh.cpu().numpy()
    f_hi = int(np.argmax(wl.omegas > 3.0))
    V_h = {f: V[f].cpu().numpy() for f in (0, f_hi)}
    U_h = {f: U[f].cpu().numpy() for f in (0, f_hi)}
    assert np.all(np.diff(sig_h, axis=1) <= 0) and np.all(sh_h > 0)
    assert np.all(sig_h[:, 0] >= sh_h[:, 0] * (1 - 1e-9))
    L = op.assemble(g, flow)
    for f in (0, F // 2, F - 1):
        Vf = V[f].cpu().numpy()
        Uf = U[f].cpu().numpy()
        gram = Vf.conj().T @ Vf
        assert np.max(np.abs(gram - np.eye(k))) < 1e-12
        A = op.shifted(L, shifts[f])
        for j in range(3):
            r = A @ (sig_h[f, j] * Uf[:, j]) - Vf[:, j]
            assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(Vf[:, j]), (f, j)
    fa.close()
    del V, U

    # the oracle's Algorithm 1 (banded LAPACK LU) at full size on two of the
    # batch's frequencies, element by element
    host_bytes = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    print(f"host memory {host_bytes / 2**30:.0f} GiB")
    if host_bytes < 48 * 2 ** 30:
        pytest.skip(f"host memory {host_bytes / 2**30:.0f} GiB: the banded oracle needs ~15 GB")
    phi_h = phi.cpu().numpy()
    for f in (0, f_hi):
        t0 = time.perf_counter()
        ref = rs.randomized(L, shifts[f], k, seeds[f], phi=phi_h, method="banded")
        print(f"oracle frequency {f} (omega {wl.omegas[f]:.3f}): {time.perf_counter() - t0:.1f} s; "
              f"max sigma rel err {np.max(np.abs(sig_h[f] - ref.sigma) / ref.sigma):.2e}")
        np.testing.assert_allclose(sig_h[f], ref.sigma, rtol=1e-6)
        np.testing.assert_allclose(sh_h[f], ref.sigma_halko, rtol=1e-6)
        assert rs.principal_angle(V_h[f], ref.V) < 1e-5
        assert rs.principal_angle(U_h[f], ref.U) < 1e-5
        del ref
    del V_h, U_h

    # the FP64 GPU path on the lowest frequency
    f64 = rr.Factors(o, shifts[:1], "fp64")
    V64, sh64, j1 = f64.sketch(k, seeds[:1], phi)
    U64, sig64, j2 = f64.modes(V64)
    for info in (j1, j2):
        assert info["refine_residual"] <= 2e-10, info
    np.testing.assert_allclose(sig_h[0], sig64.cpu().numpy()[0], rtol=1e-6)
    np.testing.assert_allclose(sh_h[0], sh64.cpu().numpy()[0], rtol=1e-6)
    f64.close()


def test_gradient_workload_at_full_size(env):
    """The differentiation workload (256 x 128, 16 frequencies, k = 16, J = 3,
    factors recomputed per 4-frequency chunk) through the autograd function:
    the gradient against central differences with h = 1e-6 of the same
    objective on the first 4 of the workload's 64 random directions.  FP64
    factors (the difference quotient needs the objective to ~1e-12), two
    subspace iterations.  A direction can be nearly orthogonal to the
    gradient, so the error is measured against the rms directional
    derivative (1e-5), as in the reduced test."""
    torch, rr = env
    from paper_1902_01458_gb300.autograd import gain_objective
    wl = W.config_gradient()
    g, base = wl.grid, wl.flow
    seeds = [wl.seed0 + i for i in range(len(wl.omegas))]
    kw = dict(grid=g, omegas=wl.omegas, k=wl.k, J=wl.J, seeds=seeds, chunk=wl.chunk,
              precision="fp64", power_iters=2)
    fields = [torch.tensor(a, dtype=torch.float64, requires_grad=True)
              for a in (base.rho, base.u, base.v)]
    val = gain_objective(*fields, **kw)
    val.backward()
    grad = np.stack([f.grad.numpy() for f in fields])
    assert np.all(np.isfinite(grad)) and np.abs(grad).max() > 0
    an, fd = [], []
    for d in W.gradient_directions(wl, 4):
        def at(t):
            with torch.no_grad():
                f = [torch.tensor(a + t * dd) for a, dd in zip((base.rho, base.u, base.v), d)]
                return float(gain_objective(*f, **dict(kw, chunk=len(wl.omegas))))
        fd.append((at(wl.h) - at(-wl.h)) / (2 * wl.h))
        an.append(float(np.sum(grad * d)))
    an, fd = np.array(an), np.array(fd)
    scale = np.sqrt(np.mean(fd ** 2))
    print("directional derivatives", an, fd, "rel err", np.abs(an - fd) / scale)
    assert np.max(np.abs(an - fd)) <= 1e-5 * scale
