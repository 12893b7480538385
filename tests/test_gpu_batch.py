"""Batch plans (rr_batch_*): problems of uneven size in one captured CUDA graph,
checked problem by problem against the FP64 oracle's Algorithm 1 on the same
seeded inputs (sigma, sigma_halko within 1e-6 relative for FP32 factors with
refinement, 1e-9 for FP64; largest principal angle of U and V within 1e-5).
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import operator as op
from oracle import resolvent as rs
from tests.gpu_util import lib, torch_cuda

pytestmark = pytest.mark.gpu

# grids with b = 36 (CUDA-core paths), b = 144 (tensor-core update and
# sweeps) and b = 192; k odd and even; several problems per (grid, k)
SMALL = [(6, 12, 3, 0.4), (5, 48, 4, 1.3), (6, 12, 4, 2.2), (4, 64, 8, 0.9),
         (5, 48, 4, 3.1), (6, 12, 3, 5.0), (4, 64, 3, 0.2), (5, 48, 8, 7.7),
         (4, 64, 8, 4.4)]


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    return torch, lib()


def _build(rr, spec):
    ops, problems = {}, []
    for i, (nx, ny, k, w) in enumerate(spec):
        if (nx, ny) not in ops:
            g = W.ns_grid(nx, ny)
            ops[(nx, ny)] = (g, W.shear_bubble_flow(g), rr.Operator(g, W.shear_bubble_flow(g)))
        problems.append({"op": ops[(nx, ny)][2], "shift": 1j * w, "k": k, "seed": 1000 + i,
                         "grid": (nx, ny)})
    return ops, problems


def _check_against_oracle(ops, problems, outputs, shifts, tol):
    for p, out, s in zip(problems, outputs, shifts):
        g, flow, _ = ops[p["grid"]]
        L = op.assemble(g, flow)
        ref = rs.randomized(L, s, p["k"], p["seed"], phi=op.phi(g, flow))
        np.testing.assert_allclose(out["sigma"].cpu().numpy(), ref.sigma, rtol=tol)
        np.testing.assert_allclose(out["sigma_halko"].cpu().numpy(), ref.sigma_halko, rtol=tol)
        assert rs.principal_angle(out["V"].cpu().numpy(), ref.V) < 1e-5
        assert rs.principal_angle(out["U"].cpu().numpy(), ref.U) < 1e-5


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-6), ("fp64", 1e-9), ("fp32_simt", 1e-6)])
def test_batch_matches_oracle(env, precision, tol):
    torch, rr = env
    ops, problems = _build(rr, SMALL)
    b = rr.Batch(problems, precision=precision)
    st, info = b.run()
    d = b.describe()
    assert d["groups"] == 3 and d["views"] == 6 and d["lanes"] == 3
    assert d["kernel_nodes"] > 0
    _check_against_oracle(ops, problems, b.outputs, [p["shift"] for p in problems], tol)
    if precision != "fp64":
        assert info["refine_residual"] <= 1e-10 or info["refine_iters"] > 0
    b.close()


def test_batch_runs_are_bitwise_reproducible_and_counted(env):
    torch, rr = env
    from paper_1902_01458_gb300 import _lib
    ops, problems = _build(rr, SMALL)
    b = rr.Batch(problems, precision="fp32", lanes=2)
    b.run()
    first = [{k: v.clone() for k, v in o.items()} for o in b.outputs]
    for o in b.outputs:  # outputs are rewritten by every run
        for v in o.values():
            v.fill_(float("nan"))
    _lib.rr_profile_start([])
    b.run()
    assert _lib.rr_launch_count() == b.describe()["kernel_nodes"]
    for a, o in zip(first, b.outputs):
        for key in a:
            assert torch.equal(a[key], o[key]), key
    b.close()


def test_batch_set_shifts_reuses_the_graph(env):
    torch, rr = env
    ops, problems = _build(rr, SMALL)
    b = rr.Batch(problems, precision="fp32")
    new = [1j * (0.5 + 0.37 * i) for i in range(len(problems))]
    b.set_shifts(new)
    st, info = b.run(check=False)
    assert st in (0, 4)
    if st == 0:
        _check_against_oracle(ops, problems, b.outputs, new, 1e-6)
    b.close()


def test_tuned_batch_matches_oracle(env):
    torch, rr = env
    spec = [(4, 64, 8, 0.7), (3, 48, 4, 2.0), (4, 64, 4, 3.3), (3, 48, 4, 0.3)]
    ops, problems = _build(rr, spec)
    b = rr.Batch(problems, precision="fp32", tune=True)
    b.run()
    d = b.describe()
    assert d["lanes"] in (1, 2) and d["tuned_ms"] > 0
    _check_against_oracle(ops, problems, b.outputs, [p["shift"] for p in problems], 1e-6)
    b.close()


def test_batch_argument_errors(env):
    torch, rr = env
    from paper_1902_01458_gb300 import _lib
    lib_ = _lib.load()
    h = ctypes.c_void_p()
    assert lib_.rr_batch_create(0, None, 1, None, ctypes.byref(h)) == 1
    ops, problems = _build(rr, SMALL[:1])
    for k in (0, 65):
        with pytest.raises(rr.RRError) as e:
            rr.Batch([dict(problems[0], k=k)], precision="fp32")
        assert e.value.status == 1
    with pytest.raises(rr.RRError) as e:
        rr.Batch(problems, precision="fp32", lanes=65)
    assert e.value.status == 1
    with pytest.raises(rr.RRError) as e:
        rr.Batch([dict(problems[0], shift=complex(float("nan"), 1.0))], precision="fp32")
    assert e.value.status == 1


def test_batched_workload_full_size_sampled(env):
    """The 128-problem uneven workload (grids 128..384 x 64..256, q = 3,
    k in {8, 16, 32, 64}, omega ~ U[0.1, 8]) as one plan.  Checked:
      * against the oracle's Algorithm 1 (banded LU) element by element: the
        first problem of each (grid, k = 64) group on the two smallest grids
        (k = 64 runs on the CUDA-core sweep in FP32) and the first problem on
        the largest grid (384 x 256, block 768);
      * for the first problem of every one of the 46 (grid, k) groups, the
        recovery identity of Eq. 8 with the oracle's sparse operator,
        A (sigma_j u_j) = v_j for the leading three modes (identity weights),
        and orthonormal forcing modes;
      * for every problem: sigma_1 >= sigma_1^Halko > 0 and unit response
        modes."""
    torch, rr = env
    spec = W.config_batched()
    ops, problems = {}, []
    for i, p in enumerate(spec):
        if (p.nx, p.ny) not in ops:
            g = W.ns_grid(p.nx, p.ny)
            flow = W.shear_bubble_flow(g)
            ops[(p.nx, p.ny)] = (g, flow, rr.Operator(g, flow))
        problems.append({"op": ops[(p.nx, p.ny)][2], "shift": 1j * p.omega, "k": p.k,
                         "seed": p.seed, "grid": (p.nx, p.ny)})
    b = rr.Batch(problems, precision="fp32")
    b.run()
    first = {}
    for i, p in enumerate(problems):
        first.setdefault((p["grid"], p["k"]), i)
    assert len(first) == 46
    by_size = sorted(ops, key=lambda g: g[0] * g[1])
    full = [first[(g, 64)] for g in by_size[:2] if (g, 64) in first]
    full.append(first[(max(ops, key=lambda g: (g[1], g[0])), 32)])
    assert len(full) == 3 and any(problems[i]["grid"] == (384, 256) for i in full)
    for i in full:
        p, out = problems[i], b.outputs[i]
        g, flow, _ = ops[p["grid"]]
        ref = rs.randomized(op.assemble(g, flow), p["shift"], p["k"], p["seed"],
                            phi=op.phi(g, flow), method="banded")
        np.testing.assert_allclose(out["sigma"].cpu().numpy(), ref.sigma, rtol=1e-6)
        np.testing.assert_allclose(out["sigma_halko"].cpu().numpy(), ref.sigma_halko, rtol=1e-6)
        assert rs.principal_angle(out["V"].cpu().numpy(), ref.V) < 1e-5
        assert rs.principal_angle(out["U"].cpu().numpy(), ref.U) < 1e-5
    Ls = {gk: op.assemble(ops[gk][0], ops[gk][1]) for gk in ops}
    for (grid, k), i in sorted(first.items()):
        p, out = problems[i], b.outputs[i]
        A = op.shifted(Ls[grid], p["shift"])
        sig = out["sigma"].cpu().numpy()
        Vh, Uh = out["V"].cpu().numpy(), out["U"].cpu().numpy()
        assert np.max(np.abs(Vh.conj().T @ Vh - np.eye(k))) < 1e-12, (grid, k)
        for j in range(min(3, k)):
            r = A @ (sig[j] * Uh[:, j]) - Vh[:, j]
            assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(Vh[:, j]), (grid, k, j)
    for p, o in zip(problems, b.outputs):
        sig = o["sigma"].cpu().numpy()
        sh = o["sigma_halko"].cpu().numpy()
        assert np.all(np.isfinite(sig)) and np.all(sh > 0)
        assert sig[0] >= sh[0] * (1 - 1e-9)
        nrm = torch.linalg.vector_norm(o["U"], dim=0).cpu().numpy()
        np.testing.assert_allclose(nrm, 1.0, rtol=1e-12)
    b.close()


def test_single_problem_batch_matches_oracle(env):
    """The smallest plan: one problem, one group, one sub-batch, one lane."""
    torch, rr = env
    ops, problems = _build(rr, [(5, 48, 6, 1.7)])
    b = rr.Batch(problems, precision="fp32", tune=True)
    b.run()
    d = b.describe()
    assert d["groups"] == 1 and d["views"] == 1 and d["lanes"] == 1
    _check_against_oracle(ops, problems, b.outputs, [problems[0]["shift"]], 1e-6)
    b.close()
