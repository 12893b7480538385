"""The two failure statuses of the boundary that ordinary inputs never reach,
forced in forms that cannot hang or fault the GPU, each followed by an
ordinary call in the same process that succeeds.

* RR_ERR_RANK: the CholeskyQR of a sketch that is exactly rank deficient.
  A weight Phi (Eq. 9) that is zero everywhere makes the test matrix, and so
  Y = R Omega, exactly zero: the Gram matrix has a zero pivot, the shifted
  fallback's shift (a multiple of its trace) is zero too, and the call must
  report the breakdown instead of returning a basis.
* RR_ERR_TIMEOUT: the bounded mbarrier waits of the tensor-core sweep.  With
  rr_debug_waits the first CTA of the next sweep launch issues no copy and
  no MMA, so its first wait runs out with nothing in flight; the kernel
  records the timeout, frees its tensor memory and returns, and the solve
  reports RR_ERR_TIMEOUT.
"""
import numpy as np
import pytest

import workloads as W
from oracle import operator as op
from oracle import resolvent as rs
from tests.gpu_util import lib, rel_err, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = torch_cuda()
    return torch, lib()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rank_deficient_sketch_reports_rank(env, precision):
    torch, rr = env
    wl = W.config_small_ns(10, 8, k=6, nfreq=1)
    o = rr.Operator(wl.grid, wl.flow)
    fa = o.factor(1j * wl.omegas, precision)
    zero_phi = torch.zeros(o.n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(rr.RRError) as e:
        fa.sketch(wl.k, [wl.seed0], zero_phi)
    assert e.value.status == 5 and "rank" in e.value.message
    # the same factors serve an ordinary sketch afterwards
    phi = op.phi(wl.grid, wl.flow)
    res = fa.randomized_resolvent(wl.k, [wl.seed0], phi=to_dev(phi, torch))
    ref = rs.randomized(op.assemble(wl.grid, wl.flow), 1j * wl.omegas[0], wl.k, wl.seed0,
                        phi=phi)
    tol = 1e-9 if precision == "fp64" else 1e-6
    np.testing.assert_allclose(res.sigma.cpu().numpy()[0], ref.sigma, rtol=tol)


def test_sweep_wait_timeout_reports_and_recovers(env):
    torch, rr = env
    from paper_1902_01458_gb300 import _lib
    g = W.ns_grid(4, 48)  # block 144: tensor-core sweep fed by TMA
    flow = W.smooth_random_flow(g, 2)
    o = rr.Operator(g, flow)
    fa = o.factor([0.8j], "fp32")
    rng = np.random.default_rng(4)
    k = 8
    b = rng.standard_normal((1, o.n, k)) + 1j * rng.standard_normal((1, o.n, k))
    bd = to_dev(b, torch)
    try:
        _lib.rr_debug_waits(2000, 1)
        with pytest.raises(rr.RRError) as e:
            fa.solve(bd)
        assert e.value.status == 6 and "timed out" in e.value.message
    finally:
        _lib.rr_debug_waits(0, 0)
    # an ordinary solve on the same factors, in the same process
    x, info = fa.solve(bd)
    A = op.shifted(op.assemble(g, flow), 0.8j)
    want = np.linalg.solve(A.toarray(), b[0])
    assert rel_err(x.cpu().numpy()[0], want) < 1e-9
    with pytest.raises(rr.RRError):
        _lib.rr_debug_waits(0, -1)
