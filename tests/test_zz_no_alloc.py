"""rr_apply_static: the operator application for callers that cannot allocate
device memory while running (their own memory pool owns the GPU, or their
loop may not pay for cudaMalloc's implicit synchronisation).  It stages the
shifts in a fixed array compiled into the library instead of a cudaMalloc'd
buffer; its results must equal rr_apply's.

Collected last on purpose, so a stop-at-first-failure run has already run
every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import lib, rel_err, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


def test_static_apply_matches_apply_on_consecutive_calls():
    torch = torch_cuda()
    rr = lib()
    from paper_1902_01458_gb300 import _lib
    g = W.ns_grid(24, 20)
    op = rr.Operator(g, W.smooth_random_flow(g, 4))
    rng = np.random.default_rng(21)
    calls = [(np.array([0.3j, 1.1 + 2.0j, -0.4j]), 5, False),
             (np.array([2.5j]), 3, True)]
    for shifts, k, adjoint in calls:
        x = to_dev(rng.standard_normal((len(shifts), g.n, k))
                   + 1j * rng.standard_normal((len(shifts), g.n, k)), torch)
        y_ref = torch.empty_like(x)
        y_static = torch.full_like(x, complex("nan"))
        _lib.rr_apply(op.handle, shifts, x, y_ref, adjoint)
        _lib.rr_apply_static(op.handle, shifts, x, y_static, adjoint)
        torch.cuda.synchronize()
        assert rel_err(y_static.cpu().numpy(), y_ref.cpu().numpy()) < 1e-13


def test_static_apply_rejects_too_many_shifts():
    torch = torch_cuda()
    rr = lib()
    from paper_1902_01458_gb300 import _lib
    g = W.ns_grid(5, 4)
    op = rr.Operator(g, W.shear_bubble_flow(g))
    shifts = np.ones(4097, dtype=np.complex128)
    x = torch.zeros(len(shifts), g.n, 1, dtype=torch.complex128, device="cuda:0")
    y = torch.zeros_like(x)
    with pytest.raises(rr.RRError) as e:
        _lib.rr_apply_static(op.handle, shifts, x, y)
    assert e.value.status == 1 and "4096" in e.value.message
