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


def test_static_apply_allocates_no_device_memory():
    """After a first call (which looks up the array's address and may load the
    library's kernels), further calls leave the device's free memory as it
    was: nothing is allocated per call."""
    torch = torch_cuda()
    rr = lib()
    from paper_1902_01458_gb300 import _lib
    g = W.ns_grid(12, 10)
    op = rr.Operator(g, W.shear_bubble_flow(g))
    rng = np.random.default_rng(5)
    shifts = np.array([0.7j, 1.9j])
    x = to_dev(rng.standard_normal((2, g.n, 4)) + 1j * rng.standard_normal((2, g.n, 4)), torch)
    y = torch.empty_like(x)
    _lib.rr_apply_static(op.handle, shifts, x, y)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    for adjoint in (False, True, False):
        _lib.rr_apply_static(op.handle, shifts, x, y, adjoint)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(0)[0] == free0


def test_static_apply_at_the_shift_limit():
    """Exactly RR_APPLY_STATIC_MAX_SHIFTS shifts (the whole fixed array) on a
    tiny grid with k = 1, checked against rr_apply."""
    torch = torch_cuda()
    rr = lib()
    from paper_1902_01458_gb300 import _lib
    g = W.ns_grid(4, 3)
    op = rr.Operator(g, W.smooth_random_flow(g, 2))
    rng = np.random.default_rng(9)
    nmax = 4096
    shifts = rng.standard_normal(nmax) * 0.1 + 1j * rng.uniform(0.1, 5.0, nmax)
    x = to_dev(rng.standard_normal((nmax, g.n, 1)) + 1j * rng.standard_normal((nmax, g.n, 1)),
               torch)
    y_ref = torch.empty_like(x)
    y_static = torch.full_like(x, complex("nan"))
    for _ in range(2):
        _lib.rr_apply(op.handle, shifts, x, y_ref)
        _lib.rr_apply_static(op.handle, shifts, x, y_static)
        torch.cuda.synchronize()
        assert rel_err(y_static.cpu().numpy(), y_ref.cpu().numpy()) < 1e-13
        shifts = shifts[::-1].copy()


def test_static_apply_refuses_a_capturing_stream():
    """Every call copies from host memory and synchronises its stream, which a
    capturing stream does not allow: the call returns RR_ERR_ARG before it
    issues any work."""
    torch = torch_cuda()
    rr = lib()
    from paper_1902_01458_gb300 import _lib
    g = W.ns_grid(5, 4)
    op = rr.Operator(g, W.shear_bubble_flow(g))
    x = torch.zeros(1, g.n, 1, dtype=torch.complex128, device="cuda:0")
    y = torch.zeros_like(x)
    _lib.rr_apply_static(op.handle, [1j], x, y)  # set-up outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.stream(s):
        graph.capture_begin()
        try:
            _lib.rr_apply_static(op.handle, [1j], x, y, stream=s)
        except rr.RRError as e:
            err = e
        finally:
            graph.capture_end()
    torch.cuda.synchronize()
    assert err is not None and err.status == 1 and "capturing" in err.message
