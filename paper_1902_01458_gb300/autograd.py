"""torch.autograd.Function around the gain gradient (rr_gain_grad).

objective(rho, U, V) = sum over frequencies of sum_{j<J} sigma_j^2, the
leading gains of the weighted resolvent (Eq. 4-5) computed by Algorithm 1
(optionally with subspace iterations), differentiable with respect to the
base-flow fields.  Frequencies are processed in chunks: the forward pass
factors one chunk at a time and keeps only the J leading triplets; the
backward pass re-factors each chunk (the factors of every frequency would
not fit in device memory together at production sizes) and accumulates the
gradient on the device.  Every step runs in librr.so; this module only
marshals arguments.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib


class _Flow:
    def __init__(self, rho, u, v):
        self.rho, self.u, self.v = rho, u, v


def _host(t):
    return np.ascontiguousarray(t.detach().to("cpu", torch.float64).numpy())


def _chunks(n, size):
    return [list(range(i, min(n, i + size))) for i in range(0, n, size)]


class GainObjective(torch.autograd.Function):
    """Differentiable sum of the leading squared gains.

    forward(rho, u, v, grid, omegas, k, J, seeds, chunk, precision,
            power_iters, phi_weighted, weights, device) -> scalar tensor
    rho, u, v: [nx, ny] float64 tensors (rho ignored by the scalar operator);
    grid: an object with the rr_grid fields; omegas: real frequencies (shift
    i*omega); seeds: one Omega seed per frequency.
    """

    @staticmethod
    def forward(ctx, rho, u, v, grid, omegas, k, J, seeds, chunk=4, precision="fp64",
                power_iters=1, phi_weighted=True, weights=None, device=0, refine_tol=1e-10,
                max_refine=10):
        flow = _Flow(_host(rho), _host(u), _host(v))
        op = _lib.Operator(grid, flow, weights=weights, device=device)
        phi = op.phi() if phi_weighted else None
        omegas = np.asarray(omegas, dtype=np.float64).ravel()
        seeds = [int(s) for s in np.asarray(seeds).ravel()]
        total = torch.zeros((), dtype=torch.float64, device=f"cuda:{device}")
        saved = []
        fa = None
        for idx in _chunks(omegas.size, chunk):
            shifts = 1j * omegas[idx]
            if fa is not None and fa.F == len(idx):
                fa.refactor(shifts)
            else:
                if fa is not None:
                    fa.close()
                fa = op.factor(shifts, precision)
            res = fa.randomized_resolvent(k, [seeds[i] for i in idx], phi=phi,
                                          power_iters=power_iters, refine_tol=refine_tol,
                                          max_refine=max_refine)
            sig = res.sigma[:, :J].contiguous()
            total = total + (sig ** 2).sum()
            saved.append((idx, res.U[:, :, :J].contiguous(), res.V[:, :, :J].contiguous(), sig))
        if fa is not None:
            fa.close()
        ctx.op, ctx.saved, ctx.omegas, ctx.J = op, saved, omegas, J
        ctx.in_dev = [t.device for t in (rho, u, v)]
        ctx.precision, ctx.device = precision, device
        ctx.refine = (refine_tol, max_refine)
        return total

    @staticmethod
    def backward(ctx, gout):
        op = ctx.op
        grad = torch.zeros(3, op.nx, op.ny, dtype=torch.float64, device=f"cuda:{ctx.device}")
        fa = None
        for idx, U, V, sig in ctx.saved:
            shifts = 1j * ctx.omegas[idx]
            if fa is not None and fa.F == len(idx):
                fa.refactor(shifts)
            else:
                if fa is not None:
                    fa.close()
                fa = op.factor(shifts, ctx.precision)
            fa.gain_grad(ctx.J, U, V, sig, grad, *ctx.refine)
        if fa is not None:
            fa.close()
        grad = grad * gout.to(grad.device)
        g = [grad[i].to(ctx.in_dev[i]) for i in range(3)]
        return (g[0], g[1], g[2]) + (None,) * 13


def gain_objective(rho, u, v, grid, omegas, k, J, seeds, chunk=4, precision="fp64",
                   power_iters=1, phi_weighted=True, weights=None, device=0, refine_tol=1e-10,
                   max_refine=10):
    return GainObjective.apply(rho, u, v, grid, omegas, k, J, seeds, chunk, precision,
                               power_iters, phi_weighted, weights, device, refine_tol,
                               max_refine)
