"""Oracle: gradient of the summed leading gains with respect to the base flow.
Test infrastructure only.

The paper does not differentiate its gains; this module defines the
derivative the CUDA path computes.  For a simple singular value sigma_j of
the weighted resolvent R = W^{1/2} A^{-1} W^{-1/2}, A = s I - L(theta), with
unit singular vectors u_j, v_j (Eq. 5), first-order perturbation theory gives

    d sigma_j = Re(u_j^H dR v_j),   dR = W^{1/2} A^{-1} dL A^{-1} W^{-1/2}

(dA = -dL).  With a_j = A^{-H} W^{1/2} u_j and b_j = A^{-1} W^{-1/2} v_j,

    d/dtheta sum_{s} sum_{j<J} sigma_j^2 = sum_s sum_{j<J} 2 sigma_j Re(a_j^H (dL/dtheta) b_j).

theta runs over the base-flow values rho, U, V at every interior node.  The
derivative of the assembled matrix dL/dtheta is taken here from the assembly
itself by a five-point central difference in theta (exact for the terms
affine in theta, fourth order for the rational terms in rho), so that this
module needs no hand-derived chain rule: the CUDA path differentiates the
stencil formulas by hand, this module differentiates the matrix numerically.
Tiny grids only (dense SVD, one matrix derivative per node and field).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import operator as op
from . import resolvent as rs

FIELDS = ("rho", "u", "v")


def _with(flow, field: str, p: int, delta: float):
    arrs = {f: np.array(getattr(flow, f), dtype=np.float64, copy=True) for f in FIELDS}
    arrs[field].reshape(-1)[p] += delta
    return dataclasses.replace(flow, **arrs)


def dL_dtheta(grid, flow, field: str, p: int, h: float = 1e-3):
    """dL / d(field at node p) by a five-point central difference of the assembly."""
    Ls = [op.assemble(grid, _with(flow, field, p, c * h)) for c in (2, 1, -1, -2)]
    return (-Ls[0] + 8.0 * Ls[1] - 8.0 * Ls[2] + Ls[3]) / (12.0 * h)


def objective(grid, flow, shifts, J: int, weights=None) -> float:
    """sum over shifts of sum_{j<J} sigma_j^2, sigma from the exact SVD."""
    L = op.assemble(grid, flow)
    return float(sum(np.sum(rs.exact_svd(L, s, weights)[0][:J] ** 2) for s in shifts))


def sandwich_vectors(L, s, U, V, weights=None):
    """a_j = A^{-H} W^{1/2} u_j and b_j = A^{-1} W^{-1/2} v_j for the columns
    of U and V (dense LU of A = s I - L)."""
    n = L.shape[0]
    wh = np.ones(n) if weights is None else np.sqrt(np.asarray(weights, dtype=np.float64))
    lu = rs.DenseLU(op.shifted(L, s))
    a = lu.solve_adjoint(U * wh[:, None])
    b = lu.solve(V / wh[:, None])
    return a, b


def gain_grad_triplets(grid, flow, shifts, triplets, J: int, weights=None,
                       fields=FIELDS) -> np.ndarray:
    """sum_s sum_{j<J} 2 sigma_j Re(a_j^H dL b_j) for given triplets
    [(sigma, U, V) per shift]; returns [3, nx, ny] (rho, U, V)."""
    L = op.assemble(grid, flow)
    npts = grid.nx * grid.ny
    grad = np.zeros((3, npts))
    ab = []
    for s, (sig, U, V) in zip(shifts, triplets):
        a, b = sandwich_vectors(L, s, U[:, :J], V[:, :J], weights)
        ab.append((np.asarray(sig[:J], dtype=np.float64), a, b))
    for fi, field in enumerate(FIELDS):
        if field not in fields:
            continue
        if field == "rho" and grid.q == 1:
            continue  # the scalar operator does not involve rho
        for p in range(npts):
            M = dL_dtheta(grid, flow, field, p)
            tot = 0.0
            for sig, a, b in ab:
                Mb = M @ b
                tot += float(np.sum(2.0 * sig * np.real(np.sum(a.conj() * Mb, axis=0))))
            grad[fi, p] = tot
    return grad.reshape(3, grid.nx, grid.ny)


def gain_grad(grid, flow, shifts, J: int, weights=None, fields=FIELDS) -> np.ndarray:
    """Gradient of objective() with the exact singular triplets."""
    L = op.assemble(grid, flow)
    trip = []
    for s in shifts:
        S, U, V = rs.exact_svd(L, s, weights)
        trip.append((S[:J], U[:, :J], V[:, :J]))
    return gain_grad_triplets(grid, flow, shifts, trip, J, weights, fields)
