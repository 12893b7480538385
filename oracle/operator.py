"""Oracle: discrete linearised operator L (Sec. II.A, Eq. 1) and sketch
weight Phi (Sec. III.C, Eq. 9).  Test infrastructure only.

The paper gives no discrete equations for its operator.  The operators here
follow the reading fixed for this project:

* scalar advection-diffusion (q = 1):
      L phi = -U d_x phi - V d_y phi + (1/Re) (d_xx + d_yy) phi - s_s phi
* isothermal compressible Navier-Stokes in (rho', u', v') (q = 3), with
  p = c^2 rho, c^2 = 1/M^2, linearised about (rho, U, V):
      rho': -(U.grad) rho' - rho' div U - u'.grad rho - rho div u'
      u'  : -(U.grad) u' - (u'.grad) U - (c^2/rho) grad rho'
            + (c^2 rho'/rho^2) grad rho
            + (1/(rho Re)) (lap u' + 1/3 grad div u')
            - (rho'/rho^2)(1/Re)(lap U + 1/3 grad div U)
  plus the sponge -s_s q' on every variable.

Discretisation: 2nd-order central differences on nx x ny interior nodes with
homogeneous Dirichlet ghost nodes (or periodic y); the cross derivative is
the 4-corner stencil.  Derivatives of the base flow use the same central
differences and first-order one-sided differences at the first/last node
(second derivatives reuse the neighbouring node's 3-point stencil there).

The matrix is built from Kronecker products of 1-D difference matrices, a
construction independent of the per-node stencil evaluation of the CUDA path.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------- 1-D pieces
def d1_unknown(n: int, h: float, periodic: bool = False) -> sp.csr_matrix:
    """Central first difference acting on unknowns with zero ghost values."""
    e = np.ones(n)
    m = sp.diags([-e[:-1], e[:-1]], [-1, 1], shape=(n, n), format="lil")
    if periodic:
        m[0, n - 1] = -1.0
        m[n - 1, 0] = 1.0
    return (m / (2.0 * h)).tocsr()


def d2_unknown(n: int, h: float, periodic: bool = False) -> sp.csr_matrix:
    """3-point second difference acting on unknowns with zero ghost values."""
    e = np.ones(n)
    m = sp.diags([e[:-1], -2.0 * e, e[:-1]], [-1, 0, 1], shape=(n, n),
                 format="lil")
    if periodic:
        m[0, n - 1] = 1.0
        m[n - 1, 0] = 1.0
    return (m / (h * h)).tocsr()


def d1_field(n: int, h: float, periodic: bool = False) -> np.ndarray:
    """First derivative of a known field: central, one-sided at the ends."""
    m = np.zeros((n, n))
    for i in range(n):
        if periodic:
            m[i, (i + 1) % n] += 1.0 / (2 * h)
            m[i, (i - 1) % n] -= 1.0 / (2 * h)
        elif i == 0:
            m[i, 0], m[i, 1] = -1.0 / h, 1.0 / h
        elif i == n - 1:
            m[i, n - 2], m[i, n - 1] = -1.0 / h, 1.0 / h
        else:
            m[i, i - 1], m[i, i + 1] = -1.0 / (2 * h), 1.0 / (2 * h)
    return m


def d2_field(n: int, h: float, periodic: bool = False) -> np.ndarray:
    """Second derivative of a known field; the end nodes reuse the stencil
    centred on their inner neighbour."""
    m = np.zeros((n, n))
    for i in range(n):
        if periodic:
            m[i, (i - 1) % n] += 1.0 / h ** 2
            m[i, i] += -2.0 / h ** 2
            m[i, (i + 1) % n] += 1.0 / h ** 2
        else:
            c = min(max(i, 1), n - 2)
            m[i, c - 1] += 1.0 / h ** 2
            m[i, c] += -2.0 / h ** 2
            m[i, c + 1] += 1.0 / h ** 2
    return m


# ------------------------------------------------------------ field helpers
def field_derivatives(grid, f: np.ndarray) -> dict:
    """Derivatives of a base-flow field f[nx, ny] with the field stencils."""
    bx1 = d1_field(grid.nx, grid.dx)
    by1 = d1_field(grid.ny, grid.dy, grid.periodic_y)
    bx2 = d2_field(grid.nx, grid.dx)
    by2 = d2_field(grid.ny, grid.dy, grid.periodic_y)
    fx = bx1 @ f
    fy = f @ by1.T
    return {
        "x": fx,
        "y": fy,
        "xx": bx2 @ f,
        "yy": f @ by2.T,
        "xy": (bx1 @ f) @ by1.T,
    }


def sponge(grid) -> np.ndarray:
    """Sponge strength s_s[nx, ny] = s_max * xi^2 in the outer layer.

    The layer is the outer `sponge_frac` of the domain length at each of the
    four boundaries; xi in [0, 1] is the normalised depth into the layer, and
    where two layers overlap the larger value is taken.  A periodic y
    direction has no layer.
    """
    X, Y = grid.mesh()
    out = np.zeros_like(X)
    if grid.sponge_max == 0.0:
        return out
    lx = grid.sponge_frac * (grid.x1 - grid.x0)
    xi = np.maximum(np.maximum((grid.x0 + lx - X) / lx,
                               (X - (grid.x1 - lx)) / lx), 0.0)
    xi = np.minimum(xi, 1.0)
    out = np.maximum(out, grid.sponge_max * xi ** 2)
    if not grid.periodic_y:
        ly = grid.sponge_frac * (grid.y1 - grid.y0)
        eta = np.maximum(np.maximum((grid.y0 + ly - Y) / ly,
                                    (Y - (grid.y1 - ly)) / ly), 0.0)
        eta = np.minimum(eta, 1.0)
        out = np.maximum(out, grid.sponge_max * eta ** 2)
    return out


# --------------------------------------------------------------- assembly
def assemble(grid, flow) -> sp.csr_matrix:
    """Sparse L (N x N, real) for the grid kind, unknown order ((ix*ny)+iy)*q+c."""
    nx, ny = grid.nx, grid.ny
    Ix = sp.identity(nx, format="csr")
    Iy = sp.identity(ny, format="csr")
    Dx = sp.kron(d1_unknown(nx, grid.dx), Iy, format="csr")
    Dy = sp.kron(Ix, d1_unknown(ny, grid.dy, grid.periodic_y), format="csr")
    Dxx = sp.kron(d2_unknown(nx, grid.dx), Iy, format="csr")
    Dyy = sp.kron(Ix, d2_unknown(ny, grid.dy, grid.periodic_y), format="csr")
    Dxy = sp.kron(d1_unknown(nx, grid.dx),
                  d1_unknown(ny, grid.dy, grid.periodic_y), format="csr")
    lap = Dxx + Dyy

    def dg(a):
        return sp.diags(np.asarray(a, dtype=np.float64).ravel(), 0,
                        format="csr")

    U, V, R = flow.u, flow.v, flow.rho
    sig = sponge(grid)
    adv = -(dg(U) @ Dx + dg(V) @ Dy)

    if grid.q == 1:
        nu = 1.0 / grid.re
        return (adv + nu * lap - dg(sig)).tocsr()

    c2 = 1.0 / grid.mach ** 2
    re = grid.re
    dU = field_derivatives(grid, U)
    dV = field_derivatives(grid, V)
    dR = field_derivatives(grid, R)
    divU = dU["x"] + dV["y"]
    visc = dg(1.0 / (R * re))
    # base-flow viscous force, per unit mass, that multiplies -rho'/rho
    fu = (dU["xx"] + dU["yy"] + (dU["xx"] + dV["xy"]) / 3.0) / re
    fv = (dV["xx"] + dV["yy"] + (dU["xy"] + dV["yy"]) / 3.0) / re

    blk = [[None] * 3 for _ in range(3)]
    blk[0][0] = adv - dg(divU) - dg(sig)
    blk[0][1] = -dg(dR["x"]) - dg(R) @ Dx
    blk[0][2] = -dg(dR["y"]) - dg(R) @ Dy
    blk[1][0] = (-c2 * dg(1.0 / R) @ Dx + c2 * dg(dR["x"] / R ** 2)
                 - dg(fu / R ** 2))
    blk[1][1] = adv - dg(dU["x"]) + visc @ (lap + Dxx / 3.0) - dg(sig)
    blk[1][2] = -dg(dU["y"]) + visc @ (Dxy / 3.0)
    blk[2][0] = (-c2 * dg(1.0 / R) @ Dy + c2 * dg(dR["y"] / R ** 2)
                 - dg(fv / R ** 2))
    blk[2][1] = -dg(dV["x"]) + visc @ (Dxy / 3.0)
    blk[2][2] = adv - dg(dV["y"]) + visc @ (lap + Dyy / 3.0) - dg(sig)

    L = None
    for a in range(3):
        for b in range(3):
            e = sp.csr_matrix(([1.0], ([a], [b])), shape=(3, 3))
            term = sp.kron(blk[a][b], e, format="csr")
            L = term if L is None else L + term
    L = L.tocsr()
    L.eliminate_zeros()
    return L


def shifted(L: sp.spmatrix, s: complex) -> sp.csc_matrix:
    """s I - L as a complex sparse matrix."""
    n = L.shape[0]
    return (s * sp.identity(n, dtype=np.complex128, format="csc")
            - L.astype(np.complex128)).tocsc()


def phi(grid, flow) -> np.ndarray:
    """Eq. (9): Phi_j = ||grad v_j|| at each grid point j (Frobenius norm of
    the 2x2 velocity-gradient tensor, same field differences as L), returned
    stacked over the q variables to length N."""
    dU = field_derivatives(grid, flow.u)
    dV = field_derivatives(grid, flow.v)
    p = np.sqrt(dU["x"] ** 2 + dU["y"] ** 2 + dV["x"] ** 2 + dV["y"] ** 2)
    return np.repeat(p.ravel(), grid.q)
