"""Oracle: discrete linearised operator L (Sec. II.A, Eq. 1) and sketch
weight Phi (Sec. III.D, Eq. 9).  Test infrastructure only.

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
* bi-global isothermal Navier-Stokes in (rho', u', v', w') (q = 4): the
  perturbations vary as exp(i kz z) about a flow (rho, U, V, W = 0) that does
  not depend on z (Sec. III.A/B: a spanwise wavenumber kz), so d/dz -> i kz:
      rho': as above - rho i kz w'
      u', v': as above with lap -> lap - kz^2 and div u' -> div u' + i kz w'
      w'  : -(U.grad) w' - (c^2/rho) i kz rho'
            + (1/(rho Re)) (lap w' - kz^2 w' + 1/3 i kz (div u' + i kz w'))
  L is complex; at kz = 0 it is the (rho, u, v) operator plus a decoupled
  advection-diffusion equation for w'.

Discretisation: 2nd-order central differences on nx x ny interior nodes with
homogeneous Dirichlet ghost nodes (or periodic y); the cross derivative is
the 4-corner stencil.  Optionally (Sec. III.A's far-field / outlet closure)
a variable's ghost node on a side equals the adjacent interior node
(Neumann); grid.neumann holds the variable bit masks of the sides x0, x1,
y0, y1, and each variable gets difference matrices with its own closure.  Derivatives of the base flow use the same central
differences and first-order one-sided differences at the first/last node
(second derivatives reuse the neighbouring node's 3-point stencil there).

The matrix is built from Kronecker products of 1-D difference matrices, a
construction independent of the per-node stencil evaluation of the CUDA path.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------- 1-D pieces
def d1_unknown(n: int, h: float, periodic: bool = False, neu_lo: bool = False,
               neu_hi: bool = False) -> sp.csr_matrix:
    """Central first difference acting on unknowns; the ghost value beyond
    each end is zero, or (neu_lo / neu_hi) the end node's own value."""
    e = np.ones(n)
    m = sp.diags([-e[:-1], e[:-1]], [-1, 1], shape=(n, n), format="lil")
    if periodic:
        m[0, n - 1] = -1.0
        m[n - 1, 0] = 1.0
    if neu_lo:   # (u_1 - u_ghost) with u_ghost = u_0
        m[0, 0] += -1.0
    if neu_hi:   # (u_ghost - u_{n-2}) with u_ghost = u_{n-1}
        m[n - 1, n - 1] += 1.0
    return (m / (2.0 * h)).tocsr()


def d2_unknown(n: int, h: float, periodic: bool = False, neu_lo: bool = False,
               neu_hi: bool = False) -> sp.csr_matrix:
    """3-point second difference acting on unknowns; ghost values as in
    d1_unknown."""
    e = np.ones(n)
    m = sp.diags([e[:-1], -2.0 * e, e[:-1]], [-1, 0, 1], shape=(n, n),
                 format="lil")
    if periodic:
        m[0, n - 1] = 1.0
        m[n - 1, 0] = 1.0
    if neu_lo:
        m[0, 0] += 1.0
    if neu_hi:
        m[n - 1, n - 1] += 1.0
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
def variable_operators(grid, var: int) -> dict:
    """Difference matrices (nx*ny square) acting on variable `var`, with that
    variable's closure on each side."""
    nx, ny = grid.nx, grid.ny
    masks = getattr(grid, "neumann", (0, 0, 0, 0))
    x0, x1, y0, y1 = (bool((int(m) >> var) & 1) for m in masks)
    Ix = sp.identity(nx, format="csr")
    Iy = sp.identity(ny, format="csr")
    d1x = d1_unknown(nx, grid.dx, False, x0, x1)
    d1y = d1_unknown(ny, grid.dy, grid.periodic_y, y0, y1)
    ops = {
        "Dx": sp.kron(d1x, Iy, format="csr"),
        "Dy": sp.kron(Ix, d1y, format="csr"),
        "Dxx": sp.kron(d2_unknown(nx, grid.dx, False, x0, x1), Iy, format="csr"),
        "Dyy": sp.kron(Ix, d2_unknown(ny, grid.dy, grid.periodic_y, y0, y1), format="csr"),
        "Dxy": sp.kron(d1x, d1y, format="csr"),
    }
    ops["lap"] = ops["Dxx"] + ops["Dyy"]
    return ops


def assemble(grid, flow) -> sp.csr_matrix:
    """Sparse L (N x N, real) for the grid kind, unknown order ((ix*ny)+iy)*q+c."""
    ops = [variable_operators(grid, v) for v in range(grid.q)]
    lap = ops[0]["lap"]

    def dg(a):
        return sp.diags(np.asarray(a, dtype=np.float64).ravel(), 0,
                        format="csr")

    U, V, R = flow.u, flow.v, flow.rho
    sig = sponge(grid)

    def adv(v):  # -(U d_x + V d_y) acting on variable v
        return -(dg(U) @ ops[v]["Dx"] + dg(V) @ ops[v]["Dy"])

    if grid.q == 1:
        nu = 1.0 / grid.re
        return (adv(0) + nu * lap - dg(sig)).tocsr()

    if grid.q == 4:
        return _assemble_kz(grid, flow, ops, adv, dg, sig)
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

    # blk[a][b]: equation a acting on variable b (b's difference matrices)
    o0, o1, o2 = ops
    blk = [[None] * 3 for _ in range(3)]
    blk[0][0] = adv(0) - dg(divU) - dg(sig)
    blk[0][1] = -dg(dR["x"]) - dg(R) @ o1["Dx"]
    blk[0][2] = -dg(dR["y"]) - dg(R) @ o2["Dy"]
    blk[1][0] = (-c2 * dg(1.0 / R) @ o0["Dx"] + c2 * dg(dR["x"] / R ** 2)
                 - dg(fu / R ** 2))
    blk[1][1] = adv(1) - dg(dU["x"]) + visc @ (o1["lap"] + o1["Dxx"] / 3.0) - dg(sig)
    blk[1][2] = -dg(dU["y"]) + visc @ (o2["Dxy"] / 3.0)
    blk[2][0] = (-c2 * dg(1.0 / R) @ o0["Dy"] + c2 * dg(dR["y"] / R ** 2)
                 - dg(fv / R ** 2))
    blk[2][1] = -dg(dV["x"]) + visc @ (o1["Dxy"] / 3.0)
    blk[2][2] = adv(2) - dg(dV["y"]) + visc @ (o2["lap"] + o2["Dyy"] / 3.0) - dg(sig)

    L = None
    for a in range(3):
        for b in range(3):
            e = sp.csr_matrix(([1.0], ([a], [b])), shape=(3, 3))
            term = sp.kron(blk[a][b], e, format="csr")
            L = term if L is None else L + term
    L = L.tocsr()
    L.eliminate_zeros()
    return L


def _assemble_kz(grid, flow, ops, adv, dg, sig) -> sp.csr_matrix:
    """Complex L(kz) of the bi-global operator, (rho', u', v', w')."""
    U, V, R = flow.u, flow.v, flow.rho
    c2 = 1.0 / grid.mach ** 2
    re = grid.re
    kz = float(grid.kz)
    ik = 1j * kz
    dU = field_derivatives(grid, U)
    dV = field_derivatives(grid, V)
    dR = field_derivatives(grid, R)
    divU = dU["x"] + dV["y"]
    visc = dg(1.0 / (R * re))
    fu = (dU["xx"] + dU["yy"] + (dU["xx"] + dV["xy"]) / 3.0) / re
    fv = (dV["xx"] + dV["yy"] + (dU["xy"] + dV["yy"]) / 3.0) / re
    n = grid.npts
    eye = sp.identity(n, format="csr")
    o0, o1, o2, o3 = ops
    blk = [[None] * 4 for _ in range(4)]
    # continuity: -(U.grad) rho' - rho' div U - u'.grad rho - rho (div u' + i kz w')
    blk[0][0] = adv(0) - dg(divU) - dg(sig)
    blk[0][1] = -dg(dR["x"]) - dg(R) @ o1["Dx"]
    blk[0][2] = -dg(dR["y"]) - dg(R) @ o2["Dy"]
    blk[0][3] = -ik * dg(R)
    # x momentum: the 2-D terms, lap -> lap - kz^2, div u' -> div u' + i kz w'
    blk[1][0] = (-c2 * dg(1.0 / R) @ o0["Dx"] + c2 * dg(dR["x"] / R ** 2)
                 - dg(fu / R ** 2))
    blk[1][1] = (adv(1) - dg(dU["x"]) + visc @ (o1["lap"] - kz ** 2 * eye + o1["Dxx"] / 3.0)
                 - dg(sig))
    blk[1][2] = -dg(dU["y"]) + visc @ (o2["Dxy"] / 3.0)
    blk[1][3] = visc @ (ik / 3.0 * o3["Dx"])
    # y momentum
    blk[2][0] = (-c2 * dg(1.0 / R) @ o0["Dy"] + c2 * dg(dR["y"] / R ** 2)
                 - dg(fv / R ** 2))
    blk[2][1] = -dg(dV["x"]) + visc @ (o1["Dxy"] / 3.0)
    blk[2][2] = (adv(2) - dg(dV["y"]) + visc @ (o2["lap"] - kz ** 2 * eye + o2["Dyy"] / 3.0)
                 - dg(sig))
    blk[2][3] = visc @ (ik / 3.0 * o3["Dy"])
    # z momentum (W = 0): -(U.grad) w' - (c^2/rho) i kz rho'
    #   + (1/(rho Re)) (lap w' - kz^2 w' + 1/3 i kz (div u' + i kz w'))
    blk[3][0] = -ik * c2 * dg(1.0 / R)
    blk[3][1] = visc @ (ik / 3.0 * o1["Dx"])
    blk[3][2] = visc @ (ik / 3.0 * o2["Dy"])
    blk[3][3] = adv(3) + visc @ (o3["lap"] - (4.0 / 3.0) * kz ** 2 * eye) - dg(sig)
    L = None
    for a in range(4):
        for b in range(4):
            e = sp.csr_matrix(([1.0], ([a], [b])), shape=(4, 4))
            term = sp.kron(sp.csr_matrix(blk[a][b], dtype=np.complex128), e, format="csr")
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
