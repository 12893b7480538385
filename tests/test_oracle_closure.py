"""Pins of the oracle's Neumann boundary closure (Sec. III.A: Neumann pressure
at the far field, Neumann for every variable at the outlet), each fixed by
mathematics independent of the assembly:
  * pure diffusion with the closure on every side, on the x sides only, or at
    the outlet only has closed-form eigenpairs (cosine / sine products of the
    1-D second difference with ghost = end value, or ghost = 0), so
    L v = lambda v is checked for the analytic v and lambda, and the
    resolvent gains are 1/|s - lambda|;
  * constants are in the null space of all-Neumann diffusion;
  * for the Navier-Stokes operator, the closure changes only rows of
    boundary points and only columns of the variables whose bit is set on
    that side (the routing of the per-variable masks).
"""
import numpy as np

import workloads as W
from oracle import operator as op
from oracle import resolvent as rs


def _diffusion_grid(nx, ny, neumann, re=2.0):
    return W.Grid(kind=W.KIND_ADVDIFF, nx=nx, ny=ny, x0=0.0, x1=3.0, y0=-1.0, y1=1.0,
                  re=re, neumann=neumann)


def _modes_1d(n, h, lo, hi):
    """Eigenpairs of the 1-D 3-point second difference on n nodes with ghost
    = end value (Neumann, lo/hi True) or ghost = 0 (Dirichlet)."""
    i = np.arange(n)
    out = []
    for p in range(n):
        if lo and hi:       # DCT-II: cos(p pi (i + 1/2) / n)
            v = np.cos(p * np.pi * (i + 0.5) / n)
            lam = -4.0 / h ** 2 * np.sin(p * np.pi / (2 * n)) ** 2
        elif not lo and not hi:
            v = np.sin((p + 1) * np.pi * (i + 1) / (n + 1))
            lam = -4.0 / h ** 2 * np.sin((p + 1) * np.pi / (2 * (n + 1))) ** 2
        elif hi:            # Dirichlet at the start, Neumann at the end
            v = np.sin((2 * p + 1) * np.pi * (i + 1) / (2 * n + 1))
            lam = -4.0 / h ** 2 * np.sin((2 * p + 1) * np.pi / (2 * (2 * n + 1))) ** 2
        else:
            v = np.sin((2 * p + 1) * np.pi * (n - i) / (2 * n + 1))
            lam = -4.0 / h ** 2 * np.sin((2 * p + 1) * np.pi / (2 * (2 * n + 1))) ** 2
        out.append((lam, v))
    return out


def _check_eigenpairs(neumann):
    g = _diffusion_grid(7, 5, neumann)
    nu = 1.0 / g.re
    L = op.assemble(g, W.zero_flow(g)).toarray()
    mx = _modes_1d(g.nx, g.dx, bool(neumann[0] & 1), bool(neumann[1] & 1))
    my = _modes_1d(g.ny, g.dy, bool(neumann[2] & 1), bool(neumann[3] & 1))
    lams = []
    for lx, vx in mx:
        for ly, vy in my:
            v = np.outer(vx, vy).ravel()
            lam = nu * (lx + ly)
            np.testing.assert_allclose(L @ v, lam * v, atol=1e-11 * np.abs(lam) + 1e-12)
            lams.append(lam)
    return L, np.array(lams)


def test_all_sides_neumann_diffusion_eigenpairs_and_gains():
    L, lam = _check_eigenpairs((1, 1, 1, 1))
    import scipy.sparse as sp
    for s in (0.7j, 0.3 + 2.0j):
        sig = np.sort(1.0 / np.abs(s - lam))[::-1]
        S, U, V = rs.exact_svd(sp.csr_matrix(L), s)
        np.testing.assert_allclose(S[:10], sig[:10], rtol=1e-12)


def test_mixed_and_outlet_only_closures_eigenpairs():
    _check_eigenpairs((1, 1, 0, 0))   # Neumann in x, Dirichlet in y
    _check_eigenpairs((0, 1, 0, 0))   # outlet only
    _check_eigenpairs((1, 0, 0, 1))   # inlet and top


def test_constants_span_the_null_space_of_all_neumann_diffusion():
    g = _diffusion_grid(9, 6, (1, 1, 1, 1))
    L = op.assemble(g, W.zero_flow(g))
    assert np.max(np.abs(L @ np.ones(g.n))) < 1e-12
    # and the Dirichlet operator is not singular on constants
    g0 = _diffusion_grid(9, 6, (0, 0, 0, 0))
    assert np.max(np.abs(op.assemble(g0, W.zero_flow(g0)) @ np.ones(g0.n))) > 1.0


def test_ns_closure_touches_only_boundary_rows_and_masked_variables():
    nx, ny, q = 8, 7, 3
    masks = W.PAPER_NEUMANN
    g1 = W.ns_grid(nx, ny, neumann=masks)
    g0 = W.ns_grid(nx, ny)
    flow = W.smooth_random_flow(g0, 3)
    D = (op.assemble(g1, flow) - op.assemble(g0, flow)).tocoo()
    assert D.nnz > 0
    for r, c, val in zip(D.row, D.col, D.data):
        if abs(val) < 1e-14:
            continue
        pr, pc, var = r // q, c // q, c % q
        ix, iy = divmod(pr, ny)
        jx, jy = divmod(pc, ny)
        sides = []
        if ix == 0:
            sides.append(0)
        if ix == nx - 1:
            sides.append(1)
        if iy == 0:
            sides.append(2)
        if iy == ny - 1:
            sides.append(3)
        assert sides, "closure changed an interior row"
        # the column is the row's point or a boundary neighbour of it, and its
        # variable has the Neumann bit on a side the row lies on
        assert abs(ix - jx) <= 1 and abs(iy - jy) <= 1
        assert any((masks[sd] >> var) & 1 for sd in sides)
    # the velocity columns change only at the outlet (bit set on x1 alone)
    for r, c, val in zip(D.row, D.col, D.data):
        if abs(val) > 1e-14 and c % q in (1, 2):
            assert (r // q) // ny == nx - 1
