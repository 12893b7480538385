"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module holds no arithmetic of the method: it only describes grids,
evaluates the analytic synthetic base flows on them, and lists the
frequencies and seeds of each workload.  The paper's airfoil base flow
(Sec. III.A, an LES mean of a NACA 0012 wing at Re=23,000, M=0.3) is not
available, so every workload here is synthetic: a tanh shear layer with a
Gaussian recirculation bubble, which reproduces the ingredients that make the
airfoil resolvent interesting (strong shear, reverse flow, a sponge at the
boundaries).

Unknowns are ordered by streamwise column: n = ((ix * ny) + iy) * q + c, so
the block of column ix is contiguous with size b = q * ny.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

KIND_ADVDIFF = 1  # scalar linearised advection-diffusion, q = 1
KIND_NS2D = 3     # isothermal compressible Navier-Stokes (rho, u, v), q = 3
KIND_NS2D_KZ = 4  # bi-global: (rho, u, v, w) ~ exp(i kz z) about a z-invariant flow, q = 4


@dataclasses.dataclass(frozen=True)
class Grid:
    kind: int
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    re: float
    mach: float = 0.0
    sponge_max: float = 0.0
    sponge_frac: float = 0.1
    periodic_y: bool = False
    # boundary closure: per side (x0, x1, y0, y1) a bit mask over the q
    # variables whose ghost node equals the adjacent interior node (Neumann);
    # clear bits keep the zero (Dirichlet) ghost
    neumann: tuple = (0, 0, 0, 0)
    # spanwise wavenumber of the bi-global operator (KIND_NS2D_KZ)
    kz: float = 0.0

    @property
    def q(self) -> int:
        return {KIND_ADVDIFF: 1, KIND_NS2D_KZ: 4}.get(self.kind, 3)

    @property
    def b(self) -> int:
        return self.q * self.ny

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.q

    @property
    def npts(self) -> int:
        return self.nx * self.ny

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / (self.nx + 1)

    @property
    def dy(self) -> float:
        if self.periodic_y:
            return (self.y1 - self.y0) / self.ny
        return (self.y1 - self.y0) / (self.ny + 1)

    def coords(self):
        """Interior node coordinates (x[nx], y[ny]).

        Dirichlet directions hold nx interior nodes at spacing L/(n+1); a
        periodic y direction holds ny nodes at spacing L/ny starting at y0.
        """
        x = self.x0 + self.dx * np.arange(1, self.nx + 1)
        if self.periodic_y:
            y = self.y0 + self.dy * np.arange(self.ny)
        else:
            y = self.y0 + self.dy * np.arange(1, self.ny + 1)
        return x, y

    def mesh(self):
        x, y = self.coords()
        return np.meshgrid(x, y, indexing="ij")  # arrays [nx, ny]


@dataclasses.dataclass
class BaseFlow:
    """Base-flow fields on the interior nodes, each [nx, ny] float64."""
    rho: np.ndarray
    u: np.ndarray
    v: np.ndarray


@dataclasses.dataclass
class Workload:
    name: str
    grid: Grid
    flow: BaseFlow
    omegas: np.ndarray      # real frequencies; shift s = i * omega
    k: int
    seed0: int              # Omega seed of frequency j is seed0 + j
    phi_weighted: bool      # base-flow-weighted Gaussian columns (Eq. 9)


def shear_bubble_flow(grid: Grid) -> BaseFlow:
    """Synthetic separated base flow.

    U = U_s(y) (1 - G) - 0.2 G with U_s = (1 + tanh(y / 0.5)) / 2 and the
    recirculation bubble G = exp(-((x-6)/3)^2 - ((y+0.5)/0.75)^2); V = 0,
    rho = 1.  The reverse velocity peaks at exactly -0.2 at the bubble centre.
    """
    X, Y = grid.mesh()
    us = 0.5 * (1.0 + np.tanh(Y / 0.5))
    g = np.exp(-((X - 6.0) / 3.0) ** 2 - ((Y + 0.5) / 0.75) ** 2)
    u = us * (1.0 - g) - 0.2 * g
    return BaseFlow(rho=np.ones_like(X), u=u, v=np.zeros_like(X))


def tanh_shear_flow(grid: Grid) -> BaseFlow:
    """U = tanh(y), V = 0 (scalar advection-diffusion workload)."""
    X, Y = grid.mesh()
    return BaseFlow(rho=np.ones_like(X), u=np.tanh(Y), v=np.zeros_like(X))


def zero_flow(grid: Grid, v_const: float = 0.0) -> BaseFlow:
    X, _ = grid.mesh()
    return BaseFlow(rho=np.ones_like(X), u=np.zeros_like(X),
                    v=np.full_like(X, v_const))


def smooth_random_flow(grid: Grid, seed: int, amp: float = 0.05) -> BaseFlow:
    """Shear-bubble flow plus a smooth seeded perturbation of rho, U and V.

    Used for the general (rho != 1, V != 0) operator terms.
    """
    rng = np.random.default_rng(seed)
    base = shear_bubble_flow(grid)
    X, Y = grid.mesh()
    out = []
    for f in (base.rho, base.u, base.v):
        a, b, c, d = rng.uniform(0.3, 1.2, size=4)
        ph = rng.uniform(0, 2 * math.pi, size=2)
        out.append(f + amp * np.sin(a * X + ph[0]) * np.cos(b * Y + ph[1])
                   + amp * 0.5 * np.cos(c * X) * np.sin(d * Y))
    return BaseFlow(rho=out[0], u=out[1], v=out[2])


def log_omegas(n: int, lo: float = 0.1, hi: float = 5.0) -> np.ndarray:
    return np.exp(np.linspace(math.log(lo), math.log(hi), n))


# Sec. III.A's closure in (rho', u', v'): Neumann pressure (= rho' in the
# isothermal model) with Dirichlet velocities at the far field, Neumann for
# every variable at the outlet x1
PAPER_NEUMANN = (1, 7, 1, 1)


def ns_grid(nx: int, ny: int, re: float = 500.0, mach: float = 0.3,
            neumann: tuple = (0, 0, 0, 0)) -> Grid:
    return Grid(kind=KIND_NS2D, nx=nx, ny=ny, x0=0.0, x1=20.0, y0=-5.0,
                y1=5.0, re=re, mach=mach, sponge_max=1.0, sponge_frac=0.1,
                neumann=tuple(neumann))


def kz_grid(nx: int, ny: int, kz: float, re: float = 500.0, mach: float = 0.3,
            neumann: tuple = (0, 0, 0, 0)) -> Grid:
    """The bi-global operator (rho, u, v, w) at spanwise wavenumber kz on the
    same domain and sponge as ns_grid (Sec. III.A/B: k_z L_c in {0, 20 pi})."""
    return Grid(kind=KIND_NS2D_KZ, nx=nx, ny=ny, x0=0.0, x1=20.0, y0=-5.0,
                y1=5.0, re=re, mach=mach, sponge_max=1.0, sponge_frac=0.1,
                neumann=tuple(neumann), kz=float(kz))


def config_tiny() -> Workload:
    """Scalar advection-diffusion, 32x32 on [0,10]x[-5,5], Re=100, w=0.5, k=10."""
    g = Grid(kind=KIND_ADVDIFF, nx=32, ny=32, x0=0.0, x1=10.0, y0=-5.0,
             y1=5.0, re=100.0)
    return Workload("advdiff-32x32-k10", g, tanh_shear_flow(g),
                    np.array([0.5]), 10, 1000, False)


def config_fp64() -> Workload:
    """Isothermal NS about the shear-bubble flow, 256x128 (N=98,304, b=384),
    32 frequencies log-spaced in [0.1, 5], k=16 base-flow-weighted columns."""
    g = ns_grid(256, 128)
    return Workload("ns2d-256x128-k16", g, shear_bubble_flow(g),
                    log_omegas(32), 16, 1000, True)


def config_mixed() -> Workload:
    """Same operator on 512x256 (N=393,216, b=768), 64 frequencies, k=32."""
    g = ns_grid(512, 256)
    return Workload("ns2d-512x256-k32", g, shear_bubble_flow(g),
                    log_omegas(64), 32, 1000, True)


def config_small_ns(nx: int = 24, ny: int = 20, k: int = 8,
                    nfreq: int = 3) -> Workload:
    """Small NS case the oracle finishes in seconds (several tiles + ragged tail)."""
    g = ns_grid(nx, ny)
    return Workload(f"ns2d-{nx}x{ny}-k{k}", g, shear_bubble_flow(g),
                    log_omegas(nfreq, 0.3, 3.0), k, 1000, True)


@dataclasses.dataclass(frozen=True)
class GradientWorkload:
    grid: Grid
    flow: BaseFlow
    omegas: np.ndarray      # real frequencies; shift s = i * omega
    k: int                  # sketch columns
    J: int                  # objective: sum over omega of sum_{j<J} sigma_j^2
    chunk: int              # frequencies per factorisation chunk
    seed0: int              # Omega seed of frequency j is seed0 + j
    h: float                # central-difference step
    ndir: int               # random base-flow directions
    dir_seed: int           # generator seed of the directions


def config_gradient() -> GradientWorkload:
    """Differentiation workload: d(sum_omega sum_{j<=3} sigma_j^2)/d(rho, U, V)
    on the 256x128 NS grid about the shear-bubble flow, 16 frequencies
    log-spaced in [0.1, 5], k = 16, factors per 4-frequency chunk, checked by
    central differences (h = 1e-6) on 64 standard-normal field directions."""
    g = ns_grid(256, 128)
    return GradientWorkload(g, shear_bubble_flow(g), log_omegas(16), 16, 3, 4, 1000,
                            1e-6, 64, 77)


def gradient_directions(wl: GradientWorkload, n: int | None = None) -> np.ndarray:
    """The first n (default all) random directions [n, 3, nx, ny]."""
    rng = np.random.default_rng(wl.dir_seed)
    n = wl.ndir if n is None else n
    return rng.standard_normal((n, 3, wl.grid.nx, wl.grid.ny))


@dataclasses.dataclass(frozen=True)
class BatchProblem:
    nx: int
    ny: int
    k: int
    omega: float            # shift s = i * omega
    seed: int               # Omega seed


def config_batched(nprob: int = 128, seed: int = 1234,
                   nx_set=(128, 256, 384), ny_set=(64, 128, 192, 256),
                   k_set=(8, 16, 32, 64), omega_lo: float = 0.1,
                   omega_hi: float = 8.0) -> list[BatchProblem]:
    """Uneven batch: nprob NS problems (q = 3, shear-bubble base flow) with
    (nx, ny, k) drawn uniformly from the sets and omega ~ U[omega_lo,
    omega_hi], from one seeded generator; Omega seed of problem i is 1000 + i.
    The defaults are the 128-problem batching workload."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nprob):
        out.append(BatchProblem(nx=int(rng.choice(nx_set)), ny=int(rng.choice(ny_set)),
                                k=int(rng.choice(k_set)),
                                omega=float(rng.uniform(omega_lo, omega_hi)), seed=1000 + i))
    return out
