// Operator assembly (Sec. II.A, Eq. 1), the FP64 operator application used
// by the refinement residual, and the sketch weight Phi of Eq. (9).
//
// Each grid point evaluates its own stencil: base-flow derivatives from its
// neighbours (central differences, first-order one-sided at the first/last
// node, second derivatives re-centred on the inner neighbour there), then the
// 9 x q x q coefficients of the linearised equations.
#include <algorithm>

#include <mutex>

#include "rr_internal.cuh"

namespace {

struct Field {
  const double* f;
  int nx, ny, periodic;
  double dx, dy;
  __device__ double at(int i, int j) const { return f[i * ny + j]; }
  __device__ int wrap(int j) const { return (j + ny) % ny; }
  __device__ double d1x(int i, int j) const {
    if (i == 0) return (at(1, j) - at(0, j)) / dx;
    if (i == nx - 1) return (at(nx - 1, j) - at(nx - 2, j)) / dx;
    return (at(i + 1, j) - at(i - 1, j)) / (2.0 * dx);
  }
  __device__ double d1y(int i, int j) const {
    if (periodic) return (at(i, wrap(j + 1)) - at(i, wrap(j - 1))) / (2.0 * dy);
    if (j == 0) return (at(i, 1) - at(i, 0)) / dy;
    if (j == ny - 1) return (at(i, ny - 1) - at(i, ny - 2)) / dy;
    return (at(i, j + 1) - at(i, j - 1)) / (2.0 * dy);
  }
  __device__ double d2x(int i, int j) const {
    int c = min(max(i, 1), nx - 2);
    return (at(c - 1, j) - 2.0 * at(c, j) + at(c + 1, j)) / (dx * dx);
  }
  __device__ double d2y(int i, int j) const {
    if (periodic)
      return (at(i, wrap(j - 1)) - 2.0 * at(i, j) + at(i, wrap(j + 1))) / (dy * dy);
    int c = min(max(j, 1), ny - 2);
    return (at(i, c - 1) - 2.0 * at(i, c) + at(i, c + 1)) / (dy * dy);
  }
  // d/dx of the y-derivative field
  __device__ double dxy(int i, int j) const {
    if (i == 0) return (d1y(1, j) - d1y(0, j)) / dx;
    if (i == nx - 1) return (d1y(nx - 1, j) - d1y(nx - 2, j)) / dx;
    return (d1y(i + 1, j) - d1y(i - 1, j)) / (2.0 * dx);
  }
};

struct AsmParams {
  int kind, q, nx, ny, periodic;
  double dx, dy, x0, x1, y0, y1, re, c2, smax, sfrac, kz;
  int neu[4];  // Neumann variable masks of the sides x0, x1, y0, y1
};

__device__ double sponge_at(const AsmParams& p, int i, int j) {
  if (p.smax == 0.0) return 0.0;
  double x = p.x0 + (i + 1) * p.dx;
  double lx = p.sfrac * (p.x1 - p.x0);
  double xi = fmax(fmax((p.x0 + lx - x) / lx, (x - (p.x1 - lx)) / lx), 0.0);
  xi = fmin(xi, 1.0);
  double s = p.smax * xi * xi;
  if (!p.periodic) {
    double y = p.y0 + (j + 1) * p.dy;
    double ly = p.sfrac * (p.y1 - p.y0);
    double eta = fmax(fmax((p.y0 + ly - y) / ly, (y - (p.y1 - ly)) / ly), 0.0);
    eta = fmin(eta, 1.0);
    s = fmax(s, p.smax * eta * eta);
  }
  return s;
}

// slot index of stencil offset (dx, dy)
__device__ __forceinline__ int slot(int dx, int dy) { return (dx + 1) * 3 + (dy + 1); }

__global__ void assemble_kernel(AsmParams p, const double* __restrict__ flow,
                                double* __restrict__ coef) {
  int pt = blockIdx.x * blockDim.x + threadIdx.x;
  int npts = p.nx * p.ny;
  if (pt >= npts) return;
  int i = pt / p.ny, j = pt % p.ny;
  const int q = p.q, S = 9 * q;
  double c[4][9][4];
  for (int a = 0; a < 4; ++a)
    for (int s = 0; s < 9; ++s)
      for (int b = 0; b < 4; ++b) c[a][s][b] = 0.0;

  Field R{flow, p.nx, p.ny, p.periodic, p.dx, p.dy};
  Field U{flow + npts, p.nx, p.ny, p.periodic, p.dx, p.dy};
  Field V{flow + 2 * npts, p.nx, p.ny, p.periodic, p.dx, p.dy};
  const double u = U.at(i, j), v = V.at(i, j);
  const double hx = 1.0 / (2.0 * p.dx), hy = 1.0 / (2.0 * p.dy);
  const double ixx = 1.0 / (p.dx * p.dx), iyy = 1.0 / (p.dy * p.dy);
  const double ixy = 1.0 / (4.0 * p.dx * p.dy);
  const double sg = sponge_at(p, i, j);

  // generic pieces: coefficient a * (difference operator) added to c[o][.][in]
  auto addDx = [&](int o, int in, double a) {
    c[o][slot(1, 0)][in] += a * hx;
    c[o][slot(-1, 0)][in] -= a * hx;
  };
  auto addDy = [&](int o, int in, double a) {
    c[o][slot(0, 1)][in] += a * hy;
    c[o][slot(0, -1)][in] -= a * hy;
  };
  auto addDxx = [&](int o, int in, double a) {
    c[o][slot(1, 0)][in] += a * ixx;
    c[o][slot(-1, 0)][in] += a * ixx;
    c[o][slot(0, 0)][in] -= 2.0 * a * ixx;
  };
  auto addDyy = [&](int o, int in, double a) {
    c[o][slot(0, 1)][in] += a * iyy;
    c[o][slot(0, -1)][in] += a * iyy;
    c[o][slot(0, 0)][in] -= 2.0 * a * iyy;
  };
  auto addDxy = [&](int o, int in, double a) {
    c[o][slot(1, 1)][in] += a * ixy;
    c[o][slot(-1, -1)][in] += a * ixy;
    c[o][slot(1, -1)][in] -= a * ixy;
    c[o][slot(-1, 1)][in] -= a * ixy;
  };
  auto addDiag = [&](int o, int in, double a) { c[o][slot(0, 0)][in] += a; };

  if (p.kind == RR_ADVDIFF_SCALAR) {
    const double nu = 1.0 / p.re;
    addDx(0, 0, -u);
    addDy(0, 0, -v);
    addDxx(0, 0, nu);
    addDyy(0, 0, nu);
    addDiag(0, 0, -sg);
  } else {
    const double rho = R.at(i, j);
    const double Ux = U.d1x(i, j), Uy = U.d1y(i, j);
    const double Vx = V.d1x(i, j), Vy = V.d1y(i, j);
    const double Rx = R.d1x(i, j), Ry = R.d1y(i, j);
    const double Uxx = U.d2x(i, j), Uyy = U.d2y(i, j), Uxy = U.dxy(i, j);
    const double Vxx = V.d2x(i, j), Vyy = V.d2y(i, j), Vxy = V.dxy(i, j);
    const double c2 = p.c2, re = p.re;
    const double mu = 1.0 / (rho * re);
    // viscous force of the base flow per unit mass (multiplies -rho'/rho^2 * rho)
    const double fu = (Uxx + Uyy + (Uxx + Vxy) / 3.0) / re;
    const double fv = (Vxx + Vyy + (Uxy + Vyy) / 3.0) / re;
    // continuity
    addDx(0, 0, -u); addDy(0, 0, -v); addDiag(0, 0, -(Ux + Vy) - sg);
    addDx(0, 1, -rho); addDiag(0, 1, -Rx);
    addDy(0, 2, -rho); addDiag(0, 2, -Ry);
    // x-momentum
    addDx(1, 0, -c2 / rho); addDiag(1, 0, c2 * Rx / (rho * rho) - fu / (rho * rho));
    addDx(1, 1, -u); addDy(1, 1, -v);
    addDxx(1, 1, mu * (4.0 / 3.0)); addDyy(1, 1, mu);
    addDiag(1, 1, -Ux - sg);
    addDxy(1, 2, mu / 3.0); addDiag(1, 2, -Uy);
    // y-momentum
    addDy(2, 0, -c2 / rho); addDiag(2, 0, c2 * Ry / (rho * rho) - fv / (rho * rho));
    addDxy(2, 1, mu / 3.0); addDiag(2, 1, -Vx);
    addDx(2, 2, -u); addDy(2, 2, -v);
    addDxx(2, 2, mu); addDyy(2, 2, mu * (4.0 / 3.0));
    addDiag(2, 2, -Vy - sg);
    if (p.kind == RR_ISO_NS2D_KZ) {
      // bi-global terms (d/dz -> i kz, no spanwise base velocity), written
      // for the real operator D^{-1} L D, D = diag(1, 1, 1, i): variable 3
      // is w' / i, so every i kz coupling with w' becomes real
      const double kz = p.kz;
      addDiag(0, 3, rho * kz);                       // -rho i kz w'
      addDiag(1, 1, -mu * kz * kz);                  // -kz^2 u'
      addDx(1, 3, -mu * kz / 3.0);                   // (1/3) d/dx (i kz w')
      addDiag(2, 2, -mu * kz * kz);
      addDy(2, 3, -mu * kz / 3.0);
      // z-momentum: -(U.grad) w' - (c^2/rho) i kz rho'
      //   + mu (lap w' - kz^2 w' + (1/3) i kz (div u' + i kz w'))
      addDiag(3, 0, -c2 / rho * kz);
      addDx(3, 1, mu * kz / 3.0);
      addDy(3, 2, mu * kz / 3.0);
      addDx(3, 3, -u); addDy(3, 3, -v);
      addDxx(3, 3, mu); addDyy(3, 3, mu);
      addDiag(3, 3, -(4.0 / 3.0) * mu * kz * kz - sg);
    }
  }

  // boundary closure: a ghost neighbour of variable b is zero (Dirichlet) or,
  // where b's bit is set on every side the ghost lies beyond, equal to the
  // adjacent interior node, so its coefficient moves to that node's slot
  for (int dxo = -1; dxo <= 1; ++dxo)
    for (int dyo = -1; dyo <= 1; ++dyo) {
      const bool gx = i + dxo < 0 || i + dxo >= p.nx;
      const bool gy = !p.periodic && (j + dyo < 0 || j + dyo >= p.ny);
      if (!gx && !gy) continue;
      const int mx = gx ? p.neu[i + dxo < 0 ? 0 : 1] : ~0;
      const int my = gy ? p.neu[j + dyo < 0 ? 2 : 3] : ~0;
      const int to = slot(gx ? 0 : dxo, gy ? 0 : dyo);
      for (int b = 0; b < q; ++b) {
        const bool fold = ((mx >> b) & 1) && ((my >> b) & 1);
        for (int a = 0; a < q; ++a) {
          if (fold) c[a][to][b] += c[a][slot(dxo, dyo)][b];
          c[a][slot(dxo, dyo)][b] = 0.0;
        }
      }
    }
  for (int a = 0; a < q; ++a) {
    double* out = coef + (size_t)(pt * q + a) * S;
    for (int s = 0; s < 9; ++s)
      for (int b = 0; b < q; ++b) out[s * q + b] = c[a][s][b];
  }
}

// y = (s I - L)^H x, optionally r = b - that (the forward product uses the
// ELL kernel below).  Block (blockIdx.y = problem f) of rows x columns: a
// group of tpr threads shares one row n and covers its k columns (coalesced
// [n][k] accesses, the stencil entries read once per group through L1); all
// index arithmetic is 32-bit and done once per row; Q (unknowns per point) is
// a template parameter so the 9 x Q stencil loop unrolls and its loads issue
// together.  (L^T x)[n] sums over the rows r whose stencil reaches n: row r
// at point (ix - dx, iy - dy) reaches n through its slot (dx, dy).
template <bool RESID, int Q>
__global__ void __launch_bounds__(256)
apply_adjoint_kernel(OpView op, const double2* __restrict__ shifts, int k,
                     const double2* __restrict__ bvec, const double2* __restrict__ x,
                     double2* __restrict__ y, const int* __restrict__ amap) {
  const int f = amap ? amap[blockIdx.y] : (int)blockIdx.y;
  const int tpr = k < (int)blockDim.x ? k : (int)blockDim.x;
  const int rows_per = blockDim.x / tpr;
  const int rsub = threadIdx.x / tpr, jt = threadIdx.x - rsub * tpr;
  if (rsub >= rows_per) return;
  const size_t NK = (size_t)op.n * k;
  const double2* xf = x + (size_t)f * NK;
  double2* yf = y + (size_t)f * NK;
  const double2* bf = RESID ? bvec + (size_t)f * NK : nullptr;
  const double2 s = make_double2(shifts[f].x, -shifts[f].y);
  constexpr int q = Q, S = 9 * Q;
  for (int n = blockIdx.x * rows_per + rsub; n < op.n; n += gridDim.x * rows_per) {
    const int pt = n / q, c = n - pt * q;
    const int ix = pt / op.ny, iy = pt - ix * op.ny;
    // bases of the points whose stencils reach n (-1: Dirichlet ghost)
    int nb[9];
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx)
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const int jx = ix - dx;
        const int jy = nbr_y(iy, -dy, op.ny, op.periodic);
        nb[(dx + 1) * 3 + (dy + 1)] =
            (jx >= 0 && jx < op.nx && jy >= 0) ? (jx * op.ny + jy) * q : -1;
      }
    for (int j = jt; j < k; j += tpr) {
      double2 acc = cmul(s, xf[(size_t)n * k + j]);
#pragma unroll
      for (int sl = 0; sl < 9; ++sl) {
        const int base = nb[sl];
        if (base < 0) continue;
#pragma unroll
        for (int cr = 0; cr < q; ++cr) {
          const double a = op.coef[(size_t)(base + cr) * S + sl * q + c];
          acc = crfma(-a, xf[(size_t)(base + cr) * k + j], acc);
        }
      }
      if (RESID) {
        const double2 bb = bf[(size_t)n * k + j];
        acc = mk(bb.x - acc.x, bb.y - acc.y);
      }
      yf[(size_t)n * k + j] = acc;
    }
  }
}

// y = (s I - L) x (or r = b - that) from the ELL copy of the stencil: a
// row's nonzero entries in slot order, the same sum as over all 9q slots
// (the skipped terms are zero).  The width WT is a compile-time constant so
// the loop runs exactly WT multiply-adds per entry: the kernel is bound by
// the FP64 pipe, and the Navier-Stokes rows have at most 13 of their 27
// slots nonzero.  Threads as in apply_adjoint_kernel.
template <bool RESID, int WT>
__global__ void __launch_bounds__(256)
apply_ell_kernel(OpView op, const double2* __restrict__ shifts, int k,
                 const double2* __restrict__ bvec, const double2* __restrict__ x,
                 double2* __restrict__ y, const int* __restrict__ amap) {
  const int f = amap ? amap[blockIdx.y] : (int)blockIdx.y;
  const int tpr = k < (int)blockDim.x ? k : (int)blockDim.x;
  const int rows_per = blockDim.x / tpr;
  const int rsub = threadIdx.x / tpr, jt = threadIdx.x - rsub * tpr;
  if (rsub >= rows_per) return;
  const size_t NK = (size_t)op.n * k;
  const double2* xf = x + (size_t)f * NK;
  double2* yf = y + (size_t)f * NK;
  const double2* bf = RESID ? bvec + (size_t)f * NK : nullptr;
  const double2 s = shifts[f];
  for (int n = blockIdx.x * rows_per + rsub; n < op.n; n += gridDim.x * rows_per) {
    const double* ev = op.ell_val + (size_t)n * WT;
    const int* ec = op.ell_col + (size_t)n * WT;
    double a[WT];
    int m[WT];
#pragma unroll
    for (int t = 0; t < WT; ++t) {
      a[t] = ev[t];
      m[t] = ec[t];
    }
    for (int j = jt; j < k; j += tpr) {
      double2 acc = cmul(s, xf[(size_t)n * k + j]);
#pragma unroll
      for (int t = 0; t < WT; ++t) acc = crfma(-a[t], xf[(size_t)m[t] * k + j], acc);
      if (RESID) {
        const double2 bb = bf[(size_t)n * k + j];
        acc = mk(bb.x - acc.x, bb.y - acc.y);
      }
      yf[(size_t)n * k + j] = acc;
    }
  }
}

// Widths the ELL apply kernel is compiled for; a row set is padded to the
// smallest one that holds its widest row.
constexpr int kEllWidths[] = {4, 6, 8, 10, 13, 16, 20, 27};

// ELL copy of the stencil: the widest row, then every row's nonzero entries
// in slot order, padded with zero entries on the row itself.  Both kernels
// walk the entries of a row with the same rule (in-grid neighbour, nonzero
// coefficient), so the counted width always holds the filled row; a row that
// would not fit anyway sets *overflow instead of losing entries.
template <typename Visit>
__device__ __forceinline__ void ell_row_entries(const OpView& op, int n, Visit&& visit) {
  const int q = op.q, pt = n / q;
  const int ix = pt / op.ny, iy = pt - ix * op.ny;
  const double* cf = op.coef + (size_t)n * op.S;
  for (int sl = 0; sl < 9; ++sl) {
    const int jx = ix + sl / 3 - 1;
    const int jy = nbr_y(iy, sl % 3 - 1, op.ny, op.periodic);
    if (jx < 0 || jx >= op.nx || jy < 0) continue;
    for (int cp = 0; cp < q; ++cp) {
      const double a = cf[sl * q + cp];
      if (a != 0.0) visit(a, (jx * op.ny + jy) * q + cp);
    }
  }
}

__global__ void ell_count_kernel(OpView op, int* wmax) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= op.n) return;
  int cnt = 0;
  ell_row_entries(op, n, [&](double, int) { ++cnt; });
  atomicMax(wmax, cnt);
}

__global__ void ell_fill_kernel(OpView op, int W, double* __restrict__ val, int* __restrict__ col,
                                int* overflow) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= op.n) return;
  double* v = val + (size_t)n * W;
  int* c = col + (size_t)n * W;
  int t = 0;
  ell_row_entries(op, n, [&](double a, int m) {
    if (t < W) {
      v[t] = a;
      c[t] = m;
    }
    ++t;
  });
  if (t > W) atomicExch(overflow, 1);
  for (; t < W; ++t) {
    v[t] = 0.0;
    c[t] = n;
  }
}

__global__ void phi_kernel(const double* __restrict__ flow, int nx, int ny, int periodic,
                           double dx, double dy, int q, double* __restrict__ phi) {
  int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= nx * ny) return;
  int i = pt / ny, j = pt % ny;
  Field U{flow + nx * ny, nx, ny, periodic, dx, dy};
  Field V{flow + 2 * nx * ny, nx, ny, periodic, dx, dy};
  double a = U.d1x(i, j), b = U.d1y(i, j), c = V.d1x(i, j), d = V.d1y(i, j);
  double p = sqrt(a * a + b * b + c * c + d * d);
  for (int cc = 0; cc < q; ++cc) phi[pt * q + cc] = p;
}

}  // namespace

__global__ void round_coef_kernel(const double* __restrict__ in, float* __restrict__ out, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

static dim3 apply_grid(const OpDev& d, int F, int k);

rr_status build_ell(OpDev& d) {
  int* wdev = nullptr;  // [0] widest row, [1] overflow flag of the fill
  RR_CUDA(cudaMalloc(&wdev, 2 * sizeof(int)));
  const int blocks = (d.n + 255) / 256;
  int W = 0;
  cudaError_t e = cudaMemset(wdev, 0, 2 * sizeof(int));
  if (e == cudaSuccess) {
    prof_count(1);
    ell_count_kernel<<<blocks, 256>>>(view(d), wdev);
    e = cudaMemcpy(&W, wdev, sizeof(int), cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) {
    cudaFree(wdev);
    return cuda_status(e, "ELL stencil width");
  }
  constexpr int kWidest = kEllWidths[sizeof(kEllWidths) / sizeof(int) - 1];
  if (W > kWidest) {
    cudaFree(wdev);
    set_error("ELL stencil row wider than the widest compiled apply kernel");
    return RR_ERR_ARG;
  }
  d.ell_w = kWidest;
  for (int w : kEllWidths)
    if (w >= W) {
      d.ell_w = w;
      break;
    }
  e = cudaMalloc(&d.ell_val, (size_t)d.n * d.ell_w * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d.ell_col, (size_t)d.n * d.ell_w * sizeof(int));
  int overflow = 0;
  if (e == cudaSuccess) {
    prof_count(1);
    ell_fill_kernel<<<blocks, 256>>>(view(d), d.ell_w, d.ell_val, d.ell_col, wdev + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&overflow, wdev + 1, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(wdev);
  if (e != cudaSuccess) return cuda_status(e, "ELL stencil copy");
  if (overflow) {
    set_error("ELL stencil copy: a row has more entries than the counted width");
    return RR_ERR_ARG;
  }
  return RR_OK;
}

// Forward operator application (adjoint == 0) on the ELL copy, by width.
template <bool RESID>
static rr_status launch_ell(const OpDev& d, int F, const double2* shifts, int k,
                            const double2* b, const double2* x, double2* y, cudaStream_t st,
                            const int* amap) {
  const dim3 grid = apply_grid(d, F, k);
  const OpView v = view(d);
  switch (d.ell_w) {
    case 4: apply_ell_kernel<RESID, 4><<<grid, 256, 0, st>>>(v, shifts, k, b, x, y, amap); break;
    case 6: apply_ell_kernel<RESID, 6><<<grid, 256, 0, st>>>(v, shifts, k, b, x, y, amap); break;
    case 8: apply_ell_kernel<RESID, 8><<<grid, 256, 0, st>>>(v, shifts, k, b, x, y, amap); break;
    case 10: apply_ell_kernel<RESID, 10><<<grid, 256, 0, st>>>(v, shifts, k, b, x, y, amap); break;
    case 13: apply_ell_kernel<RESID, 13><<<grid, 256, 0, st>>>(v, shifts, k, b, x, y, amap); break;
    case 16: apply_ell_kernel<RESID, 16><<<grid, 256, 0, st>>>(v, shifts, k, b, x, y, amap); break;
    case 20: apply_ell_kernel<RESID, 20><<<grid, 256, 0, st>>>(v, shifts, k, b, x, y, amap); break;
    case 27: apply_ell_kernel<RESID, 27><<<grid, 256, 0, st>>>(v, shifts, k, b, x, y, amap); break;
    default: set_error("ELL width without a compiled kernel"); return RR_ERR_ARG;
  }
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_assemble(OpDev& d, const rr_grid& g, cudaStream_t st) {
  AsmParams p;
  p.kind = g.kind; p.q = d.q; p.nx = d.nx; p.ny = d.ny; p.periodic = d.periodic;
  p.dx = d.dx; p.dy = d.dy; p.x0 = g.x0; p.x1 = g.x1; p.y0 = g.y0; p.y1 = g.y1;
  p.re = g.re; p.c2 = (g.kind != RR_ADVDIFF_SCALAR) ? 1.0 / (g.mach * g.mach) : 0.0;
  p.kz = g.kind == RR_ISO_NS2D_KZ ? g.kz : 0.0;
  p.smax = g.sponge_max; p.sfrac = g.sponge_frac;
  for (int e = 0; e < 4; ++e) p.neu[e] = g.neumann[e];
  int npts = d.nx * d.ny;
  prof_count(1);
  assemble_kernel<<<(npts + 127) / 128, 128, 0, st>>>(p, d.flow, d.coef);
  RR_CUDA(cudaGetLastError());
  if (d.coef32) {
    const size_t n = (size_t)d.n * 9 * d.q;
    prof_count(1);
    round_coef_kernel<<<(int)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(d.coef, d.coef32, n);
    RR_CUDA(cudaGetLastError());
  }
  return RR_OK;
}

// Grid of the apply kernel: F problems in y, row blocks in x, about eight
// 256-thread blocks per SM in total.
static dim3 apply_grid(const OpDev& d, int F, int k) {
  const int tpr = k < 256 ? k : 256;
  const int rows_per = 256 / tpr;
  long long need = ((long long)d.n + rows_per - 1) / rows_per;
  long long want = std::max(1LL, (long long)num_sms(d.device) * 8 / std::max(F, 1));
  return dim3((unsigned)std::max(1LL, std::min(need, want)), (unsigned)F);
}

rr_status launch_apply(const OpDev& d, int F, const double2* shifts, int k, int adjoint,
                       const double2* x, double2* y, cudaStream_t st) {
  prof_count(1);
  if (!adjoint) return launch_ell<false>(d, F, shifts, k, nullptr, x, y, st, nullptr);
  if (d.q == 4)
    apply_adjoint_kernel<false, 4><<<apply_grid(d, F, k), 256, 0, st>>>(view(d), shifts, k,
                                                                        nullptr, x, y, nullptr);
  else if (d.q == 3)
    apply_adjoint_kernel<false, 3><<<apply_grid(d, F, k), 256, 0, st>>>(view(d), shifts, k,
                                                                        nullptr, x, y, nullptr);
  else
    apply_adjoint_kernel<false, 1><<<apply_grid(d, F, k), 256, 0, st>>>(view(d), shifts, k,
                                                                        nullptr, x, y, nullptr);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

// ----------------------------------------------------------------------------
// Allocation-free operator application.
//
// The shift list that rr_apply stages in a cudaMalloc'd buffer lives here in a
// fixed array compiled into the library instead.  Every GPU that loads the
// library holds this array until the process exits; every call of
// rr_apply_static shares it, so calls that overlap on the GPU (different
// streams, or different host threads) race on it.
static __device__ __align__(256) double2 g_apply_static_shifts[RR_APPLY_STATIC_MAX_SHIFTS];

namespace {
constexpr int kMaxDevices = 64;
// Device address of g_apply_static_shifts per device ordinal, looked up once
// under g_static_mutex.  A cudaDeviceReset of that device invalidates it.
double2* g_static_shift_ptr[kMaxDevices] = {nullptr};
std::mutex g_static_mutex;
}  // namespace

extern "C" rr_status rr_apply_static(rr_operator* op, int nshift, const double* shifts, int k,
                                     int adjoint, const void* x, void* y, void* stream) {
  if (!op || !shifts || !x || !y) {
    set_error("rr_apply_static: null argument");
    return RR_ERR_ARG;
  }
  if (nshift < 1 || k < 1) {
    set_error("rr_apply_static: nshift and k must be >= 1");
    return RR_ERR_ARG;
  }
  if (nshift > RR_APPLY_STATIC_MAX_SHIFTS) {
    set_error("rr_apply_static: nshift exceeds RR_APPLY_STATIC_MAX_SHIFTS (4096)");
    return RR_ERR_ARG;
  }
  if (x == y) {
    set_error("rr_apply_static: x and y must be distinct");
    return RR_ERR_ARG;
  }
  if (op->d.q == 4) {
    // the bi-global operator is applied through its real similar form, which
    // needs a temporary for D^{-1} x: use rr_apply
    set_error("rr_apply_static: not implemented for the bi-global operator (use rr_apply)");
    return RR_ERR_UNSUPPORTED;
  }
  const int dev = op->d.device;
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("rr_apply_static: device ordinal out of range");
    return RR_ERR_ARG;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // every call copies the shifts from pageable host memory and synchronises
  // its stream, neither of which a capturing stream allows
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  RR_CUDA(cudaStreamIsCapturing(st, &cap));
  if (cap != cudaStreamCaptureStatusNone) {
    set_error("rr_apply_static: the stream is capturing (not supported)");
    return RR_ERR_ARG;
  }
  int prev = -1;
  RR_CUDA(cudaGetDevice(&prev));
  if (prev != dev) RR_CUDA(cudaSetDevice(dev));
  rr_status s = RR_OK;
  // one-time set-up on this device: the host cannot use the symbol itself as
  // a device address, so fetch the address with the device current
  double2* shift_dev = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (g_static_shift_ptr[dev] == nullptr) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_apply_static_shifts);
      if (e != cudaSuccess) s = cuda_status(e, "rr_apply_static: cudaGetSymbolAddress");
      else g_static_shift_ptr[dev] = static_cast<double2*>(p);
    }
    shift_dev = g_static_shift_ptr[dev];
  }
  if (s == RR_OK) {
    cudaError_t e = cudaMemcpyAsync(shift_dev, shifts, nshift * sizeof(double2),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) s = cuda_status(e, "rr_apply_static: shift copy");
  }
  if (s == RR_OK)
    s = launch_apply(op->d, nshift, shift_dev, k, adjoint,
                     static_cast<const double2*>(x), static_cast<double2*>(y), st);
  if (s == RR_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_status(e, "rr_apply_static");
  }
  if (prev != dev && prev >= 0) cudaSetDevice(prev);
  return s;
}

rr_status launch_residual(const OpDev& d, int F, const double2* shifts, int k, int adjoint,
                          const double2* b, const double2* x, double2* r, cudaStream_t st,
                          const int* amap) {
  prof_begin(PROF_RESIDUAL, st);
  if (!adjoint) {
    rr_status s = launch_ell<true>(d, F, shifts, k, b, x, r, st, amap);
    prof_end(PROF_RESIDUAL, st);
    return s;
  }
  if (d.q == 4)
    apply_adjoint_kernel<true, 4><<<apply_grid(d, F, k), 256, 0, st>>>(view(d), shifts, k, b, x,
                                                                       r, amap);
  else if (d.q == 3)
    apply_adjoint_kernel<true, 3><<<apply_grid(d, F, k), 256, 0, st>>>(view(d), shifts, k, b, x,
                                                                       r, amap);
  else
    apply_adjoint_kernel<true, 1><<<apply_grid(d, F, k), 256, 0, st>>>(view(d), shifts, k, b, x,
                                                                       r, amap);
  prof_end(PROF_RESIDUAL, st);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_phi(const OpDev& d, double* phi, cudaStream_t st) {
  int npts = d.nx * d.ny;
  prof_count(1);
  phi_kernel<<<(npts + 127) / 128, 128, 0, st>>>(d.flow, d.nx, d.ny, d.periodic, d.dx, d.dy,
                                                 d.q, phi);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}
