// Gradient of the summed leading gains with respect to the base flow.
//
// For a simple singular value sigma_j of R = W^{1/2} A^{-1} W^{-1/2},
// A = s I - L, first-order perturbation of the SVD (Eq. 5) gives
// d sigma_j = Re(u_j^H dR v_j) with dR = W^{1/2} A^{-1} dL A^{-1} W^{-1/2},
// so with a_j = A^{-H} W^{1/2} u_j and b_j = A^{-1} W^{-1/2} v_j
//
//   d/dtheta sum_f sum_{j<J} sigma_j^2 = sum_f sum_{j<J} 2 sigma_j Re(a_j^H dL/dtheta b_j).
//
// The two solves reuse the stored factors; this file holds the reverse of the
// per-point assembly (operator.cu): the sensitivity of every stencil
// coefficient, Cbar[n][slot] = sum 2 sigma Re(conj(a[n]) b[nbr(n, slot)]),
// folded through the coefficient formulas into sensitivities of the local
// base-flow quantities (value, first, second and cross differences of rho, U,
// V at each point), and a gather that applies the transposed difference
// stencils to land on the nodal fields.
#include "rr_internal.cuh"

namespace {

struct GradParams {
  int kind, q, nx, ny, periodic, npts;
  double dx, dy, re, c2;
  int neu[4];  // Neumann variable masks of the sides x0, x1, y0, y1
};

// local base-flow quantities per field: value, d/dx, d/dy, d2/dx2, d2/dy2, d2/dxdy
enum { F_VAL = 0, F_DX = 1, F_DY = 2, F_DXX = 3, F_DYY = 4, F_DXY = 5, NFEAT = 6 };
// operator kinds in the assembly: Dx, Dy, Dxx, Dyy, Dxy, diagonal
enum { O_X = 0, O_Y = 1, O_XX = 2, O_YY = 3, O_XY = 4, O_D = 5, NOPS = 6 };

__device__ __forceinline__ int slot(int dx, int dy) { return (dx + 1) * 3 + (dy + 1); }

// Sensitivities of the base-flow quantities at one grid point:
// featbar[pt][field * 6 + feature], fields rho, U, V.
__global__ void grad_local_kernel(GradParams p, const double* __restrict__ flow, int F, int J,
                                  int N, const double2* __restrict__ A,
                                  const double2* __restrict__ B, const double* __restrict__ sigma,
                                  int sstride, double* __restrict__ featbar) {
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= p.npts) return;
  const int i = pt / p.ny, j = pt % p.ny, q = p.q;
  // neighbour point of every slot for every variable: -1 for a Dirichlet
  // ghost, the adjacent interior point for a Neumann ghost (the closure of
  // the assembly)
  int nb[3][9];
  for (int dxo = -1; dxo <= 1; ++dxo)
    for (int dyo = -1; dyo <= 1; ++dyo) {
      const int jx = i + dxo;
      const int jy = nbr_y(j, dyo, p.ny, p.periodic);
      const bool gx = jx < 0 || jx >= p.nx, gy = jy < 0;
      const int mx = gx ? p.neu[jx < 0 ? 0 : 1] : ~0;
      const int my = gy ? p.neu[j + dyo < 0 ? 2 : 3] : ~0;
      for (int in = 0; in < q; ++in) {
        const bool keep = ((mx >> in) & 1) && ((my >> in) & 1);
        nb[in][slot(dxo, dyo)] = keep ? (gx ? i : jx) * p.ny + (gy ? j : jy) : -1;
      }
    }
  const double hx = 1.0 / (2.0 * p.dx), hy = 1.0 / (2.0 * p.dy);
  const double ixx = 1.0 / (p.dx * p.dx), iyy = 1.0 / (p.dy * p.dy);
  const double ixy = 1.0 / (4.0 * p.dx * p.dy);

  // G[o][in][op]: sensitivity of the coefficient a in "a * op" added to
  // equation o acting on variable in (the adjoint of the add* helpers)
  double G[3][3][NOPS];
  for (int o = 0; o < q; ++o)
    for (int in = 0; in < q; ++in) {
      double C[9];
      const int n = pt * q + o;
      for (int s = 0; s < 9; ++s) {
        double acc = 0.0;
        if (nb[in][s] >= 0) {
          const int m = nb[in][s] * q + in;
          for (int f = 0; f < F; ++f) {
            const double2* Af = A + ((size_t)f * N + n) * J;
            const double2* Bf = B + ((size_t)f * N + m) * J;
            for (int jj = 0; jj < J; ++jj) {
              double2 a = Af[jj], b = Bf[jj];
              acc += 2.0 * sigma[(size_t)f * sstride + jj] * (a.x * b.x + a.y * b.y);
            }
          }
        }
        C[s] = acc;
      }
      G[o][in][O_X] = hx * (C[slot(1, 0)] - C[slot(-1, 0)]);
      G[o][in][O_Y] = hy * (C[slot(0, 1)] - C[slot(0, -1)]);
      G[o][in][O_XX] = ixx * (C[slot(1, 0)] + C[slot(-1, 0)] - 2.0 * C[slot(0, 0)]);
      G[o][in][O_YY] = iyy * (C[slot(0, 1)] + C[slot(0, -1)] - 2.0 * C[slot(0, 0)]);
      G[o][in][O_XY] = ixy * (C[slot(1, 1)] + C[slot(-1, -1)] - C[slot(1, -1)] - C[slot(-1, 1)]);
      G[o][in][O_D] = C[slot(0, 0)];
    }

  double fb[3][NFEAT];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < NFEAT; ++b) fb[a][b] = 0.0;
  double(&rb)[NFEAT] = fb[0];
  double(&ub)[NFEAT] = fb[1];
  double(&vb)[NFEAT] = fb[2];

  if (p.kind == RR_ADVDIFF_SCALAR) {
    // L = -U Dx - V Dy + nu lap - s_s
    ub[F_VAL] -= G[0][0][O_X];
    vb[F_VAL] -= G[0][0][O_Y];
  } else {
    const int npts = p.npts;
    const double* R = flow;
    // the same one-sided / re-centred differences as the assembly
    auto at = [&](const double* f, int ii, int jj) { return f[ii * p.ny + jj]; };
    auto d1x = [&](const double* f) {
      if (i == 0) return (at(f, 1, j) - at(f, 0, j)) / p.dx;
      if (i == p.nx - 1) return (at(f, p.nx - 1, j) - at(f, p.nx - 2, j)) / p.dx;
      return (at(f, i + 1, j) - at(f, i - 1, j)) / (2.0 * p.dx);
    };
    auto d1y = [&](const double* f) {
      if (p.periodic)
        return (at(f, i, (j + 1) % p.ny) - at(f, i, (j - 1 + p.ny) % p.ny)) / (2.0 * p.dy);
      if (j == 0) return (at(f, i, 1) - at(f, i, 0)) / p.dy;
      if (j == p.ny - 1) return (at(f, i, p.ny - 1) - at(f, i, p.ny - 2)) / p.dy;
      return (at(f, i, j + 1) - at(f, i, j - 1)) / (2.0 * p.dy);
    };
    const double rho = R[pt];
    const double Rx = d1x(R), Ry = d1y(R);
    const double* U = flow + npts;
    const double* V = flow + 2 * npts;
    const double c2 = p.c2, re = p.re;
    const double ir2 = 1.0 / (rho * rho), ir3 = ir2 / rho;
    // values of the base-flow viscous force fu, fv: the rho' coefficient
    // (c2 Rx - fu)/rho^2 depends on rho through them too
    double fu, fv;
    {
      auto d2x = [&](const double* f) {
        int c = min(max(i, 1), p.nx - 2);
        return (at(f, c - 1, j) - 2.0 * at(f, c, j) + at(f, c + 1, j)) / (p.dx * p.dx);
      };
      auto d2y = [&](const double* f) {
        if (p.periodic)
          return (at(f, i, (j - 1 + p.ny) % p.ny) - 2.0 * at(f, i, j) +
                  at(f, i, (j + 1) % p.ny)) / (p.dy * p.dy);
        int c = min(max(j, 1), p.ny - 2);
        return (at(f, i, c - 1) - 2.0 * at(f, i, c) + at(f, i, c + 1)) / (p.dy * p.dy);
      };
      auto d1y_at = [&](const double* f, int ii) {
        if (p.periodic)
          return (at(f, ii, (j + 1) % p.ny) - at(f, ii, (j - 1 + p.ny) % p.ny)) / (2.0 * p.dy);
        if (j == 0) return (at(f, ii, 1) - at(f, ii, 0)) / p.dy;
        if (j == p.ny - 1) return (at(f, ii, p.ny - 1) - at(f, ii, p.ny - 2)) / p.dy;
        return (at(f, ii, j + 1) - at(f, ii, j - 1)) / (2.0 * p.dy);
      };
      auto dxy = [&](const double* f) {
        if (i == 0) return (d1y_at(f, 1) - d1y_at(f, 0)) / p.dx;
        if (i == p.nx - 1) return (d1y_at(f, p.nx - 1) - d1y_at(f, p.nx - 2)) / p.dx;
        return (d1y_at(f, i + 1) - d1y_at(f, i - 1)) / (2.0 * p.dx);
      };
      const double Uxx = d2x(U), Uyy = d2y(U), Uxy = dxy(U);
      const double Vxx = d2x(V), Vyy = d2y(V), Vxy = dxy(V);
      fu = (Uxx + Uyy + (Uxx + Vxy) / 3.0) / re;
      fv = (Vxx + Vyy + (Uxy + Vyy) / 3.0) / re;
    }
    double mub = 0.0, fub = 0.0, fvb = 0.0;
    // continuity: -U Dx - V Dy - (Ux + Vy) - s_s | -rho Dx - Rx | -rho Dy - Ry
    ub[F_VAL] -= G[0][0][O_X];
    vb[F_VAL] -= G[0][0][O_Y];
    ub[F_DX] -= G[0][0][O_D];
    vb[F_DY] -= G[0][0][O_D];
    rb[F_VAL] -= G[0][1][O_X];
    rb[F_DX] -= G[0][1][O_D];
    rb[F_VAL] -= G[0][2][O_Y];
    rb[F_DY] -= G[0][2][O_D];
    // x-momentum
    rb[F_VAL] += G[1][0][O_X] * c2 * ir2;                   // -c2/rho Dx
    rb[F_DX] += G[1][0][O_D] * c2 * ir2;                    // (c2 Rx - fu)/rho^2
    fub -= G[1][0][O_D] * ir2;
    rb[F_VAL] -= 2.0 * G[1][0][O_D] * (c2 * Rx - fu) * ir3;
    ub[F_VAL] -= G[1][1][O_X];
    vb[F_VAL] -= G[1][1][O_Y];
    mub += G[1][1][O_XX] * (4.0 / 3.0) + G[1][1][O_YY];
    ub[F_DX] -= G[1][1][O_D];
    mub += G[1][2][O_XY] / 3.0;
    ub[F_DY] -= G[1][2][O_D];
    // y-momentum
    rb[F_VAL] += G[2][0][O_Y] * c2 * ir2;
    rb[F_DY] += G[2][0][O_D] * c2 * ir2;
    fvb -= G[2][0][O_D] * ir2;
    rb[F_VAL] -= 2.0 * G[2][0][O_D] * (c2 * Ry - fv) * ir3;
    mub += G[2][1][O_XY] / 3.0;
    vb[F_DX] -= G[2][1][O_D];
    ub[F_VAL] -= G[2][2][O_X];
    vb[F_VAL] -= G[2][2][O_Y];
    mub += G[2][2][O_XX] + G[2][2][O_YY] * (4.0 / 3.0);
    vb[F_DY] -= G[2][2][O_D];
    // mu = 1/(rho re); fu = (Uxx + Uyy + (Uxx + Vxy)/3)/re; fv likewise
    rb[F_VAL] -= mub * ir2 / re;
    ub[F_DXX] += fub * (4.0 / 3.0) / re;
    ub[F_DYY] += fub / re;
    vb[F_DXY] += fub / (3.0 * re);
    vb[F_DXX] += fvb / re;
    vb[F_DYY] += fvb * (4.0 / 3.0) / re;
    ub[F_DXY] += fvb / (3.0 * re);
  }
  double* out = featbar + (size_t)pt * 3 * NFEAT;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < NFEAT; ++b) out[a * NFEAT + b] = fb[a][b];
}

// weight of node t in the first difference at node i (assembly's rule)
__device__ __forceinline__ double w1(int i, int t, int n, double h, int periodic) {
  if (periodic) {
    double r = 0.0;
    if (t == (i + 1) % n) r += 1.0 / (2.0 * h);
    if (t == (i - 1 + n) % n) r -= 1.0 / (2.0 * h);
    return r;
  }
  if (i == 0) return t == 1 ? 1.0 / h : (t == 0 ? -1.0 / h : 0.0);
  if (i == n - 1) return t == n - 1 ? 1.0 / h : (t == n - 2 ? -1.0 / h : 0.0);
  return t == i + 1 ? 1.0 / (2.0 * h) : (t == i - 1 ? -1.0 / (2.0 * h) : 0.0);
}

// weight of node t in the second difference at node i
__device__ __forceinline__ double w2(int i, int t, int n, double h, int periodic) {
  int lo, c, hi;
  if (periodic) {
    c = i; lo = (i - 1 + n) % n; hi = (i + 1) % n;
  } else {
    c = min(max(i, 1), n - 2); lo = c - 1; hi = c + 1;
  }
  double r = 0.0;
  if (t == lo) r += 1.0;
  if (t == hi) r += 1.0;
  if (t == c) r -= 2.0;
  return r / (h * h);
}

// grad[field][node] += sum over points whose local quantities read the node
__global__ void grad_gather_kernel(GradParams p, const double* __restrict__ featbar,
                                   double* __restrict__ grad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 3 * p.npts) return;
  const int fld = e / p.npts, node = e % p.npts;
  const int it = node / p.ny, jt = node % p.ny;
  const int ry = p.periodic ? 1 : 2;
  double acc = 0.0;
  for (int di = -2; di <= 2; ++di) {
    const int i = it + di;
    if (i < 0 || i >= p.nx) continue;
    const double ex = i == it ? 1.0 : 0.0;
    const double wx1 = w1(i, it, p.nx, p.dx, 0), wx2 = w2(i, it, p.nx, p.dx, 0);
    for (int dj = -ry; dj <= ry; ++dj) {
      int j = jt + dj;
      if (p.periodic) j = (j + p.ny) % p.ny;
      else if (j < 0 || j >= p.ny) continue;
      const double ey = j == jt ? 1.0 : 0.0;
      const double wy1 = w1(j, jt, p.ny, p.dy, p.periodic);
      const double wy2 = w2(j, jt, p.ny, p.dy, p.periodic);
      const double* fb = featbar + ((size_t)(i * p.ny + j) * 3 + fld) * NFEAT;
      acc += fb[F_VAL] * ex * ey + fb[F_DX] * wx1 * ey + fb[F_DY] * ex * wy1 +
             fb[F_DXX] * wx2 * ey + fb[F_DYY] * ex * wy2 + fb[F_DXY] * wx1 * wy1;
    }
  }
  grad[e] += acc;
}

}  // namespace

rr_status launch_gain_grad(const OpDev& d, const rr_grid& g, int F, int J, const double2* A,
                           const double2* B, const double* sigma, int sstride, double* featbar,
                           double* grad, cudaStream_t st) {
  GradParams p;
  p.kind = d.kind; p.q = d.q; p.nx = d.nx; p.ny = d.ny; p.periodic = d.periodic;
  p.npts = d.nx * d.ny;
  p.dx = d.dx; p.dy = d.dy; p.re = g.re;
  p.c2 = d.kind == RR_ISO_NS2D ? 1.0 / (g.mach * g.mach) : 0.0;
  for (int e = 0; e < 4; ++e) p.neu[e] = g.neumann[e];
  prof_count(2);
  grad_local_kernel<<<(p.npts + 127) / 128, 128, 0, st>>>(p, d.flow, F, J, d.n, A, B, sigma,
                                                          sstride, featbar);
  RR_CUDA(cudaGetLastError());
  grad_gather_kernel<<<(3 * p.npts + 255) / 256, 256, 0, st>>>(p, featbar, grad);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}
