// Dense FP64 kernels of Algorithm 1 around the solves: the Gaussian test
// matrix (first step, Eq. 9), CholeskyQR2 (economy QR, third step), the SVD
// of the small k x N matrix B via its k x k R factor (fifth step), and the
// recovery of sigma_j and u_j by column norms (Eq. 8, seventh and eighth
// steps), plus the sorting and phase normalisation of the outputs.
#include <cmath>

#include "rr_internal.cuh"

namespace {

// ------------------------------------------------------------- Philox 4x32-10
// Salmon et al., SC'11: ten rounds of two 32x32->64 multiplies, the key
// bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k.x += W0; k.y += W1; }
    uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Test-matrix entry (n, j) of problem f from one Philox-4x32-10 block with
// key seeds[f], counter (n, j, 0, 0).  kind 0: Box-Muller normal from the
// four words; kind 1: Rademacher sign, -1 iff bit 0 of w0 is set; kind 2:
// sparse Rademacher, +-mag iff w1 < thresh (thresh = floor(d 2^32), mag =
// 1/sqrt(d)), else 0.
__global__ void philox_kernel(int F, int N, int k, const uint64_t* __restrict__ seeds,
                              const double* __restrict__ phi, const double* __restrict__ wis,
                              double2* __restrict__ out, int kind, uint64_t thresh, double mag) {
  const size_t total = (size_t)F * N * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t NK = (size_t)N * k;
    int f = (int)(e / NK);
    size_t rem = e - (size_t)f * NK;
    uint32_t n = (uint32_t)(rem / k);
    uint32_t j = (uint32_t)(rem - (size_t)n * k);
    uint64_t s = seeds[f];
    uint4 w = philox4x32_10(make_uint4(n, j, 0u, 0u),
                            make_uint2((uint32_t)(s & 0xFFFFFFFFu), (uint32_t)(s >> 32)));
    double g;
    if (kind == 0) {
      uint64_t m1 = ((uint64_t)(w.x >> 5) << 26) + (w.y >> 6);
      uint64_t m2 = ((uint64_t)(w.z >> 5) << 26) + (w.w >> 6);
      double u1 = ((double)m1 + 1.0) * 0x1p-53;
      double u2 = (double)m2 * 0x1p-53;
      g = sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
    } else if (kind == 1) {
      g = (w.x & 1u) ? -1.0 : 1.0;
    } else {
      g = ((uint64_t)w.y < thresh) ? ((w.x & 1u) ? -mag : mag) : 0.0;
    }
    if (phi) g *= phi[n];
    if (wis) g *= wis[n];
    out[e] = make_double2(g, 0.0);
  }
}

__global__ void scale_rows_kernel(int F, int N, int k, const double* __restrict__ w,
                                  double2* __restrict__ x) {
  const size_t total = (size_t)F * N * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t n = (e / k) % N;
    double a = w[n];
    double2 v = x[e];
    x[e] = make_double2(v.x * a, v.y * a);
  }
}

// rows of variable 3 of every point (q = 4) times i (sign > 0) or -i: the
// similarity D = diag(1, 1, 1, i) between the bi-global L and its real form
__global__ void kz_phase_kernel(int F, int N, int k, int sign, double2* __restrict__ x) {
  const size_t total = (size_t)F * N * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t n = (e / k) % N;
    if ((n & 3) != 3) continue;
    const double2 v = x[e];
    x[e] = sign > 0 ? make_double2(-v.y, v.x) : make_double2(v.y, -v.x);
  }
}

__global__ void d2f_kernel(size_t n, const double2* __restrict__ in, float2* __restrict__ out) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    out[e] = make_float2((float)in[e].x, (float)in[e].y);
}

__global__ void f2d_kernel(size_t n, const float2* __restrict__ in, double2* __restrict__ out,
                           int acc) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    double2 v = make_double2((double)in[e].x, (double)in[e].y);
    if (acc) { v.x += out[e].x; v.y += out[e].y; }
    out[e] = v;
  }
}

// The conversions on the problems amap[0..Fa) only: grid (blocks, Fa),
// a grid-stride loop within problem amap[blockIdx.y].
__global__ void d2f_map_kernel(size_t nk, const int* __restrict__ amap,
                               const double2* __restrict__ in, float2* __restrict__ out) {
  const size_t o = (size_t)amap[blockIdx.y] * nk;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nk;
       e += (size_t)gridDim.x * blockDim.x)
    out[o + e] = make_float2((float)in[o + e].x, (float)in[o + e].y);
}

__global__ void f2d_map_kernel(size_t nk, const int* __restrict__ amap,
                               const float2* __restrict__ in, double2* __restrict__ out, int acc) {
  const size_t o = (size_t)amap[blockIdx.y] * nk;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nk;
       e += (size_t)gridDim.x * blockDim.x) {
    double2 v = make_double2((double)in[o + e].x, (double)in[o + e].y);
    if (acc) { v.x += out[o + e].x; v.y += out[o + e].y; }
    out[o + e] = v;
  }
}

// Per-column sum of squares, partials over row blocks: part[slot][blk][j]
// (slot = blockIdx.y, problem active_problem(amap, slot)).
__global__ void colnorm2_part_kernel(int N, int k, int nblk, const double2* __restrict__ x,
                                     double* __restrict__ part, const int* __restrict__ amap) {
  extern __shared__ double red[];
  const int f = active_problem(amap, blockIdx.y), blk = blockIdx.x;
  const int rows_per = (N + nblk - 1) / nblk;
  const int n0 = blk * rows_per, n1 = min(N, n0 + rows_per);
  const double2* xf = x + (size_t)f * N * k;
  // thread t handles column j = t % k over rows strided by blockDim/k
  const int j = threadIdx.x % k;
  const int lane_rows = blockDim.x / k;
  const int rsub = threadIdx.x / k;
  double s = 0.0;
  if (rsub < lane_rows)
    for (int n = n0 + rsub; n < n1; n += lane_rows) {
      double2 v = xf[(size_t)n * k + j];
      s += v.x * v.x + v.y * v.y;
    }
  red[threadIdx.x] = (rsub < lane_rows) ? s : 0.0;
  __syncthreads();
  if (threadIdx.x < k) {
    double t = 0.0;
    for (int r = 0; r < lane_rows; ++r) t += red[r * k + threadIdx.x];
    part[((size_t)blockIdx.y * nblk + blk) * k + threadIdx.x] = t;
  }
}

__global__ void colnorm2_reduce_kernel(int F, int k, int nblk, const double* __restrict__ part,
                                       double* __restrict__ out, const int* __restrict__ amap) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= F * k) return;
  int sl = e / k, j = e % k;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[((size_t)sl * nblk + b) * k + j];
  out[(size_t)active_problem(amap, sl) * k + j] = sqrt(s);
}

// Gram partials part[f][blk][a][c] = sum_n conj(Y[n][a]) Y[n][c].
constexpr int GRAM_ROWS = 32;
__global__ void gram_part_kernel(int N, int k, int nblk, const double2* __restrict__ Y,
                                 double2* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* Ys = reinterpret_cast<double2*>(smem_raw);  // [GRAM_ROWS][k]
  const int f = blockIdx.y, blk = blockIdx.x;
  const int rows_per = (N + nblk - 1) / nblk;
  const int n0 = blk * rows_per, n1 = min(N, n0 + rows_per);
  const double2* Yf = Y + (size_t)f * N * k;
  // G is Hermitian: only the pairs a <= c (k (k+1)/2 of them) are formed
  const int kk = k * k, nup = k * (k + 1) / 2;
  double2 acc[9];
  int pa[9], pc[9];
  const int npair = (nup + blockDim.x - 1) / blockDim.x;  // <= 9 for k <= 64
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    acc[t] = make_double2(0.0, 0.0);
    int rem = threadIdx.x + t * blockDim.x, a = 0;
    while (a < k && rem >= k - a) {
      rem -= k - a;
      ++a;
    }
    pa[t] = a;
    pc[t] = a + rem;
  }
  for (int nb = n0; nb < n1; nb += GRAM_ROWS) {
    const int rows = min(GRAM_ROWS, n1 - nb);
    for (int e = threadIdx.x; e < GRAM_ROWS * k; e += blockDim.x) {
      int r = e / k;
      Ys[e] = (r < rows) ? Yf[(size_t)nb * k + e] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      if (t >= npair) break;
      if (threadIdx.x + t * blockDim.x >= nup) break;
      const int a = pa[t], c = pc[t];
      double2 s = acc[t];
      for (int r = 0; r < rows; ++r) s = cfmac(Ys[r * k + a], Ys[r * k + c], s);
      acc[t] = s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    if (t >= npair || threadIdx.x + t * blockDim.x >= nup) break;
    part[((size_t)f * nblk + blk) * kk + pa[t] * k + pc[t]] = acc[t];
  }
}

__global__ void gram_reduce_kernel(int F, int k, int nblk, const double2* __restrict__ part,
                                   double2* __restrict__ G) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int kk = k * k;
  if (e >= F * kk) return;
  int f = e / kk, p = e % kk;
  const int a = p / k, c = p - a * k;
  // only the upper triangle was formed: G[c][a] = conj(G[a][c])
  const int src = a <= c ? p : c * k + a;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nblk; ++b) s = cadd(s, part[((size_t)f * nblk + b) * kk + src]);
  if (a > c) s.y = -s.y;
  G[e] = s;
}

// Cholesky G (+ shift) = R^H R (R upper) and R^{-1}; one CTA per problem.
// bad[f] = 1 on a non-positive pivot.  cond[f] = max|R_jj| / min|R_jj|.
__global__ void cholesky_kernel(int k, const double2* __restrict__ Gall, double2* __restrict__ Rall,
                                double2* __restrict__ Riall, int* __restrict__ bad,
                                double shift_rel, double* __restrict__ cond) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* A = reinterpret_cast<double2*>(smem_raw);  // [k][k]
  __shared__ double s_shift;
  __shared__ int s_bad;
  const int f = blockIdx.x, kk = k * k;
  const double2* G = Gall + (size_t)f * kk;
  for (int e = threadIdx.x; e < kk; e += blockDim.x) A[e] = G[e];
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int j = 0; j < k; ++j) tr += G[j * k + j].x;
    s_shift = shift_rel * tr;
    s_bad = 0;
  }
  __syncthreads();
  if (threadIdx.x < k) A[threadIdx.x * k + threadIdx.x].x += s_shift;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      double d = A[j * k + j].x;
      if (!(d > 0.0) || !isfinite(d)) { s_bad = 1; d = 1e-300; }
      double r = sqrt(d);
      A[j * k + j] = make_double2(r, 0.0);
    }
    __syncthreads();
    const double rinv = 1.0 / A[j * k + j].x;
    for (int c = j + 1 + threadIdx.x; c < k; c += blockDim.x)
      A[j * k + c] = make_double2(A[j * k + c].x * rinv, A[j * k + c].y * rinv);
    __syncthreads();
    // A[i][c] -= conj(R[j][i]) R[j][c] for j < i <= c
    const int rem = k - j - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      int i = j + 1 + e / rem, c = j + 1 + e % rem;
      if (c >= i) {
        double2 a = A[j * k + i], bb = A[j * k + c];
        double2 v = A[i * k + c];
        v.x -= a.x * bb.x + a.y * bb.y;
        v.y -= a.x * bb.y - a.y * bb.x;
        A[i * k + c] = v;
      }
    }
    __syncthreads();
  }
  double2* R = Rall + (size_t)f * kk;
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    int i = e / k, c = e % k;
    R[e] = (c >= i) ? A[e] : make_double2(0.0, 0.0);
  }
  // R^{-1}: thread per column, back substitution
  double2* Ri = Riall + (size_t)f * kk;
  if (threadIdx.x < k) {
    const int c = threadIdx.x;
    for (int i = k - 1; i >= 0; --i) {
      double2 s = (i == c) ? make_double2(1.0, 0.0) : make_double2(0.0, 0.0);
      if (i <= c)
        for (int m = i + 1; m <= c; ++m) s = csub(s, cmul(A[i * k + m], Ri[m * k + c]));
      else
        s = make_double2(0.0, 0.0);
      Ri[i * k + c] = (i <= c) ? make_double2(s.x / A[i * k + i].x, s.y / A[i * k + i].x)
                               : make_double2(0.0, 0.0);
    }
  }
  if (threadIdx.x == 0) {
    double mx = 0.0, mn = 1e300;
    for (int j = 0; j < k; ++j) {
      double d = fabs(A[j * k + j].x);
      mx = fmax(mx, d);
      mn = fmin(mn, d);
    }
    if (cond) cond[f] = mx / fmax(mn, 1e-300);
    if (s_bad) bad[f] = 1;
  }
}

// out[f][n][:] = Y[f][n][:] . S[f] (k x k); in place allowed (rows staged).
// out = Y S per problem (S k x k row-major).
__global__ void right_mul_kernel(int N, int k, int RB, const double2* Y,
                                 const double2* __restrict__ Sall, double2* out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* S = reinterpret_cast<double2*>(smem_raw);  // [k][k]
  double2* Yr = S + k * k;                             // [RB][k]
  const int f = blockIdx.y;
  const int kk = k * k;
  for (int e = threadIdx.x; e < kk; e += blockDim.x) S[e] = Sall[(size_t)f * kk + e];
  const double2* Yf = Y + (size_t)f * N * k;
  double2* of = out + (size_t)f * N * k;
  for (int n0 = blockIdx.x * RB; n0 < N; n0 += gridDim.x * RB) {
    const int rows = min(RB, N - n0);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * k; e += blockDim.x) Yr[e] = Yf[(size_t)n0 * k + e];
    __syncthreads();
    for (int e = threadIdx.x; e < rows * k; e += blockDim.x) {
      int r = e / k, j = e % k;
      double2 s = make_double2(0.0, 0.0);
      for (int m = 0; m < k; ++m) s = cfma(Yr[r * k + m], S[m * k + j], s);
      of[(size_t)n0 * k + e] = s;
    }
  }
}

// out = Y S with S upper triangular (S[m][j] = 0 for m > j, as the inverse
// Cholesky factors are): column j sums m <= j only, in the same order as the
// dense kernel.  A thread takes the column pair (j, k-1-j), so every thread
// runs k+1 multiply-adds and the FP64 work halves.
__global__ void right_mul_upper_kernel(int N, int k, int RB, const double2* Y,
                                       const double2* __restrict__ Sall, double2* out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* S = reinterpret_cast<double2*>(smem_raw);  // [k][k]
  double2* Yr = S + k * k;                             // [RB][k]
  const int f = blockIdx.y;
  const int kk = k * k, kh = (k + 1) / 2;
  for (int e = threadIdx.x; e < kk; e += blockDim.x) S[e] = Sall[(size_t)f * kk + e];
  const double2* Yf = Y + (size_t)f * N * k;
  double2* of = out + (size_t)f * N * k;
  for (int n0 = blockIdx.x * RB; n0 < N; n0 += gridDim.x * RB) {
    const int rows = min(RB, N - n0);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * k; e += blockDim.x) Yr[e] = Yf[(size_t)n0 * k + e];
    __syncthreads();
    for (int e = threadIdx.x; e < rows * kh; e += blockDim.x) {
      const int r = e / kh, j1 = e - r * kh, j2 = k - 1 - j1;
      const double2* yr = Yr + r * k;
      double2 s1 = make_double2(0.0, 0.0), s2 = make_double2(0.0, 0.0);
      for (int m = 0; m <= j1; ++m) s1 = cfma(yr[m], S[m * k + j1], s1);
      of[(size_t)(n0 + r) * k + j1] = s1;
      if (j2 != j1) {
        for (int m = 0; m <= j2; ++m) s2 = cfma(yr[m], S[m * k + j2], s2);
        of[(size_t)(n0 + r) * k + j2] = s2;
      }
    }
  }
}

__global__ void small_mul_kernel(int k, const double2* __restrict__ A, const double2* __restrict__ B,
                                 double2* __restrict__ C) {
  const int f = blockIdx.x, kk = k * k;
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    int i = e / k, j = e % k;
    double2 s = make_double2(0.0, 0.0);
    for (int m = 0; m < k; ++m) s = cfma(A[(size_t)f * kk + i * k + m], B[(size_t)f * kk + m * k + j], s);
    C[(size_t)f * kk + e] = s;
  }
}

// One-sided Jacobi SVD of a k x k matrix R = Ul diag(sigma) Vr^H, applied to
// the columns of M = R^H (M J = Vr Sigma with J = Ul).  One warp per column
// pair, round-robin ordering, one CTA per problem; sigma sorted descending.
__global__ void jacobi_svd_kernel(int k, int kp, const double2* __restrict__ Rall,
                                  double* __restrict__ sig_out, double2* __restrict__ Ul_out,
                                  double2* __restrict__ Vr_out, int* __restrict__ sweeps_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* A = reinterpret_cast<double2*>(smem_raw);  // column-major [kp cols][kp rows]
  double2* J = A + kp * kp;                            // column-major
  double* nrm = reinterpret_cast<double*>(J + kp * kp);  // [kp]
  int* order = reinterpret_cast<int*>(nrm + kp);        // [kp]
  __shared__ int s_rot;
  const int f = blockIdx.x, kk = k * k;
  const double2* R = Rall + (size_t)f * kk;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int npair = kp / 2;
  // M = R^H: M[row i][col c] = conj(R[c][i]); column c of M stored at A[c*kp + i]
  for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) {
    int c = e / kp, i = e % kp;
    A[e] = (c < k && i < k) ? cconj(R[c * k + i]) : make_double2(0.0, 0.0);
    J[e] = (c == i) ? make_double2(1.0, 0.0) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int step = 0; step < kp - 1; ++step) {
      if (warp < npair) {
        int p, q;
        if (warp == 0) { p = kp - 1; q = step; }
        else {
          p = (step + warp) % (kp - 1);
          q = (step - warp + (kp - 1)) % (kp - 1);
        }
        if (p > q) { int t = p; p = q; q = t; }
        double al = 0.0, be = 0.0;
        double2 ga = make_double2(0.0, 0.0);
        for (int i = lane; i < kp; i += 32) {
          double2 x = A[p * kp + i], y = A[q * kp + i];
          al += x.x * x.x + x.y * x.y;
          be += y.x * y.x + y.y * y.y;
          ga = cfmac(x, y, ga);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga.x += __shfl_xor_sync(0xffffffffu, ga.x, o);
          ga.y += __shfl_xor_sync(0xffffffffu, ga.y, o);
        }
        double g = sqrt(ga.x * ga.x + ga.y * ga.y);
        if (g > 1e-15 * sqrt(al * be) && g > 1e-300) {
          double zeta = (be - al) / (2.0 * g);
          double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          double2 ph = make_double2(ga.x / g, -ga.y / g);  // e^{-i phi}
          for (int i = lane; i < kp; i += 32) {
            double2 x = A[p * kp + i], y = cmul(ph, A[q * kp + i]);
            A[p * kp + i] = make_double2(c * x.x - s * y.x, c * x.y - s * y.y);
            A[q * kp + i] = make_double2(s * x.x + c * y.x, s * x.y + c * y.y);
            double2 u = J[p * kp + i], v = cmul(ph, J[q * kp + i]);
            J[p * kp + i] = make_double2(c * u.x - s * v.x, c * u.y - s * v.y);
            J[q * kp + i] = make_double2(s * u.x + c * v.x, s * u.y + c * v.y);
          }
          if (lane == 0) atomicAdd(&s_rot, 1);
        }
      }
      __syncthreads();
    }
    if (s_rot == 0) break;
    __syncthreads();
  }
  // column norms and descending order (stable by index)
  for (int c = threadIdx.x; c < kp; c += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < kp; ++i) s += cabs2(A[c * kp + i]);
    nrm[c] = (c < k) ? sqrt(s) : -1.0;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    int rank = 0;
    for (int m = 0; m < k; ++m)
      if (nrm[m] > nrm[c] || (nrm[m] == nrm[c] && m < c)) ++rank;
    order[rank] = c;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    int i = e / k, jn = e % k;  // output row i, output column jn
    int c = order[jn];
    double sg = nrm[c];
    Ul_out[(size_t)f * kk + e] = J[c * kp + i];
    double2 a = A[c * kp + i];
    Vr_out[(size_t)f * kk + e] = (sg > 0.0) ? make_double2(a.x / sg, a.y / sg) : make_double2(0.0, 0.0);
  }
  for (int jn = threadIdx.x; jn < k; jn += blockDim.x) sig_out[(size_t)f * k + jn] = nrm[order[jn]];
  if (threadIdx.x == 0 && sweeps_out) sweeps_out[f] = sweep;
}

__global__ void col_scale_kernel(int F, int N, int k, const double2* __restrict__ in,
                                 const double* __restrict__ sigma, double2* __restrict__ out) {
  const size_t total = (size_t)F * N * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int j = (int)(e % k);
    int f = (int)(e / ((size_t)N * k));
    double s = sigma[(size_t)f * k + j];
    double inv = s > 0.0 ? 1.0 / s : 0.0;
    double2 v = in[e];
    out[e] = make_double2(v.x * inv, v.y * inv);
  }
}

// Largest |V[n][j]|^2 per column with its lowest index: partials.
__global__ void colmax_part_kernel(int N, int k, int nblk, const double2* __restrict__ V,
                                   double* __restrict__ pv, int* __restrict__ pi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* rv = reinterpret_cast<double*>(smem_raw);
  int* ri = reinterpret_cast<int*>(rv + blockDim.x);
  const int f = blockIdx.y, blk = blockIdx.x;
  const int rows_per = (N + nblk - 1) / nblk;
  const int n0 = blk * rows_per, n1 = min(N, n0 + rows_per);
  const double2* Vf = V + (size_t)f * N * k;
  const int j = threadIdx.x % k, lane_rows = blockDim.x / k, rsub = threadIdx.x / k;
  double bv = -1.0;
  int bi = N;
  if (rsub < lane_rows)
    for (int n = n0 + rsub; n < n1; n += lane_rows) {
      double a = cabs2(Vf[(size_t)n * k + j]);
      if (a > bv) { bv = a; bi = n; }
    }
  rv[threadIdx.x] = bv;
  ri[threadIdx.x] = bi;
  __syncthreads();
  if (threadIdx.x < k) {
    double v = -1.0;
    int ix = N;
    for (int r = 0; r < lane_rows; ++r) {
      double a = rv[r * k + threadIdx.x];
      int b = ri[r * k + threadIdx.x];
      if (a > v || (a == v && b < ix)) { v = a; ix = b; }
    }
    pv[((size_t)f * nblk + blk) * k + threadIdx.x] = v;
    pi[((size_t)f * nblk + blk) * k + threadIdx.x] = ix;
  }
}

// Sort by sigma descending (stable) and phase-normalise; writes permuted copies.
__global__ void finish_small_kernel(int N, int k, int nblk, const double* __restrict__ pv,
                                    const int* __restrict__ pi, const double2* __restrict__ V,
                                    double* __restrict__ sigma, int* __restrict__ rank_out,
                                    double2* __restrict__ phase_out) {
  const int f = blockIdx.x;
  __shared__ double sg[64];
  const int j = threadIdx.x;
  if (j < k) sg[j] = sigma[(size_t)f * k + j];
  __syncthreads();
  if (j < k) {
    double v = -1.0;
    int ix = N;
    for (int b = 0; b < nblk; ++b) {
      double a = pv[((size_t)f * nblk + b) * k + j];
      int i = pi[((size_t)f * nblk + b) * k + j];
      if (a > v || (a == v && i < ix)) { v = a; ix = i; }
    }
    double2 e = V[((size_t)f * N + ix) * k + j];
    double m = sqrt(e.x * e.x + e.y * e.y);
    phase_out[(size_t)f * k + j] = (m > 0.0) ? make_double2(e.x / m, -e.y / m) : make_double2(1.0, 0.0);
    int rank = 0;
    for (int m2 = 0; m2 < k; ++m2)
      if (sg[m2] > sg[j] || (sg[m2] == sg[j] && m2 < j)) ++rank;
    rank_out[(size_t)f * k + j] = rank;
  }
  __syncthreads();
  if (j < k) sigma[(size_t)f * k + rank_out[(size_t)f * k + j]] = sg[j];
}

__global__ void permute_phase_kernel(int F, int N, int k, const int* __restrict__ rank,
                                     const double2* __restrict__ phase, const double2* __restrict__ in,
                                     double2* __restrict__ out) {
  const size_t total = (size_t)F * N * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int j = (int)(e % k);
    size_t rowbase = e - j;
    int f = (int)(e / ((size_t)N * k));
    int rj = rank[(size_t)f * k + j];
    out[rowbase + rj] = cmul(in[e], phase[(size_t)f * k + j]);
  }
}

int grid1d(size_t total, int threads) {
  size_t b = (total + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

rr_status launch_philox(int F, int N, int k, const uint64_t* seeds, const double* phi,
                        const double* wis, double2* out, cudaStream_t st, int kind,
                        double density) {
  uint64_t thresh = 0;
  double mag = 1.0;
  if (kind == 2) {
    thresh = (uint64_t)std::floor(density * 4294967296.0);
    mag = 1.0 / std::sqrt(density);
  }
  prof_count(1);
  philox_kernel<<<grid1d((size_t)F * N * k, 256), 256, 0, st>>>(F, N, k, seeds, phi, wis, out,
                                                                 kind, thresh, mag);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_scale_rows(int F, int N, int k, const double* w, double2* x, cudaStream_t st) {
  if (!w) return RR_OK;
  prof_count(1);
  scale_rows_kernel<<<grid1d((size_t)F * N * k, 256), 256, 0, st>>>(F, N, k, w, x);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_kz_phase(int F, int N, int k, int q, int sign, double2* x, cudaStream_t st) {
  if (q != 4) return RR_OK;
  prof_count(1);
  kz_phase_kernel<<<grid1d((size_t)F * N * k, 256), 256, 0, st>>>(F, N, k, sign, x);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_convert_d2f(size_t n, const double2* in, float2* out, cudaStream_t st) {
  prof_count(1);
  d2f_kernel<<<grid1d(n, 256), 256, 0, st>>>(n, in, out);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_convert_f2d(size_t n, const float2* in, double2* out, int acc, cudaStream_t st) {
  prof_count(1);
  f2d_kernel<<<grid1d(n, 256), 256, 0, st>>>(n, in, out, acc);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_convert_d2f_map(int Fa, const int* amap, size_t nk, const double2* in,
                                 float2* out, cudaStream_t st) {
  if (Fa <= 0) return RR_OK;
  prof_count(1);
  const int bx = (int)std::min<size_t>((nk + 255) / 256, 1024);
  d2f_map_kernel<<<dim3(bx, Fa), 256, 0, st>>>(nk, amap, in, out);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_convert_f2d_map(int Fa, const int* amap, size_t nk, const float2* in,
                                 double2* out, int acc, cudaStream_t st) {
  if (Fa <= 0) return RR_OK;
  prof_count(1);
  const int bx = (int)std::min<size_t>((nk + 255) / 256, 1024);
  f2d_map_kernel<<<dim3(bx, Fa), 256, 0, st>>>(nk, amap, in, out, acc);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_colnorm2(int F, int N, int k, const double2* x, double* part, int nblk,
                          double* out, cudaStream_t st, const int* amap) {
  int threads = (256 / k) * k;
  prof_count(1);
  colnorm2_part_kernel<<<dim3(nblk, F), threads, threads * sizeof(double), st>>>(N, k, nblk, x, part,
                                                                                 amap);
  prof_count(1);
  colnorm2_reduce_kernel<<<(F * k + 127) / 128, 128, 0, st>>>(F, k, nblk, part, out, amap);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_gram(int F, int N, int k, const double2* Y, double2* part, int nblk, double2* G,
                      cudaStream_t st) {
  size_t smem = (size_t)GRAM_ROWS * k * sizeof(double2);
  prof_begin(PROF_GRAM, st);
  gram_part_kernel<<<dim3(nblk, F), 256, smem, st>>>(N, k, nblk, Y, part);
  prof_end(PROF_GRAM, st);
  prof_count(1);
  gram_reduce_kernel<<<(F * k * k + 127) / 128, 128, 0, st>>>(F, k, nblk, part, G);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_cholesky(int F, int k, const double2* G, double2* R, double2* Rinv, int* bad,
                          double shift_rel, double* cond, cudaStream_t st) {
  size_t smem = (size_t)k * k * sizeof(double2);
  static bool attr = false;
  if (!attr) {
    RR_CUDA(cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 96 * 1024));
    attr = true;
  }
  prof_begin(PROF_SMALL, st);
  cholesky_kernel<<<F, 256, smem, st>>>(k, G, R, Rinv, bad, shift_rel, cond);
  prof_end(PROF_SMALL, st);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_right_mul(int F, int N, int k, const double2* Y, const double2* S, double2* out,
                           cudaStream_t st, int upper) {
  int RB = 64;
  size_t smem = ((size_t)k * k + (size_t)RB * k) * sizeof(double2);
  static bool attr = false;
  if (!attr) {
    RR_CUDA(cudaFuncSetAttribute(right_mul_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 160 * 1024));
    RR_CUDA(cudaFuncSetAttribute(right_mul_upper_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    attr = true;
  }
  int nb = (N + RB - 1) / RB;
  if (nb > 152 * 4 / (F > 0 ? F : 1) + 1) nb = 152 * 4 / (F > 0 ? F : 1) + 1;
  prof_begin(PROF_RIGHTMUL, st);
  if (upper)
    right_mul_upper_kernel<<<dim3(nb, F), 256, smem, st>>>(N, k, RB, Y, S, out);
  else
    right_mul_kernel<<<dim3(nb, F), 256, smem, st>>>(N, k, RB, Y, S, out);
  prof_end(PROF_RIGHTMUL, st);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_small_mul(int F, int k, const double2* A, const double2* B, double2* C,
                           cudaStream_t st) {
  prof_count(1);
  small_mul_kernel<<<F, 256, 0, st>>>(k, A, B, C);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_jacobi_svd(int F, int k, const double2* R, double* sigma, double2* Ul,
                            double2* Vr, int* sweeps, cudaStream_t st) {
  int kp = (k + 1) & ~1;
  if (kp < 2) kp = 2;
  size_t smem = 2 * (size_t)kp * kp * sizeof(double2) + kp * (sizeof(double) + sizeof(int));
  static bool attr = false;
  if (!attr) {
    RR_CUDA(cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 160 * 1024));
    attr = true;
  }
  int threads = 32 * (kp / 2);
  if (threads < 64) threads = 64;
  prof_begin(PROF_SMALL, st);
  jacobi_svd_kernel<<<F, threads, smem, st>>>(k, kp, R, sigma, Ul, Vr, sweeps);
  prof_end(PROF_SMALL, st);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_col_scale(int F, int N, int k, const double2* in, const double* sigma,
                           double2* out, cudaStream_t st) {
  prof_count(1);
  col_scale_kernel<<<grid1d((size_t)F * N * k, 256), 256, 0, st>>>(F, N, k, in, sigma, out);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

// Sort (sigma descending) and phase-normalise U and V in place; tmpU/tmpV are
// [F][N][k] scratch, part holds nblk*k doubles + ints per problem, small holds
// the ranks and phases.
rr_status launch_finish_modes(int F, int N, int k, double2* U, double2* V, double* sigma,
                              double2* tmpU, double2* tmpV, double* part, int nblk,
                              int* rank, double2* phase, cudaStream_t st) {
  int threads = (256 / k) * k;
  double* pv = part;
  int* pi = reinterpret_cast<int*>(part + (size_t)F * nblk * k);
  prof_count(1);
  colmax_part_kernel<<<dim3(nblk, F), threads, threads * (sizeof(double) + sizeof(int)), st>>>(
      N, k, nblk, V, pv, pi);
  prof_count(1);
  finish_small_kernel<<<F, 64, 0, st>>>(N, k, nblk, pv, pi, V, sigma, rank, phase);
  size_t total = (size_t)F * N * k;
  prof_count(1);
  permute_phase_kernel<<<grid1d(total, 256), 256, 0, st>>>(F, N, k, rank, phase, U, tmpU);
  prof_count(1);
  permute_phase_kernel<<<grid1d(total, 256), 256, 0, st>>>(F, N, k, rank, phase, V, tmpV);
  RR_CUDA(cudaMemcpyAsync(U, tmpU, total * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  RR_CUDA(cudaMemcpyAsync(V, tmpV, total * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

namespace {
__global__ void axpy_kernel(size_t n, const double2* __restrict__ d, double2* __restrict__ x) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    x[e] = cadd(x[e], d[e]);
}
}  // namespace

rr_status launch_axpy(size_t n, const double2* d, double2* x, cudaStream_t st) {
  prof_count(1);
  axpy_kernel<<<grid1d(n, 256), 256, 0, st>>>(n, d, x);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}
