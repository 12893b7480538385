// Block factorisation of the block-tridiagonal s I - L, one factorisation per
// shift reused by every later solve (Sec. III.A).
//
// With the unknowns ordered by streamwise column, s I - L has diagonal blocks
// D_i, sub-diagonal blocks A_i = -L_{i,i-1} and super-diagonal blocks
// C_i = -L_{i,i+1} (b x b, A_i and C_i with at most 3q entries per row).  The
// block LU is
//     S_0 = D_0,  G_i = S_i^{-1},  X_i = G_i C_i,  S_{i+1} = D_{i+1} - A_{i+1} X_i.
// G_i is formed explicitly by blocked Gauss-Jordan elimination with partial
// pivoting (the block-sweep operator applied one panel of NB columns at a
// time), so every later solve is a dense block product instead of a pair of
// triangular solves.  Per panel K = [k0, k0+nb):
//   panel    : pivots from an LU of the tall panel M[k0:b, K]; T = M[K,K];
//              M[K,K] <- T^{-1};  M[I,K] <- -M[I,K] T^{-1}  (I = rows not in K)
//   rowblock : row swaps in the other columns; B <- M[K,R] (saved);
//              M[K,R] <- T^{-1} B
//   update   : M[I,R] <- M[I,R] + M[I,K] B    (= D - C A^{-1} B)
// After the last panel M = (P S)^{-1}; S^{-1} is M with its columns permuted.
#include <algorithm>

#include "rr_internal.cuh"

namespace {

constexpr int PANEL_THREADS = 512;

__device__ __forceinline__ int slotx(int dx, int dy) { return (dx + 1) * 3 + (dy + 1); }

// M = D_i (+ L_{i,i-1} X_{i-1} for i > 0), i.e. S_i = D_i - A_i X_{i-1}.
template <typename T>
__global__ void schur_kernel(OpView op, const double2* __restrict__ shifts, int i,
                             const C_t<T>* __restrict__ Xprev, size_t xstride,
                             C_t<T>* __restrict__ M) {
  using C = C_t<T>;
  const int b = op.b, q = op.q;
  const int r = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = blockIdx.z;
  if (c >= b) return;
  const int iy = r / q;
  const size_t nrow = (size_t)i * b + r;
  const double* cf = op.coef + nrow * op.S;
  C val = czero<C>();
  if (r == c) val = mk((T)shifts[f].x, (T)shifts[f].y);
  for (int dy = -1; dy <= 1; ++dy) {
    int jy = nbr_y(iy, dy, op.ny, op.periodic);
    if (jy < 0) continue;
    for (int cp = 0; cp < q; ++cp) {
      int m = jy * q + cp;
      if (m == c) val.x -= (T)cf[slotx(0, dy) * q + cp];
    }
  }
  if (i > 0) {
    const C* Xp = Xprev + (size_t)f * xstride;
    for (int dy = -1; dy <= 1; ++dy) {
      int jy = nbr_y(iy, dy, op.ny, op.periodic);
      if (jy < 0) continue;
      for (int cp = 0; cp < q; ++cp) {
        T a = (T)cf[slotx(-1, dy) * q + cp];
        if (a != (T)0) val = crfma(a, Xp[(size_t)(jy * q + cp) * b + c], val);
      }
    }
  }
  M[(size_t)f * b * b + (size_t)r * b + c] = val;
}

// argmax reduction helper: larger value wins, lower index on ties
template <typename T>
__device__ __forceinline__ void amax_merge(T& v, int& i, T v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

template <typename T, int NB>
__global__ void __launch_bounds__(PANEL_THREADS)
gj_panel_kernel(int b, int k0, int nbk, C_t<T>* __restrict__ Mall, int* __restrict__ ipiv_all,
                int* __restrict__ perm_all, int* __restrict__ flag) {
  using C = C_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int PS = NB + 1;  // padded row stride: column walks hit distinct banks
  C* P = reinterpret_cast<C*>(smem_raw);  // [b][PS]
  __shared__ C Ui[NB][NB + 1], Li[NB][NB + 1], Ti[NB][NB + 1];
  __shared__ T red_v[PANEL_THREADS / 32];
  __shared__ int red_i[PANEL_THREADS / 32];
  __shared__ int s_piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int f = blockIdx.x;
  C* M = Mall + (size_t)f * b * b;
  int* perm = perm_all + (size_t)f * b;
  int* ipiv = ipiv_all + f * 32;

  for (int e = tid; e < b * nbk; e += nt) {
    int r = e / nbk, c = e - r * nbk;
    P[r * PS + c] = M[(size_t)r * b + k0 + c];
  }
  __syncthreads();

  // unblocked right-looking LU with partial pivoting on rows [k0, b)
  for (int j = 0; j < nbk; ++j) {
    const int top = k0 + j;
    T bv = (T)-1;
    int bi = b;
    for (int r = top + tid; r < b; r += nt) amax_merge(bv, bi, cabs2(P[r * PS + j]), r);
    for (int o = 16; o > 0; o >>= 1) {
      T v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      amax_merge(bv, bi, v2, i2);
    }
    if ((tid & 31) == 0) { red_v[tid >> 5] = bv; red_i[tid >> 5] = bi; }
    __syncthreads();
    if (tid < 32) {
      int nw = nt >> 5;
      bv = tid < nw ? red_v[tid] : (T)-1;
      bi = tid < nw ? red_i[tid] : b;
      for (int o = 16; o > 0; o >>= 1) {
        T v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        amax_merge(bv, bi, v2, i2);
      }
      if (tid == 0) {
        if (bi >= b) bi = top;
        s_piv = bi;
        ipiv[j] = bi;
        if (!(bv > (T)0)) flag[f] = 1;
        if (bi != top) {
          int t = perm[top];
          perm[top] = perm[bi];
          perm[bi] = t;
        }
      }
    }
    __syncthreads();
    const int p = s_piv;
    if (p != top)
      for (int c = tid; c < nbk; c += nt) {
        C t = P[top * PS + c];
        P[top * PS + c] = P[p * PS + c];
        P[p * PS + c] = t;
      }
    __syncthreads();
    C piv = P[top * PS + j];
    if (cabs2(piv) == (T)0) piv = mk(sizeof(T) == 8 ? (T)1e-150 : (T)1e-18, (T)0);
    const C pinv = cinv(piv);
    for (int r = top + 1 + tid; r < b; r += nt) {
      C l = cmul(P[r * PS + j], pinv);
      P[r * PS + j] = l;
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c > j && c < nbk) P[r * PS + c] = csub(P[r * PS + c], cmul(l, P[top * PS + c]));
    }
    __syncthreads();
  }

  // inverses of U11 and of the unit lower L11, then T^{-1} = U11^{-1} L11^{-1}
  if (tid < nbk) {
    const int c = tid;
    for (int i = 0; i < NB; ++i) { Ui[i][c] = czero<C>(); Li[i][c] = czero<C>(); }
    for (int i = c; i >= 0; --i) {
      C s = (i == c) ? mk((T)1, (T)0) : czero<C>();
      for (int m = i + 1; m <= c; ++m) s = csub(s, cmul(P[(k0 + i) * PS + m], Ui[m][c]));
      Ui[i][c] = cmul(s, cinv(P[(k0 + i) * PS + i]));
    }
    Li[c][c] = mk((T)1, (T)0);
    for (int i = c + 1; i < nbk; ++i) {
      C s = czero<C>();
      for (int m = c; m < i; ++m) s = csub(s, cmul(P[(k0 + i) * PS + m], Li[m][c]));
      Li[i][c] = s;
    }
  }
  __syncthreads();
  for (int e = tid; e < nbk * nbk; e += nt) {
    int i = e / nbk, c = e - i * nbk;
    C s = czero<C>();
    for (int m = max(i, c); m < nbk; ++m) s = cfma(Ui[i][m], Li[m][c], s);
    Ti[i][c] = s;
  }
  __syncthreads();

  // rows: K -> T^{-1};  above -> -row T^{-1};  below (holding L21) -> -row L11^{-1}
  for (int r = tid; r < b; r += nt) {
    if (r >= k0 && r < k0 + nbk) {
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c < nbk) P[r * PS + c] = Ti[r - k0][c];
      continue;
    }
    C v[NB];
#pragma unroll
    for (int m = 0; m < NB; ++m) v[m] = (m < nbk) ? P[r * PS + m] : czero<C>();
    const bool above = r < k0;
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      if (c >= nbk) continue;
      C s = czero<C>();
#pragma unroll
      for (int m = 0; m < NB; ++m)
        if (m < nbk) s = cfma(v[m], above ? Ti[m][c] : Li[m][c], s);
      P[r * PS + c] = cneg(s);
    }
  }
  __syncthreads();
  for (int e = tid; e < b * nbk; e += nt) {
    int r = e / nbk, c = e - r * nbk;
    M[(size_t)r * b + k0 + c] = P[r * PS + c];
  }
}

// Row swaps + B save + M[K,R] <- T^{-1} B for the columns outside the panel.
template <typename T, int NB>
__global__ void gj_rowblock_kernel(int b, int k0, int nbk, C_t<T>* __restrict__ Mall,
                                   const int* __restrict__ ipiv_all, C_t<T>* __restrict__ Ball) {
  using C = C_t<T>;
  __shared__ C Ts[NB][NB + 1];
  __shared__ int piv[NB];
  const int f = blockIdx.y;
  C* M = Mall + (size_t)f * b * b;
  C* B = Ball + (size_t)f * NB * b;
  for (int e = threadIdx.x; e < nbk * nbk; e += blockDim.x) {
    int i = e / nbk, c = e - i * nbk;
    Ts[i][c] = M[(size_t)(k0 + i) * b + k0 + c];
  }
  if (threadIdx.x < nbk) piv[threadIdx.x] = ipiv_all[f * 32 + threadIdx.x];
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= b || (c >= k0 && c < k0 + nbk)) return;
  for (int j = 0; j < nbk; ++j) {
    int p = piv[j];
    if (p != k0 + j) {
      C t = M[(size_t)(k0 + j) * b + c];
      M[(size_t)(k0 + j) * b + c] = M[(size_t)p * b + c];
      M[(size_t)p * b + c] = t;
    }
  }
  C v[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    v[j] = (j < nbk) ? M[(size_t)(k0 + j) * b + c] : czero<C>();
    if (j < nbk) B[(size_t)j * b + c] = v[j];
  }
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    if (i >= nbk) continue;
    C s = czero<C>();
#pragma unroll
    for (int j = 0; j < NB; ++j)
      if (j < nbk) s = cfma(Ts[i][j], v[j], s);
    M[(size_t)(k0 + i) * b + c] = s;
  }
}

// Trailing update M[I,R] += M[I,K] B on 64 x 64 tiles (16 x 16 threads, 4 x 4 each).
template <typename T, int NB>
__global__ void __launch_bounds__(256)
gj_update_kernel(int b, int k0, int nbk, C_t<T>* __restrict__ Mall, const C_t<T>* __restrict__ Ball) {
  using C = C_t<T>;
  __shared__ C As[64][NB + 1];
  __shared__ C Bs[NB][64];
  const int f = blockIdx.z;
  C* M = Mall + (size_t)f * b * b;
  const C* B = Ball + (size_t)f * NB * b;
  const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < 64 * NB; e += 256) {
    int rr = e / NB, m = e - rr * NB;
    int r = r0 + rr;
    As[rr][m] = (r < b && m < nbk) ? M[(size_t)r * b + k0 + m] : czero<C>();
  }
  for (int e = tid; e < NB * 64; e += 256) {
    int m = e / 64, cc = e - m * 64;
    int c = c0 + cc;
    Bs[m][cc] = (c < b && m < nbk) ? B[(size_t)m * b + c] : czero<C>();
  }
  __syncthreads();
  C acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int d = 0; d < 4; ++d) acc[a][d] = czero<C>();
#pragma unroll 4
  for (int m = 0; m < NB; ++m) {
    C av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = As[ty + 16 * a][m];
#pragma unroll
    for (int d = 0; d < 4; ++d) bv[d] = Bs[m][tx + 16 * d];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int d = 0; d < 4; ++d) acc[a][d] = cfma(av[a], bv[d], acc[a][d]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int r = r0 + ty + 16 * a;
    if (r >= b || (r >= k0 && r < k0 + nbk)) continue;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      int c = c0 + tx + 16 * d;
      if (c >= b || (c >= k0 && c < k0 + nbk)) continue;
      size_t o = (size_t)r * b + c;
      M[o] = cadd(M[o], acc[a][d]);
    }
  }
}

// G_i[:, perm[c]] = M[:, c];  X_i = G_i C_i with C_i = -L_{i,i+1}.
template <typename T>
__global__ void gj_finalize_kernel(OpView op, int i, int RB, const C_t<T>* __restrict__ Mall,
                                   const int* __restrict__ perm_all, C_t<T>* __restrict__ Gi,
                                   size_t gstride, C_t<T>* __restrict__ Xi, size_t xstride) {
  using C = C_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = op.b, q = op.q;
  C* Gs = reinterpret_cast<C*>(smem_raw);          // [RB][b]
  int* ps = reinterpret_cast<int*>(Gs + (size_t)RB * b);  // [b]
  const int f = blockIdx.y;
  const int r0 = blockIdx.x * RB;
  const C* M = Mall + (size_t)f * b * b;
  for (int c = threadIdx.x; c < b; c += blockDim.x) ps[c] = perm_all[(size_t)f * b + c];
  __syncthreads();
  for (int e = threadIdx.x; e < RB * b; e += blockDim.x) {
    int rr = e / b, c = e - rr * b;
    int r = r0 + rr;
    if (r < b) Gs[rr * b + ps[c]] = M[(size_t)r * b + c];
  }
  __syncthreads();
  C* G = Gi + (size_t)f * gstride;
  for (int e = threadIdx.x; e < RB * b; e += blockDim.x) {
    int rr = e / b, c = e - rr * b;
    int r = r0 + rr;
    if (r < b) G[(size_t)r * b + c] = Gs[rr * b + c];
  }
  if (Xi == nullptr) return;
  C* X = Xi + (size_t)f * xstride;
  for (int e = threadIdx.x; e < RB * b; e += blockDim.x) {
    int rr = e / b, c = e - rr * b;
    int r = r0 + rr;
    if (r >= b) continue;
    const int iyc = c / q, cc = c - iyc * q;
    C s = czero<C>();
    for (int dy = -1; dy <= 1; ++dy) {
      int iym = nbr_y(iyc, -dy, op.ny, op.periodic);
      if (iym < 0) continue;
      for (int cm = 0; cm < q; ++cm) {
        int m = iym * q + cm;
        T a = (T)op.coef[((size_t)i * b + m) * op.S + slotx(1, dy) * q + cc];
        if (a != (T)0) s = crfma(a, Gs[rr * b + m], s);
      }
    }
    X[(size_t)r * b + c] = cneg(s);
  }
}

__global__ void iota_kernel(int* perm, int b, int F) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < b * F) perm[e] = e % b;
}

// Widest panel whose tall slab (b x NB) plus the static NB x NB scratch fits
// the 227 KB of shared memory a CTA may use.
template <typename T>
int panel_nb(int b) {
  const size_t csz = sizeof(C_t<T>);
  const size_t cap = 227 * 1024 - 2048;
  for (int nb = 32; nb >= 8; nb >>= 1)
    if ((size_t)b * (nb + 1) * csz + 3 * (size_t)nb * (nb + 1) * csz <= cap) return nb;
  return 8;
}

template <typename T, int NB>
rr_status factor_impl(rr_factors* fa) {
  using C = C_t<T>;
  const OpDev& d = fa->op->d;
  const OpView ov = view(d);
  const int b = d.b, nx = d.nx, F = fa->F;
  cudaStream_t st = fa->stream;
  C* M = reinterpret_cast<C*>(fa->M);
  C* G = reinterpret_cast<C*>(fa->G);
  C* X = reinterpret_cast<C*>(fa->X);
  C* Bbuf = reinterpret_cast<C*>(fa->Bbuf);
  const size_t bb = (size_t)b * b;
  const size_t gstride = (size_t)nx * bb;          // per problem
  const size_t xstride = (size_t)(nx > 1 ? nx - 1 : 1) * bb;

  const size_t psmem = (size_t)b * (NB + 1) * sizeof(C);
  RR_CUDA(cudaFuncSetAttribute(gj_panel_kernel<T, NB>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
  int RB = 4;
  while (RB > 1 && (size_t)RB * b * sizeof(C) + b * sizeof(int) > 160 * 1024) RB >>= 1;
  const size_t fsmem = (size_t)RB * b * sizeof(C) + b * sizeof(int);
  RR_CUDA(cudaFuncSetAttribute(gj_finalize_kernel<T>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));

  for (int i = 0; i < nx; ++i) {
    iota_kernel<<<(b * F + 255) / 256, 256, 0, st>>>(fa->perm, b, F);
    prof_count(1);
    dim3 gs((b + 127) / 128, b, F);
    const C* Xprev = (i > 0) ? X + (size_t)(i - 1) * bb : nullptr;
    prof_begin(PROF_SCHUR, st);
    schur_kernel<T><<<gs, 128, 0, st>>>(ov, fa->shifts, i, Xprev, xstride, M);
    prof_end(PROF_SCHUR, st);
    for (int k0 = 0; k0 < b; k0 += NB) {
      const int nbk = std::min(NB, b - k0);
      prof_begin(PROF_PANEL, st);
      gj_panel_kernel<T, NB><<<F, PANEL_THREADS, psmem, st>>>(b, k0, nbk, M, fa->ipiv,
                                                             fa->perm, fa->flag);
      prof_end(PROF_PANEL, st);
      prof_begin(PROF_ROWBLOCK, st);
      gj_rowblock_kernel<T, NB><<<dim3((b + 127) / 128, F), 128, 0, st>>>(b, k0, nbk, M,
                                                                          fa->ipiv, Bbuf);
      prof_end(PROF_ROWBLOCK, st);
      prof_begin(PROF_UPDATE, st);
      gj_update_kernel<T, NB><<<dim3((b + 63) / 64, (b + 63) / 64, F), 256, 0, st>>>(
          b, k0, nbk, M, Bbuf);
      prof_end(PROF_UPDATE, st);
    }
    C* Xi = (i + 1 < nx) ? X + (size_t)i * bb : nullptr;
    prof_begin(PROF_FINALIZE, st);
    gj_finalize_kernel<T><<<dim3((b + RB - 1) / RB, F), 256, fsmem, st>>>(
        ov, i, RB, M, fa->perm, G + (size_t)i * bb, gstride, Xi, xstride);
    prof_end(PROF_FINALIZE, st);
    RR_CUDA(cudaGetLastError());
  }
  return RR_OK;
}

template <typename T>
rr_status factor_dispatch(rr_factors* fa) {
  switch (panel_nb<T>(fa->op->d.b)) {
    case 32: return factor_impl<T, 32>(fa);
    case 16: return factor_impl<T, 16>(fa);
    default: return factor_impl<T, 8>(fa);
  }
}

}  // namespace

int factor_panel_width(int prec, int b) {
  return prec == RR_FP64 ? panel_nb<double>(b) : panel_nb<float>(b);
}

rr_status launch_factor(rr_factors* fa) {
  if (fa->prec == RR_FP64) return factor_dispatch<double>(fa);
  return factor_dispatch<float>(fa);
}
