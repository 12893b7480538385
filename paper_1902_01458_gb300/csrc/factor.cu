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
#include <cuda.h>

#include <algorithm>
#include <type_traits>

#include "rr_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int PANEL_THREADS = 512;

__device__ __forceinline__ int slotx(int dx, int dy) { return (dx + 1) * 3 + (dy + 1); }

// M = D_i (+ L_{i,i-1} X_{i-1} for i > 0), i.e. S_i = D_i - A_i X_{i-1}.  One
// CTA per (SCHUR_Y grid points in y = SCHUR_Y * q rows, column tile, problem):
// the rows of X_{i-1} its rows couple to (the y neighbours, SCHUR_Y + 2
// points) are staged once in shared memory, so every X row is read from
// memory about once instead of once per coupled row; a row's stencil
// coefficients are uniform across the CTA (broadcast loads).
// one thread per column of the tile: the block has CB threads
constexpr int SCHUR_Y = 8;
template <typename T> struct SchurCfg { static constexpr int CB = sizeof(T) == 4 ? 256 : 128; };
template <typename T>
__host__ __device__ constexpr size_t schur_smem(int q) {
  return (size_t)(SCHUR_Y + 2) * q * SchurCfg<T>::CB * sizeof(C_t<T>);
}

template <typename T>
__global__ void __launch_bounds__(SchurCfg<T>::CB)
schur_kernel(OpView op, const double2* __restrict__ shifts, int i,
             const C_t<T>* __restrict__ Xprev, size_t xstride, C_t<T>* __restrict__ M) {
  using C = C_t<T>;
  constexpr int CB = SchurCfg<T>::CB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Xs = reinterpret_cast<C*>(smem_raw);  // [(SCHUR_Y + 2) * q][CB]
  const int b = op.b, q = op.q, ny = op.ny;
  const int f = blockIdx.z;
  const int y0 = blockIdx.x * SCHUR_Y;
  const int c0 = blockIdx.y * CB;
  const C sh = mk((T)shifts[f].x, (T)shifts[f].y);
  const C* Xp = Xprev ? Xprev + (size_t)f * xstride : nullptr;
  C* Mf = M + (size_t)f * b * b;
  const int ny_blk = min(SCHUR_Y, ny - y0);
  // stage X rows of y points y0 - 1 .. y0 + ny_blk (slot k <-> point y0 - 1 + k)
  if (Xp) {
    const int nslots = (ny_blk + 2) * q;
    for (int e = threadIdx.x; e < nslots * CB; e += CB) {
      const int sl = e / CB, cc = e - sl * CB;
      const int pt = sl / q, comp = sl - pt * q;
      // point y0 - 1 + pt, wrapped when y is periodic (outside the grid
      // otherwise: never read, its coupling coefficient is absent)
      const int yy = op.periodic ? (y0 - 1 + pt + ny) % ny : y0 - 1 + pt;
      const int c = c0 + cc;
      C v = czero<C>();
      if (c < b && yy >= 0 && yy < ny) v = Xp[(size_t)(yy * q + comp) * b + c];
      Xs[sl * CB + cc] = v;
    }
    __syncthreads();
  }
  // The CTA's rows (ny_blk points x q variables) share their stencil
  // coefficients: stage them once, with the neighbour point of every y
  // offset (-1: a Dirichlet ghost), so the per-entry loop reads shared
  // memory only.
  __shared__ T cA[SCHUR_Y * 4][12];  // coupling to column i-1 (slot dx = -1), term (dy, cp)
  __shared__ T cD[SCHUR_Y * 4][12];  // diagonal block D_i (slot dx = 0)
  __shared__ int jyt[SCHUR_Y][3];    // neighbour y of point y0 + ly at dy = -1, 0, 1
  const int nt3 = 3 * q;
  for (int e = threadIdx.x; e < ny_blk * q * nt3; e += blockDim.x) {
    const int lr = e / nt3, t = e - lr * nt3;
    const int ly = lr / q, comp = lr - ly * q;
    const int iy = y0 + ly, dy = t / q - 1, cp = t - (t / q) * q;
    const int jy = nbr_y(iy, dy, ny, op.periodic);
    const size_t cf = ((size_t)i * b + iy * q + comp) * op.S;
    cA[lr][t] = (jy >= 0 && Xp) ? coefv<T>(op, cf + slotx(-1, dy) * q + cp) : (T)0;
    cD[lr][t] = jy >= 0 ? coefv<T>(op, cf + slotx(0, dy) * q + cp) : (T)0;
  }
  for (int e = threadIdx.x; e < ny_blk * 3; e += blockDim.x)
    jyt[e / 3][e % 3] = nbr_y(y0 + e / 3, e % 3 - 1, ny, op.periodic);
  __syncthreads();
  const int c = c0 + threadIdx.x;
  if (c >= b) return;
  const int jc = c / q, cc = c - jc * q;  // column c = variable cc of point jc
  for (int ly = 0; ly < ny_blk; ++ly) {
    const int iy = y0 + ly;
    for (int comp = 0; comp < q; ++comp) {
      const int r = iy * q + comp, lr = ly * q + comp;
      C val = (r == c) ? sh : czero<C>();
      // D_i: the row's entries at column c (one per y offset landing on jc)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
        if (jyt[ly][dy] == jc) val.x -= cD[lr][dy * q + cc];
      if (Xp) {
#pragma unroll
        for (int t = 0; t < 12; ++t) {  // 3 y neighbours x q <= 4 variables
          if (t >= nt3) break;
          const T av = cA[lr][t];
          // slot of point iy + dy: ly + 1 + dy (periodic wrap stays in the
          // staged range because the staged points are y0 - 1 .. y0 + ny_blk)
          const int dy = t / q - 1, cp = t - (t / q) * q;
          if (av != (T)0) val = crfma(av, Xs[((ly + 1 + dy) * q + cp) * CB + threadIdx.x], val);
        }
      }
      Mf[(size_t)r * b + c] = val;
    }
  }
}

// argmax reduction helper: larger value wins, lower index on ties
template <typename T>
__device__ __forceinline__ void amax_merge(T& v, int& i, T v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

// Pivoted panel step.  The tall panel M[:, K] sits in shared memory by
// original row ("slot"); the LU with partial pivoting over slots >= k0 never
// moves data: each step picks the largest remaining |.|^2 of column j (lowest
// slot on ties), marks that slot as the j-th pivot and eliminates column j
// from the other remaining slots, with one block barrier per step (every
// warp reduces the per-warp candidates itself).  Warp 0 then replays the
// choices as the equivalent sequence of row interchanges (ipiv, as the row
// block kernel applies them to the other columns) and the final position of
// every slot, and the transformed panel is written back in that order:
//   pivot rows  -> T^{-1} = U11^{-1} L11^{-1}
//   rows above  -> -row T^{-1}
//   other rows  -> -(their multipliers) L11^{-1}   (= -M[I,K] T^{-1})
template <typename T, int NB>
__global__ void __launch_bounds__(PANEL_THREADS)
gj_panel_kernel(int b, int k0, int nbk, C_t<T>* __restrict__ Mall, int* __restrict__ ipiv_all,
                int* __restrict__ perm_all, int* __restrict__ flag) {
  using C = C_t<T>;
  constexpr int PS = NB + 1;  // padded row stride: column walks hit distinct banks
  constexpr int NW = PANEL_THREADS / 32;
  constexpr int MAXOWN = (1024 + PANEL_THREADS - 1) / PANEL_THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);  // [b][PS] by slot
  __shared__ C Ui[NB][NB + 1], Li[NB][NB + 1], Ti[NB][NB + 1];
  __shared__ T red_v[2][NW];  // per-step candidates, double buffered by step parity
  __shared__ int red_i[2][NW];
  __shared__ int chosen[NB];
  __shared__ int sigK[NB];            // slot that ends at position k0 + j
  __shared__ int nkPos[32], nkSlot[32];
  __shared__ int s_nk;
  __shared__ unsigned touched[32];    // positions outside K that receive another slot
  const int tid = threadIdx.x, nt = PANEL_THREADS;
  const int lane = tid & 31, warp = tid >> 5;
  const int f = blockIdx.x;
  C* M = Mall + (size_t)f * b * b;
  int* perm = perm_all + (size_t)f * b;
  int* ipiv = ipiv_all + f * 32;

  for (int e = tid; e < b * nbk; e += nt) {
    int r = e / nbk, c = e - r * nbk;
    P[r * PS + c] = M[(size_t)r * b + k0 + c];
  }
  if (tid < 32) touched[tid] = 0u;
  unsigned done = 0u;  // bit t: slot k0 + tid + t*nt already pivoted
  __syncthreads();

  for (int j = 0; j < nbk; ++j) {
    T bv = (T)-1;
    int bi = b;
#pragma unroll
    for (int t = 0; t < MAXOWN; ++t) {
      int r = k0 + tid + t * nt;
      if (r < b && !(done & (1u << t))) amax_merge(bv, bi, cabs2(P[r * PS + j]), r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      amax_merge(bv, bi, v2, i2);
    }
    // one barrier per step: it publishes the candidates and orders the
    // owner's elimination of step j-1 on the pivot row before its reads
    // below; the other rows are only ever touched by their owner thread
    if (lane == 0) { red_v[j & 1][warp] = bv; red_i[j & 1][warp] = bi; }
    __syncthreads();
    bv = lane < NW ? red_v[j & 1][lane] : (T)-1;
    bi = lane < NW ? red_i[j & 1][lane] : b;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T v2 = __shfl_xor_sync(0xffffffffu, bv, o);
      int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      amax_merge(bv, bi, v2, i2);
    }
    const int p = bi < b ? bi : k0 + j;  // (bi >= b cannot happen while slots remain)
    if (tid == 0) {
      chosen[j] = p;
      if (!(bv > (T)0)) flag[f] = 1;
    }
    C piv = P[p * PS + j];
    if (cabs2(piv) == (T)0) piv = mk(sizeof(T) == 8 ? (T)1e-150 : (T)1e-18, (T)0);
    const C pinv = cinv(piv);
#pragma unroll
    for (int t = 0; t < MAXOWN; ++t) {
      int r = k0 + tid + t * nt;
      if (r >= b || (done & (1u << t))) continue;
      if (r == p) { done |= 1u << t; continue; }
      C l = cmul(P[r * PS + j], pinv);
      P[r * PS + j] = l;
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c > j && c < nbk) P[r * PS + c] = csub(P[r * PS + c], cmul(l, P[p * PS + c]));
    }
  }
  __syncthreads();

  // warp 0: replay the choices as row interchanges (position a = k0 + j with
  // the current position q of the chosen slot), tracking where slots end
  if (warp == 0) {
    int kc = (lane < nbk) ? k0 + lane : -1;  // slot now at position k0 + lane
    int np = -1, nc = -1, cnt = 0;           // touched position outside K and its slot
    for (int j = 0; j < nbk; ++j) {
      const int sj = chosen[j];
      unsigned bK = __ballot_sync(0xffffffffu, lane < nbk && kc == sj);
      unsigned bN = __ballot_sync(0xffffffffu, np >= 0 && nc == sj);
      int q, ql;
      bool inK;
      if (bK) {
        ql = __ffs(bK) - 1;
        q = k0 + ql;
        inK = true;
      } else if (bN) {
        ql = __ffs(bN) - 1;
        q = __shfl_sync(0xffffffffu, np, ql);
        inK = false;
      } else {
        ql = cnt++;
        q = sj;
        inK = false;
        if (lane == ql) { np = sj; nc = sj; }
      }
      const int ca = __shfl_sync(0xffffffffu, kc, j);
      const int cq = inK ? __shfl_sync(0xffffffffu, kc, ql) : __shfl_sync(0xffffffffu, nc, ql);
      if (lane == j) kc = cq;
      if (inK && lane == ql) kc = ca;
      if (!inK && lane == ql) nc = ca;
      if (lane == 0) ipiv[j] = q;
      __syncwarp();
    }
    // perm undergoes the same interchanges: every position that received
    // another slot takes that slot's old entry (all reads before any write,
    // instead of a chain of dependent global swaps)
    const bool movedK = lane < nbk && kc != k0 + lane;
    const int pk = movedK ? perm[kc] : 0;
    const int pn = lane < cnt ? perm[nc] : 0;
    __syncwarp();
    if (movedK) perm[k0 + lane] = pk;
    if (lane < cnt) perm[np] = pn;
    if (lane < nbk) sigK[lane] = kc;
    if (lane < cnt) {
      nkPos[lane] = np;
      nkSlot[lane] = nc;
      atomicOr(&touched[np >> 5], 1u << (np & 31));
    }
    if (lane == 0) s_nk = cnt;
  }

  // inverses of U11 (warp 0) and of the unit lower L11 (warp 1) in parallel,
  // rows = chosen slots in order, one column per lane; then
  // T^{-1} = U11^{-1} L11^{-1}
  if (warp == 0 && lane < nbk) {
    const int c = lane;
    for (int i = 0; i < NB; ++i) Ui[i][c] = czero<C>();
    for (int i = c; i >= 0; --i) {
      const C* row = P + chosen[i] * PS;
      C sacc = (i == c) ? mk((T)1, (T)0) : czero<C>();
      for (int m = i + 1; m <= c; ++m) sacc = csub(sacc, cmul(row[m], Ui[m][c]));
      Ui[i][c] = cmul(sacc, cinv(row[i]));
    }
  } else if (warp == 1 && lane < nbk) {
    const int c = lane;
    for (int i = 0; i < NB; ++i) Li[i][c] = czero<C>();
    Li[c][c] = mk((T)1, (T)0);
    for (int i = c + 1; i < nbk; ++i) {
      const C* row = P + chosen[i] * PS;
      C sacc = czero<C>();
      for (int m = c; m < i; ++m) sacc = csub(sacc, cmul(row[m], Li[m][c]));
      Li[i][c] = sacc;
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

  // transform every slot in place
  for (int r = tid; r < b; r += nt) {
    int jpiv = -1;
    if (r >= k0)
      for (int j = 0; j < nbk; ++j)
        if (chosen[j] == r) jpiv = j;
    if (jpiv >= 0) {
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c < nbk) P[r * PS + c] = Ti[jpiv][c];
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
  // write back by position: K positions take their pivot slot, touched
  // positions outside K take the displaced slot, the rest keep their own
  const int nk = s_nk;
  for (int e = tid; e < b * nbk; e += nt) {
    int a = e / nbk, c = e - a * nbk;
    int slot = a;
    if (a >= k0 && a < k0 + nbk) {
      slot = sigK[a - k0];
    } else if (touched[a >> 5] & (1u << (a & 31))) {
      for (int t = 0; t < nk; ++t)
        if (nkPos[t] == a) slot = nkSlot[t];
    }
    M[(size_t)a * b + k0 + c] = P[slot * PS + c];
  }
}

// Row swaps + B save + M[K,R] <- T^{-1} B for the columns outside the panel.
// Warp 0 first turns the panel's sequence of swaps into the net movement of
// at most 2*NB rows; every thread then moves its column with independent
// loads (all issued before any store) instead of a chain of dependent swaps.
template <typename T, int NB>
__host__ __device__ constexpr int rb_threads() {
  return (NB * 128 * (int)sizeof(C_t<T>) > 32768) ? 32768 / (NB * (int)sizeof(C_t<T>)) : 128;
}
template <typename T, int NB>
__global__ void __launch_bounds__(128)
gj_rowblock_kernel(int b, int k0, int nbk, C_t<T>* __restrict__ Mall,
                   const int* __restrict__ ipiv_all, C_t<T>* __restrict__ Ball) {
  using C = C_t<T>;
  __shared__ C Ts[NB][NB + 1];
  __shared__ int srcK[NB];       // original row now at position k0 + j
  __shared__ int nkPos[32], nkSrc[32];
  __shared__ int s_nk;
  constexpr int RBT = rb_threads<T, NB>();
  __shared__ C W[NB][RBT];        // values moving to positions outside K
  const int f = blockIdx.y;
  C* M = Mall + (size_t)f * b * b;
  C* B = Ball + (size_t)f * NB * b;
  for (int e = threadIdx.x; e < nbk * nbk; e += blockDim.x) {
    int i = e / nbk, c = e - i * nbk;
    Ts[i][c] = M[(size_t)(k0 + i) * b + k0 + c];
  }
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int j = lane; j < NB; j += 32) srcK[j] = k0 + j;
    // the panel's interchanges, one per lane, read once (not one dependent
    // global load per step of the serial loop below)
    const int piv_l = lane < nbk ? ipiv_all[f * 32 + lane] : 0;
    int myPos = -1, myCont = -1, nk = 0;
    __syncwarp();
    for (int j = 0; j < nbk; ++j) {
      const int a = k0 + j;
      const int p = __shfl_sync(0xffffffffu, piv_l, j);
      if (p == a) continue;
      if (p < k0 + nbk) {
        if (lane == 0) {
          int t = srcK[j];
          srcK[j] = srcK[p - k0];
          srcK[p - k0] = t;
        }
        __syncwarp();
        continue;
      }
      unsigned hit = __ballot_sync(0xffffffffu, myPos == p);
      int owner;
      if (hit) {
        owner = __ffs(hit) - 1;
      } else {
        owner = nk;
        if (lane == owner) { myPos = p; myCont = p; }
        ++nk;
      }
      int kc = srcK[j];
      int oc = __shfl_sync(0xffffffffu, myCont, owner);
      if (lane == owner) myCont = kc;
      __syncwarp();
      if (lane == 0) srcK[j] = oc;
      __syncwarp();
    }
    if (lane < nk) { nkPos[lane] = myPos; nkSrc[lane] = myCont; }
    if (lane == 0) s_nk = nk;
  }
  __syncthreads();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= b || (c >= k0 && c < k0 + nbk)) return;
  const int nk = s_nk;
  C v[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) v[j] = (j < nbk) ? M[(size_t)srcK[j] * b + c] : czero<C>();
  for (int t = 0; t < nk; ++t) W[t][threadIdx.x] = M[(size_t)nkSrc[t] * b + c];
  for (int t = 0; t < nk; ++t) M[(size_t)nkPos[t] * b + c] = W[t][threadIdx.x];
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < nbk) B[(size_t)j * b + c] = v[j];
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

// Trailing update M[I,R] += M[I,K] B on 64 x 64 tiles (16 x 16 threads, 4 x 4
// each) for the columns [c_begin, c_end) outside K and outside [ex_lo, ex_hi).
template <typename T, int NB>
__global__ void __launch_bounds__(256)
gj_update_kernel(int b, int k0, int nbk, int c_begin, int c_end, int ex_lo, int ex_hi,
                 C_t<T>* __restrict__ Mall, const C_t<T>* __restrict__ Ball) {
  using C = C_t<T>;
  __shared__ C As[64][NB + 1];
  __shared__ C Bs[NB][64];
  const int f = blockIdx.z;
  C* M = Mall + (size_t)f * b * b;
  const C* B = Ball + (size_t)f * NB * b;
  const int r0 = blockIdx.y * 64, c0 = c_begin + blockIdx.x * 64;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < 64 * NB; e += 256) {
    int rr = e / NB, m = e - rr * NB;
    int r = r0 + rr;
    As[rr][m] = (r < b && m < nbk) ? M[(size_t)r * b + k0 + m] : czero<C>();
  }
  for (int e = tid; e < NB * 64; e += 256) {
    int m = e / 64, cc = e - m * 64;
    int c = c0 + cc;
    Bs[m][cc] = (c < c_end && m < nbk) ? B[(size_t)m * b + c] : czero<C>();
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
      if (c >= c_end || (c >= k0 && c < k0 + nbk) || (c >= ex_lo && c < ex_hi)) continue;
      size_t o = (size_t)r * b + c;
      M[o] = cadd(M[o], acc[a][d]);
    }
  }
}

// ---------------------------------------------------------------------------
// Trailing update on the tensor cores (FP32 factors, 32-column panels):
// M[I,R] += M[I,K] B as a real GEMM on tcgen05.mma kind::tf32.
//
// A tile is 128 rows of M[., K] read interleaved (re, im) as 64 K-major reals;
// the right operand is B expanded to B~ with rows (Re, -Im), (Im, Re) per
// complex column, so one real product gives the complex one.  FP32 accuracy
// comes from the 3xTF32 split (hi.hi + hi.lo + lo.hi into one FP32 TMEM
// accumulator).  One CTA per item (problem, tile of 64 complex columns,
// group of row tiles): it expands B~ once and streams the item's row tiles
// of M through a warp-specialised pipeline:
//   warp 10     loads the raw A tile of row tile t+1 by TMA (3-D map over M)
//               and issues the 24 MMAs of tile t into accumulator t & 1,
//   warps 8-9   split the raw A tile into the hi / lo operand tiles,
//   warps 0-7   prefetch the M rows of tile t (coalesced, whole 512-byte tile
//               rows per warp instruction), move accumulator t & 1 through a
//               shared staging tile and add it to M in place (rows in K,
//               columns in K and in [ex_lo, ex_hi) untouched),
// so the HBM traffic of tile t overlaps the split and MMAs of tile t+1.
// Every mbarrier wait is bounded; a timeout sets *err and the CTA winds down
// (in-flight MMAs drain, TMEM is freed).
constexpr int UTC_RT = 128;                                   // rows per tile
constexpr int UTC_CT = 64;                                    // complex columns per tile
constexpr uint32_t UTC_LBO = 128, UTC_SBO = 2048;             // 64 reals of K
constexpr uint32_t UTC_OP_BYTES = UTC_RT * 64 * 4;            // 32 KB operand tile
constexpr int UTC_STAGE_LD = 2 * UTC_CT + 4;                  // staging row pitch (floats)
constexpr uint32_t UTC_STAGE_BYTES = UTC_RT * UTC_STAGE_LD * 4;
constexpr int UTC_EPI = 256, UTC_CONV = 64;                   // epilogue / split threads
constexpr int UTC_THREADS = UTC_EPI + UTC_CONV + 32;          // + MMA warp
// B~ hi/lo, A hi/lo, the raw A tile (TMA destination) and the staging tile
constexpr size_t UTC_SMEM = 5 * (size_t)UTC_OP_BYTES + UTC_STAGE_BYTES + 128;
constexpr uint32_t UTC_WAIT_TRIES = 1u << 22;

// bounded wait; gives up at once when another thread has aborted
__device__ __forceinline__ bool utc_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t t = 0; t < UTC_WAIT_TRIES; ++t) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void utc_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tc::smem_u32(bar)) : "memory");
}

// barrier among the 256 epilogue threads only
__device__ __forceinline__ void utc_epi_sync() {
  asm volatile("bar.sync 1, %0;\n" ::"n"(UTC_EPI) : "memory");
}

__global__ void __launch_bounds__(UTC_THREADS, 1)
gj_update_tc_kernel(const __grid_constant__ CUtensorMap tmapM, int b, int k0, int nbk, int c_begin,
                    int c_end, int ex_lo, int ex_hi, float2* __restrict__ Mall,
                    const float2* __restrict__ Ball, int F, int nct, int nrg, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t raw_full, a_full, mma_done[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_sh;
  volatile int* abort_flag = &abort_sh;
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  unsigned char* Bhi = base;
  unsigned char* Blo = base + UTC_OP_BYTES;
  unsigned char* Ahi = base + 2 * UTC_OP_BYTES;
  unsigned char* Alo = base + 3 * UTC_OP_BYTES;
  const float* Araw = reinterpret_cast<const float*>(base + 4 * UTC_OP_BYTES);  // [128][64]
  float* stage = reinterpret_cast<float*>(base + 5 * UTC_OP_BYTES);  // [128][UTC_STAGE_LD]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool is_epi = tid < UTC_EPI;
  const bool is_conv = tid >= UTC_EPI && tid < UTC_EPI + UTC_CONV;
  const bool is_mma = tid == UTC_EPI + UTC_CONV;
  const int nrt = (b + UTC_RT - 1) / UTC_RT;
  const int rpg = (nrt + nrg - 1) / nrg;  // row tiles per row group
  const int nitems = nct * F * nrg;

  if (warp == 0) tc::tmem_alloc(&tmem_base, 256);
  if (tid == 0) {
    tc::mbar_init(&raw_full, 1);
    tc::mbar_init(&a_full, UTC_CONV);
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&mma_done[q], 1);
      tc::mbar_init(&acc_empty[q], UTC_EPI);
    }
    abort_sh = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tc::idesc_tf32(UTC_RT, 2 * UTC_CT);
  uint64_t dBhi = 0, dBlo = 0, dAhi = 0, dAlo = 0;
  if (is_mma) {
    dBhi = tc::smem_desc(tc::smem_u32(Bhi), UTC_LBO, UTC_SBO);
    dBlo = tc::smem_desc(tc::smem_u32(Blo), UTC_LBO, UTC_SBO);
    dAhi = tc::smem_desc(tc::smem_u32(Ahi), UTC_LBO, UTC_SBO);
    dAlo = tc::smem_desc(tc::smem_u32(Alo), UTC_LBO, UTC_SBO);
  }
  int g = 0;           // row tiles of this CTA so far (all items)
  int issued = 0;      // tiles whose MMAs were issued (MMA thread)
  int tma_issued = 0;  // raw A tiles requested (MMA thread)
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int rg = it % nrg, fc = it / nrg;
    const int f = fc / nct, ct = fc - f * nct;
    const int rt0 = rg * rpg, rt1 = min(nrt, rt0 + rpg);
    const int c0 = c_begin + ct * UTC_CT;
    float2* M = Mall + (size_t)f * b * b;
    // every earlier tile's MMAs are complete here (their epilogues waited
    // for them before this barrier), so B~ may be overwritten
    __syncthreads();
    if ((is_epi || is_conv) && !*abort_flag) {
      const float2* B = Ball + (size_t)f * 32 * b;
      for (int e = tid; e < UTC_CT * 16; e += UTC_EPI + UTC_CONV) {
        const int j = e & (UTC_CT - 1), p = e / UTC_CT;
        const int c = c0 + j, m0 = 2 * p, m1 = m0 + 1;
        const bool cv = c < c_end;
        const float2 t0 = (cv && m0 < nbk) ? B[(size_t)m0 * b + c] : make_float2(0.f, 0.f);
        const float2 t1 = (cv && m1 < nbk) ? B[(size_t)m1 * b + c] : make_float2(0.f, 0.f);
        float4 h0, l0;
        tc::split_tf32(t0.x, h0.x, l0.x);
        tc::split_tf32(-t0.y, h0.y, l0.y);
        tc::split_tf32(t1.x, h0.z, l0.z);
        tc::split_tf32(-t1.y, h0.w, l0.w);
        const float4 h1 = make_float4(-h0.y, h0.x, -h0.w, h0.z);
        const float4 l1 = make_float4(-l0.y, l0.x, -l0.w, l0.z);
        const int n0 = 2 * j, n1 = n0 + 1;
        const uint32_t o0 = (uint32_t)(n0 >> 3) * UTC_SBO + (uint32_t)p * UTC_LBO + (uint32_t)(n0 & 7) * 16;
        const uint32_t o1 = (uint32_t)(n1 >> 3) * UTC_SBO + (uint32_t)p * UTC_LBO + (uint32_t)(n1 & 7) * 16;
        *reinterpret_cast<float4*>(Bhi + o0) = h0;
        *reinterpret_cast<float4*>(Blo + o0) = l0;
        *reinterpret_cast<float4*>(Bhi + o1) = h1;
        *reinterpret_cast<float4*>(Blo + o1) = l1;
      }
      tc::fence_async_smem();
    }
    __syncthreads();
    if (is_mma && !*abort_flag && rt0 < rt1) {  // raw A tile of the item's first row tile
      tc::mbar_expect_tx(&raw_full, UTC_OP_BYTES);
      tc::tma_load_3d(base + 4 * UTC_OP_BYTES, &tmapM, 2 * k0, rt0 * UTC_RT, f, &raw_full);
      ++tma_issued;
    }
    for (int rt = rt0; rt < rt1; ++rt, ++g) {
      const int q = g & 1;
      const uint32_t ph = (uint32_t)(g >> 1) & 1u;  // phase of tile g on the barriers q
      if (is_conv) {
        // raw A tile (row-major 128 x 64 floats: rows rt*128.., the 32 panel
        // columns; zero beyond b) -> TF32 hi / lo tiles in the K-major
        // core-matrix layout.  Each 8-lane phase takes a diagonal: rows
        // 8G + a and K groups ((a + D) & 7) + 8H for a = 0..7, so both the
        // raw reads (slot p mod 8) and the core-matrix writes (slot i mod 8)
        // hit 8 distinct 16-byte bank slots.
        const int ci = tid - UTC_EPI;
        bool ok = !*abort_flag;
        if (ok) ok = utc_wait(&raw_full, (uint32_t)g & 1u, abort_flag);
        // the A operand tiles are free once tile g-1's MMAs are complete
        if (ok && g >= 1) ok = utc_wait(&mma_done[(g - 1) & 1], (uint32_t)((g - 1) >> 1) & 1u, abort_flag);
        if (ok) {
#pragma unroll 8
          for (int s = 0; s < 32; ++s) {
            const int a = lane & 7;
            const int combo = ((ci >> 5) * 32 + s) * 4 + (lane >> 3);  // 0 .. 255
            const int i = 8 * (combo & 15) + a;                         // row
            const int p = ((a + (combo >> 5)) & 7) + 8 * ((combo >> 4) & 1);  // K group
            const float4 v = *reinterpret_cast<const float4*>(Araw + i * 64 + 4 * p);
            float4 h, l;
            tc::split_tf32(v.x, h.x, l.x);
            tc::split_tf32(v.y, h.y, l.y);
            tc::split_tf32(v.z, h.z, l.z);
            tc::split_tf32(v.w, h.w, l.w);
            const uint32_t off = (uint32_t)(i >> 3) * UTC_SBO + (uint32_t)p * UTC_LBO + (uint32_t)(i & 7) * 16;
            *reinterpret_cast<float4*>(Ahi + off) = h;
            *reinterpret_cast<float4*>(Alo + off) = l;
          }
          tc::fence_async_smem();
        }
        utc_arrive(&a_full);
      } else if (is_mma) {
        bool ok = !*abort_flag;
        if (ok) ok = utc_wait(&a_full, (uint32_t)g & 1u, abort_flag);
        if (ok && rt + 1 < rt1) {  // the raw tile has been split: fetch the next one
          tc::mbar_expect_tx(&raw_full, UTC_OP_BYTES);
          tc::tma_load_3d(base + 4 * UTC_OP_BYTES, &tmapM, 2 * k0, (rt + 1) * UTC_RT, f, &raw_full);
          ++tma_issued;
        }
        if (ok && g >= 2) ok = utc_wait(&acc_empty[q], (uint32_t)((g - 2) >> 1) & 1u, abort_flag);
        if (ok) {
          tc::fence_after_sync();
          const uint32_t acc = tmem + (uint32_t)q * (2 * UTC_CT);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const uint64_t koff = (uint64_t)((kk * 2 * UTC_LBO) >> 4);
            tc::mma_tf32(acc, dAhi + koff, dBhi + koff, idesc, kk > 0 ? 1u : 0u);
            tc::mma_tf32(acc, dAhi + koff, dBlo + koff, idesc, 1u);
            tc::mma_tf32(acc, dAlo + koff, dBhi + koff, idesc, 1u);
          }
          tc::mma_commit(&mma_done[q]);
          issued = g + 1;
        }
      } else if (is_epi) {
        // 1. prefetch: warp w owns tile rows 16w..16w+15; lane l the complex
        //    columns c0 + 2l, c0 + 2l + 1 (whole 512-byte tile rows per load)
        const int cl = c0 + 2 * lane;
        const bool cval = cl < c_end && !(cl >= k0 && cl < k0 + nbk) && !(cl >= ex_lo && cl < ex_hi);
        float4 cm[16];
        unsigned rvalid = 0u;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int r = rt * UTC_RT + 16 * warp + u;
          const bool v = cval && r < b && !(r >= k0 && r < k0 + nbk);
          rvalid |= (v ? 1u : 0u) << u;
          cm[u] = v ? *reinterpret_cast<const float4*>(M + (size_t)r * b + cl)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        bool ok = !*abort_flag;
        if (ok) ok = utc_wait(&mma_done[q], ph, abort_flag);
        // 2. the previous tile's staging reads are complete
        utc_epi_sync();
        if (ok) {
          // 3. accumulator -> staging: thread = TMEM lane (tile row), 64 of
          //    the 128 real columns per warp (half h)
          tc::fence_after_sync();
          const int wq = warp & 3, h = warp >> 2;
          const int row = wq * 32 + lane;
          float* srow = stage + row * UTC_STAGE_LD + h * 64;
#pragma unroll
          for (int grp = 0; grp < 4; ++grp) {
            float v[16];
            const uint32_t ta = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)q * (2 * UTC_CT) +
                                (uint32_t)(h * 64 + grp * 16);
            tc::tmem_ld16(ta, v);
#pragma unroll
            for (int u = 0; u < 4; ++u)
              *reinterpret_cast<float4*>(srow + grp * 16 + 4 * u) =
                  make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
          }
          tc::fence_before_sync();
        }
        utc_arrive(&acc_empty[q]);
        // 4. staging complete; 5. add and store the owned rows
        utc_epi_sync();
        if (ok) {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            if (!(rvalid & (1u << u))) continue;
            const int row = 16 * warp + u;
            const float4 a = *reinterpret_cast<const float4*>(stage + row * UTC_STAGE_LD + 4 * lane);
            float4 m = cm[u];
            m.x += a.x;
            m.y += a.y;
            m.z += a.z;
            m.w += a.w;
            *reinterpret_cast<float4*>(M + (size_t)(rt * UTC_RT + row) * b + cl) = m;
          }
        }
      }
    }
  }
  if (is_mma && issued > 0) {
    // the last commit covers every MMA issued: drain before TMEM is freed
    const int last = issued - 1;
    tc::mbar_wait(&mma_done[last & 1], (uint32_t)(last >> 1) & 1u, UTC_WAIT_TRIES);
  }
  if (is_mma && tma_issued > 0) {
    // a raw tile still in flight (after an abort) lands before the CTA exits
    const int last = tma_issued - 1;
    tc::mbar_wait(&raw_full, (uint32_t)last & 1u, UTC_WAIT_TRIES);
  }
  if (tid == 0 && *abort_flag) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
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
        T a = coefv<T>(op, ((size_t)i * b + m) * op.S + slotx(1, dy) * q + cc);
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
  // complex double keeps NB <= 16 so the static NB x NB scratch stays small
  for (int nb = (csz == 16 ? 16 : 32); nb >= 8; nb >>= 1)
    if ((size_t)b * (nb + 1) * csz + 3 * (size_t)nb * (nb + 1) * csz <= cap) return nb;
  return 8;
}

template <typename T>
void launch_schur(const OpView& ov, const double2* shifts, int i, const C_t<T>* Xprev,
                  size_t xstride, C_t<T>* M, int F, cudaStream_t st) {
  constexpr int CB = SchurCfg<T>::CB;
  const size_t smem = Xprev ? schur_smem<T>(ov.q) : 0;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(schur_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)schur_smem<T>(4));
    attr = true;
  }
  dim3 gs((ov.ny + SCHUR_Y - 1) / SCHUR_Y, (ov.b + CB - 1) / CB, F);
  schur_kernel<T><<<gs, CB, smem, st>>>(ov, shifts, i, Xprev, xstride, M);
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
  const size_t xstride = bb;  // X_i is transient: one b x b block per problem

  const size_t psmem = (size_t)b * (NB + 1) * sizeof(C);
  RR_CUDA(cudaFuncSetAttribute(gj_panel_kernel<T, NB>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
  int RB = 4;
  while (RB > 1 && (size_t)RB * b * sizeof(C) + b * sizeof(int) > 160 * 1024) RB >>= 1;
  const size_t fsmem = (size_t)RB * b * sizeof(C) + b * sizeof(int);
  RR_CUDA(cudaFuncSetAttribute(gj_finalize_kernel<T>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem));

  // look-ahead: panel p+1 runs on a second stream while the trailing update
  // of panel p proceeds on the main stream (disjoint columns of M)
  cudaStream_t st2 = fa->stream2;
  const int P = (b + NB - 1) / NB;
  // FP32 factors with 32-column panels, b % 8 == 0 (16-byte aligned rows)
  // and b >= 128 (the TMA map of M) update on the tensor cores;
  // RR_FP32_SIMT and FP64 on the CUDA cores
  constexpr bool tc_shape = std::is_same<T, float>::value && NB == 32;
  const bool use_tc = tc_shape && tc_prec(fa->prec) && b % 8 == 0 && b >= UTC_RT &&
                      fa->tma_m_ok && fa->tune_update != 1;
  if (use_tc)
    RR_CUDA(cudaFuncSetAttribute(gj_update_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)UTC_SMEM));
  auto update = [&](int k0, int nbk, int cb, int ce, int exl, int exh) {
    prof_begin(PROF_UPDATE, st);
    if constexpr (tc_shape) {
      if (use_tc) {
        // one CTA per item (not persistent): CTAs retire after one column
        // tile, so the look-ahead panel kernel on the second stream finds
        // free SMs while the update runs
        // a slice of one column tile (the next panel's columns) splits its
        // row tiles over CTAs: it is on the look-ahead critical path
        const int nct = (ce - cb + UTC_CT - 1) / UTC_CT;
        const int nrg = nct == 1 ? (b + UTC_RT - 1) / UTC_RT : 1;
        const int grid = nct * F * nrg;
        gj_update_tc_kernel<<<grid, UTC_THREADS, UTC_SMEM, st>>>(
            *reinterpret_cast<const CUtensorMap*>(fa->tmap[2]), b, k0, nbk, cb, ce, exl, exh,
            reinterpret_cast<float2*>(M),
            reinterpret_cast<const float2*>(Bbuf), F, nct, nrg, fa->flag + F);
        prof_end(PROF_UPDATE, st);
        return;
      }
    }
    const int ntile = (ce - cb + 63) / 64;
    gj_update_kernel<T, NB><<<dim3(ntile, (b + 63) / 64, F), 256, 0, st>>>(
        b, k0, nbk, cb, ce, exl, exh, M, Bbuf);
    prof_end(PROF_UPDATE, st);
  };
  auto panel = [&](int p, cudaStream_t s) {
    const int k0 = p * NB, nbk = std::min(NB, b - k0);
    prof_begin(PROF_PANEL, s);
    gj_panel_kernel<T, NB><<<F, PANEL_THREADS, psmem, s>>>(b, k0, nbk, M, fa->ipiv, fa->perm,
                                                          fa->flag);
    prof_end(PROF_PANEL, s);
  };
  // (factor_cols > 0 stops after that many columns: autotuner timing only)
  const int ncols = fa->factor_cols > 0 ? std::min(fa->factor_cols, nx) : nx;
  for (int i = 0; i < ncols; ++i) {
    iota_kernel<<<(b * F + 255) / 256, 256, 0, st>>>(fa->perm, b, F);
    prof_count(1);
    const C* Xprev = (i > 0) ? X : nullptr;
    prof_begin(PROF_SCHUR, st);
    launch_schur<T>(ov, fa->shifts, i, Xprev, xstride, M, F, st);
    prof_end(PROF_SCHUR, st);
    panel(0, st);
    for (int p = 0; p < P; ++p) {
      const int k0 = p * NB, nbk = std::min(NB, b - k0);
      prof_begin(PROF_ROWBLOCK, st);
      constexpr int RBT = rb_threads<T, NB>();
      gj_rowblock_kernel<T, NB><<<dim3((b + RBT - 1) / RBT, F), RBT, 0, st>>>(
          b, k0, nbk, M, fa->ipiv, Bbuf);
      prof_end(PROF_ROWBLOCK, st);
      if (p + 1 < P && st2 != nullptr) {
        const int n0 = k0 + nbk, n1 = std::min(b, n0 + NB);
        update(k0, nbk, n0, n1, 0, 0);
        RR_CUDA(cudaEventRecord(fa->ev_next, st));
        RR_CUDA(cudaStreamWaitEvent(st2, fa->ev_next, 0));
        panel(p + 1, st2);
        RR_CUDA(cudaEventRecord(fa->ev_panel, st2));
        update(k0, nbk, 0, b, n0, n1);
        RR_CUDA(cudaStreamWaitEvent(st, fa->ev_panel, 0));
      } else {
        update(k0, nbk, 0, b, 0, 0);
        if (p + 1 < P) panel(p + 1, st);
      }
    }
    C* Xi = (i + 1 < nx) ? X : nullptr;
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

rr_status launch_schur_f32(rr_factors* fa, int i, cudaStream_t st) {
  const OpDev& d = fa->op->d;
  const int b = d.b;
  float2* X = reinterpret_cast<float2*>(fa->X);
  prof_begin(PROF_SCHUR, st);
  launch_schur<float>(view(d), fa->shifts, i, i > 0 ? X : nullptr, (size_t)b * b,
                      reinterpret_cast<float2*>(fa->M), fa->F, st);
  prof_end(PROF_SCHUR, st);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

rr_status launch_factor(rr_factors* fa) {
  if (fa->prec == RR_FP64) return factor_dispatch<double>(fa);
  if (factor_wide_ok(fa) && fa->tune_update != 1) return launch_factor_wide(fa);
  return factor_dispatch<float>(fa);
}
