// Wide block factorisation of the Schur blocks for FP32 factors: the explicit
// inverse G_i = S_i^{-1} of Sec. III.A's one-factorisation-per-shift scheme
// (S_0 = D_0, X_i = G_i C_i, S_{i+1} = D_{i+1} - A_{i+1} X_i), formed by
// Gauss-Jordan elimination with partial pivoting in two levels so that the
// bulk of the work is a rank-128 complex update on the tensor cores.
//
// Pivoting is implicit: rows are never moved.  Column j is eliminated with
// the pivot row p_j (the largest |.| among rows not yet pivoted, lowest row on
// ties) by the elementary transformation E_j (row p_j scaled by 1/m_pj,
// m_pj times it subtracted from every other row; column j then holds E_j's
// column p_j, the in-place inverse).  After all b columns the work matrix is
// M = Q^T S^{-1} Q^T with (Q x)_j = x_{p_j}, so S^{-1}[j, p_m] = M[p_j, m].
//
// Levels, for every slab of W = 128 columns [c0, c1):
//   inner, per panel K of 16 columns:
//     panel  : one CTA per problem holds the tall panel M[:, K] in registers
//              (one row per thread), first applies the previous panel's
//              transformation to it, then the 16 eliminations, recording the
//              pivot rows P (gjw_panel_kernel);
//     update : the transformations of K applied to the rest of the slab but
//              the next panel, M[r, m] += M[r, K] * M_old[P, m] for rows r not
//              in P and M[P, m] = M[P, K] * M_old[P, m] (the pivot rows take
//              T^{-1} B itself: adding (T^{-1} - I) B to B would cancel when
//              T^{-1} is small), in FP32 on the CUDA cores, beside the next
//              panel on a third stream (gjw_slab_update_kernel);
//   outer:
//     gather : B = M[P_slab, outside the slab] (the pivot rows, saved before
//              they change);
//     update : the composed transformation of the slab's 128 eliminations
//              applied at once, M[r, outside] += M[r, slab] * B (r not in
//              P_slab), M[P_slab, outside] = M[P_slab, slab] * B, as a complex
//              GEMM on tcgen05 with the operands split into TF32 or BF16
//              pieces (FP32-level products, FP32 accumulation in TMEM;
//              gjw_gemm_kernel).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "rr_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int GW_W = 128;   // slab width (rank of the outer update)
constexpr int GW_NB = 16;   // panel width (rank of the slab update)
constexpr int GW_PANEL_MAX = 768;  // rows a panel CTA holds (two per thread)

// ------------------------------------------------------------------- panel
// Eliminates columns K = [k0, k0 + nbk) of every row of M (problem =
// blockIdx.x), one row per thread, the row's 16 entries of K held in
// registers.  When kp0 >= 0 the previous panel [kp0, kp0 + 16) of the same
// slab was factored last and its transformation has reached every slab
// column except its own and K (gjw_slab_update_kernel); the kernel applies
// it to K first:
//   x += M[r, Kp] B   (rows not pivoted in Kp),   x = M[r, Kp] B   (its pivot rows),
// B = the rows of Kp's pivots at K before this step.  Then per column j:
// each warp finds its best eligible row (largest |.|^2, lowest row on ties)
// and the winning lane publishes that whole row in shared memory; after one
// block barrier every warp reduces the per-warp candidates itself, reads the
// pivot row from shared memory and eliminates (candidates double-buffered
// by step parity).  Outputs: the columns K of M, rowpiv[r] = pivot column of
// the rows pivoted here, pivslot[k0 + j] = pivot row of column k0 + j.
constexpr int GW_PANEL_THREADS = GW_PANEL_MAX;  // one row per thread up to 768 rows

// rotate a held row left by one place (column c + 1 moves to register c)
__device__ __forceinline__ void gjw_rotate(float2 (&x)[GW_NB]) {
  const float2 first = x[0];
#pragma unroll
  for (int c = 0; c + 1 < GW_NB; ++c) x[c] = x[c + 1];
  x[GW_NB - 1] = first;
}

// staged panel rows: 16 complex padded to 18 (row pitch 144 bytes, so the
// threads of a warp, one row each, spread over the banks)
constexpr int GW_STAGE_LD = GW_NB + 2;

// the 16 columns [c, c + ncol) of every row of M into the stage (zero
// beyond ncol), each warp reading whole 128-byte row segments
__device__ __forceinline__ void gjw_stage_cols(float2* stage, const float2* M, int b, int c,
                                               int ncol) {
  for (int e = threadIdx.x; e < b * (GW_NB / 2); e += blockDim.x) {
    const int row = e / (GW_NB / 2), u = e - row * (GW_NB / 2);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (2 * u < ncol) v = reinterpret_cast<const float4*>(M + (size_t)row * b + c)[u];
    *reinterpret_cast<float4*>(&stage[row * GW_STAGE_LD + 2 * u]) = v;
  }
}

__global__ void __launch_bounds__(GW_PANEL_THREADS, 1)
gjw_panel_kernel(int b, int k0, int nbk, int kp0, float2* __restrict__ Mall,
                 int* __restrict__ rowpiv_all, int* __restrict__ pivslot_all,
                 int* __restrict__ flag) {
  constexpr int NB = GW_NB;
  constexpr int MAXW = GW_PANEL_THREADS / 32;
  __shared__ __align__(16) float2 cand[2][MAXW][NB];
  __shared__ float candv[2][MAXW];
  __shared__ int candi[2][MAXW];
  __shared__ int piv_sm[NB];
  __shared__ __align__(16) float2 Bp[NB][NB];   // Kp's pivot rows at K
  extern __shared__ __align__(16) float2 stage[];  // [b][GW_STAGE_LD]
  const int f = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int nw = blockDim.x >> 5;
  const bool a0 = t < b;
  float2* M = Mall + (size_t)f * b * b;
  int* rowpiv = rowpiv_all + (size_t)f * b;

  float2 x0[NB];
  gjw_stage_cols(stage, M, b, k0, nbk);
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NB; ++c)
    x0[c] = a0 ? stage[t * GW_STAGE_LD + c] : make_float2(0.f, 0.f);
  const int rp = a0 ? rowpiv[t] : -1;
  if (kp0 >= 0) {
    const bool prevpiv = rp >= kp0 && rp < kp0 + NB;
    if (prevpiv) {
#pragma unroll
      for (int c = 0; c < NB; ++c) Bp[rp - kp0][c] = x0[c];
    }
    __syncthreads();  // B published; every row taken from the stage
    gjw_stage_cols(stage, M, b, kp0, NB);
    __syncthreads();
    if (a0) {
      if (prevpiv) {
#pragma unroll
        for (int c = 0; c < NB; ++c) x0[c] = make_float2(0.f, 0.f);
      }
#pragma unroll 1
      for (int j = 0; j < NB; ++j) {
        const float2 a = stage[t * GW_STAGE_LD + j];
#pragma unroll
        for (int c = 0; c < NB; ++c) x0[c] = cfma(a, Bp[j][c], x0[c]);
      }
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c >= nbk) x0[c] = make_float2(0.f, 0.f);
    }
  }
  bool e0 = a0 && rp < 0;
  int col0 = -1;

  // The step loop stays rolled (an unrolled one overflows the instruction
  // cache: every warp would run the whole straight-line program once).  The
  // held rows are kept rotated so that the column being eliminated is always
  // register 0: after each step every row (and so the published pivot row)
  // rotates left by one, and after nbk == NB steps the order is the original
  // one again (a ragged last panel rotates the rest at the end).
#pragma unroll 1
  for (int j = 0; j < nbk; ++j) {
    const int buf = j & 1;
    // this thread's best eligible row, then the warp's, in two warp
    // reductions: the largest key (the bits of a non-negative float order
    // like the float; ineligible rows key 0), then the lowest row holding it
    const float bv0 = e0 ? x0[0].x * x0[0].x + x0[0].y * x0[0].y : -1.f;
    const int mine = a0 ? t : 0x7fffffff;
    const unsigned key = bv0 >= 0.f ? __float_as_uint(bv0) + 1u : 0u;
    const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
    const int bi = (int)__reduce_min_sync(0xffffffffu, key == kmax ? (unsigned)mine : 0x7fffffffu);
    const float bv = kmax == 0u ? -1.f : __uint_as_float(kmax - 1u);
    if (bi == mine && bi != 0x7fffffff) {
      // 16-byte stores: the shared-memory pipe is the step's bottleneck
      float4* dst = reinterpret_cast<float4*>(cand[buf][warp]);
#pragma unroll
      for (int c = 0; c < NB; c += 2) dst[c / 2] = make_float4(x0[c].x, x0[c].y, x0[c + 1].x, x0[c + 1].y);
      candv[buf][warp] = bv;
      candi[buf][warp] = bi;
    }
    __syncthreads();
    // every warp reduces the per-warp candidates the same way; the winning
    // warp is the lowest lane holding the winner
    const float cv = lane < nw ? candv[buf][lane] : -2.f;
    const unsigned ck = cv >= 0.f ? __float_as_uint(cv) + 1u : 0u;
    const unsigned cmax = __reduce_max_sync(0xffffffffu, ck);
    const unsigned ci = lane < nw ? (unsigned)candi[buf][lane] : 0x7fffffffu;
    const int pi = (int)__reduce_min_sync(0xffffffffu, ck == cmax ? ci : 0x7fffffffu);
    const int pw = __ffs(__ballot_sync(0xffffffffu, ck == cmax && ci == (unsigned)pi)) - 1;
    const float pv = cmax == 0u ? -1.f : __uint_as_float(cmax - 1u);
    if (t == 0) {
      piv_sm[j] = pi;
      if (!(pv > 0.f)) flag[f] = 1;
    }
    // the pivot row in registers (16-byte loads, broadcast to the warp)
    float2 prow[NB];
    {
      const float4* src = reinterpret_cast<const float4*>(cand[buf][pw]);
#pragma unroll
      for (int c = 0; c < NB; c += 2) {
        const float4 v = src[c / 2];
        prow[c] = make_float2(v.x, v.y);
        prow[c + 1] = make_float2(v.z, v.w);
      }
    }
    float2 piv = prow[0];
    if (piv.x * piv.x + piv.y * piv.y == 0.f) piv = make_float2(1e-18f, 0.f);
    const float pd = piv.x * piv.x + piv.y * piv.y;
    const float ipd = __frcp_rn(pd);
    const float2 pinv = make_float2(piv.x * ipd, -piv.y * ipd);
    // every held row: x -= (x_0 / pivot) * pivot row, x_0 <- -x_0 / pivot;
    // the pivot row itself is scaled by 1/pivot, its x_0 <- 1/pivot
    if (t != pi) {
      const float2 m0 = cmul(x0[0], pinv);
#pragma unroll
      for (int c = 1; c < NB; ++c) {
        const float2 p = prow[c];
        x0[c].x = fmaf(-m0.x, p.x, fmaf(m0.y, p.y, x0[c].x));
        x0[c].y = fmaf(-m0.x, p.y, fmaf(-m0.y, p.x, x0[c].y));
      }
      x0[0] = make_float2(-m0.x, -m0.y);
    } else {
#pragma unroll
      for (int c = 1; c < NB; ++c) x0[c] = cmul(prow[c], pinv);
      x0[0] = pinv;
      e0 = false;
      col0 = j;
    }
    gjw_rotate(x0);
  }
  // a ragged panel (nbk < NB steps) rotates the remaining NB - nbk places
#pragma unroll 1
  for (int j = nbk; j < NB; ++j) gjw_rotate(x0);
  // panel columns back in place (through shared memory, coalesced); pivot
  // bookkeeping
  __syncthreads();  // the stage is free (the pre-step's reads are done)
  if (a0) {
#pragma unroll
    for (int c = 0; c < NB; ++c) stage[t * GW_STAGE_LD + c] = x0[c];
  }
  if (a0 && col0 >= 0) rowpiv[t] = k0 + col0;
  __syncthreads();
  for (int e = t; e < b * (NB / 2); e += blockDim.x) {
    const int row = e / (NB / 2), u = e - row * (NB / 2);
    if (2 * u < nbk)
      reinterpret_cast<float4*>(M + (size_t)row * b + k0)[u] =
          *reinterpret_cast<const float4*>(&stage[row * GW_STAGE_LD + 2 * u]);
  }
  if (t < nbk) pivslot_all[(size_t)f * b + k0 + t] = piv_sm[t];
}

// ------------------------------------------------------------- slab update
// The transformation of panel K = [k0, k0 + nbk) applied to the slab's other
// columns, except the next panel's [kn0, kn0 + 16) (kn0 < 0: none), which
// that panel's kernel updates itself:
//   M[r, m] += M[r, K] B[:, m]      rows r not pivoted in K,
//   M[r, m]  = M[r, K] B[:, m]      the pivot rows of K (T^{-1} B itself),
// B[j][m] = M[pivslot[k0 + j], m] before this step.  A cluster of SU_CL CTAs
// owns one 16-column group of the slab for one problem, each CTA a range of
// rows: every CTA reads B for the group's columns, then a cluster barrier,
// then the CTAs write their rows (pivot rows included), so no B entry is
// read after it was overwritten and no other cluster touches these columns.
// Exact FP32 on the CUDA cores: a rank-16 contraction is bound by moving the
// columns, not by its flops.
constexpr int SU_THREADS = 256, SU_RT = 64, SU_CL = 4;

__device__ __forceinline__ void su_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

__global__ void __launch_bounds__(SU_THREADS)
gjw_slab_update_kernel(int b, int k0, int nbk, int kn0, int c0, int c1, float2* __restrict__ Mall,
                       const int* __restrict__ rowpiv_all, const int* __restrict__ pivslot_all) {
  constexpr int NB = GW_NB;
  __shared__ float2 Bs[NB][NB + 1];
  __shared__ float2 As[SU_RT][NB + 1];
  const int f = blockIdx.y;
  const int gsel = blockIdx.x / SU_CL, chunk = blockIdx.x % SU_CL;  // cluster = gsel
  // gsel-th 16-column group of [c0, c1) that is neither K nor the next
  // panel (the same for every CTA of the cluster)
  int cs = -1;
  for (int g = 0, cnt = 0; c0 + NB * g < c1; ++g) {
    const int c = c0 + NB * g;
    if (c == k0 || c == kn0) continue;
    if (cnt++ == gsel) {
      cs = c;
      break;
    }
  }
  if (cs < 0) return;  // the whole cluster returns
  const int nc = min(NB, c1 - cs);
  const int rows_per = (b + SU_CL * SU_RT - 1) / (SU_CL * SU_RT) * SU_RT;
  const int rbeg = chunk * rows_per, rend = min(b, rbeg + rows_per);
  float2* M = Mall + (size_t)f * b * b;
  const int* rowpiv = rowpiv_all + (size_t)f * b;
  const int* piv = pivslot_all + (size_t)f * b + k0;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;  // ty: 0 .. 15
  for (int e = tid; e < NB * NB; e += SU_THREADS) {
    const int j = e / NB, c = e - j * NB;
    Bs[j][c] = (j < nbk && c < nc) ? M[(size_t)piv[j] * b + cs + c] : make_float2(0.f, 0.f);
  }
  // every CTA of the cluster has read B before any of them writes a row
  // (pivot rows included); the barrier also orders this CTA's Bs
  su_cluster_sync();
  // Row tiles of SU_RT rows, software-pipelined: the old values and K's
  // entries of tile t + 1 are loaded into registers while tile t is computed.
  constexpr int RI = SU_RT / 16, AI = SU_RT * NB / SU_THREADS;
  float2 old[RI], anext[AI];
  auto load = [&](int r0) {
#pragma unroll
    for (int i = 0; i < RI; ++i) {
      const int r = r0 + ty + 16 * i;
      const bool live = r < rend && tx < nc;
      const int rp = live ? rowpiv[r] : -1;
      const bool pivot = rp >= k0 && rp < k0 + NB;
      old[i] = (live && !pivot) ? M[(size_t)r * b + cs + tx] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < AI; ++u) {
      const int e = tid + u * SU_THREADS, rr = e / NB, k = e - rr * NB, r = r0 + rr;
      anext[u] = (r < rend && k < nbk) ? M[(size_t)r * b + k0 + k] : make_float2(0.f, 0.f);
    }
  };
  if (rbeg < rend) load(rbeg);
#pragma unroll 1
  for (int r0 = rbeg; r0 < rend; r0 += SU_RT) {
#pragma unroll
    for (int u = 0; u < AI; ++u) {
      const int e = tid + u * SU_THREADS, rr = e / NB, k = e - rr * NB;
      As[rr][k] = anext[u];
    }
    float2 acc[RI];
#pragma unroll
    for (int i = 0; i < RI; ++i) acc[i] = old[i];
    __syncthreads();
    if (r0 + SU_RT < rend) load(r0 + SU_RT);
#pragma unroll
    for (int i = 0; i < RI; ++i) {
      const int rr = ty + 16 * i, r = r0 + rr;
#pragma unroll
      for (int k = 0; k < NB; ++k) acc[i] = cfma(As[rr][k], Bs[k][tx], acc[i]);
      if (r < rend && tx < nc) M[(size_t)r * b + cs + tx] = acc[i];
    }
    __syncthreads();
  }
}

// launch of the slab update: ngroups column groups x SU_CL-CTA clusters
rr_status launch_slab_update(int b, int k0, int nbk, int kn0, int c0, int c1, int ngroups, int F,
                             float2* M, const int* rowpiv, const int* pivslot, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ngroups * SU_CL, F, 1);
  cfg.blockDim = dim3(SU_THREADS, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = SU_CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  RR_CUDA(cudaLaunchKernelEx(&cfg, gjw_slab_update_kernel, b, k0, nbk, kn0, c0, c1, M, rowpiv,
                             pivslot));
  return RR_OK;
}

// Outer-update right operand: Bout[f][c][m] = M[P_{c0+c}][m] for m outside
// [c0, c1) and c < c1 - c0; zero elsewhere (rows up to GW_W).
__global__ void gjw_gather_kernel(int b, int c0, int c1, const float2* __restrict__ Mall,
                                  const int* __restrict__ pivslot_all, float2* __restrict__ Bout) {
  const int f = blockIdx.y;
  const int c = blockIdx.x;  // 0 .. GW_W - 1
  const float2* M = Mall + (size_t)f * b * b;
  float2* dst = Bout + ((size_t)f * GW_W + c) * b;
  const bool row_ok = c < c1 - c0;
  const int p = row_ok ? pivslot_all[(size_t)f * b + c0 + c] : 0;
  for (int m = threadIdx.x; m < b; m += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (row_ok && (m < c0 || m >= c1)) v = M[(size_t)p * b + m];
    dst[m] = v;
  }
}

// --------------------------------------------------------------- tensor GEMM
// C[f][rows][cols] (+)= A[f] B[f] for complex FP32 data:
//   A = M[f][:, ka .. ka + Kc)          (b x Kc, from M by TMA)
//   B = Wbuf[f][0..Kc)[cols]            (Kc x b rows by TMA: the slab's pivot rows)
// rows pivoted in [ka, ka + Kc) are overwritten with the product, the other
// rows accumulate it, and the columns [ka, ka + Kc) are left alone.
// Items (problem, 128-row tile, 64-column tile) over the column tiles of up
// to two ranges; persistent CTAs take items round-robin.  Per item the
// contraction runs in chunks of 16 complex columns of A (32 reals of K):
//   control warp : TMA of the raw A chunk (128 x 32 floats) and B chunk (16 x
//                  64 complex) into a 4-stage ring, and the MMAs of each
//                  converted chunk into the item's TMEM accumulator (two, by
//                  item parity);
//   8 converter warps: split the raw chunk into operand pieces (K-major
//                  core-matrix tiles; B expanded to the real 128 x 32 matrix
//                  with rows (Re, -Im), (Im, Re) so one real GEMM gives the
//                  complex product), double-buffered;
//   8 epilogue warps: prefetch the item's rows of C, read the accumulator
//                  (TMEM lane = row) and add it in place,
// so the epilogue of item t overlaps the chunks of item t + 1.  Every wait is
// bounded (tries polls); a timeout sets *err, every role winds down, and the
// control thread drains its copies and MMAs before TMEM is freed.
using tc::SPLIT_BF16X3;
using tc::SPLIT_BF16X6;
using tc::SPLIT_TF32X3;
template <int SPLIT> struct SplitCfg : tc::SplitCfg<SPLIT> {
  static constexpr int KSTEPS = tc::ksteps32<SPLIT>();
};

// piece products (A piece, B piece) in the order they are accumulated: the
// first three are hi.hi, hi.lo, lo.hi (x3 splits); BF16x6 adds the three
// products of the next order, hi.lo2, lo.lo, lo2.hi
__device__ __forceinline__ int prod_a(int pr) { return pr == 2 || pr == 4 ? 1 : pr == 5 ? 2 : 0; }
__device__ __forceinline__ int prod_b(int pr) { return pr == 1 || pr == 4 ? 1 : pr == 3 ? 2 : 0; }

constexpr int GG_RT = 128, GG_CT = 64, GG_KC = 16;  // rows, complex cols, complex K per chunk
constexpr int GG_STAGES = 4;
constexpr uint32_t GG_RAW_A = GG_RT * 2 * GG_KC * 4;  // 16 KB
constexpr uint32_t GG_RAW_B = GG_KC * GG_CT * 8;      // 8 KB
constexpr uint32_t GG_RAW_STAGE = GG_RAW_A + GG_RAW_B;
constexpr int GG_EPI = 256, GG_CONV = 256;
constexpr int GG_THREADS = GG_EPI + GG_CONV + 32;
constexpr uint32_t GG_LBO = 128;

template <int SPLIT>
__host__ __device__ constexpr uint32_t gg_piece_bytes() {
  return (uint32_t)GG_RT * 2 * GG_KC * SplitCfg<SPLIT>::ESZ;  // 128 rows x 32 reals
}
template <int SPLIT>
__host__ __device__ constexpr uint32_t gg_sbo() {
  return tc::sbo32<SPLIT>();  // 32 reals of K per row
}
template <int SPLIT>
__host__ __device__ constexpr uint32_t gg_opbuf_bytes() {
  return 2 * SplitCfg<SPLIT>::PIECES * gg_piece_bytes<SPLIT>();  // A pieces + B pieces
}
template <int SPLIT>
__host__ __device__ constexpr size_t gg_smem_bytes() {
  return 2 * (size_t)gg_opbuf_bytes<SPLIT>() + (size_t)GG_STAGES * GG_RAW_STAGE + 1024;
}

struct GemmArgs {
  int b, F, ka, Kc;            // K range [ka, ka + Kc) of M's columns, Kc % 16 == 0
  int x0, x1, y0, y1;          // column tiles [x0, x1) and [y0, y1) (64 complex each)
  float2* M;
  const int* rowpiv;           // [F][b]
  int* err;
  uint32_t tries;
};

__device__ __forceinline__ bool gg_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                        uint32_t tries) {
  for (uint32_t t = 0; t < tries; ++t) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void gg_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tc::smem_u32(bar)) : "memory");
}

template <int SPLIT>
__global__ void __launch_bounds__(GG_THREADS, 1)
gjw_gemm_kernel(const __grid_constant__ CUtensorMap tmapA, const __grid_constant__ CUtensorMap tmapB,
                GemmArgs g) {
  using Cfg = SplitCfg<SPLIT>;
  constexpr int PIECES = Cfg::PIECES;
  constexpr uint32_t PB = gg_piece_bytes<SPLIT>();
  constexpr uint32_t OPB = gg_opbuf_bytes<SPLIT>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t full_bar[GG_STAGES], opready[2], opfree[2], accfull[2], accempty[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_sh;
  volatile int* abort_flag = &abort_sh;
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* ops = base;                    // 2 operand buffers
  unsigned char* raw = base + 2 * OPB;          // GG_STAGES raw stages
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool is_epi = tid < GG_EPI;
  const bool is_conv = tid >= GG_EPI && tid < GG_EPI + GG_CONV;
  const bool is_ctrl = tid == GG_EPI + GG_CONV;
  const int b = g.b;
  const int nrt = (b + GG_RT - 1) / GG_RT;
  const int n1 = g.x1 - g.x0, nct = n1 + (g.y1 - g.y0);
  const int nitems = g.F * nrt * nct;
  const int nk = g.Kc / GG_KC;
  const int my_items = nitems > (int)blockIdx.x
                           ? (nitems - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                           : 0;
  auto item = [&](int t, int& f, int& rt, int& ctile) {
    const int it = (int)blockIdx.x + t * (int)gridDim.x;
    const int ct = it % nct;
    rt = (it / nct) % nrt;
    f = it / (nct * nrt);
    ctile = ct < n1 ? g.x0 + ct : g.y0 + (ct - n1);
  };

  if (warp == 0) tc::tmem_alloc(&tmem_base, 256);
  if (tid == 0) {
    for (int s = 0; s < GG_STAGES; ++s) tc::mbar_init(&full_bar[s], 1);
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&opready[q], GG_CONV);
      tc::mbar_init(&opfree[q], 1);
      tc::mbar_init(&accfull[q], 1);
      tc::mbar_init(&accempty[q], GG_EPI);
    }
    tc::mbar_init(&drain, 1);
    abort_sh = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (is_ctrl) {
    // ---------------------------------------------------- control thread
    const uint32_t idesc = SPLIT == SPLIT_TF32X3 ? tc::idesc_tf32(GG_RT, 2 * GG_CT)
                                                 : tc::idesc_bf16(GG_RT, 2 * GG_CT);
    int p_t = 0, p_kc = 0, issued = 0;
    int pf = 0, prt = 0, pct = 0;
    if (my_items > 0) item(0, pf, prt, pct);
    auto issue_next = [&]() {
      if (p_t >= my_items) return;
      const int s = issued % GG_STAGES;
      unsigned char* st = raw + s * GG_RAW_STAGE;
      tc::mbar_expect_tx(&full_bar[s], GG_RAW_STAGE);
      tc::tma_load_3d(st, &tmapA, 2 * (g.ka + p_kc * GG_KC), prt * GG_RT, pf, &full_bar[s]);
      tc::tma_load_3d(st + GG_RAW_A, &tmapB, 2 * pct * GG_CT, p_kc * GG_KC, pf, &full_bar[s]);
      ++issued;
      if (++p_kc == nk) {
        p_kc = 0;
        if (++p_t < my_items) item(p_t, pf, prt, pct);
      }
    };
    for (int q = 0; q < GG_STAGES; ++q) issue_next();
    int gch = 0;
    bool ok = true;
    for (int t = 0; t < my_items && ok; ++t) {
      const int a = t & 1;
      if (t >= 2) ok = gg_wait(&accempty[a], (uint32_t)((t - 2) >> 1) & 1u, abort_flag, g.tries);
      for (int kc = 0; kc < nk && ok; ++kc, ++gch) {
        const int q = gch & 1;
        ok = gg_wait(&opready[q], (uint32_t)(gch >> 1) & 1u, abort_flag, g.tries);
        if (!ok) break;
        issue_next();  // raw stage of chunk gch has been converted: refill it
        tc::fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)a * (2 * GG_CT);
        const uint32_t ob = tc::smem_u32(ops + q * OPB);
#pragma unroll
        for (int ks = 0; ks < Cfg::KSTEPS; ++ks) {
#pragma unroll
          for (int pr = 0; pr < Cfg::NPROD; ++pr) {
            const int pa = prod_a(pr), pb = prod_b(pr);
            const uint64_t da = tc::smem_desc(ob + pa * PB + ks * 2 * GG_LBO, GG_LBO, gg_sbo<SPLIT>());
            const uint64_t db = tc::smem_desc(ob + (PIECES + pb) * PB + ks * 2 * GG_LBO, GG_LBO,
                                              gg_sbo<SPLIT>());
            const uint32_t accum = (kc > 0 || ks > 0 || pr > 0) ? 1u : 0u;
            if (SPLIT == SPLIT_TF32X3) tc::mma_tf32(acc, da, db, idesc, accum);
            else tc::mma_bf16(acc, da, db, idesc, accum);
          }
        }
        tc::mma_commit(&opfree[q]);
        if (kc == nk - 1) tc::mma_commit(&accfull[a]);
      }
    }
    if (!ok) {
      *abort_flag = 1;
      // copies still in flight: the last GG_STAGES issued chunks
      for (int c = max(0, issued - GG_STAGES); c < issued; ++c)
        tc::mbar_wait(&full_bar[c % GG_STAGES], (uint32_t)(c / GG_STAGES) & 1u, 1u << 22);
    }
    // every MMA this thread issued completes before TMEM is freed
    tc::mma_commit(&drain);
    tc::mbar_wait(&drain, 0, 1u << 22);
  } else if (is_conv) {
    // -------------------------------------------------------- converters
    const int ct_id = tid - GG_EPI;
    int gch = 0;
    bool ok = true;
    for (int t = 0; t < my_items && ok; ++t) {
      int f, rt, ctile;
      item(t, f, rt, ctile);
      for (int kc = 0; kc < nk; ++kc, ++gch) {
        const int s = gch % GG_STAGES, q = gch & 1;
        ok = gg_wait(&full_bar[s], (uint32_t)(gch / GG_STAGES) & 1u, abort_flag, g.tries);
        if (ok && gch >= 2) ok = gg_wait(&opfree[q], (uint32_t)((gch - 2) >> 1) & 1u, abort_flag, g.tries);
        if (!ok) break;
        const float* RA = reinterpret_cast<const float*>(raw + s * GG_RAW_STAGE);
        const float2* RB = reinterpret_cast<const float2*>(raw + s * GG_RAW_STAGE + GG_RAW_A);
        unsigned char* ob = ops + q * OPB;
        unsigned char* pa[3] = {ob, ob + PB, ob + 2 * PB};
        unsigned char* pbp[3] = {ob + PIECES * PB, ob + (PIECES + 1) * PB, ob + (PIECES + 2) * PB};
        // A: 128 rows x 8 units of 4 reals; rotated order for distinct banks
        for (int it = ct_id; it < GG_RT * 8; it += GG_CONV) {
          const int row = (it & 7) + 8 * (it >> 6);
          const int p = (((it >> 3) & 7) + row) & 7;
          const float4 v = *reinterpret_cast<const float4*>(RA + row * 32 + 4 * p);
          tc::store_split<SPLIT>(v, pa, tc::kmajor_off32<SPLIT>(row, 4 * p));
        }
        // B: 64 complex columns j x 8 pairs of K rows -> real rows 2j, 2j+1
        for (int it = ct_id; it < GG_CT * 8; it += GG_CONV) {
          const int j = it % GG_CT, pp = it / GG_CT;
          const float2 t0 = RB[(2 * pp) * GG_CT + j], t1 = RB[(2 * pp + 1) * GG_CT + j];
          tc::store_split<SPLIT>(make_float4(t0.x, -t0.y, t1.x, -t1.y), pbp, tc::kmajor_off32<SPLIT>(2 * j, 4 * pp));
          tc::store_split<SPLIT>(make_float4(t0.y, t0.x, t1.y, t1.x), pbp, tc::kmajor_off32<SPLIT>(2 * j + 1, 4 * pp));
        }
        tc::fence_async_smem();
        gg_arrive(&opready[q]);
      }
    }
    if (!ok) *abort_flag = 1;
  } else if (is_epi) {
    // ---------------------------------------------------------- epilogue
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its quadrant) in two
    // 16-lane blocks, complex columns 32 (w / 4) .. + 31 of the tile, with
    // the 16x256b fragment: thread t holds rows base + t/4 and base + t/4 + 8
    // and complex columns 4 r + t % 4 (r = 0..7), so every global access of
    // a warp covers 8 rows x 32 contiguous bytes
    const int lq = warp & 3, half = warp >> 2;
    bool ok = true;
    for (int t = 0; t < my_items && ok; ++t) {
      int f, rt, ctile;
      item(t, f, rt, ctile);
      const int a = t & 1;
      const int cb = ctile * GG_CT + half * 32 + (lane & 3);  // + 4 r
      float2* Mf = g.M + (size_t)f * b * b;
      const int* rpf = g.rowpiv + (size_t)f * b;
      int row[4];
      bool add[4];
      float2 cm[4][8];
#pragma unroll
      for (int u = 0; u < 4; ++u) {  // u = 2 * sub-block + (second row)
        row[u] = rt * GG_RT + lq * 32 + 16 * (u >> 1) + (lane >> 2) + 8 * (u & 1);
        // a pivot row of the contraction's columns takes the product itself
        // (E[p, P] B = T^{-1} B); every other row adds it
        const int rp = row[u] < b ? rpf[row[u]] : -1;
        add[u] = !(rp >= g.ka && rp < g.ka + g.Kc);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int c = cb + 4 * r;
          cm[u][r] = (row[u] < b && add[u] && c < b) ? Mf[(size_t)row[u] * b + c]
                                                      : make_float2(0.f, 0.f);
        }
      }
      ok = gg_wait(&accfull[a], (uint32_t)(t >> 1) & 1u, abort_flag, g.tries);
      if (!ok) break;
      tc::fence_after_sync();
#pragma unroll
      for (int sb = 0; sb < 2; ++sb) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float v[16];
          tc::tmem_ld_16x256b_x4(tmem + ((uint32_t)(lq * 32 + 16 * sb) << 16) +
                                     (uint32_t)a * (2 * GG_CT) + (uint32_t)(half * 64 + hh * 32),
                                 v);
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            cm[2 * sb][4 * hh + r].x += v[4 * r];
            cm[2 * sb][4 * hh + r].y += v[4 * r + 1];
            cm[2 * sb + 1][4 * hh + r].x += v[4 * r + 2];
            cm[2 * sb + 1][4 * hh + r].y += v[4 * r + 3];
          }
        }
      }
      tc::fence_before_sync();
      gg_arrive(&accempty[a]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (row[u] >= b) continue;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          // the contraction's own columns (the slab) keep their values
          const int c = cb + 4 * r;
          if (c < b && !(c >= g.ka && c < g.ka + g.Kc)) Mf[(size_t)row[u] * b + c] = cm[u][r];
        }
      }
    }
    if (!ok) *abort_flag = 1;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicExch(g.err, 1);
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// ---------------------------------------------------------------- finalize
// G_i[j][p_m] = M[p_j][m] (S^{-1} from the implicitly pivoted work matrix),
// X_i = G_i C_i with C_i = -L_{i,i+1} (at most 3q entries per column).  A CTA
// gathers RB rows into shared memory (scattering the columns), writes them
// as rows of G_i and forms the same rows of X_i; each thread owns fixed
// columns of X_i, so the (up to 3q) coupling coefficients of a column are
// loaded once and reused for all RB rows.
constexpr int FIN_THREADS = 256, FIN_CPT = 4;  // columns per thread (b <= 1024)

__global__ void __launch_bounds__(FIN_THREADS)
gjw_finalize_kernel(OpView op, int i, int RB, const float2* __restrict__ Mall,
                    const int* __restrict__ pivslot_all, float2* __restrict__ Gi, size_t gstride,
                    float2* __restrict__ Xi, size_t xstride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = op.b, q = op.q;
  float2* Gs = reinterpret_cast<float2*>(smem_raw);        // [RB][b]
  int* ps = reinterpret_cast<int*>(Gs + (size_t)RB * b);   // [b]
  const int f = blockIdx.y;
  const int r0 = blockIdx.x * RB;
  const int nr = min(RB, b - r0);
  const float2* M = Mall + (size_t)f * b * b;
  for (int c = threadIdx.x; c < b; c += FIN_THREADS) ps[c] = pivslot_all[(size_t)f * b + c];
  __syncthreads();
  for (int e = threadIdx.x; e < nr * b; e += FIN_THREADS) {
    const int rr = e / b, c = e - rr * b;
    Gs[rr * b + ps[c]] = M[(size_t)ps[r0 + rr] * b + c];
  }
  __syncthreads();
  float2* G = Gi + (size_t)f * gstride;
  for (int e = threadIdx.x; e < nr * b; e += FIN_THREADS) {
    const int rr = e / b, c = e - rr * b;
    G[(size_t)(r0 + rr) * b + c] = Gs[rr * b + c];
  }
  if (Xi == nullptr) return;
  float2* X = Xi + (size_t)f * xstride;
#pragma unroll
  for (int k = 0; k < FIN_CPT; ++k) {
    const int c = threadIdx.x + k * FIN_THREADS;
    if (c >= b) break;
    // the coupling of column c: entries L[(i, m), (i + 1, c)] for the rows m
    // of the y neighbours of c's point
    const int iyc = c / q, cc = c - iyc * q;
    int mm[12];  // 3 y neighbours x q <= 4 variables
    float aa[12];
#pragma unroll
    for (int t = 0; t < 12; ++t) {
      mm[t] = 0;
      aa[t] = 0.f;
      if (t < 3 * q) {
        const int dy = t / q - 1, cm = t - (t / q) * q;
        const int iym = nbr_y(iyc, -dy, op.ny, op.periodic);
        if (iym >= 0) {
          mm[t] = iym * q + cm;
          aa[t] = op.coef32[((size_t)i * b + mm[t]) * op.S + (2 * 3 + (dy + 1)) * q + cc];
        }
      }
    }
    for (int rr = 0; rr < nr; ++rr) {
      float2 s = make_float2(0.f, 0.f);
#pragma unroll
      for (int t = 0; t < 12; ++t)
        if (aa[t] != 0.f) s = crfma(aa[t], Gs[rr * b + mm[t]], s);
      X[(size_t)(r0 + rr) * b + c] = make_float2(-s.x, -s.y);
    }
  }
}

__global__ void gjw_rowpiv_init_kernel(int* rowpiv, int n) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) rowpiv[e] = -1;
}

template <int SPLIT>
rr_status launch_gemm(rr_factors* fa, const CUtensorMap* ta, const CUtensorMap* tb, int ka, int Kc,
                      int x0, int x1, int y0, int y1, cudaStream_t st) {
  const OpDev& d = fa->op->d;
  GemmArgs a;
  a.b = d.b;
  a.F = fa->F;
  a.ka = ka;
  a.Kc = Kc;
  a.x0 = x0; a.x1 = x1; a.y0 = y0; a.y1 = y1;
  a.M = reinterpret_cast<float2*>(fa->M);
  a.rowpiv = fa->rowpiv;
  a.err = fa->flag + fa->F;
  a.tries = wait_tries();
  const int nrt = (d.b + GG_RT - 1) / GG_RT;
  const long items = (long)fa->F * nrt * ((x1 - x0) + (y1 - y0));
  if (items <= 0) return RR_OK;
  // small launches (up to 8 items per SM): one wave of persistent CTAs;
  // large ones: about four items per CTA, so CTAs retire during the launch
  // and the second stream's panels find SMs as they free up
  const long nsm = num_sms(d.device);
  const int grid = (int)(items <= 8 * nsm ? std::min<long>(items, nsm) : (items + 3) / 4);
  static bool attr = false;
  if (!attr) {
    RR_CUDA(cudaFuncSetAttribute(gjw_gemm_kernel<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gg_smem_bytes<SPLIT>()));
    attr = true;
  }
  prof_begin(PROF_UPDATE, st);
  gjw_gemm_kernel<SPLIT><<<grid, GG_THREADS, gg_smem_bytes<SPLIT>(), st>>>(*ta, *tb, a);
  prof_end(PROF_UPDATE, st);
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

template <int SPLIT>
rr_status factor_wide_impl(rr_factors* fa) {
  const OpDev& d = fa->op->d;
  const OpView ov = view(d);
  const int b = d.b, nx = d.nx, F = fa->F;
  cudaStream_t st = fa->stream;
  float2* M = reinterpret_cast<float2*>(fa->M);
  float2* G = reinterpret_cast<float2*>(fa->G);
  float2* X = reinterpret_cast<float2*>(fa->X);
  const size_t bb = (size_t)b * b;
  const CUtensorMap* tA = reinterpret_cast<const CUtensorMap*>(fa->wmap[0]);
  const CUtensorMap* tBout = reinterpret_cast<const CUtensorMap*>(fa->wmap[1]);
  const int RB = 8;
  const size_t fsmem = (size_t)RB * b * sizeof(float2) + b * sizeof(int);
  RR_CUDA(cudaFuncSetAttribute(gjw_finalize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)fsmem));
  const int nct_all = (b + GG_CT - 1) / GG_CT;
  const int pthreads = (b + 31) & ~31;  // one row per thread
  const size_t psmem = (size_t)b * GW_STAGE_LD * sizeof(float2);
  RR_CUDA(cudaFuncSetAttribute(gjw_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)psmem));
  const int ncols = fa->factor_cols > 0 ? std::min(fa->factor_cols, nx) : nx;
  for (int i = 0; i < ncols; ++i) {
    prof_count(1);
    gjw_rowpiv_init_kernel<<<(F * b + 255) / 256, 256, 0, st>>>(fa->rowpiv, F * b);
    rr_status s = launch_schur_f32(fa, i, st);
    if (s != RR_OK) return s;
    // Inner factorisation of one slab: the panels in order on stream sx,
    // each panel's update of the rest of the slab on stream sy.  Panel p+1
    // applies panel p's transformation to its own columns itself, so it
    // waits only for the slab update of panel p-1 (which reaches its
    // columns) and runs beside the slab update of panel p (disjoint
    // columns; the rows pivoted in p+1 change rowpiv from "none" to a
    // column outside panel p, which that update reads as "not a pivot of p"
    // either way).  The slab updates run in order on sy; sx joins sy at the
    // end.
    auto inner = [&](int c0, cudaStream_t sx, cudaStream_t sy) -> rr_status {
      const int c1 = std::min(b, c0 + GW_W);
      const int npan = (c1 - c0 + GW_NB - 1) / GW_NB;
      cudaEvent_t* ev_pan = fa->ev_w;      // [4] ring: panel p done (on sx)
      cudaEvent_t* ev_upd = fa->ev_w + 4;  // [4] ring: slab update of panel p done (on sy)
      bool used = false;                   // sy took work (it joined sx's order by an event)
      for (int p = 0; p < npan; ++p) {
        const int k0 = c0 + p * GW_NB, nbk = std::min(GW_NB, c1 - k0);
        if (p >= 2) RR_CUDA(cudaStreamWaitEvent(sx, ev_upd[(p - 2) & 3], 0));
        prof_begin(PROF_PANEL, sx);
        gjw_panel_kernel<<<F, pthreads, psmem, sx>>>(b, k0, nbk, p > 0 ? k0 - GW_NB : -1, M,
                                                     fa->rowpiv, fa->pivslot, fa->flag);
        prof_end(PROF_PANEL, sx);
        RR_CUDA(cudaGetLastError());
        // the slab's columns outside this panel and the next one
        const int kn0 = p + 1 < npan ? k0 + GW_NB : -1;
        const int ngroups = npan - 1 - (kn0 >= 0 ? 1 : 0);
        if (ngroups > 0) {
          RR_CUDA(cudaEventRecord(ev_pan[p & 3], sx));
          RR_CUDA(cudaStreamWaitEvent(sy, ev_pan[p & 3], 0));
          prof_begin(PROF_INNER, sy);
          rr_status ls = launch_slab_update(b, k0, nbk, kn0, c0, c1, ngroups, F, M, fa->rowpiv,
                                            fa->pivslot, sy);
          prof_end(PROF_INNER, sy);
          if (ls != RR_OK) return ls;
          RR_CUDA(cudaEventRecord(ev_upd[p & 3], sy));
          used = true;
        }
      }
      if (used) {
        RR_CUDA(cudaEventRecord(fa->ev_w[8], sy));
        RR_CUDA(cudaStreamWaitEvent(sx, fa->ev_w[8], 0));
      }
      return RR_OK;
    };
    // Look-ahead: once the next slab's columns have received this slab's
    // rank-128 update, the next slab's inner factorisation runs on the second
    // (high-priority) stream while the rank-128 update of the remaining
    // columns proceeds on the main stream; the two touch disjoint columns of
    // M (rowpiv entries of the next slab's pivot rows change meanwhile, but
    // only from "not pivoted" to a column outside this slab, which the main
    // stream's update reads as "not a pivot of this slab" either way).  The
    // next slab's pivot rows are gathered on the main stream after both.
    cudaStream_t st2 = fa->stream2;
    cudaStream_t st3 = fa->stream3;
    if ((s = inner(0, st, st3)) != RR_OK) return s;
    for (int c0 = 0; c0 < b; c0 += GW_W) {
      const int c1 = std::min(b, c0 + GW_W);
      if (c1 >= b && c0 == 0) break;  // one slab: no outer update
      prof_begin(PROF_ROWBLOCK, st);
      gjw_gather_kernel<<<dim3(GW_W, F), 256, 0, st>>>(b, c0, c1, M, fa->pivslot,
                                                      reinterpret_cast<float2*>(fa->Wbuf));
      prof_end(PROF_ROWBLOCK, st);
      const int s0 = c0 / GG_CT, s1 = (c1 + GG_CT - 1) / GG_CT;
      if (c1 < b) {
        const int n1 = std::min(b, c1 + GW_W);
        const int u1 = (n1 + GG_CT - 1) / GG_CT;  // tiles [s1, u1): the next slab
        if ((s = launch_gemm<SPLIT>(fa, tA, tBout, c0, GW_W, s1, u1, 0, 0, st)) != RR_OK) return s;
        if (st2 != nullptr) {
          RR_CUDA(cudaEventRecord(fa->ev_next, st));
          RR_CUDA(cudaStreamWaitEvent(st2, fa->ev_next, 0));
          if ((s = inner(c1, st2, st3)) != RR_OK) return s;
          RR_CUDA(cudaEventRecord(fa->ev_panel, st2));
          if ((s = launch_gemm<SPLIT>(fa, tA, tBout, c0, GW_W, 0, s0, u1, nct_all, st)) != RR_OK)
            return s;
          RR_CUDA(cudaStreamWaitEvent(st, fa->ev_panel, 0));
        } else {
          if ((s = launch_gemm<SPLIT>(fa, tA, tBout, c0, GW_W, 0, s0, u1, nct_all, st)) != RR_OK)
            return s;
          if ((s = inner(c1, st, st3)) != RR_OK) return s;
        }
      } else {
        if ((s = launch_gemm<SPLIT>(fa, tA, tBout, c0, GW_W, 0, s0, 0, 0, st)) != RR_OK) return s;
      }
    }
    float2* Xi = (i + 1 < nx) ? X : nullptr;
    prof_begin(PROF_FINALIZE, st);
    gjw_finalize_kernel<<<dim3((b + RB - 1) / RB, F), FIN_THREADS, fsmem, st>>>(
        ov, i, RB, M, fa->pivslot, G + (size_t)i * bb, (size_t)nx * bb, Xi, bb);
    prof_end(PROF_FINALIZE, st);
    RR_CUDA(cudaGetLastError());
  }
  return RR_OK;
}

}  // namespace

// The wide path needs FP32 factors, an even block of at most 768 rows (one
// panel row per thread) and at least 64, and the TMA maps of M and of the
// gathered pivot rows.
bool factor_wide_ok(const rr_factors* fa) {
  const int b = fa->op->d.b;
  return fa->wide_ok && b >= 64 && b <= GW_PANEL_MAX && (b % 8) == 0 &&
         (fa->prec == RR_FP32 || fa->prec == RR_FP32_BF16X3 || fa->prec == RR_FP32_BF16X6);
}

rr_status launch_factor_wide(rr_factors* fa) {
  switch (fa->prec) {
    case RR_FP32_BF16X3: return factor_wide_impl<SPLIT_BF16X3>(fa);
    case RR_FP32_BF16X6: return factor_wide_impl<SPLIT_BF16X6>(fa);
    default: return factor_wide_impl<SPLIT_TF32X3>(fa);
  }
}
