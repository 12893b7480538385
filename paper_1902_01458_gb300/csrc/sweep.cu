// Block forward/back sweeps with the stored factors: the linear solves of
// Algorithm 1 (Sec. II.B, second, fourth and sixth steps), all reusing the
// one factorisation of s I - L (Sec. III.A).
//
// With G_i = S_i^{-1} and C_i = -L_{i,i+1} (at most 3q entries per row):
// Normal solve (s I - L) y = f:
//   forward  z_0 = G_0 f_0,      z_i = G_i (f_i + L_{i,i-1} z_{i-1})
//   backward y_{n-1} = z_{n-1},  y_i = z_i - G_i (C_i y_{i+1})
// Adjoint solve (s I - L)^H w = g:
//   forward  h_0 = g_0,          h_{i+1} = g_{i+1} - C_i^H (G_i^H h_i)
//   backward w_{n-1} = G^H h,    w_i = G_i^H (h_i + L_{i+1,i}^T w_{i+1})
// Only G_i is stored; every step is one dense (b x b) x (b x k) product
// streamed from HBM, plus a sparse coupling product formed by a small kernel
// into a b x k staging block before (or after) it.  One launch per streamwise
// column covers all F problems of the batch.
#include <algorithm>
#include <type_traits>

#include <cuda.h>

#include "rr_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int SW_THREADS = 256;  // each thread owns a 4 x 2 output tile: RT * kp = 2048

enum { FWD = 0, BWD = 1, ADJ_FWD = 2, ADJ_BWD = 3 };
enum { EPI_STORE = 0, EPI_SUB = 1, EPI_TMP = 2 };

__device__ __forceinline__ int slotv(int dx, int dy) { return (dx + 1) * 3 + (dy + 1); }

// Staged right-hand side t (b x k per problem):
//   FWD     (i > 0)      t = in_i + L_{i,i-1} out_{i-1}
//   BWD                  t = C_i out_{i+1} = -L_{i,i+1} out_{i+1}
//   ADJ_BWD (i < nx-1)   t = in_i + L_{i+1,i}^T out_{i+1}
// Grid (ceil(b k / blockDim), active problems): problem f =
// active_problem(amap, blockIdx.y), 32-bit indices within the problem.
template <typename T, int MODE>
__global__ void sweep_rhs_kernel(OpView op, int i, int k, const C_t<T>* in, const C_t<T>* out,
                                 C_t<T>* __restrict__ tbuf, size_t tstride,
                                 const int* __restrict__ amap) {
  using C = C_t<T>;
  const int b = op.b, q = op.q;
  const size_t NK = (size_t)op.n * k;
  const int f = active_problem(amap, blockIdx.y);
  {
    const int rem = blockIdx.x * blockDim.x + threadIdx.x;
    if (rem >= b * k) return;
    const int m = rem / k, j = rem - m * k;
    const C* outf = out + (size_t)f * NK;
    size_t row = (size_t)i * b + m;
    C v = czero<C>();
    if (MODE == FWD) {
      v = in[(size_t)f * NK + row * k + j];
      int iy = m / q;
      const size_t cf = row * op.S;
      for (int dy = -1; dy <= 1; ++dy) {
        int jy = nbr_y(iy, dy, op.ny, op.periodic);
        if (jy < 0) continue;
        for (int cp = 0; cp < q; ++cp) {
          T a = coefv<T>(op, cf + slotv(-1, dy) * q + cp);
          if (a != (T)0) v = crfma(a, outf[((size_t)(i - 1) * b + jy * q + cp) * k + j], v);
        }
      }
    } else if (MODE == BWD) {
      int iy = m / q;
      const size_t cf = row * op.S;
      for (int dy = -1; dy <= 1; ++dy) {
        int jy = nbr_y(iy, dy, op.ny, op.periodic);
        if (jy < 0) continue;
        for (int cp = 0; cp < q; ++cp) {
          T a = coefv<T>(op, cf + slotv(1, dy) * q + cp);
          if (a != (T)0) v = crfma(-a, outf[((size_t)(i + 1) * b + jy * q + cp) * k + j], v);
        }
      }
    } else {
      v = in[(size_t)f * NK + row * k + j];
      int iym = m / q, cm = m - iym * q;
      for (int dy = -1; dy <= 1; ++dy) {
        int iyr = nbr_y(iym, -dy, op.ny, op.periodic);
        if (iyr < 0) continue;
        for (int cr = 0; cr < q; ++cr) {
          size_t rrow = (size_t)(i + 1) * b + iyr * q + cr;
          T a = coefv<T>(op, rrow * op.S + slotv(-1, dy) * q + cm);
          if (a != (T)0) v = crfma(a, outf[rrow * k + j], v);
        }
      }
    }
    tbuf[(size_t)f * tstride + (size_t)m * k + j] = v;
  }
}

// h_{i+1} -= C_i^H t, i.e. h_{i+1}[c] += sum_m L[(i,m),(i+1,c)] t[m] (L real).
// Grid (ceil(b k / blockDim), F) as sweep_rhs_kernel.
template <typename T>
__global__ void adj_couple_kernel(OpView op, int i, int k, const C_t<T>* __restrict__ tbuf,
                                  size_t tstride, C_t<T>* h, const int* __restrict__ amap) {
  using C = C_t<T>;
  const int b = op.b, q = op.q;
  const size_t NK = (size_t)op.n * k;
  const int f = active_problem(amap, blockIdx.y);
  {
    const int rem = blockIdx.x * blockDim.x + threadIdx.x;
    if (rem >= b * k) return;
    const int c = rem / k, j = rem - c * k;
    const int iyc = c / q, cc = c - iyc * q;
    const C* tf = tbuf + (size_t)f * tstride;
    size_t idx = (size_t)f * NK + ((size_t)(i + 1) * b + c) * k + j;
    C v = h[idx];
    for (int dy = -1; dy <= 1; ++dy) {
      int iym = nbr_y(iyc, -dy, op.ny, op.periodic);
      if (iym < 0) continue;
      for (int cm = 0; cm < q; ++cm) {
        int m = iym * q + cm;
        T a = coefv<T>(op, ((size_t)i * b + m) * op.S + slotv(1, dy) * q + cc);
        if (a != (T)0) v = crfma(a, tf[(size_t)m * k + j], v);
      }
    }
    h[idx] = v;
  }
}

// Asynchronous global->shared copy of one complex element (cp.async;
// zero-filled when pred is false).
template <typename C>
__device__ __forceinline__ void cp_async_elem(C* smem, const C* gmem, bool pred) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  if constexpr (sizeof(C) == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(pred ? 16 : 0));
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(pred ? 8 : 0));
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// acc[r][j] = sum_m op(G)[r][m] rhs[m][j] with op = identity or conjugate
// transpose.  rhs is b x k (row stride k) at rhs + f * rstride.  The
// contraction is staged through ST shared-memory stages filled by cp.async
// while the previous stage is consumed; each thread owns a 4 x 2 register
// tile of the RT x kp output.  Epilogue: store to block ob of out, subtract
// from it, or store to the staging block tmp.
template <typename T, bool TRANS, int EPI, int KC, int ST>
__global__ void __launch_bounds__(SW_THREADS)
sweep_step_kernel(int b, int k, int kp, int RT, size_t NK, int ob,
                  const C_t<T>* __restrict__ Mat, size_t mstride, const C_t<T>* rhs,
                  size_t rstride, C_t<T>* out, C_t<T>* tmp, size_t tstride) {
  using C = C_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* base = reinterpret_cast<C*>(smem_raw);
  const int ms_elems = TRANS ? KC * (RT + 1) : RT * (KC + 1);
  const int stage_elems = ms_elems + KC * kp;
  const int f = blockIdx.y;
  const int r0 = blockIdx.x * RT;
  const C* Mf = Mat + (size_t)f * mstride;
  const C* rf = rhs + (size_t)f * rstride;
  const int tid = threadIdx.x;
  const int TX = kp >> 1, TY = SW_THREADS / TX;
  const int tx = tid % TX, ty = tid / TX;

  auto load_stage = [&](int stage, int m0) {
    C* Ms = base + stage * stage_elems;
    C* Ts = Ms + ms_elems;
    if (!TRANS) {
      for (int e = tid; e < RT * KC; e += SW_THREADS) {
        int rr = e / KC, mm = e - rr * KC;
        int r = r0 + rr, m = m0 + mm;
        bool ok = r < b && m < b;
        cp_async_elem(&Ms[rr * (KC + 1) + mm], ok ? Mf + (size_t)r * b + m : Mf, ok);
      }
    } else {
      for (int e = tid; e < RT * KC; e += SW_THREADS) {
        int mm = e / RT, rr = e - mm * RT;
        int r = r0 + rr, m = m0 + mm;
        bool ok = r < b && m < b;
        cp_async_elem(&Ms[mm * (RT + 1) + rr], ok ? Mf + (size_t)m * b + r : Mf, ok);
      }
    }
    for (int e = tid; e < KC * kp; e += SW_THREADS) {
      int mm = e / kp, j = e - mm * kp;
      int m = m0 + mm;
      bool ok = m < b && j < k;
      cp_async_elem(&Ts[mm * kp + j], ok ? rf + (size_t)m * k + j : rf, ok);
    }
  };

  C acc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = czero<C>();

  const int nch = (b + KC - 1) / KC;
#pragma unroll
  for (int s = 0; s < ST - 1; ++s) {
    if (s < nch) load_stage(s, s * KC);
    cp_async_commit();
  }
  for (int c = 0; c < nch; ++c) {
    cp_async_wait<ST - 2>();
    __syncthreads();
    if (c + ST - 1 < nch) load_stage((c + ST - 1) % ST, (c + ST - 1) * KC);
    cp_async_commit();
    const C* Ms = base + (c % ST) * stage_elems;
    const C* Ts = Ms + ms_elems;
#pragma unroll 4
    for (int mm = 0; mm < KC; ++mm) {
      C a[4], bv[2];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        a[i] = TRANS ? cconj(Ms[mm * (RT + 1) + ty + TY * i]) : Ms[(ty + TY * i) * (KC + 1) + mm];
      bv[0] = Ts[mm * kp + tx];
      bv[1] = Ts[mm * kp + tx + TX];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        acc[i][0] = cfma(a[i], bv[0], acc[i][0]);
        acc[i][1] = cfma(a[i], bv[1], acc[i][1]);
      }
    }
  }
  cp_async_wait<0>();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = r0 + ty + TY * i;
    if (r >= b) continue;
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      int j = tx + TX * jj;
      if (j >= k) continue;
      if (EPI == EPI_TMP) {
        tmp[(size_t)f * tstride + (size_t)r * k + j] = acc[i][jj];
      } else {
        size_t idx = (size_t)f * NK + ((size_t)ob * b + r) * k + j;
        if (EPI == EPI_STORE) out[idx] = acc[i][jj];
        else out[idx] = csub(out[idx], acc[i][jj]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Tensor-core sweep step (complex FP32 factors, tcgen05 kind::tf32).
//
// The complex product acc = op(G) t (128 rows of G per CTA, all k columns)
// is one real GEMM: the interleaved rows of op(G) are the K-major A operand
// (K = 2 * 32 reals per chunk) and the right-hand side chunk is expanded to
// the 2k x 64 real matrix Bt with rows (Re t, -Im t, ...) and (Im t, Re t, ...),
// so D = A Bt^T holds (Re, Im) pairs of the complex result.  FP32 accuracy
// comes from splitting every operand into a round-to-nearest TF32 part and
// its remainder, A Bt ~ Ahi Bhi + Ahi Blo + Alo Bhi (3 MMAs per K step).
// Raw tiles arrive by cp.async (double-buffered); one thread issues the MMAs
// into a TMEM accumulator and commits them to an mbarrier; warps 0-3 read the
// 128 x 2k accumulator back with tcgen05.ld.  Waits are bounded: on timeout
// the kernel sets *err, drains its copies, frees TMEM and returns.
constexpr int TC_RT = 128, TC_KC = 32, TC_THREADS = 256;
constexpr uint32_t TC_LBO = 128, TC_SBO = 2048;   // 64 reals of K per 8-row group
constexpr uint32_t TC_WAIT_TRIES = 1u << 22;

__host__ __device__ constexpr size_t tc_smem_bytes(int kp, bool trans) {
  return 2 * 32768 + 2 * (size_t)(2 * kp / 8) * TC_SBO +
         2 * (size_t)((trans ? TC_KC * (TC_RT + 1) : TC_RT * (TC_KC + 1)) + TC_KC * kp) * 8;
}

template <bool TRANS, int EPI>
__global__ void __launch_bounds__(TC_THREADS, 1)
sweep_tc_kernel(int b, int k, int kp, size_t NK, int ob, const float2* __restrict__ Mat,
                size_t mstride, const float2* rhs, size_t rstride, float2* out, float2* tmp,
                size_t tstride, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_ok;
  const int N = 2 * kp;
  const uint32_t bt_bytes = (uint32_t)(N / 8) * TC_SBO;
  // operand tiles start on a 1 KB boundary (the launch adds 1 KB of slack)
  unsigned char* A_hi = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* A_lo = A_hi + 32768;
  unsigned char* B_hi = A_lo + 32768;
  unsigned char* B_lo = B_hi + bt_bytes;
  float2* raw = reinterpret_cast<float2*>(B_lo + bt_bytes);
  const int raw_ms = TRANS ? TC_KC * (TC_RT + 1) : TC_RT * (TC_KC + 1);
  const int raw_elems = raw_ms + TC_KC * kp;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int f = blockIdx.y;
  const int r0 = blockIdx.x * TC_RT;
  const float2* Mf = Mat + (size_t)f * mstride;
  const float2* rf = rhs + (size_t)f * rstride;
  const uint32_t ncols = N <= 32 ? 32u : (N <= 64 ? 64u : 128u);

  if (warp == 0) tc::tmem_alloc(&tmem_base, ncols);
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    s_ok = 1;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  auto load_raw = [&](int stage, int m0) {
    float2* Ms = raw + stage * raw_elems;
    float2* Ts = Ms + raw_ms;
    if (!TRANS) {
      for (int e = tid; e < TC_RT * TC_KC; e += TC_THREADS) {
        int rr = e / TC_KC, mm = e - rr * TC_KC;
        int r = r0 + rr, m = m0 + mm;
        bool ok = r < b && m < b;
        cp_async_elem(&Ms[rr * (TC_KC + 1) + mm], ok ? Mf + (size_t)r * b + m : Mf, ok);
      }
    } else {
      for (int e = tid; e < TC_RT * TC_KC; e += TC_THREADS) {
        int mm = e / TC_RT, rr = e - mm * TC_RT;
        int r = r0 + rr, m = m0 + mm;
        bool ok = r < b && m < b;
        cp_async_elem(&Ms[mm * (TC_RT + 1) + rr], ok ? Mf + (size_t)m * b + r : Mf, ok);
      }
    }
    for (int e = tid; e < TC_KC * kp; e += TC_THREADS) {
      int mm = e / kp, j = e - mm * kp;
      int m = m0 + mm;
      bool ok = m < b && j < k;
      cp_async_elem(&Ts[mm * kp + j], ok ? rf + (size_t)m * k + j : rf, ok);
    }
  };

  const int nch = (b + TC_KC - 1) / TC_KC;
  const uint32_t idesc = tc::idesc_tf32(TC_RT, N);
  load_raw(0, 0);
  cp_async_commit();
  for (int c = 0; c < nch; ++c) {
    cp_async_wait<0>();
    __syncthreads();
    if (c + 1 < nch) load_raw((c + 1) & 1, (c + 1) * TC_KC);
    cp_async_commit();
    if (c > 0) {  // the MMAs of chunk c-1 still read the operand tiles
      if (tid == 0 && !tc::mbar_wait(&mbar, (c - 1) & 1, TC_WAIT_TRIES)) s_ok = 0;
      __syncthreads();
      if (!s_ok) break;
      tc::fence_after_sync();
    }
    const float2* Ms = raw + (c & 1) * raw_elems;
    const float2* Ts = Ms + raw_ms;
    for (int it = tid; it < TC_RT * 16; it += TC_THREADS) {
      const int r = it % TC_RT, p = it / TC_RT;
      float2 g0, g1;
      if (!TRANS) {
        g0 = Ms[r * (TC_KC + 1) + 2 * p];
        g1 = Ms[r * (TC_KC + 1) + 2 * p + 1];
      } else {
        g0 = Ms[(2 * p) * (TC_RT + 1) + r];
        g1 = Ms[(2 * p + 1) * (TC_RT + 1) + r];
        g0.y = -g0.y;
        g1.y = -g1.y;
      }
      float4 h, l;
      tc::split_tf32(g0.x, h.x, l.x);
      tc::split_tf32(g0.y, h.y, l.y);
      tc::split_tf32(g1.x, h.z, l.z);
      tc::split_tf32(g1.y, h.w, l.w);
      const uint32_t off = (uint32_t)(r >> 3) * TC_SBO + (uint32_t)p * TC_LBO + (uint32_t)(r & 7) * 16;
      *reinterpret_cast<float4*>(A_hi + off) = h;
      *reinterpret_cast<float4*>(A_lo + off) = l;
    }
    for (int it = tid; it < kp * 16; it += TC_THREADS) {
      const int j = it % kp, p = it / kp;
      const float2 t0 = Ts[(2 * p) * kp + j], t1 = Ts[(2 * p + 1) * kp + j];
      float4 h0, l0, h1, l1;
      tc::split_tf32(t0.x, h0.x, l0.x);
      tc::split_tf32(-t0.y, h0.y, l0.y);
      tc::split_tf32(t1.x, h0.z, l0.z);
      tc::split_tf32(-t1.y, h0.w, l0.w);
      h1 = make_float4(-h0.y, h0.x, -h0.w, h0.z);
      l1 = make_float4(-l0.y, l0.x, -l0.w, l0.z);
      const int n0 = 2 * j, n1 = 2 * j + 1;
      const uint32_t o0 = (uint32_t)(n0 >> 3) * TC_SBO + (uint32_t)p * TC_LBO + (uint32_t)(n0 & 7) * 16;
      const uint32_t o1 = (uint32_t)(n1 >> 3) * TC_SBO + (uint32_t)p * TC_LBO + (uint32_t)(n1 & 7) * 16;
      *reinterpret_cast<float4*>(B_hi + o0) = h0;
      *reinterpret_cast<float4*>(B_lo + o0) = l0;
      *reinterpret_cast<float4*>(B_hi + o1) = h1;
      *reinterpret_cast<float4*>(B_lo + o1) = l1;
    }
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a_hi = tc::smem_u32(A_hi), a_lo = tc::smem_u32(A_lo);
      const uint32_t b_hi = tc::smem_u32(B_hi), b_lo = tc::smem_u32(B_lo);
#pragma unroll
      for (int prod = 0; prod < 3; ++prod) {
        const uint32_t ab = prod == 2 ? a_lo : a_hi;
        const uint32_t bb = prod == 1 ? b_lo : b_hi;
#pragma unroll
        for (int ks = 0; ks < 8; ++ks) {
          const uint64_t ad = tc::smem_desc(ab + ks * 2 * TC_LBO, TC_LBO, TC_SBO);
          const uint64_t bd = tc::smem_desc(bb + ks * 2 * TC_LBO, TC_LBO, TC_SBO);
          tc::mma_tf32(tmem, ad, bd, idesc, (c > 0 || prod > 0 || ks > 0) ? 1u : 0u);
        }
      }
      tc::mma_commit(&mbar);
    }
  }
  cp_async_wait<0>();
  if (s_ok) {
    if (tid == 0 && !tc::mbar_wait(&mbar, (nch - 1) & 1, TC_WAIT_TRIES)) s_ok = 0;
    __syncthreads();
  }
  tc::fence_after_sync();
  if (s_ok && warp < 4) {
    const int r = r0 + warp * 32 + lane;
    for (int cc = 0; cc < N / 16; ++cc) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 16), v);
      if (r >= b) continue;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int j = cc * 8 + t;
        if (j >= k) continue;
        const float2 a = make_float2(v[2 * t], v[2 * t + 1]);
        if (EPI == EPI_TMP) {
          tmp[(size_t)f * tstride + (size_t)r * k + j] = a;
        } else {
          const size_t idx = (size_t)f * NK + ((size_t)ob * b + r) * k + j;
          if (EPI == EPI_STORE) out[idx] = a;
          else out[idx] = csub(out[idx], a);
        }
      }
    }
  }
  if (!s_ok && tid == 0) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// Tensor-core sweep step fed by TMA, with the contraction split over KS CTAs.
//
// Same arithmetic as sweep_tc_kernel, on chunks of 16 complex columns.  The
// raw 128 x 16 complex tiles of G_i (or of G_i^H) arrive by 3-D TMA (one
// tensor map over all factors, coordinate 2 = problem * nx + column), and the
// matching 16 right-hand-side rows by a 1-D bulk copy, into a 4-stage ring
// guarded by mbarriers.  The split into TF32 hi/lo operand tiles is
// double-buffered so the tensor core works on chunk c while the threads
// split chunk c+1.  CTA (row tile, part) handles the chunks
// [part*cpp, (part+1)*cpp) and writes a partial 128 x k block;
// sweep_combine_kernel adds the KS partials in a fixed order and applies the
// step's epilogue.  All waits are bounded (flag *err).
constexpr int TC2_KC = 16;                                // complex columns per chunk
constexpr int TC2_STAGES = 4;
constexpr uint32_t TC2_SBO = 1024;                        // 32 reals of K per 8-row group
constexpr uint32_t TC2_TILE_BYTES = TC_RT * TC2_KC * 8;   // 16 KB raw tile
constexpr uint32_t TC2_A_BYTES = TC_RT * 2 * TC2_KC * 4;  // 16 KB operand tile

__host__ __device__ constexpr uint32_t tc2_stage_bytes(int kp) {
  return (TC2_TILE_BYTES + (uint32_t)TC2_KC * kp * 8 + 1023u) & ~1023u;
}
// one operand piece: A is 128 rows, B~ is 2 kp rows, of 32 reals of K
template <int SPLIT>
__host__ __device__ constexpr uint32_t tc2_a_piece() { return (TC_RT / 8) * tc::sbo32<SPLIT>(); }
template <int SPLIT>
__host__ __device__ constexpr uint32_t tc2_b_piece(int kp) {
  return (uint32_t)(2 * kp / 8) * tc::sbo32<SPLIT>();
}
template <int SPLIT>
__host__ __device__ constexpr uint32_t tc2_buf_bytes(int kp) {
  return tc::SplitCfg<SPLIT>::PIECES * (tc2_a_piece<SPLIT>() + tc2_b_piece<SPLIT>(kp));
}
template <int SPLIT>
__host__ __device__ constexpr size_t tc2_smem_bytes(int kp) {
  return 2 * (size_t)tc2_buf_bytes<SPLIT>(kp) + (size_t)TC2_STAGES * tc2_stage_bytes(kp);
}

__device__ __forceinline__ bool tc_poll(uint64_t* bar, uint32_t parity, uint32_t tries) {
  return tc::mbar_wait(bar, parity, tries);
}

constexpr int TC2_CONV = 512;                 // converter threads (warps 0-15)
constexpr int TC2_THREADS = TC2_CONV + 32;    // + control warp 16 (TMA producer, MMA issuer)

template <bool TRANS, int SPLIT>
__global__ void __launch_bounds__(TC2_THREADS, 1)
sweep_tc2_kernel(const __grid_constant__ CUtensorMap tmap, int b, int k, int kp, int blk,
                 int nx, int nrt, int KS, int cpp, const float2* rhs, size_t rstride,
                 float2* __restrict__ part, int F, int Fa, const int* __restrict__ amap, int* err,
                 uint32_t tries, int stall) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t full_bar[TC2_STAGES];
  __shared__ uint64_t mma_bar[2];
  __shared__ uint32_t tmem_base;
  constexpr int PIECES = tc::SplitCfg<SPLIT>::PIECES;
  constexpr bool X6 = SPLIT == tc::SPLIT_BF16X6;
  const int N = 2 * kp;
  const uint32_t a_piece = tc2_a_piece<SPLIT>();
  const uint32_t bt_bytes = tc2_b_piece<SPLIT>(kp);
  const uint32_t buf_bytes = tc2_buf_bytes<SPLIT>(kp);  // pieces of A and B of one chunk
  unsigned char* ops = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* raw = ops + 2 * buf_bytes;  // TC2_STAGES stages, 1 KB aligned
  const uint32_t stage_bytes = tc2_stage_bytes(kp);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool ctrl = (tid == TC2_CONV);  // the one thread that feeds TMA and the tensor core
  const int nch = (b + TC2_KC - 1) / TC2_KC;
  const int nitems = nrt * KS * Fa;  // over the active problems
  const int my_items = nitems > (int)blockIdx.x
                           ? (nitems - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                           : 0;
  // x3 splits, per K step two MMAs: A_hi x [B_hi | B_lo] (N = 2 * 2k, both
  // hi products in one pass over A_hi) and A_lo x B_hi.  Up to 32 columns
  // (3N <= 256) two accumulator sets (even and odd K steps) keep consecutive
  // MMAs independent and the epilogue adds six partial sums; with 64 columns
  // one set of 3N = 384 columns takes every K step.  Set layout: [hi.hi |
  // hi.lo | lo.hi], 3N columns.  BF16 x6 (up to 32 columns), per K step three
  // MMAs into one set of 6N columns: p0 x [q0 | q1 | q2], p1 x [q0 | q1], p2 x q0.
  const uint32_t ncols = X6 ? (6 * N <= 128 ? 128u : 6 * N <= 256 ? 256u : 512u)
                            : ((N <= 32) ? 256u : 512u);
  // work item t of this CTA -> (problem, row tile, contraction part)
  auto item = [&](int t, int& f, int& rt, int& ks) {
    const int it = (int)blockIdx.x + t * (int)gridDim.x;
    rt = it % nrt;
    ks = (it / nrt) % KS;
    f = active_problem(amap, it / (nrt * KS));
  };
  auto item_len = [&](int ks) { return min(nch, ks * cpp + cpp) - ks * cpp; };

  if (warp == 0) tc::tmem_alloc(&tmem_base, ncols);
  if (tid == 0) {
    for (int s = 0; s < TC2_STAGES; ++s) tc::mbar_init(&full_bar[s], 1);
    tc::mbar_init(&mma_bar[0], 1);
    tc::mbar_init(&mma_bar[1], 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t set_cols = (uint32_t)(3 * N <= 128 ? 128 : 256);  // one accumulator set
  const bool two_sets = !X6 && 3 * N <= 256;
  const int nprod = (X6 || two_sets) ? 6 : 3;  // partial sums the epilogue adds

  // control thread: the stream of chunks of all this CTA's items.  With
  // stall set (a diagnostic of the bounded waits) the first CTA issues
  // nothing at all, so its first wait runs out with no copy or MMA in flight.
  const bool stalled = stall && blockIdx.x == 0;
  int p_item = 0, p_lc = 0, issued = 0, p_f = 0, p_rt = 0, p_ks = 0, p_len = 0;
  int committed = 0;  // chunks whose MMAs have been committed (control thread)
  if (ctrl && my_items > 0) {
    item(0, p_f, p_rt, p_ks);
    p_len = item_len(p_ks);
  }
  auto issue_next = [&]() {
    if (stalled || p_item >= my_items) return;
    const int m0 = (p_ks * cpp + p_lc) * TC2_KC;
    const int s = issued % TC2_STAGES;
    const uint32_t rhs_bytes = (uint32_t)(min(TC2_KC, b - m0) * k * 8);
    unsigned char* st = raw + s * stage_bytes;
    const int zblk = p_f * nx + blk;
    tc::mbar_expect_tx(&full_bar[s], TC2_TILE_BYTES + rhs_bytes);
    if (!TRANS) tc::tma_load_3d(st, &tmap, 2 * m0, p_rt * TC_RT, zblk, &full_bar[s]);
    else tc::tma_load_3d(st, &tmap, 2 * p_rt * TC_RT, m0, zblk, &full_bar[s]);
    tc::bulk_load(st + TC2_TILE_BYTES, rhs + (size_t)p_f * rstride + (size_t)m0 * k, rhs_bytes,
                  &full_bar[s]);
    ++issued;
    if (++p_lc == p_len) {
      p_lc = 0;
      if (++p_item < my_items) {
        item(p_item, p_f, p_rt, p_ks);
        p_len = item_len(p_ks);
      }
    }
  };
  if (ctrl)
    for (int q = 0; q < TC2_STAGES; ++q) issue_next();
  // operand descriptors of both buffers (piece 0 of A and the pieces of A
  // and of the stacked B~); a K step (32 bytes) advances 256 bytes
  constexpr uint32_t SBO = tc::sbo32<SPLIT>();
  uint64_t dA[2][3], dB[2];
  if (ctrl)
    for (int q = 0; q < 2; ++q) {
      const uint32_t a0 = tc::smem_u32(ops + q * buf_bytes);
      for (int pc = 0; pc < PIECES; ++pc) dA[q][pc] = tc::smem_desc(a0 + pc * a_piece, TC_LBO, SBO);
      dB[q] = tc::smem_desc(a0 + PIECES * a_piece, TC_LBO, SBO);
    }
  auto idesc = [](int n) {
    return SPLIT == tc::SPLIT_TF32X3 ? tc::idesc_tf32(TC_RT, n) : tc::idesc_bf16(TC_RT, n);
  };
  const uint32_t id1 = idesc(N), id2 = idesc(2 * N), id3 = idesc(3 * N);
  auto mma = [](uint32_t d, uint64_t a, uint64_t bb, uint32_t id, uint32_t acc) {
    if (SPLIT == tc::SPLIT_TF32X3) tc::mma_tf32(d, a, bb, id, acc);
    else tc::mma_bf16(d, a, bb, id, acc);
  };
  int g = 0;  // chunks consumed so far (global over this CTA's items)
  bool failed = false;
  for (int t = 0; t < my_items && !failed; ++t) {
    int f, rt, ks;
    item(t, f, rt, ks);
    const int nl = item_len(ks);
    for (int lc = 0; lc < nl; ++lc, ++g) {
      const int s = g % TC2_STAGES, q = g & 1;
      bool ok = true;
      if (tid < TC2_CONV) {
        ok = tc_poll(&full_bar[s], (g / TC2_STAGES) & 1, tries);
        if (ok && g >= 2) ok = tc_poll(&mma_bar[q], ((g - 2) >> 1) & 1, tries);  // buffer q is free
        tc::fence_after_sync();
        unsigned char* ob = ops + q * buf_bytes;
        unsigned char* ap[3] = {ob, ob + a_piece, ob + 2 * a_piece};
        unsigned char* bp[3] = {ob + PIECES * a_piece, ob + PIECES * a_piece + bt_bytes,
                                ob + PIECES * a_piece + 2 * bt_bytes};
        const float* R = reinterpret_cast<const float*>(raw + s * stage_bytes);
        const float2* Rt = reinterpret_cast<const float2*>(raw + s * stage_bytes + TC2_TILE_BYTES);
        if (ok) {
          // rotated item order keeps the 16-byte reads and writes conflict-free
          for (int it = tid; it < TC_RT * 8; it += TC2_CONV) {
            const int r = (it & 7) + 8 * (it >> 6);
            const int p = (((it >> 3) & 7) + r) & 7;
            float4 gv;
            if (!TRANS) {
              gv = *reinterpret_cast<const float4*>(R + r * 32 + 4 * p);
            } else {
              const float2 a = *reinterpret_cast<const float2*>(R + (2 * p) * 256 + 2 * r);
              const float2 c = *reinterpret_cast<const float2*>(R + (2 * p + 1) * 256 + 2 * r);
              gv = make_float4(a.x, -a.y, c.x, -c.y);
            }
            tc::store_split<SPLIT>(gv, ap, tc::kmajor_off32<SPLIT>(r, 4 * p));
          }
          // B~ rows 2j (x_r, -x_i) and 2j + 1 (x_i, x_r) of column j: consecutive
          // threads take consecutive rows, so each 8-thread phase of the
          // 16-byte stores covers the eight row slots of a core matrix
          const int m0 = (ks * cpp + lc) * TC2_KC;
          for (int it = tid; it < 2 * kp * 8; it += TC2_CONV) {
            const int row = it % (2 * kp), p = it / (2 * kp), j = row >> 1;
            const int ma = m0 + 2 * p, mb = ma + 1;
            const float2 t0 = (j < k && ma < b) ? Rt[(2 * p) * k + j] : make_float2(0.f, 0.f);
            const float2 t1 = (j < k && mb < b) ? Rt[(2 * p + 1) * k + j] : make_float2(0.f, 0.f);
            const float4 v = (row & 1) ? make_float4(t0.y, t0.x, t1.y, t1.x)
                                       : make_float4(t0.x, -t0.y, t1.x, -t1.y);
            tc::store_split<SPLIT>(v, bp, tc::kmajor_off32<SPLIT>(row, 4 * p));
          }
        }
        tc::fence_async_smem();
      }
      failed = __syncthreads_or(ok ? 0 : 1) != 0;
      if (failed) break;
      if (ctrl) {
        tc::fence_after_sync();
        issue_next();  // stage s has been split: refill it
#pragma unroll
        for (int kk = 0; kk < tc::ksteps32<SPLIT>(); ++kk) {
          const uint64_t koff = (uint64_t)(kk * 2 * TC_LBO >> 4);
          if (X6) {
            const uint32_t acc = (lc > 0 || kk > 0) ? 1u : 0u;
            mma(tmem, dA[q][0] + koff, dB[q] + koff, id3, acc);
            mma(tmem + 3 * N, dA[q][1] + koff, dB[q] + koff, id2, acc);
            mma(tmem + 5 * N, dA[q][2] + koff, dB[q] + koff, id1, acc);
          } else {
            const uint32_t set = tmem + (two_sets ? (uint32_t)(kk & 1) * set_cols : 0u);
            const uint32_t acc = (lc > 0 || kk > (two_sets ? 1 : 0)) ? 1u : 0u;
            mma(set, dA[q][0] + koff, dB[q] + koff, id2, acc);
            mma(set + 2 * N, dA[q][1] + koff, dB[q] + koff, id1, acc);
          }
        }
        tc::mma_commit(&mma_bar[q]);
        ++committed;
      }
    }
    if (failed) break;
    // item done: wait for its last MMAs, then move the accumulator to its slot
    bool ok = (tid < TC2_CONV) ? tc_poll(&mma_bar[(g - 1) & 1], ((g - 1) >> 1) & 1, tries) : true;
    failed = __syncthreads_or(ok ? 0 : 1) != 0;
    if (failed) break;
    tc::fence_after_sync();
    if (tid < TC2_CONV) {
      // 16x256b fragments: warp w reads lanes 32 (w % 4) + 16 sb + [0, 16)
      // (sb = (w / 4) & 1) and float columns 32 hh + [0, 32) (hh = w / 8) of
      // each partial product; thread t holds rows t/4 and t/4 + 8 and complex
      // columns 4 r + t % 4, so four consecutive threads write 32 contiguous
      // bytes of a row (whole sectors)
      const int lq = warp & 3, sb = (warp >> 2) & 1;
      float2* pf = part + ((size_t)ks * F + f) * (size_t)b * k;
      for (int hh = warp >> 3; hh < (N + 31) / 32; hh += 2) {
        float v[16], w[16];
        const uint32_t ta =
            tmem + ((uint32_t)(lq * 32 + 16 * sb) << 16) + (uint32_t)(hh * 32);
        tc::tmem_ld_16x256b_x4(ta, v);
#pragma unroll
        for (int a = 1; a < 6; ++a) {  // the partial products
          // x3: sets 0/1 x {hi.hi, hi.lo, lo.hi} (one set: a < 3); x6:
          // p0.q0..2, p1.q0..1, p2.q0
          if (a >= nprod) break;
          const uint32_t col = (X6 || !two_sets)
                                   ? (uint32_t)(a * N)
                                   : (uint32_t)(a / 3) * set_cols + (uint32_t)(a % 3) * N;
          tc::tmem_ld_16x256b_x4(ta + col, w);
#pragma unroll
          for (int tt = 0; tt < 16; ++tt) v[tt] += w[tt];
        }
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int r = rt * TC_RT + lq * 32 + 16 * sb + (lane >> 2) + 8 * h2;
          if (r >= b) continue;
#pragma unroll
          for (int rr = 0; rr < 4; ++rr) {
            const int j = hh * 16 + 4 * rr + (lane & 3);
            if (j < k)
              pf[(size_t)r * k + j] = make_float2(v[4 * rr + 2 * h2], v[4 * rr + 2 * h2 + 1]);
          }
        }
      }
    }
    tc::fence_before_sync();  // accumulator reads complete before the next item's MMAs
  }
  if (failed && ctrl) {
    atomicExch(err, 1);
    // drain the copies still in flight before the CTA's shared memory goes,
    // and the last committed MMAs before their tensor memory is freed
    for (int qq = g; qq < issued; ++qq)
      tc::mbar_wait(&full_bar[qq % TC2_STAGES], (qq / TC2_STAGES) & 1, TC_WAIT_TRIES);
    if (committed > 0) {
      const int last = committed - 1;
      tc::mbar_wait(&mma_bar[last & 1], (uint32_t)(last >> 1) & 1u, TC_WAIT_TRIES);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// Sum the KS partial products in a fixed order and apply the step epilogue.
// Grid (ceil(b k / blockDim), active problems): problem f =
// active_problem(amap, blockIdx.y).
template <int EPI>
__global__ void sweep_combine_kernel(int F, int b, int k, int KS, size_t NK, int ob,
                                     const float2* __restrict__ part, float2* out, float2* tmp,
                                     size_t tstride, const int* __restrict__ amap) {
  const size_t total = (size_t)F * b * k;
  const int f = active_problem(amap, blockIdx.y);
  {
    const int rem = blockIdx.x * blockDim.x + threadIdx.x;
    if (rem >= b * k) return;
    const size_t e = (size_t)f * b * k + rem;
    float2 s = part[e];
    for (int q = 1; q < KS; ++q) s = cadd(s, part[(size_t)q * total + e]);
    if (EPI == EPI_TMP) {
      tmp[(size_t)f * tstride + rem] = s;
    } else {
      const size_t idx = (size_t)f * NK + (size_t)ob * b * k + rem;
      if (EPI == EPI_STORE) out[idx] = s;
      else out[idx] = csub(out[idx], s);
    }
  }
}

// One launch of the TMA-fed tensor-core sweep step in the factors' operand
// split (partial products into Pbuf).
template <bool TRANS, int SPLIT, typename C>
rr_status launch_tc2(const CUtensorMap* tm, int grid_x, int b, int k, int kp, int blk, int nx,
                     int nrt, int KS, int cpp, const C* rhs, size_t rstride, rr_factors* fa,
                     cudaStream_t st) {
  const size_t smem = tc2_smem_bytes<SPLIT>(kp) + 1024;
  static size_t attr = 0;  // dynamic shared memory opted in so far
  if (smem > attr) {
    RR_CUDA(cudaFuncSetAttribute(sweep_tc2_kernel<TRANS, SPLIT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = smem;
  }
  sweep_tc2_kernel<TRANS, SPLIT><<<grid_x, TC2_THREADS, smem, st>>>(
      *tm, b, k, kp, blk, nx, nrt, KS, cpp, reinterpret_cast<const float2*>(rhs), rstride,
      reinterpret_cast<float2*>(fa->Pbuf), fa->F, active_count(fa), fa->amap, fa->flag + fa->F,
      wait_tries(), take_stall());
  return RR_OK;
}

}  // namespace

// The split tensor-core sweep (sweep_tc2_kernel) serves FP32 factors with an
// even block of at least 128 and an even k of at most 64 columns (32 for the
// BF16 x6 split, whose six products need 6N accumulator columns); only this
// path runs on a subset of the problems.
bool sweep_tc2_ok(const rr_factors* fa, int k) {
  const int kmax = fa->prec == RR_FP32_BF16X6 ? 32 : 64;
  return tc_prec(fa->prec) && k <= kmax && fa->tma_ok && (k % 2) == 0;
}

namespace {

template <typename T> struct SweepCfg;
template <> struct SweepCfg<float> { static constexpr int KC = 32, ST = 3; };
template <> struct SweepCfg<double> { static constexpr int KC = 16, ST = 2; };

template <typename T, bool TRANS, int EPI>
rr_status gemm_step(rr_factors* fa, int k, int kp, int RT, int ob, int blk, const C_t<T>* Mat,
                    size_t mstride, const C_t<T>* rhs, size_t rstride, C_t<T>* out, C_t<T>* tmp,
                    size_t tstride) {
  using C = C_t<T>;
  constexpr int KC = SweepCfg<T>::KC, ST = SweepCfg<T>::ST;
  const OpDev& d = fa->op->d;
  const int b = d.b, F = fa->F, Fa = active_count(fa);
  const size_t NK = (size_t)d.n * k;
  cudaStream_t st = fa->stream;
  if constexpr (std::is_same<T, float>::value) {
    if (sweep_tc2_ok(fa, k)) {
      const int nrt = (b + TC_RT - 1) / TC_RT;
      const int nch = (b + TC2_KC - 1) / TC2_KC;
      const int nsm = num_sms(d.device);
      // split count: the smallest whose items fill the persistent CTAs to
      // 85 % (each split adds a partial block to write and combine), else
      // the best balance.  The partial buffer holds 4 F b 64 complex, so up
      // to 256 / k splits fit; few active problems (refinement corrections)
      // take more splits to keep the SMs busy.
      const int ks_max = std::min(16, std::max(1, 256 / k));
      int KS = 1;
      double best = 0.0;
      for (int ksc = 1; ksc <= ks_max && ksc <= nch; ++ksc) {
        const int cppc = (nch + ksc - 1) / ksc;
        const int ksr = (nch + cppc - 1) / cppc;
        if (ksr > ks_max) continue;
        const long items = (long)nrt * Fa * ksr;
        const long waves = (items + nsm - 1) / nsm;
        const double eff = (double)items / (double)(waves * nsm);
        if (eff >= 0.85) {
          KS = ksr;
          break;
        }
        if (eff > best + 1e-9) { best = eff; KS = ksr; }
      }
      if (fa->tune_ks > 0) {  // tuned split count (at most the 4 partial buffers)
        const int cppc = (nch + std::min(fa->tune_ks, 4) - 1) / std::min(fa->tune_ks, 4);
        KS = (nch + cppc - 1) / cppc;
      }
      const int cpp = (nch + KS - 1) / KS;
      const int nitems = nrt * Fa * KS;
      const int grid_x = std::min(nitems, nsm);
      const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(fa->tmap[TRANS ? 1 : 0]);
      prof_begin(PROF_SWEEP, st);
      rr_status ls;
      switch (fa->prec) {
        case RR_FP32_BF16X3:
          ls = launch_tc2<TRANS, tc::SPLIT_BF16X3>(tm, grid_x, b, k, kp, blk, d.nx, nrt, KS, cpp,
                                                  rhs, rstride, fa, st);
          break;
        case RR_FP32_BF16X6:
          ls = launch_tc2<TRANS, tc::SPLIT_BF16X6>(tm, grid_x, b, k, kp, blk, d.nx, nrt, KS, cpp,
                                                  rhs, rstride, fa, st);
          break;
        default:
          ls = launch_tc2<TRANS, tc::SPLIT_TF32X3>(tm, grid_x, b, k, kp, blk, d.nx, nrt, KS, cpp,
                                                  rhs, rstride, fa, st);
      }
      if (ls != RR_OK) return ls;
      const dim3 cgrid((b * k + 255) / 256, Fa);
      sweep_combine_kernel<EPI><<<cgrid, 256, 0, st>>>(
          F, b, k, KS, NK, ob, reinterpret_cast<const float2*>(fa->Pbuf), out, tmp, tstride,
          fa->amap);
      prof_end(PROF_SWEEP, st);
      prof_count(1);
      RR_CUDA(cudaGetLastError());
      return RR_OK;
    }
    if (fa->amap) {  // the active-problem list exists only on the split sweep path
      set_error("sweep: active-problem list on a path without it");
      return RR_ERR_ARG;
    }
    if (tc_prec(fa->prec) && kp <= 32) {
      const size_t smem = tc_smem_bytes(kp, TRANS) + 1024;
      static size_t tc_attr = 0;  // dynamic shared memory opted in so far
      if (smem > tc_attr) {
        RR_CUDA(cudaFuncSetAttribute(sweep_tc_kernel<TRANS, EPI>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        tc_attr = smem;
      }
      dim3 grid((b + TC_RT - 1) / TC_RT, F);
      prof_begin(PROF_SWEEP, st);
      sweep_tc_kernel<TRANS, EPI><<<grid, TC_THREADS, smem, st>>>(
          b, k, kp, NK, ob, Mat, mstride, rhs, rstride, out, tmp, tstride, fa->flag + F);
      prof_end(PROF_SWEEP, st);
      cudaError_t le = cudaGetLastError();
      if (le != cudaSuccess) {
        cudaFuncAttributes fat;
        cudaFuncGetAttributes(&fat, sweep_tc_kernel<TRANS, EPI>);
        char buf[256];
        snprintf(buf, sizeof buf,
                 "sweep_tc launch (grid %u x %u, smem %zu, static %zu, max dyn %d, regs %d, "
                 "max threads %d): %s",
                 grid.x, grid.y, smem, fat.sharedSizeBytes, fat.maxDynamicSharedSizeBytes,
                 fat.numRegs, fat.maxThreadsPerBlock, cudaGetErrorString(le));
        set_error(buf);
        return RR_ERR_CUDA;
      }
      return RR_OK;
    }
  }
  static bool attr_set = false;
  if (!attr_set) {
    RR_CUDA(cudaFuncSetAttribute(sweep_step_kernel<T, TRANS, EPI, KC, ST>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr_set = true;
  }
  const size_t ms_elems = TRANS ? (size_t)KC * (RT + 1) : (size_t)RT * (KC + 1);
  const size_t smem = (size_t)ST * (ms_elems + (size_t)KC * kp) * sizeof(C);
  dim3 grid((b + RT - 1) / RT, F);
  prof_begin(PROF_SWEEP, st);
  sweep_step_kernel<T, TRANS, EPI, KC, ST><<<grid, SW_THREADS, smem, st>>>(
      b, k, kp, RT, NK, ob, Mat, mstride, rhs, rstride, out, tmp, tstride);
  prof_end(PROF_SWEEP, st);
  return RR_OK;
}

template <typename T, int MODE>
void stage_rhs(rr_factors* fa, int i, int k, const C_t<T>* in, const C_t<T>* out, C_t<T>* tb) {
  const OpDev& d = fa->op->d;
  const dim3 grid((d.b * k + 255) / 256, active_count(fa));
  prof_count(1);
  sweep_rhs_kernel<T, MODE><<<grid, 256, 0, fa->stream>>>(view(d), i, k, in, out, tb,
                                                          (size_t)d.b * k, fa->amap);
}

template <typename T>
rr_status solve_impl(rr_factors* fa, int k, int adjoint, const void* bv, void* xv, void* tmpv) {
  using C = C_t<T>;
  const OpDev& d = fa->op->d;
  const int b = d.b, nx = d.nx, F = fa->F;
  int kp = 8;
  while (kp < k) kp <<= 1;
  const int RT = 2048 / kp;
  const size_t bb = (size_t)b * b;
  const size_t NK = (size_t)d.n * k;
  const C* G = reinterpret_cast<const C*>(fa->G);
  const size_t gstride = (size_t)nx * bb;
  const C* bin = reinterpret_cast<const C*>(bv);
  C* x = reinterpret_cast<C*>(xv);
  C* tb = reinterpret_cast<C*>(fa->Tbuf);                     // [F][b][k]
  C* tb2 = tb + (size_t)F * b * 64;                           // [F][b][k]
  const size_t tstride = (size_t)b * k;
  rr_status s;
  if (!adjoint) {
    for (int i = 0; i < nx; ++i) {
      const C* rhs = bin;
      size_t rstride = NK;
      if (i > 0) {
        stage_rhs<T, FWD>(fa, i, k, bin, x, tb);
        rhs = tb;
        rstride = tstride;
      }
      if ((s = gemm_step<T, false, EPI_STORE>(fa, k, kp, RT, i, i, G + i * bb, gstride, rhs, rstride,
                                             x, nullptr, 0)) != RR_OK)
        return s;
    }
    for (int i = nx - 2; i >= 0; --i) {
      stage_rhs<T, BWD>(fa, i, k, nullptr, x, tb);
      if ((s = gemm_step<T, false, EPI_SUB>(fa, k, kp, RT, i, i, G + i * bb, gstride, tb, tstride, x,
                                           nullptr, 0)) != RR_OK)
        return s;
    }
  } else {
    C* h = reinterpret_cast<C*>(tmpv);
    if (!fa->amap) {
      RR_CUDA(cudaMemcpyAsync(h, bin, (size_t)F * NK * sizeof(C), cudaMemcpyDeviceToDevice,
                              fa->stream));
    } else {
      for (int a = 0; a < fa->Fa; ++a) {
        const size_t o = (size_t)fa->amap_h[a] * NK;
        RR_CUDA(cudaMemcpyAsync(h + o, bin + o, NK * sizeof(C), cudaMemcpyDeviceToDevice,
                                fa->stream));
      }
    }
    for (int i = 0; i + 1 < nx; ++i) {
      if ((s = gemm_step<T, true, EPI_TMP>(fa, k, kp, RT, 0, i, G + i * bb, gstride,
                                          h + (size_t)i * b * k, NK, nullptr, tb2, tstride)) !=
          RR_OK)
        return s;
      prof_count(1);
      adj_couple_kernel<T><<<dim3((b * k + 255) / 256, active_count(fa)), 256, 0, fa->stream>>>(
          view(d), i, k, tb2, tstride, h, fa->amap);
    }
    for (int i = nx - 1; i >= 0; --i) {
      const C* rhs = h + (size_t)i * b * k;
      size_t rstride = NK;
      if (i + 1 < nx) {
        stage_rhs<T, ADJ_BWD>(fa, i, k, h, x, tb);
        rhs = tb;
        rstride = tstride;
      }
      if ((s = gemm_step<T, true, EPI_STORE>(fa, k, kp, RT, i, i, G + i * bb, gstride, rhs, rstride,
                                            x, nullptr, 0)) != RR_OK)
        return s;
    }
  }
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

}  // namespace

rr_status launch_solve_lo(rr_factors* fa, int k, int adjoint, const void* b, void* x, void* tmp) {
  if (fa->prec == RR_FP64) return solve_impl<double>(fa, k, adjoint, b, x, tmp);
  return solve_impl<float>(fa, k, adjoint, b, x, tmp);
}
