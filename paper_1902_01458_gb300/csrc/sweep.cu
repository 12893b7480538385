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

#include "rr_internal.cuh"

namespace {

constexpr int SW_THREADS = 256;  // each thread owns a 4 x 2 output tile: RT * kp = 2048

enum { FWD = 0, BWD = 1, ADJ_FWD = 2, ADJ_BWD = 3 };
enum { EPI_STORE = 0, EPI_SUB = 1, EPI_TMP = 2 };

__device__ __forceinline__ int slotv(int dx, int dy) { return (dx + 1) * 3 + (dy + 1); }

// Staged right-hand side t (b x k per problem):
//   FWD     (i > 0)      t = in_i + L_{i,i-1} out_{i-1}
//   BWD                  t = C_i out_{i+1} = -L_{i,i+1} out_{i+1}
//   ADJ_BWD (i < nx-1)   t = in_i + L_{i+1,i}^T out_{i+1}
template <typename T, int MODE>
__global__ void sweep_rhs_kernel(OpView op, int i, int k, const C_t<T>* in, const C_t<T>* out,
                                 C_t<T>* __restrict__ tbuf, size_t tstride, int F) {
  using C = C_t<T>;
  const int b = op.b, q = op.q;
  const size_t NK = (size_t)op.n * k;
  const size_t total = (size_t)F * b * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int f = (int)(e / ((size_t)b * k));
    int rem = (int)(e - (size_t)f * b * k);
    int m = rem / k, j = rem - m * k;
    const C* outf = out + (size_t)f * NK;
    size_t row = (size_t)i * b + m;
    C v = czero<C>();
    if (MODE == FWD) {
      v = in[(size_t)f * NK + row * k + j];
      int iy = m / q;
      const double* cf = op.coef + row * op.S;
      for (int dy = -1; dy <= 1; ++dy) {
        int jy = nbr_y(iy, dy, op.ny, op.periodic);
        if (jy < 0) continue;
        for (int cp = 0; cp < q; ++cp) {
          T a = (T)cf[slotv(-1, dy) * q + cp];
          if (a != (T)0) v = crfma(a, outf[((size_t)(i - 1) * b + jy * q + cp) * k + j], v);
        }
      }
    } else if (MODE == BWD) {
      int iy = m / q;
      const double* cf = op.coef + row * op.S;
      for (int dy = -1; dy <= 1; ++dy) {
        int jy = nbr_y(iy, dy, op.ny, op.periodic);
        if (jy < 0) continue;
        for (int cp = 0; cp < q; ++cp) {
          T a = (T)cf[slotv(1, dy) * q + cp];
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
          T a = (T)op.coef[rrow * op.S + slotv(-1, dy) * q + cm];
          if (a != (T)0) v = crfma(a, outf[rrow * k + j], v);
        }
      }
    }
    tbuf[(size_t)f * tstride + (size_t)m * k + j] = v;
  }
}

// h_{i+1} -= C_i^H t, i.e. h_{i+1}[c] += sum_m L[(i,m),(i+1,c)] t[m] (L real).
template <typename T>
__global__ void adj_couple_kernel(OpView op, int i, int k, const C_t<T>* __restrict__ tbuf,
                                  size_t tstride, C_t<T>* h, int F) {
  using C = C_t<T>;
  const int b = op.b, q = op.q;
  const size_t NK = (size_t)op.n * k;
  const size_t total = (size_t)F * b * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    int f = (int)(e / ((size_t)b * k));
    int rem = (int)(e - (size_t)f * b * k);
    int c = rem / k, j = rem - c * k;
    const int iyc = c / q, cc = c - iyc * q;
    const C* tf = tbuf + (size_t)f * tstride;
    size_t idx = (size_t)f * NK + ((size_t)(i + 1) * b + c) * k + j;
    C v = h[idx];
    for (int dy = -1; dy <= 1; ++dy) {
      int iym = nbr_y(iyc, -dy, op.ny, op.periodic);
      if (iym < 0) continue;
      for (int cm = 0; cm < q; ++cm) {
        int m = iym * q + cm;
        T a = (T)op.coef[((size_t)i * b + m) * op.S + slotv(1, dy) * q + cc];
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

template <typename T> struct SweepCfg;
template <> struct SweepCfg<float> { static constexpr int KC = 32, ST = 3; };
template <> struct SweepCfg<double> { static constexpr int KC = 16, ST = 2; };

template <typename T, bool TRANS, int EPI>
rr_status gemm_step(rr_factors* fa, int k, int kp, int RT, int ob, const C_t<T>* Mat,
                    size_t mstride, const C_t<T>* rhs, size_t rstride, C_t<T>* out, C_t<T>* tmp,
                    size_t tstride) {
  using C = C_t<T>;
  constexpr int KC = SweepCfg<T>::KC, ST = SweepCfg<T>::ST;
  const OpDev& d = fa->op->d;
  const int b = d.b, F = fa->F;
  const size_t NK = (size_t)d.n * k;
  cudaStream_t st = fa->stream;
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
  const size_t total = (size_t)fa->F * d.b * k;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 8192);
  prof_count(1);
  sweep_rhs_kernel<T, MODE><<<blocks, 256, 0, fa->stream>>>(view(d), i, k, in, out, tb,
                                                            (size_t)d.b * k, fa->F);
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
      if ((s = gemm_step<T, false, EPI_STORE>(fa, k, kp, RT, i, G + i * bb, gstride, rhs, rstride,
                                             x, nullptr, 0)) != RR_OK)
        return s;
    }
    for (int i = nx - 2; i >= 0; --i) {
      stage_rhs<T, BWD>(fa, i, k, nullptr, x, tb);
      if ((s = gemm_step<T, false, EPI_SUB>(fa, k, kp, RT, i, G + i * bb, gstride, tb, tstride, x,
                                           nullptr, 0)) != RR_OK)
        return s;
    }
  } else {
    C* h = reinterpret_cast<C*>(tmpv);
    RR_CUDA(cudaMemcpyAsync(h, bin, (size_t)F * NK * sizeof(C), cudaMemcpyDeviceToDevice,
                            fa->stream));
    const size_t total = (size_t)F * b * k;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 8192);
    for (int i = 0; i + 1 < nx; ++i) {
      if ((s = gemm_step<T, true, EPI_TMP>(fa, k, kp, RT, 0, G + i * bb, gstride,
                                          h + (size_t)i * b * k, NK, nullptr, tb2, tstride)) !=
          RR_OK)
        return s;
      prof_count(1);
      adj_couple_kernel<T><<<blocks, 256, 0, fa->stream>>>(view(d), i, k, tb2, tstride, h, F);
    }
    for (int i = nx - 1; i >= 0; --i) {
      const C* rhs = h + (size_t)i * b * k;
      size_t rstride = NK;
      if (i + 1 < nx) {
        stage_rhs<T, ADJ_BWD>(fa, i, k, h, x, tb);
        rhs = tb;
        rstride = tstride;
      }
      if ((s = gemm_step<T, true, EPI_STORE>(fa, k, kp, RT, i, G + i * bb, gstride, rhs, rstride,
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
