// Block forward/back sweeps with the stored factors: the linear solves of
// Algorithm 1 (Sec. II.B, second, fourth and sixth steps), all reusing the
// one factorisation of s I - L (Sec. III.A).
//
// Normal solve (s I - L) y = f:
//   forward  z_0 = G_0 f_0,     z_i = G_i (f_i + L_{i,i-1} z_{i-1})
//   backward y_{n-1} = z_{n-1}, y_i = z_i - X_i y_{i+1}
// Adjoint solve (s I - L)^H w = g:
//   forward  h_0 = g_0,         h_{i+1} = g_{i+1} - X_i^H h_i
//   backward w_{n-1} = G^H h,   w_i = G_i^H (h_i + L_{i+1,i}^T w_{i+1})
// Each step is a dense (b x b) x (b x k) product streamed from HBM.  The
// sparse coupling term of the forward/adjoint-backward steps is formed once
// per column by a small kernel into a b x k staging block, which the product
// kernel then reads like any other right-hand side.  One launch per
// streamwise column covers all F problems of the batch.
#include <algorithm>

#include "rr_internal.cuh"

namespace {

constexpr int SW_THREADS = 256;
constexpr int SW_OUT = 8;    // outputs per thread: RT * kp = 2048
constexpr int SW_KC = 32;    // chunk of the contraction dimension

enum { FWD = 0, BWD = 1, ADJ_FWD = 2, ADJ_BWD = 3 };

__device__ __forceinline__ int slotv(int dx, int dy) { return (dx + 1) * 3 + (dy + 1); }

// t = in_i + L_{i,i-1} out_{i-1}      (FWD, i > 0)
// t = in_i + L_{i+1,i}^T out_{i+1}    (ADJ_BWD, i < nx-1)
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
    const C* inf = in + (size_t)f * NK;
    const C* outf = out + (size_t)f * NK;
    size_t row = (size_t)i * b + m;
    C v = inf[row * k + j];
    if (MODE == FWD) {
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
    } else {
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

// acc[r][j] = sum_m op(Mat)[r][m] rhs[m][j]; epilogue by MODE.
// rhs is b x k (row stride k) at rhs + f * rstride.
template <typename T, int MODE>
__global__ void __launch_bounds__(SW_THREADS)
sweep_step_kernel(int b, int k, int kp, int RT, size_t NK, int ob,
                  const C_t<T>* __restrict__ Mat, size_t mstride, const C_t<T>* rhs,
                  size_t rstride, C_t<T>* out) {
  using C = C_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Ms = reinterpret_cast<C*>(smem_raw);   // [RT][KC+1]
  C* Ts = Ms + RT * (SW_KC + 1);            // [KC][kp]
  const int f = blockIdx.y;
  const int r0 = blockIdx.x * RT;
  const C* Mf = Mat + (size_t)f * mstride;
  const C* rf = rhs + (size_t)f * rstride;
  C* outf = out + (size_t)f * NK;
  const int tid = threadIdx.x;

  C acc[SW_OUT];
#pragma unroll
  for (int t = 0; t < SW_OUT; ++t) acc[t] = czero<C>();

  for (int m0 = 0; m0 < b; m0 += SW_KC) {
    for (int e = tid; e < SW_KC * kp; e += SW_THREADS) {
      int mm = e / kp, j = e - mm * kp;
      int m = m0 + mm;
      Ts[mm * kp + j] = (m < b && j < k) ? rf[(size_t)m * k + j] : czero<C>();
    }
    if (MODE == FWD || MODE == BWD) {
      for (int e = tid; e < RT * SW_KC; e += SW_THREADS) {
        int rr = e / SW_KC, mm = e - rr * SW_KC;
        int r = r0 + rr, m = m0 + mm;
        Ms[rr * (SW_KC + 1) + mm] = (r < b && m < b) ? Mf[(size_t)r * b + m] : czero<C>();
      }
    } else {
      for (int e = tid; e < RT * SW_KC; e += SW_THREADS) {
        int mm = e / RT, rr = e - mm * RT;
        int r = r0 + rr, m = m0 + mm;
        Ms[rr * (SW_KC + 1) + mm] =
            (r < b && m < b) ? cconj(Mf[(size_t)m * b + r]) : czero<C>();
      }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < SW_OUT; ++t) {
      int o = tid + t * SW_THREADS;
      int rr = o / kp, j = o - rr * kp;
      const C* mrow = Ms + rr * (SW_KC + 1);
      C a = acc[t];
#pragma unroll 8
      for (int mm = 0; mm < SW_KC; ++mm) a = cfma(mrow[mm], Ts[mm * kp + j], a);
      acc[t] = a;
    }
    __syncthreads();
  }
#pragma unroll
  for (int t = 0; t < SW_OUT; ++t) {
    int o = tid + t * SW_THREADS;
    int rr = o / kp, j = o - rr * kp;
    int r = r0 + rr;
    if (r >= b || j >= k) continue;
    size_t idx = ((size_t)ob * b + r) * k + j;
    if (MODE == FWD || MODE == ADJ_BWD) {
      outf[idx] = acc[t];
    } else {
      outf[idx] = csub(outf[idx], acc[t]);
    }
  }
}

template <typename T, int MODE>
rr_status step(rr_factors* fa, int i, int k, int kp, int RT, const C_t<T>* Mat, size_t mstride,
               const C_t<T>* in, C_t<T>* out) {
  using C = C_t<T>;
  const OpDev& d = fa->op->d;
  const int b = d.b, F = fa->F;
  const size_t NK = (size_t)d.n * k;
  cudaStream_t st = fa->stream;
  static bool attr_set = false;
  if (!attr_set) {
    RR_CUDA(cudaFuncSetAttribute(sweep_step_kernel<T, MODE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  // right-hand side block of this step
  const C* rhs;
  size_t rstride = NK;
  int ob = i;
  if (MODE == FWD) {
    if (i == 0) {
      rhs = in;
    } else {
      C* tb = reinterpret_cast<C*>(fa->Tbuf);
      size_t tstride = (size_t)b * k;
      size_t total = (size_t)F * b * k;
      int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
      prof_count(1);
      sweep_rhs_kernel<T, FWD><<<blocks, 256, 0, st>>>(view(d), i, k, in, out, tb, tstride, F);
      rhs = tb;
      rstride = tstride;
    }
    if (i == 0) rhs = in;  // block 0 of the input
  } else if (MODE == ADJ_BWD) {
    if (i + 1 == d.nx) {
      rhs = in + (size_t)i * b * k;
    } else {
      C* tb = reinterpret_cast<C*>(fa->Tbuf);
      size_t tstride = (size_t)b * k;
      size_t total = (size_t)F * b * k;
      int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
      prof_count(1);
      sweep_rhs_kernel<T, ADJ_BWD><<<blocks, 256, 0, st>>>(view(d), i, k, in, out, tb, tstride, F);
      rhs = tb;
      rstride = tstride;
    }
  } else if (MODE == BWD) {
    rhs = out + (size_t)(i + 1) * b * k;
  } else {  // ADJ_FWD
    rhs = out + (size_t)i * b * k;
    ob = i + 1;
  }
  size_t smem = ((size_t)RT * (SW_KC + 1) + (size_t)SW_KC * kp) * sizeof(C);
  dim3 grid((b + RT - 1) / RT, F);
  prof_begin(PROF_SWEEP, st);
  sweep_step_kernel<T, MODE><<<grid, SW_THREADS, smem, st>>>(b, k, kp, RT, NK, ob, Mat, mstride,
                                                             rhs, rstride, out);
  prof_end(PROF_SWEEP, st);
  return RR_OK;
}

template <typename T>
rr_status solve_impl(rr_factors* fa, int k, int adjoint, const void* bv, void* xv, void* tmpv) {
  using C = C_t<T>;
  const OpDev& d = fa->op->d;
  const int b = d.b, nx = d.nx;
  int kp = 8;
  while (kp < k) kp <<= 1;
  const int RT = (SW_THREADS * SW_OUT) / kp;
  const size_t bb = (size_t)b * b;
  const C* G = reinterpret_cast<const C*>(fa->G);
  const C* X = reinterpret_cast<const C*>(fa->X);
  const size_t gstride = (size_t)nx * bb;
  const size_t xstride = (size_t)(nx > 1 ? nx - 1 : 1) * bb;
  const C* bin = reinterpret_cast<const C*>(bv);
  C* x = reinterpret_cast<C*>(xv);
  rr_status s;
  if (!adjoint) {
    for (int i = 0; i < nx; ++i)
      if ((s = step<T, FWD>(fa, i, k, kp, RT, G + i * bb, gstride, bin, x)) != RR_OK) return s;
    for (int i = nx - 2; i >= 0; --i)
      if ((s = step<T, BWD>(fa, i, k, kp, RT, X + i * bb, xstride, bin, x)) != RR_OK) return s;
  } else {
    C* h = reinterpret_cast<C*>(tmpv);
    RR_CUDA(cudaMemcpyAsync(h, bin, (size_t)fa->F * d.n * k * sizeof(C),
                            cudaMemcpyDeviceToDevice, fa->stream));
    for (int i = 0; i + 1 < nx; ++i)
      if ((s = step<T, ADJ_FWD>(fa, i, k, kp, RT, X + i * bb, xstride, h, h)) != RR_OK) return s;
    for (int i = nx - 1; i >= 0; --i)
      if ((s = step<T, ADJ_BWD>(fa, i, k, kp, RT, G + i * bb, gstride, h, x)) != RR_OK) return s;
  }
  RR_CUDA(cudaGetLastError());
  return RR_OK;
}

}  // namespace

rr_status launch_solve_lo(rr_factors* fa, int k, int adjoint, const void* b, void* x, void* tmp) {
  if (fa->prec == RR_FP64) return solve_impl<double>(fa, k, adjoint, b, x, tmp);
  return solve_impl<float>(fa, k, adjoint, b, x, tmp);
}
