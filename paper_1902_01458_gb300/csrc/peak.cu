// Measured peaks of the arithmetic units the kernels of this library use, for
// their roofline fractions: tcgen05 MMA throughput (kind::tf32 and kind::f16
// with BF16 operands, FP32 accumulation in TMEM) and FMA throughput of the
// CUDA cores (FP64, FP32).  Each microbenchmark keeps its operands on chip
// (shared memory, TMEM, registers), so it measures the unit, not memory.
#include <algorithm>

#include "rr_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int PK_M = 128, PK_N = 256;
constexpr uint32_t PK_LBO = 128, PK_SBO = 256;  // one K step (32 bytes) per 8-row group

// One CTA per SM: one thread issues `iters` MMAs of 128 x 256 x (32 bytes of
// K) into one TMEM accumulator back to back, then waits for their completion.
template <bool BF16>
__global__ void __launch_bounds__(128, 1) mma_peak_kernel(int iters, int* err) {
  __shared__ __align__(1024) unsigned char A[PK_M * 32];
  __shared__ __align__(1024) unsigned char B[PK_N * 32];
  __shared__ uint64_t done;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x;
  // small nonzero operands (the tensor core's power depends on the data)
  for (int i = tid; i < PK_M * 8; i += blockDim.x)
    reinterpret_cast<uint32_t*>(A)[i] = BF16 ? 0x3C003C00u + (i & 7) : 0x3F800000u + (i & 255);
  for (int i = tid; i < PK_N * 8; i += blockDim.x)
    reinterpret_cast<uint32_t*>(B)[i] = BF16 ? 0x3C003C00u + (i & 3) : 0x3F800000u + (i & 127);
  if (tid < 32) tc::tmem_alloc(&tmem_base, PK_N);
  if (tid == 0) tc::mbar_init(&done, 1);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    const uint64_t da = tc::smem_desc(tc::smem_u32(A), PK_LBO, PK_SBO);
    const uint64_t db = tc::smem_desc(tc::smem_u32(B), PK_LBO, PK_SBO);
    const uint32_t idesc = BF16 ? tc::idesc_bf16(PK_M, PK_N) : tc::idesc_tf32(PK_M, PK_N);
    for (int it = 0; it < iters; ++it) {
      if (BF16) tc::mma_bf16(tmem, da, db, idesc, it > 0 ? 1u : 0u);
      else tc::mma_tf32(tmem, da, db, idesc, it > 0 ? 1u : 0u);
    }
    tc::mma_commit(&done);
    if (!tc::mbar_wait(&done, 0, 1u << 26)) atomicExch(err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid < 32) tc::tmem_dealloc(tmem, PK_N);
}

// Eight independent FMA chains per thread.
template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T x, T y, T* out) {
  T a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fma(a[c], x, y);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" rr_status rr_measure_peak(int kind, int device, double* tflops) {
  if (!tflops || kind < 0 || kind > 3) {
    set_error("rr_measure_peak: kind must be 0..3 and tflops non-null");
    return RR_ERR_ARG;
  }
  int prev = -1;
  RR_CUDA(cudaGetDevice(&prev));
  if (prev != device) RR_CUDA(cudaSetDevice(device));
  const int nsm = num_sms(device);
  int* err = nullptr;
  void* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rr_status st = RR_OK;
  auto fail = [&](cudaError_t e, const char* what) {
    if (st == RR_OK && e != cudaSuccess) st = cuda_status(e, what);
  };
  fail(cudaMalloc(&err, sizeof(int)), "rr_measure_peak");
  const int fma_blocks = nsm * 8;
  fail(cudaMalloc(&out, (size_t)fma_blocks * 256 * sizeof(double)), "rr_measure_peak");
  fail(cudaMemset(err, 0, sizeof(int)), "rr_measure_peak");
  fail(cudaEventCreate(&e0), "rr_measure_peak");
  fail(cudaEventCreate(&e1), "rr_measure_peak");
  double flops = 0.0;
  float best = 0.f;
  for (int rep = 0; rep < 6 && st == RR_OK; ++rep) {
    fail(cudaEventRecord(e0), "rr_measure_peak");
    if (kind == 0 || kind == 1) {
      const int iters = 1 << 15;
      prof_count(1);
      if (kind == 0) mma_peak_kernel<false><<<nsm, 128>>>(iters, err);
      else mma_peak_kernel<true><<<nsm, 128>>>(iters, err);
      flops = 2.0 * PK_M * PK_N * (kind == 0 ? 8 : 16) * (double)iters * nsm;
    } else {
      const int iters = 1 << 14;
      prof_count(1);
      if (kind == 2)
        fma_peak_kernel<double><<<fma_blocks, 256>>>(iters, 0.999999, 1e-7,
                                                     static_cast<double*>(out));
      else
        fma_peak_kernel<float><<<fma_blocks, 256>>>(iters, 0.9999f, 1e-4f,
                                                    static_cast<float*>(out));
      flops = 2.0 * 8 * (double)iters * fma_blocks * 256;
    }
    fail(cudaGetLastError(), "rr_measure_peak launch");
    fail(cudaEventRecord(e1), "rr_measure_peak");
    fail(cudaEventSynchronize(e1), "rr_measure_peak");
    float ms = 0.f;
    fail(cudaEventElapsedTime(&ms, e0, e1), "rr_measure_peak");
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;  // first run is a warm-up
  }
  int herr = 0;
  if (st == RR_OK) fail(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost), "rr_measure_peak");
  if (st == RR_OK && herr) {
    set_error("rr_measure_peak: the MMA loop timed out");
    st = RR_ERR_TIMEOUT;
  }
  if (st == RR_OK) *tflops = flops / (best * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(err);
  cudaFree(out);
  if (prev != device && prev >= 0) cudaSetDevice(prev);
  return st;
}
