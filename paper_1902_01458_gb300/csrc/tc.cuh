// Blackwell (sm_103a) tensor-core helpers: tcgen05 MMA with TMEM accumulators,
// shared-memory matrix descriptors, mbarriers with bounded waits.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace tc {

// ---- shared-memory matrix descriptor (K-major, no swizzle) ----------------
// A tile of R rows x K 32-bit elements is stored as 8-row x 16-byte core
// matrices: element (r, kk) at (r/8)*SBO + (kk/4)*LBO + (r%8)*16 + (kk%4)*4.
// Descriptor fields: start address, LBO (core-matrix stride along K) and SBO
// (stride between 8-row groups), all in 16-byte units; version 1; layout 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, LBO mode 0, layout type 0 (no swizzle)
}

// ---- instruction descriptor: kind::tf32, FP32 accumulate, A/B K-major ------
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4)                       // D format: F32
         | (2u << 7)                     // A format: TF32
         | (2u << 10)                    // B format: TF32
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// ---- instruction descriptor: kind::f16 with BF16 A and B, FP32 accumulate --
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)                       // D format: F32
         | (1u << 7)                     // A format: BF16
         | (1u << 10)                    // B format: BF16
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- TMEM allocation (one warp) ---------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                   smem_u32(smem_dst)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
}
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::);
}

// ---- MMA: D[tmem] (+)= A[smem] * B[smem]^T, issued by one thread -----------
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// kind::f16 MMA (BF16 operands per the instruction descriptor), FP32 accumulate
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// arrive on an mbarrier when all previously issued MMAs of this thread complete
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(mbar)));
}

// ---- mbarrier -------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(mbar)), "r"(parity));
  return ok != 0;
}
// Bounded wait: returns false after max_tries unsuccessful polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t max_tries) {
  for (uint32_t t = 0; t < max_tries; ++t)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

// arrive on an mbarrier and announce `bytes` of incoming TMA traffic
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(mbar)),
               "r"(bytes)
               : "memory");
}

// ---- TMA: 3-D tiled bulk copy global -> shared, completion on an mbarrier --
__device__ __forceinline__ void tma_load_3d(void* smem_dst, const void* tmap, int c0, int c1,
                                            int c2, uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3, %4}], [%5];\n" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(mbar))
      : "memory");
}

// ---- 1-D bulk copy global -> shared (16-byte aligned, size % 16 == 0) -----
__device__ __forceinline__ void bulk_load(void* smem_dst, const void* gsrc, uint32_t bytes,
                                          uint64_t* mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
          "r"(smem_u32(smem_dst)),
      "l"(gsrc), "r"(bytes), "r"(smem_u32(mbar))
      : "memory");
}

// ---- TMEM -> registers: 32 lanes x 16 consecutive 32-bit columns ----------
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- TMEM -> registers: 16 lanes x 64 columns (tcgen05.ld 16x256b, x8) ----
// Register 4r + j of thread t holds lane base + t/4 + 8 (j/2), column
// 8r + 2 (t%4) + (j%2): four consecutive threads cover 8 consecutive
// columns of one lane, the layout of an MMA accumulator fragment.
__device__ __forceinline__ void tmem_ld_16x256b_x8(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// the same fragment for 32 columns (x4: registers 4r + j, r = 0..3)
__device__ __forceinline__ void tmem_ld_16x256b_x4(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x4.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// TF32 split: hi = round-to-nearest TF32 of x, lo = x - hi (exact in FP32).
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  lo = x - hi;
}

// ---- FP32 operands as sums of lower-precision pieces ----------------------
// An FP32 operand x is split into pieces whose sum is x to the split's
// accuracy, and a product of two operands is the sum of the piece products
// that matter at FP32 level:
//   TF32x3: x = hi + lo (hi = TF32 rounding, lo the exact remainder, read by
//           the tensor core as TF32): hi.hi + hi.lo + lo.hi;
//   BF16x3: x = p0 + p1 (BF16 roundings of x and of the remainder; about 16
//           bits): p0.q0 + p0.q1 + p1.q0;
//   BF16x6: x = p0 + p1 + p2 (about 24 bits): the six products of order at
//           most 2, p0.q0 + p0.q1 + p1.q0 + p0.q2 + p1.q1 + p2.q0.
enum { SPLIT_TF32X3 = 0, SPLIT_BF16X3 = 1, SPLIT_BF16X6 = 2 };

template <int SPLIT> struct SplitCfg;
template <> struct SplitCfg<SPLIT_TF32X3> {
  static constexpr int PIECES = 2, ESZ = 4, NPROD = 3;
};
template <> struct SplitCfg<SPLIT_BF16X3> {
  static constexpr int PIECES = 2, ESZ = 2, NPROD = 3;
};
template <> struct SplitCfg<SPLIT_BF16X6> {
  static constexpr int PIECES = 3, ESZ = 2, NPROD = 6;
};

// K-step of one MMA: 32 bytes (8 TF32 or 16 BF16 elements); a chunk of 32
// reals of K is 4 (TF32) or 2 (BF16) steps
template <int SPLIT>
__host__ __device__ constexpr int ksteps32() { return SplitCfg<SPLIT>::ESZ == 4 ? 4 : 2; }

// Byte offset of real element (row, k), k a multiple of 4, in a K-major
// core-matrix tile holding 32 reals of K per row (8-row x 16-byte core
// matrices, LBO = 128 bytes along K, SBO = 8 core matrices (TF32) or 4
// (BF16) between 8-row groups).
template <int SPLIT>
__host__ __device__ constexpr uint32_t sbo32() {
  return (uint32_t)(32 * SplitCfg<SPLIT>::ESZ / 16) * 128u;
}
template <int SPLIT>
__device__ __forceinline__ uint32_t kmajor_off32(int row, int k) {
  constexpr int ESZ = SplitCfg<SPLIT>::ESZ;
  constexpr int EPC = 16 / ESZ;  // elements per 16-byte core row
  return (uint32_t)(row >> 3) * sbo32<SPLIT>() + (uint32_t)(k / EPC) * 128u +
         (uint32_t)(row & 7) * 16u + (uint32_t)(k % EPC) * ESZ;
}

// Split 4 consecutive reals of one row and store them as one 16-byte
// (TF32) or 8-byte (BF16) unit per piece at byte offset off of each piece.
template <int SPLIT>
__device__ __forceinline__ void store_split(float4 v, unsigned char* const* piece, uint32_t off) {
  if constexpr (SPLIT == SPLIT_TF32X3) {
    float4 h, l;
    split_tf32(v.x, h.x, l.x);
    split_tf32(v.y, h.y, l.y);
    split_tf32(v.z, h.z, l.z);
    split_tf32(v.w, h.w, l.w);
    *reinterpret_cast<float4*>(piece[0] + off) = h;
    *reinterpret_cast<float4*>(piece[1] + off) = l;
  } else {
    float r[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int p = 0; p < SplitCfg<SPLIT>::PIECES; ++p) {
      __nv_bfloat162 lo2 = __floats2bfloat162_rn(r[0], r[1]);
      __nv_bfloat162 hi2 = __floats2bfloat162_rn(r[2], r[3]);
      uint2 u;
      u.x = *reinterpret_cast<uint32_t*>(&lo2);
      u.y = *reinterpret_cast<uint32_t*>(&hi2);
      *reinterpret_cast<uint2*>(piece[p] + off) = u;
      const float2 f0 = __bfloat1622float2(lo2), f1 = __bfloat1622float2(hi2);
      r[0] -= f0.x;
      r[1] -= f0.y;
      r[2] -= f1.x;
      r[3] -= f1.y;
    }
  }
}

}  // namespace tc
