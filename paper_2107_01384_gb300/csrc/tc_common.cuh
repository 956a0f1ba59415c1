// Inline-PTX helpers for the sm_103a tensor-core kernels: mbarriers with
// bounded waits, 5th-generation tensor core MMA (tcgen05) with TMEM
// accumulators, shared-memory matrix descriptors and TMA tensor copies.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace atc {
namespace tc {

// Time limit of any wait inside a tensor-core kernel (ns of %globaltimer).
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ------------------------------------------------------------------ mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// The same test with a suspend-time hint: a thread whose phase is not
// complete sleeps (up to `ns` nanoseconds, or until the phase completes)
// instead of spinning, leaving the issue slots to the working warps.
__device__ __forceinline__ bool mbar_try_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
constexpr uint32_t kWaitSleepNs = 20000;  // 20 us per suspended try

// Wait for the phase of parity `parity` to complete; gives up after the time
// limit or when *abort becomes non-zero.  Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (mbar_try_sleep(bar, parity, kWaitSleepNs)) return true;
    if (*abort) return false;
    if (globaltimer() - t0 > kWaitLimitNs) {
      *abort = 1;
      return false;
    }
  }
}

// Time-bounded wait that ignores the abort flag (used to drain in-flight work
// before freeing TMEM or leaving the CTA).
__device__ __forceinline__ bool mbar_wait_drain(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (mbar_try_sleep(bar, parity, kWaitSleepNs)) return true;
    if (globaltimer() - t0 > kWaitLimitNs) return false;
  }
}

// Make generic-proxy shared-memory writes visible to the async proxy (tensor core, TMA).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ------------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (bf16 or fp16 inputs, FP32 accumulate)
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive once on `bar` when every previously issued MMA of this thread has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 16 consecutive 32-bit columns (this warp's lane quarter).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes (64 16-bit elements), 8-row groups 1024 bytes apart.  The tile
// base must be 1024-byte aligned; a K step of 16 elements inside the swizzle
// atom advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t desc_k128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);       // start address
  d |= (uint64_t)1u << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;              // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1u << 46;                        // descriptor version (sm_100 family)
  d |= (uint64_t)2u << 61;                        // layout: 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, A/B both K-major.
// fmt: 0 = fp16, 1 = bf16.  M in {64, 128}, N a multiple of 16 in [16, 256].
__host__ __device__ constexpr uint32_t idesc_f16(int fmt, int M, int N) {
  return (1u << 4)                       // D format: F32
         | ((uint32_t)fmt << 7)          // A format
         | ((uint32_t)fmt << 10)         // B format
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// Byte offset of element (row r, k) inside a K-major 128-byte-swizzled tile of
// 16-bit elements (64 per row): the 16-byte chunk index is XORed with r mod 8.
__device__ __forceinline__ uint32_t sw128_off(uint32_t r, uint32_t k) {
  return r * 128u + ((((k >> 3) ^ (r & 7u)) & 7u) << 4) + ((k & 7u) << 1);
}

// ----------------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
          "r"(smem_u32(smem_dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* smem_dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(smem_dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Fixed-point slices (error-free splitting in the manner of Ozaki et al.,
// as used for tensor-core GEMMs by Mukunoki et al., ICCS 2020).  With one
// power-of-two scale per operand, v = x * 2^shift and |v| < 256:
//   v ~ a0 + a1 2^-8 + a2 2^-16,  a0, a1, a2 integers, |a0| <= 256, |a1|, |a2| <= 128
// (round to nearest at each step, so |v - ...| <= 2^-17).  Every slice is an
// integer exact in bf16 and fp16, every product of two slices is exact, and
// a sum of such products is exact in FP32 while its magnitude stays below 2^24:
// the tensor-core FP32 accumulation then performs no rounding at all, whatever
// its internal rounding mode.  The products are grouped by order s + t (the
// scale 2^-8(s+t)) into five accumulators and combined outside the tensor core.
// Round to the nearest integer, ties to even, for |v| < 2^22: adding 1.5 2^23
// moves v into [2^23, 2^24), where the float spacing is 1, so the addition
// itself rounds (round-to-nearest-even); subtracting the constant is exact.
// Two FP32 additions on the full-rate pipe (the _rn intrinsics keep the
// compiler from contracting or reassociating them).
__device__ __forceinline__ float rint_small(float v) {
  return __fsub_rn(__fadd_rn(v, 12582912.0f), 12582912.0f);
}

__device__ __forceinline__ void slice3i(float v, float& a0, float& a1, float& a2) {
  a0 = rint_small(v);
  const float t = (v - a0) * 256.0f;  // exact
  a1 = rint_small(t);
  a2 = rint_small((t - a1) * 256.0f);
}

// Four slices (32-bit fixed point): v ~ a0 + a1 2^-8 + a2 2^-16 + a3 2^-24,
// |a0| <= 256, |a1|, |a2|, |a3| <= 128, |v - ...| <= 2^-25.  The products of
// order s + t >= 5 (scale <= 2^-40) are left out by the Gram kernels: they are
// below the rounding of v itself.
__device__ __forceinline__ void slice4i(float v, float& a0, float& a1, float& a2, float& a3) {
  a0 = rint_small(v);
  const float t = (v - a0) * 256.0f;  // exact
  a1 = rint_small(t);
  const float t2 = (t - a1) * 256.0f;  // exact
  a2 = rint_small(t2);
  a3 = rint_small((t2 - a2) * 256.0f);
}

// acc0 + 2^-8 acc1 + 2^-16 acc2 + 2^-24 acc3 + 2^-32 acc4 as an unevaluated
// sum s + t (s carries the leading 24 bits; the exact orders 0 and 1 enter
// through an error-free two-sum, the rest with round-to-nearest)
__device__ __forceinline__ void combine_orders(float c0, float c1, float c2, float c3, float c4, float& s, float& t) {
  const float b = c1 * 0.00390625f;
  s = c0 + b;
  const float bp = s - c0;
  const float e = (c0 - (s - bp)) + (b - bp);
  t = e + fmaf(c2, 1.52587890625e-05f, fmaf(c3, 5.9604644775390625e-08f, c4 * 2.3283064365386963e-10f));
}

// 16-bit images of slice integers (|a| <= 256, exact in bf16 and fp16).  For
// bf16 the image is the upper half of the float's bits (an integer of at most
// 8 significant bits leaves the lower 16 bits zero): one byte permute packs two.
template <bool BF16>
struct Pack;
template <>
struct Pack<true> {
  static __device__ __forceinline__ uint32_t two(float a, float b) {
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
  }
  static __device__ __forceinline__ uint16_t one(float a) { return (uint16_t)(__float_as_uint(a) >> 16); }
};
template <>
struct Pack<false> {
  static __device__ __forceinline__ uint32_t two(float a, float b) {
    return (uint32_t)__half_as_ushort(__float2half_rn(a)) | ((uint32_t)__half_as_ushort(__float2half_rn(b)) << 16);
  }
  static __device__ __forceinline__ uint16_t one(float a) { return __half_as_ushort(__float2half_rn(a)); }
};

// error-free sum of two floats: s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

}  // namespace tc

// Host: TMA map over FP32 data (k_gram_tc.cu): `rank` dimensions innermost
// first, strides[d - 1] = bytes between consecutive indices of dimension d,
// box extents per dimension, no swizzle, zero fill out of range.
int make_raw_map_f32(CUtensorMap* m, const void* base, int rank, const int64_t* dims, const int64_t* strides,
                     const uint32_t* box);
}  // namespace atc
