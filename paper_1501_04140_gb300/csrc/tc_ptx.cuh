// tc_ptx.cuh -- inline-PTX wrappers for the sm_103a tensor path: mbarriers,
// bulk (TMA-engine) copies, tensor-memory allocation and loads, and the
// tcgen05 MMA.  Every wait is bounded; a wait that runs out returns false and
// the caller records FIC_ETIMEOUT in the device status word.
#pragma once

#include <stdint.h>

#include "fic_common.cuh"

namespace fic {
namespace ptx {

__device__ inline uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ inline void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ inline void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ inline uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on the phase of the given parity: false after kWaitLimitNs.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63 && global_ns() - t0 > kWaitLimitNs) return false;
  }
}

// Non-blocking probe of the phase of the given parity.
__device__ inline bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking probe of two phases in one shared-memory round trip: true when
// both have completed.
__device__ inline bool mbar_test_wait2(uint64_t* bar0, uint32_t parity0, uint64_t* bar1,
                                       uint32_t parity1) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 q, [%3], %4;\n\t"
      "and.pred p, p, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar0)), "r"(parity0), "r"(smem_u32(bar1)), "r"(parity1)
      : "memory");
  return ok != 0;
}

// Bounded wait by spinning on test_wait (the thread never suspends): for the
// single-thread producer and MMA issuer, whose wake-up latency sits on the
// pipeline's critical path.
__device__ inline bool mbar_spin(uint64_t* bar, uint32_t parity) {
  if (mbar_test_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_test_wait(bar, parity)) return true;
    if ((i & 255) == 255 && global_ns() - t0 > kWaitLimitNs) return false;
  }
}

// mbar_spin that also gives up once `abort` is set; the flag is read only
// while the phase is still pending, so a wait that is already satisfied costs
// one round trip.
__device__ inline bool mbar_spin_abort(uint64_t* bar, uint32_t parity, const volatile int* abort) {
  if (mbar_test_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 0;; ++i) {
    if (mbar_test_wait(bar, parity)) return true;
    if ((i & 255) == 255 && (*abort || global_ns() - t0 > kWaitLimitNs)) return false;
  }
}

// 1-D bulk copy global -> shared through the TMA engine; completes `bytes`
// of the barrier's transaction count.  Addresses 16-byte aligned, size a
// multiple of 16.
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------- tensor memory
__device__ inline void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}
__device__ inline void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ inline void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ inline void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of
// 8 rows x 16 bytes; `lbo` = byte step between core matrices along K,
// `sbo` = byte step between 8-row groups.
__device__ inline uint64_t smem_desc(const void* base, uint32_t lbo, uint32_t sbo) {
  const uint64_t a = smem_u32(base);
  uint64_t d = 0;
  d |= (a >> 4) & 0x3FFFull;
  d |= ((uint64_t)((lbo >> 4) & 0x3FFF)) << 16;
  d |= ((uint64_t)((sbo >> 4) & 0x3FFF)) << 32;
  d |= 1ull << 46;  // descriptor version of the tcgen05 family
  return d;         // base offset 0, no swizzle
}

// Instruction descriptor of kind::f16: f16 A and B (K-major), f32 D.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
  return (1u << 4)                        // D format: f32
         | (0u << 7) | (0u << 10)         // A, B: f16
         | ((uint32_t)(N >> 3) << 17)     // N / 8
         | ((uint32_t)(M >> 4) << 24);    // M / 16
}

__device__ inline void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                               uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on `bar` once every tcgen05 op issued so far by this thread is done.
__device__ inline void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 8 consecutive 32-bit columns of this warp's 32 TMEM lanes as floats,
// loaded and waited for in one statement.
__device__ inline void tmem_ld8_wait(uint32_t taddr, float (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7])
      : "r"(taddr)
      : "memory");
}

// The maxima of 8 groups of 8 consecutive f32 columns (64 columns from
// taddr) of this warp's 32 TMEM lanes: m[j] = max of columns 8j .. 8j+7.
// Reducing loads (tcgen05.ld.red, sm_103a): the load path takes the maximum;
// each load also returns its 8 columns, which are not used.  The wait names
// the maxima as operands so that no use is scheduled before it.
__device__ inline void tmem_ldmax8x8_wait(uint32_t taddr, float (&m)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float v0, v1, v2, v3, v4, v5, v6, v7;
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x8.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, %8, [%9];"
        : "=f"(v0), "=f"(v1), "=f"(v2), "=f"(v3), "=f"(v4), "=f"(v5), "=f"(v6), "=f"(v7),
          "=f"(m[j])
        : "r"(taddr + 8 * j)
        : "memory");
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(m[0]), "+f"(m[1]), "+f"(m[2]), "+f"(m[3]), "+f"(m[4]), "+f"(m[5]),
                 "+f"(m[6]), "+f"(m[7])
               :
               : "memory");
}

// 32 consecutive f32 columns of this warp's 32 TMEM lanes as 4 groups of 8,
// with each group's maximum: reducing loads (tcgen05.ld.red, sm_103a).  The
// registers are valid only after tmem_wait_red().
__device__ inline void tmem_ldred32(uint32_t taddr, float (&v)[32], float (&m)[4]) {
#pragma unroll
  for (int g = 0; g < 4; ++g)
    asm volatile(
        "tcgen05.ld.red.sync.aligned.32x32b.x8.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, %8, [%9];"
        : "=f"(v[8 * g + 0]), "=f"(v[8 * g + 1]), "=f"(v[8 * g + 2]), "=f"(v[8 * g + 3]), "=f"(v[8 * g + 4]), "=f"(v[8 * g + 5]), "=f"(v[8 * g + 6]), "=f"(v[8 * g + 7]),
          "=f"(m[g])
        : "r"(taddr + 8 * g)
        : "memory");
}
__device__ inline void tmem_wait_red(float (&v)[32], float (&m)[4]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]), "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]), "+f"(v[15]), "+f"(v[16]), "+f"(v[17]), "+f"(v[18]), "+f"(v[19]), "+f"(v[20]), "+f"(v[21]), "+f"(v[22]), "+f"(v[23]), "+f"(v[24]), "+f"(v[25]), "+f"(v[26]), "+f"(v[27]), "+f"(v[28]), "+f"(v[29]), "+f"(v[30]), "+f"(v[31]),
                 "+f"(m[0]), "+f"(m[1]), "+f"(m[2]), "+f"(m[3])
               :
               : "memory");
}

// Named barrier over `count` threads (ids 1..15; 0 is __syncthreads).
__device__ inline void named_bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}


// Warpgroup register budget (all four warps of the warpgroup execute it).
// The increments of some warpgroups must be paid for by decrements of others:
// the block's total stays the registers it was launched with.
template <int N>
__device__ inline void setmaxnreg_inc() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(N));
}
template <int N>
__device__ inline void setmaxnreg_dec() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(N));
}

// Three-input minimum (sm_100 family).
__device__ inline float fmin3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Three-input maximum (sm_100 family).
__device__ inline float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

}  // namespace ptx
}  // namespace fic
