// Device helpers shared by the tcgen05 kernels: mbarriers with %globaltimer-bounded
// waits, 3-D TMA loads, shared-memory matrix descriptors (K-major, 64-byte rows, 64-byte
// swizzle), TF32 MMA issue / commit, TMEM loads, and the TF32 hi/lo split.
#pragma once

#include <cstdint>

#include "f32conv.cuh"

namespace tnt {
namespace tc {

constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok;
}
// bounded wait; false (and the status bit set) if the phase never completed
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* status) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_try(b, parity)) {
    if (gtimer() - t0 > WAIT_NS) {
      atomicOr(status, 1);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* tm, uint64_t* bar, int c0,
                                          int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(su32(dst)),
      "l"((uint64_t)tm), "r"(su32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}
// K-major operand tile, 64-byte rows, 64-byte swizzle: 8-row atoms of 512 bytes
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused here)
  d |= (uint64_t)((512u >> 4) & 0x3FFFu) << 32;  // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)4 << 61;                        // swizzle: 64 B
  return d;
}
// instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_tf32_n(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t id,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}


__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void split_tf32(float x, float* hi, float* lo) {
  const float h = tf32_rna(x);
  *hi = h;
  *lo = tf32_rna(x - h);
}
// An FP64 value is first truncated to FP32 by integer operations (f32conv.cuh; 2^-23
// relative), then split: hi + lo is within ~1.5 2^-22 of x, the split-TF32 products' own
// error, and no FP64-pipe conversion or subtraction enters the operand conversion kernels
__device__ __forceinline__ void split_tf32(double x, float* hi, float* lo) {
  split_tf32(f32_of(x), hi, lo);
}


}  // namespace tc
}  // namespace tnt
