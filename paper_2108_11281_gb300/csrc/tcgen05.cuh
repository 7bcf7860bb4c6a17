// Inline-PTX helpers for the 5th-generation tensor cores (tcgen05) shared by
// the kernels that use them: shared-memory matrix descriptors in the K-major,
// no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix), the
// kind::tf32 instruction descriptor, TF32 rounding, bounded mbarrier waits,
// the MMA and its commit.  Not part of the C ABI.
#pragma once
#include <cstdint>

namespace mlmc {
namespace tc {

__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading byte offset (between
// core matrices adjacent along K), stride byte offset (between 8-row groups),
// fixed version field 1, no swizzle.
__device__ inline uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D in F32, A and B TF32, both K-major, M x N.
__device__ inline uint32_t tf32_idesc(int m, int n) {
  uint32_t d = 0;
  d |= 1u << 4;                        // D format: F32
  d |= 2u << 7;                        // A format: TF32
  d |= 2u << 10;                       // B format: TF32
  d |= (uint32_t)(n >> 3) << 17;       // N / 8
  d |= (uint32_t)(m >> 4) << 24;       // M / 16
  return d;
}

__device__ inline float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// x = hi + lo with hi a TF32 value: three TF32 products (hi hi, hi lo, lo hi)
// then carry a product at FP32 accuracy.
__device__ inline void split_store(unsigned char *hi, unsigned char *lo, uint32_t off, float4 v) {
  float4 h = make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
  *(float4 *)(hi + off) = h;
  *(float4 *)(lo + off) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
}

__device__ inline void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Non-blocking test of phase `parity`, polled for at most `limit` SM cycles.
__device__ inline bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
    if (it > 64) __nanosleep(64);
  }
}

__device__ inline void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// Three TF32 products per term (A_hi B_hi + A_hi B_lo + A_lo B_hi): FP32 accuracy.
__device__ inline void mma_tf32x3(uint32_t tmem_d, uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl, uint32_t idesc,
                                  uint32_t acc) {
  mma_tf32(tmem_d, ah, bh, idesc, acc);
  mma_tf32(tmem_d, ah, bl, idesc, 1u);
  mma_tf32(tmem_d, al, bh, idesc, 1u);
}

__device__ inline void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ inline void tmem_alloc(uint32_t *dst_smem, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ inline void tmem_dealloc(uint32_t tmem, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

// 8 consecutive 32-bit accumulator columns of the calling warp's 32 TMEM lanes.
__device__ inline void tmem_ld8(uint32_t taddr, float out[8]) {
  uint32_t v[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int u = 0; u < 8; ++u) out[u] = __uint_as_float(v[u]);
}

}  // namespace tc
}  // namespace mlmc
