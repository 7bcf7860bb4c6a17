// Coarsest-level dense apply Y = A_L^-1 B on the 5th-generation tensor cores.
//
// The coarsest solve inside the FP32 cycle (Sec. 4: the coarsest system is
// solved directly) is a dense matrix times a block of k vectors, a real
// contraction, so it runs as a tcgen05 GEMM in FP32 accuracy:
//
//   real:    Y[n][k] = A[n][n] B[n][k]
//   complex: the same with A, B, Y complex interleaved.  With A viewed as a
//            real n x 2n matrix (re, im interleaved along j) the product is the
//            real GEMM  Yf[n][2k] = Af[n][2n] B'[2n][2k]  where row 2j of B' is
//            (re, im) of B[j] and row 2j+1 is (-im, re): then
//            Re y = Ar Br - Ai Bi and Im y = Ar Bi + Ai Br.
//
// One CTA of 128 threads owns a 128-row by `ntile`-column tile of Y and a
// slice of the contraction (K) range; its accumulator lives in tensor memory.
// Per 32-wide K step the CTA stages A[128 x 32] and B^T[ntile x 32] into
// shared memory in the K-major, no-swizzle core-matrix layout (8 rows x 16 B
// per core matrix), splitting every value into a TF32 head and an FP32 tail
// (x = hi + lo).  One elected thread issues tcgen05.mma.kind::tf32
// (M = 128, N = ntile, K = 8) three times per 8-wide sub-step,
// A_hi B_hi + A_hi B_lo + A_lo B_hi, which keeps the product at FP32 accuracy,
// and commits to the stage's mbarrier.  Two stages alternate, so the loads of
// step t+1 overlap the MMAs of step t.  The epilogue reads the accumulator
// with tcgen05.ld and writes Y (one K slice) or a partial tile that
// k_dense_sum_tc adds up in slice order.
//
// Every wait on an mbarrier is bounded (about a second): when a bound is hit
// the CTA records MLMC_ERR_TIMEOUT in *err, waits (bounded) for its own MMAs,
// releases its tensor memory and returns without writing its tile.  The
// `withhold` launch mode (tests of that path) issues no MMA and no commit, so
// the first wait runs out after `wait_cycles` with nothing in flight.
#include <cstdint>
#include <mutex>

#include "mlmc.h"
#include "mlmc_internal.cuh"
#include "tcgen05.cuh"

namespace mlmc {

namespace {

constexpr int TC_M = 128;             // rows per tile (TMEM lanes)
constexpr int TC_BK = 32;             // K elements per stage (4 MMAs of K = 8)
constexpr int TC_NT = 128;            // max columns per tile
constexpr int TC_THREADS = 128;
constexpr long long TC_WAIT_CYCLES = 2000000000LL;   // ~1 s at 2 GHz
constexpr long long TC_TEST_WAIT_CYCLES = 2000000LL;  // ~1 ms: the withheld-commit test mode

constexpr int A_BYTES = TC_M * TC_BK * 4;            // one A half (hi or lo), 16 KB
__host__ __device__ constexpr int b_bytes(int ntile) { return ntile * TC_BK * 4; }
constexpr size_t stage_smem(int ntile) { return (size_t)2 * (2 * A_BYTES + 2 * b_bytes(ntile)); }

using tc::mbar_init;
using tc::mbar_wait_bounded;
using tc::mma_commit;
using tc::mma_tf32;
using tc::smem_desc;
using tc::smem_u32;
using tc::split_store;

__device__ inline uint32_t tf32_idesc(int n) { return tc::tf32_idesc(TC_M, n); }

}  // namespace

// grid: (row tiles, column tiles, K slices).  Af: rows of `lda` floats; Bf and
// Y / partials: rows of `nf` floats.  kdim: the real contraction length (n or
// 2n); jchunk: K per slice (a multiple of TC_BK).
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_dense_apply_tc(const float *__restrict__ Af, const float *__restrict__ Bf, float *__restrict__ Y, int n,
                     int kdim, int lda, int nf, int ntile, int jchunk, int tmem_cols, int cplx, int withhold,
                     long long wait_cycles, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * TC_M, col0 = blockIdx.y * ntile;
  const int j_begin = blockIdx.z * jchunk, j_end = min(kdim, j_begin + jchunk);
  const int nsteps = j_end > j_begin ? (j_end - j_begin + TC_BK - 1) / TC_BK : 0;
  const int bb = b_bytes(ntile);
  const int sbytes = 2 * A_BYTES + 2 * bb;
  const bool avec = (lda % 4) == 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tf32_idesc(ntile);
  constexpr uint32_t LBO = 128, SBO = (TC_BK / 4) * 128;

  // One stage's tiles pass through registers: every thread first issues all its
  // global loads (A: 8 float4; B^T: up to 8 (column, K quad) pairs of 4 scalars),
  // and the loads of step t+1 are in flight while the MMAs of step t run.
  constexpr int A_IT = TC_M * TC_BK / 4 / TC_THREADS;
  constexpr int B_IT = TC_NT * (TC_BK / 4) / TC_THREADS;
  float4 ra[A_IT];
  float rb[B_IT][4];
  auto load_stage = [&](int t) {
    const int j0 = j_begin + t * TC_BK;
    // A tile: float4 e4 -> row (e4>>6)*8 + (e4&7), K quad (e4>>3)&7; its core-matrix
    // offset is exactly 16*e4, so the 16-byte shared stores are dense.
#pragma unroll
    for (int it = 0; it < A_IT; ++it) {
      const int e4 = tid + it * TC_THREADS;
      const int r = ((e4 >> 6) << 3) | (e4 & 7), kq = (e4 >> 3) & 7;
      const int gi = row0 + r, gj = j0 + 4 * kq;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gi < n) {
        const float *src = Af + (size_t)gi * lda + gj;
        if (avec && gj + 4 <= j_end) {
          v = __ldg((const float4 *)src);
        } else {
          if (gj + 0 < j_end) v.x = __ldg(src + 0);
          if (gj + 1 < j_end) v.y = __ldg(src + 1);
          if (gj + 2 < j_end) v.z = __ldg(src + 2);
          if (gj + 3 < j_end) v.w = __ldg(src + 3);
        }
      }
      ra[it] = v;
    }
    // B^T tile: (column c, K quad kq) with c fastest; four K rows per pair.
#pragma unroll
    for (int it = 0; it < B_IT; ++it) {
      const int e = tid + it * TC_THREADS;
      const int c = e % ntile, kq = e / ntile;
      const int gc = col0 + c;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int gj = j0 + 4 * kq + u;
        float x = 0.f;
        if (e < ntile * (TC_BK / 4) && gj < j_end && gc < nf) {
          if (!cplx) {
            x = __ldg(Bf + (size_t)gj * nf + gc);
          } else {
            const float *row = Bf + (size_t)(gj >> 1) * nf;
            if ((gj & 1) == 0) x = __ldg(row + gc);
            else x = (gc & 1) ? __ldg(row + gc - 1) : -__ldg(row + gc + 1);
          }
        }
        rb[it][u] = x;
      }
    }
  };
  auto store_stage = [&](unsigned char *Ahi, unsigned char *Alo, unsigned char *Bhi, unsigned char *Blo) {
#pragma unroll
    for (int it = 0; it < A_IT; ++it) split_store(Ahi, Alo, (uint32_t)(tid + it * TC_THREADS) * 16, ra[it]);
#pragma unroll
    for (int it = 0; it < B_IT; ++it) {
      const int e = tid + it * TC_THREADS;
      if (e >= ntile * (TC_BK / 4)) break;
      const int c = e % ntile, kq = e / ntile;
      const uint32_t off = (uint32_t)((((c >> 3) * (TC_BK / 4) + kq) << 7) + ((c & 7) << 4));
      split_store(Bhi, Blo, off, make_float4(rb[it][0], rb[it][1], rb[it][2], rb[it][3]));
    }
  };

  int issued = 0;      // K steps whose MMAs were committed (uniform over the CTA)
  if (nsteps > 0) load_stage(0);
  for (int t = 0; t < nsteps; ++t) {
    const int buf = t & 1;
    unsigned char *Ahi = smem + buf * sbytes, *Alo = Ahi + A_BYTES;
    unsigned char *Bhi = Ahi + 2 * A_BYTES, *Blo = Bhi + bb;
    if (t >= 2) {
      // the MMAs of step t-2 read this stage: one thread waits for their commit, the
      // others sleep in the barrier
      if (tid == 0 && !mbar_wait_bounded(&bars[buf], (uint32_t)(((t >> 1) - 1) & 1), wait_cycles)) failed = 1;
      __syncthreads();
      if (failed) break;
    }
    store_stage(Ahi, Alo, Bhi, Blo);
    // generic-proxy stores -> visible to the tensor core's async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0 && !withhold) {
      const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
      for (int s = 0; s < TC_BK / 8; ++s) {
        const uint32_t step = (uint32_t)s * 2 * LBO;     // K = 8 TF32 = two core matrices
        const uint64_t dah = smem_desc(ah + step, LBO, SBO), dal = smem_desc(al + step, LBO, SBO);
        const uint64_t dbh = smem_desc(bh + step, LBO, SBO), dbl = smem_desc(bl + step, LBO, SBO);
        mma_tf32(tmem, dah, dbh, idesc, (t > 0 || s > 0) ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, idesc, 1u);
        mma_tf32(tmem, dal, dbh, idesc, 1u);
      }
      mma_commit(&bars[buf]);
    }
    issued = t + 1;
    if (t + 1 < nsteps) load_stage(t + 1);
  }

  // drain: the last commit of each stage that nobody waited for yet
  if (issued > 0 && tid == 0) {
    const int tl = issued - 1;
    bool ok = true;
    if (!failed) {
      ok = mbar_wait_bounded(&bars[tl & 1], (uint32_t)((tl >> 1) & 1), wait_cycles);
      if (tl >= 1) ok = mbar_wait_bounded(&bars[(tl - 1) & 1], (uint32_t)(((tl - 1) >> 1) & 1), wait_cycles) && ok;
    } else {
      // a wait already failed: give the MMAs in flight one more bounded chance
      mbar_wait_bounded(&bars[tl & 1], (uint32_t)((tl >> 1) & 1), wait_cycles);
    }
    if (!ok) failed = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");

  if (!failed) {
    float *Yz = Y + (size_t)blockIdx.z * n * nf;
    const int r = row0 + warp * 32 + lane;
    for (int c0 = 0; c0 < ntile; c0 += 16) {
      uint32_t v[16];
      if (issued > 0) {
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
              "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = 0u;
      }
      const int gc = col0 + c0;
      if (r < n && gc < nf) {
        float *dst = Yz + (size_t)r * nf + gc;
        if (gc + 16 <= nf && (nf % 4) == 0) {
#pragma unroll
          for (int u = 0; u < 16; u += 4)
            *(float4 *)(dst + u) = make_float4(__uint_as_float(v[u]), __uint_as_float(v[u + 1]),
                                               __uint_as_float(v[u + 2]), __uint_as_float(v[u + 3]));
        } else {
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (gc + u < nf) dst[u] = __uint_as_float(v[u]);
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, (int)MLMC_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
  }
}

// Y = sum of the K-slice partials, added in slice order (deterministic).
__global__ void k_dense_sum_tc(const float *__restrict__ part, int slices, size_t count, float *__restrict__ Y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    float s = part[i];
    for (int z = 1; z < slices; ++z) s += part[(size_t)z * count + i];
    Y[i] = s;
  }
}

namespace {

struct TcPlan {
  int kdim, lda, nf, ntile, rtiles, ctiles, slices, jchunk, tmem_cols;
  size_t smem;
};

TcPlan plan_tc(DType t, int n, int k) {
  TcPlan p{};
  const int cplx = t == C32;
  p.kdim = cplx ? 2 * n : n;
  p.lda = p.kdim;
  p.nf = cplx ? 2 * k : k;
  const int nf16 = (p.nf + 15) / 16 * 16;
  p.ntile = nf16 < TC_NT ? nf16 : TC_NT;
  p.rtiles = (n + TC_M - 1) / TC_M;
  p.ctiles = (p.nf + p.ntile - 1) / p.ntile;
  const int tiles = p.rtiles * p.ctiles;
  int want = 152 / (tiles > 0 ? tiles : 1);
  const int most = (p.kdim + 2 * TC_BK - 1) / (2 * TC_BK);     // at least two K steps per slice
  if (want > most) want = most;
  if (want > 16) want = 16;
  if (want < 1) want = 1;
  p.jchunk = (p.kdim + want - 1) / want;
  p.jchunk = (p.jchunk + TC_BK - 1) / TC_BK * TC_BK;
  p.slices = (p.kdim + p.jchunk - 1) / p.jchunk;                 // every slice non-empty
  p.tmem_cols = 32;
  while (p.tmem_cols < p.ntile) p.tmem_cols <<= 1;
  p.smem = stage_smem(p.ntile);
  return p;
}

std::once_flag g_tc_attr_once[64];

}  // namespace

bool dense_apply_tc_ok(DType t, int n, int k) { return (t == F32 || t == C32) && n >= 1 && k >= 1; }

size_t dense_apply_tc_part_bytes(DType t, int n, int k) {
  if (!dense_apply_tc_ok(t, n, k)) return 0;
  TcPlan p = plan_tc(t, n, k);
  return p.slices > 1 ? (size_t)p.slices * n * p.nf * sizeof(float) : 0;
}

void launch_dense_apply_tc(DType t, const void *Ainv, const void *B, void *Y, int n, int k, void *part,
                           size_t part_bytes, int *err, cudaStream_t s, int withhold) {
  if (!dense_apply_tc_ok(t, n, k)) throw cuda_error{cudaErrorInvalidValue, "k_dense_apply_tc: unsupported type"};
  TcPlan p = plan_tc(t, n, k);
  if (p.slices > 1 && (part == nullptr || part_bytes < (size_t)p.slices * n * p.nf * sizeof(float)))
    throw cuda_error{cudaErrorInvalidValue, "k_dense_apply_tc: partial scratch too small"};
  if ((((uintptr_t)Ainv) | ((uintptr_t)B) | ((uintptr_t)Y) | ((uintptr_t)part)) & 15)
    throw cuda_error{cudaErrorInvalidValue, "k_dense_apply_tc: pointers must be 16-byte aligned"};
  int dev = 0;
  MLMC_CUDA(cudaGetDevice(&dev));
  std::call_once(g_tc_attr_once[dev & 63], [] {
    check_cuda(cudaFuncSetAttribute(k_dense_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)stage_smem(TC_NT)),
               "cudaFuncSetAttribute(k_dense_apply_tc)");
  });
  dim3 g(p.rtiles, p.ctiles, p.slices);
  float *out = p.slices > 1 ? (float *)part : (float *)Y;
  k_dense_apply_tc<<<g, TC_THREADS, p.smem, s>>>((const float *)Ainv, (const float *)B, out, n, p.kdim, p.lda, p.nf,
                                                  p.ntile, p.jchunk, p.tmem_cols, t == C32 ? 1 : 0, withhold ? 1 : 0,
                                                  withhold ? TC_TEST_WAIT_CYCLES : TC_WAIT_CYCLES, err);
  if (p.slices > 1) {
    size_t cnt = (size_t)n * p.nf;
    k_dense_sum_tc<<<grid_for(cnt, 256), 256, 0, s>>>((const float *)part, p.slices, cnt, (float *)Y);
  }
  MLMC_LAUNCH_CHECK("k_dense_apply_tc");
}

}  // namespace mlmc
