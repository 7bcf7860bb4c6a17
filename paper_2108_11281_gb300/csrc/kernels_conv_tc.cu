// The learned correction's 3x3 convolutions on the 5th-generation tensor cores.
//
// Activations are FP32 blocks [site][channel][k] (k columns innermost), weights
// W[c_out][c_in][3][3] (kernels_learned.cu holds the CUDA-core versions and
// the layout conventions).  A convolution layer is a contraction over
// (tap, input channel) for every (site, column) pair, so it runs as an
// implicit GEMM with the accumulators in tensor memory:
//
// k_conv_tc (forward, and backward-data with the taps mirrored and the
// weights transposed): one CTA owns the 128 pairs of `ts` = 128 / k
// consecutive sites of one lattice row.  It stages the 3 x (ts + 2) halo sites
// of its input block once in shared memory, K-major (channels along K, padded
// to a multiple of 8 with zeros) in the no-swizzle core-matrix layout, so that
// the A operand of tap (tx, ty) is the same array started (ty (ts + 2) + tx)
// sites further on: nine descriptors into one staging, no im2col copy.  B is
// the layer's weights, [out channel (padded to 16)][tap][in channel].  One
// elected thread issues tcgen05.mma.kind::tf32 (M = 128, N = 16, K = 8) three
// times per K step (TF32 head and tail of both operands: FP32 accuracy) into six
// accumulators (three products x even / odd taps: independent chains) and commits
// to an mbarrier.  The epilogue
// reads the accumulator with tcgen05.ld (warps 0-3 columns 0-7, warps 4-7
// columns 8-15 of the same lanes), applies the ReLU (forward) or the ReLU mask
// of the layer below (backward-data) and stores the output channels.
//
// k_conv_wgrad_tc (weight gradient): grad[co][ci][tap] = sum over pairs of
// gout[s][co][c] in[nb(s, tap)][ci][c].  Rows (tap, ci) (padded to 128 or 256)
// are M, the output channels N, the pairs K: per unit of one site and up to 32
// columns both operands are 16-byte rows of the activations, staged twice
// buffered; the CTA accumulates its sites in tensor memory and writes one
// partial gradient, which k_weight_reduce adds up over the CTAs in order.
//
// Every mbarrier wait is bounded (about a second): a CTA whose wait gives up
// records MLMC_ERR_TIMEOUT in *err, waits (bounded) for its own MMAs, frees its
// tensor memory and returns without writing.
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "mlmc.h"
#include "mlmc_internal.cuh"
#include "tcgen05.cuh"

namespace mlmc {

namespace {

constexpr int CT_M = 128;                 // pairs per tile (TMEM lanes)
constexpr int CT_N = 16;                  // output channels per tile (padded)
constexpr int CT_THREADS = 256;
constexpr int WG_KC = 32;                 // columns per weight-gradient unit
constexpr long long CT_WAIT_CYCLES = 2000000000LL;   // ~1 s at 2 GHz

__host__ __device__ inline int pad8(int c) { return (c + 7) / 8 * 8; }

// site of lattice point (ii, jj), or -1 outside a Dirichlet lattice
__device__ inline int conv_site(int ii, int jj, int nx, int ny, int periodic) {
  if (periodic) {
    ii = ii < 0 ? ii + nx : (ii >= nx ? ii - nx : ii);
    jj = jj < 0 ? jj + ny : (jj >= ny ? jj - ny : jj);
    return jj * nx + ii;
  }
  if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) return -1;
  return jj * nx + ii;
}

size_t conv_tc_smem(int k, int cin) {
  const int ts = CT_M / k, cip = pad8(cin);
  const size_t halo = (size_t)3 * (ts + 2) * (k / 8) * (cip / 4) * 128;
  const size_t wb = (size_t)(CT_N / 8) * (9 * cip / 4) * 128;
  return 2 * halo + 2 * wb;
}

size_t wgrad_tc_smem(int cin, int kc) {
  const int mt = (9 * pad8(cin) + CT_M - 1) / CT_M;
  const size_t a = (size_t)mt * CT_M * kc * 4, b = (size_t)CT_N * kc * 4;
  return 2 * (2 * a + 2 * b);             // two stages, TF32 head and tail
}

}  // namespace

// Loads of one staging pass are issued in batches of STAGE_BATCH 16-byte elements per
// thread (all loads of a batch in flight before the first shared store).
constexpr int STAGE_BATCH = 8;

// out[s][n][c] for tiles of 128 pairs (see the file comment), CTAs persistent over
// the tiles.  mirror = 0: forward, B[n][tap][c] = W[n][c][tap] (W is [cout][cin][9]);
// mirror = 1: backward-data, B[n][tap][c] = W[c][n][tap] (W is [cin][cout][9]) with tap
// (tx, ty) reading the site at offset (1 - tx, 1 - ty).  act (mask, optional): out =
// acc where act[s][n][c] > 0, else 0.
// K (columns) and CIP (input channels padded to 8 or 16) are compile-time, so the
// staging index arithmetic is shifts and masks: the kernel was issue-bound on it.
template <int K, int CIP, int MIRROR>
__global__ void __launch_bounds__(CT_THREADS, 2) k_conv_tc(const float *__restrict__ in, const float *__restrict__ W,
                                                        const float *__restrict__ act, float *__restrict__ out,
                                                        int nx, int ny, int cin, int cout, int periodic,
                                                        int relu, long long wait_cycles, int *err) {
  constexpr int mirror = MIRROR;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  constexpr int k = K, cip = CIP, c4n = CIP / 4, ts = CT_M / K, kg = K / 8, hw = ts + 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiles_x = nx / ts, tiles = tiles_x * ny;
  constexpr uint32_t LBO = 128u, SBO = (uint32_t)c4n * 128u;
  constexpr uint32_t halo_bytes = (uint32_t)(3 * hw * kg) * SBO;
  constexpr uint32_t BSBO = (uint32_t)(9 * c4n) * 128u, wbytes = (uint32_t)(CT_N / 8) * BSBO;
  unsigned char *Hhi = smem, *Hlo = smem + halo_bytes;
  unsigned char *Bhi = smem + 2 * halo_bytes, *Blo = Bhi + wbytes;

  if (warp == 0) tc::tmem_alloc(&tmem_base, 128);
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // weights, once per CTA: (n, tap, channel quad), zero outside cout x cin
  for (int e = tid; e < CT_N * 9 * c4n; e += CT_THREADS) {
    const int n = e / (9 * c4n), rem = e - n * (9 * c4n), tap = rem / c4n, q = rem - tap * c4n;
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = 4 * q + u;
      v[u] = 0.f;
      if (n < cout && c < cin) v[u] = mirror ? __ldg(W + ((size_t)c * cout + n) * 9 + tap)
                                             : __ldg(W + ((size_t)n * cin + c) * 9 + tap);
    }
    const uint32_t off = (uint32_t)(n >> 3) * BSBO + (uint32_t)(tap * c4n + q) * LBO + (uint32_t)(n & 7) * 16u;
    tc::split_store(Bhi, Blo, off, make_float4(v[0], v[1], v[2], v[3]));
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tc::tf32_idesc(CT_M, CT_N);
  constexpr int nel = 3 * hw * c4n * k;        // 16-byte halo elements per tile
  const uint64_t dAh = tc::smem_desc(tc::smem_u32(Hhi), LBO, SBO), dAl = tc::smem_desc(tc::smem_u32(Hlo), LBO, SBO);
  const uint64_t dBh = tc::smem_desc(tc::smem_u32(Bhi), LBO, BSBO), dBl = tc::smem_desc(tc::smem_u32(Blo), LBO, BSBO);

  uint32_t phase = 0;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, phase ^= 1u) {
    const int j = tile / tiles_x, i0 = (tile - j * tiles_x) * ts;
    // halo: (halo site, channel quad, column), columns fastest (coalesced loads)
    for (int base = 0; base < nel; base += STAGE_BATCH * CT_THREADS) {
      float4 v[STAGE_BATCH];
#pragma unroll
      for (int b = 0; b < STAGE_BATCH; ++b) {
        const int e = base + b * CT_THREADS + tid;
        v[b] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < nel) {
          const int c = e % k, rest = e / k, q = rest % c4n, h = rest / c4n;
          const int hy = h / hw, hx = h - hy * hw;
          const int site = conv_site(i0 - 1 + hx, j - 1 + hy, nx, ny, periodic);
          if (site >= 0) {
            const float *src = in + ((size_t)site * cin + 4 * q) * k + c;
            if (4 * q + 0 < cin) v[b].x = __ldg(src);
            if (4 * q + 1 < cin) v[b].y = __ldg(src + k);
            if (4 * q + 2 < cin) v[b].z = __ldg(src + 2 * k);
            if (4 * q + 3 < cin) v[b].w = __ldg(src + 3 * k);
          }
        }
      }
#pragma unroll
      for (int b = 0; b < STAGE_BATCH; ++b) {
        const int e = base + b * CT_THREADS + tid;
        if (e < nel) {
          const int c = e % k, rest = e / k, q = rest % c4n, h = rest / c4n;
          const uint32_t off = (uint32_t)(h * kg + (c >> 3)) * SBO + (uint32_t)q * LBO + (uint32_t)(c & 7) * 16u;
          tc::split_store(Hhi, Hlo, off, v[b]);
        }
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      // six independent accumulators (product hi.hi / hi.lo / lo.hi times even / odd tap),
      // so that the MMAs do not form one dependent chain through a single accumulator.
      // Descriptors are the base descriptors plus compile-time offsets (start address / 16
      // in the low bits): the single issuing thread spends little time per MMA.
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int tx = tap % 3, ty = tap / 3;
        const int dx = mirror ? 2 - tx : tx, dy = mirror ? 2 - ty : ty;
        const uint32_t hofs = (uint32_t)((dy * hw + dx) * kg) * SBO;
        const uint32_t d0 = tmem + (uint32_t)((tap & 1) * 3 * CT_N);
#pragma unroll
        for (int ks = 0; ks < cip / 8; ++ks) {
          const uint64_t a = (hofs + (uint32_t)ks * 2u * LBO) >> 4, b = ((uint32_t)(tap * c4n + 2 * ks) * LBO) >> 4;
          const uint32_t accf = (tap > 1 || ks > 0) ? 1u : 0u;
          tc::mma_tf32(d0, dAh + a, dBh + b, idesc, accf);
          tc::mma_tf32(d0 + CT_N, dAh + a, dBl + b, idesc, accf);
          tc::mma_tf32(d0 + 2 * CT_N, dAl + a, dBh + b, idesc, accf);
        }
      }
      tc::mma_commit(&bar);
      // one thread waits for the commit; the others sleep in the barrier below
      if (!tc::mbar_wait_bounded(&bar, phase, wait_cycles)) {
        failed = 1;
        // give the MMAs in flight one more bounded chance before the memory goes
        tc::mbar_wait_bounded(&bar, phase, wait_cycles);
      }
    }
    __syncthreads();
    if (failed) break;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int m = 32 * (warp & 3) + lane, n0 = (warp >> 2) * 8;
    float acc[8], part[8];
    const uint32_t lanes = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)n0;
    tc::tmem_ld8(lanes, acc);
#pragma unroll 1
    for (int q = 1; q < 6; ++q) {               // the accumulators, added in a fixed order
      tc::tmem_ld8(lanes + (uint32_t)(q * CT_N), part);
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] += part[u];
    }
    const int qs = m / k, c = m - qs * k;
    const size_t s = (size_t)j * nx + i0 + qs;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int n = n0 + u;
      if (n < cout) {
        const size_t o = (s * cout + n) * k + c;
        float v = acc[u];
        if (relu) v = fmaxf(v, 0.f);
        if (act && !(act[o] > 0.f)) v = 0.f;
        out[o] = v;
      }
    }
    // every accumulator read and every halo read of this tile is done before the next
    // tile's shared stores and MMAs
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (failed && tid == 0) atomicExch(err, (int)MLMC_ERR_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    tc::tmem_dealloc(tmem, 128);
  }
}

// Partial weight gradient of the CTA's units (site, column chunk of kc):
// partial[cta][co][ci][tap] (see the file comment).
__global__ void __launch_bounds__(CT_THREADS, 1)
    k_conv_wgrad_tc(const float *__restrict__ in, const float *__restrict__ gout, float *__restrict__ partial,
                    int nx, int ny, int k, int kc, int cin, int cout, int periodic, long long wait_cycles, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cip = pad8(cin), rows = 9 * cip, mt = (rows + CT_M - 1) / CT_M;
  const int nsite = nx * ny, chunks = k / kc, units = nsite * chunks;
  const int per = (units + gridDim.x - 1) / gridDim.x;
  const int u0 = blockIdx.x * per, u1 = min(units, u0 + per);
  const int nunits = u1 > u0 ? u1 - u0 : 0;
  const uint32_t LBO = 128u, KSBO = (uint32_t)(kc / 4) * 128u;   // 8-row groups along M / N
  const uint32_t abytes = (uint32_t)(mt * CT_M / 8) * KSBO, bbytes = (uint32_t)(CT_N / 8) * KSBO;
  const uint32_t sbytes = 2 * abytes + 2 * bbytes;

  if (warp == 0) tc::tmem_alloc(&tmem_base, 32);
  if (tid == 0) {
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tc::tf32_idesc(CT_M, CT_N);
  const int kq = kc / 4;

  int issued = 0;
  for (int t = 0; t < nunits; ++t) {
    const int buf = t & 1;
    unsigned char *Ahi = smem + buf * sbytes, *Alo = Ahi + abytes, *Bhi = Alo + abytes, *Blo = Bhi + bbytes;
    if (t >= 2) {
      // one thread waits for the MMAs of unit t - 2 (they read this buffer); the rest sleep
      if (tid == 0 && !tc::mbar_wait_bounded(&bars[buf], (uint32_t)(((t >> 1) - 1) & 1), wait_cycles)) failed = 1;
      __syncthreads();
      if (failed) break;
    }
    const int u = u0 + t, s = u / chunks, cc0 = (u - s * chunks) * kc;
    const int si = s % nx, sj = s / nx;
    // A: rows (tap, ci) of the unit, 16-byte column quads; padded rows and channels zero
    const int nela = mt * CT_M * kq;
    for (int base = 0; base < nela; base += STAGE_BATCH * CT_THREADS) {
      float4 v[STAGE_BATCH];
#pragma unroll
      for (int b = 0; b < STAGE_BATCH; ++b) {
        const int e = base + b * CT_THREADS + tid;
        v[b] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int r = e / kq, q = e - r * kq;
        if (e < nela && r < rows) {
          const int tap = r / cip, ci = r - tap * cip;
          if (ci < cin) {
            const int nb = conv_site(si + tap % 3 - 1, sj + tap / 3 - 1, nx, ny, periodic);
            if (nb >= 0) v[b] = __ldg((const float4 *)(in + ((size_t)nb * cin + ci) * k + cc0) + q);
          }
        }
      }
#pragma unroll
      for (int b = 0; b < STAGE_BATCH; ++b) {
        const int e = base + b * CT_THREADS + tid;
        const int r = e / kq, q = e - r * kq;
        if (e < nela)
          tc::split_store(Ahi, Alo, (uint32_t)(r >> 3) * KSBO + (uint32_t)q * LBO + (uint32_t)(r & 7) * 16u, v[b]);
      }
    }
    // B: rows co of the unit's output gradient
    for (int e = tid; e < CT_N * kq; e += CT_THREADS) {
      const int n = e / kq, q = e - n * kq;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (n < cout) v = __ldg((const float4 *)(gout + ((size_t)s * cout + n) * k + cc0) + q);
      tc::split_store(Bhi, Blo, (uint32_t)(n >> 3) * KSBO + (uint32_t)q * LBO + (uint32_t)(n & 7) * 16u, v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo), bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
      for (int mi = 0; mi < mt; ++mi) {
        const uint32_t am = (uint32_t)(mi * CT_M / 8) * KSBO;
        for (int ks = 0; ks < kc / 8; ++ks) {
          const uint32_t ko = (uint32_t)ks * 2u * LBO;
          tc::mma_tf32x3(tmem + (uint32_t)(mi * CT_N), tc::smem_desc(ah + am + ko, LBO, KSBO),
                         tc::smem_desc(al + am + ko, LBO, KSBO), tc::smem_desc(bh + ko, LBO, KSBO),
                         tc::smem_desc(bl + ko, LBO, KSBO), idesc, (t > 0 || ks > 0) ? 1u : 0u);
        }
      }
      tc::mma_commit(&bars[buf]);
    }
    issued = t + 1;
  }
  // drain: the last commit of each stage that nobody waited for yet
  if (issued > 0 && tid == 0) {
    const int tl = issued - 1;
    bool ok = true;
    if (!failed) {
      ok = tc::mbar_wait_bounded(&bars[tl & 1], (uint32_t)((tl >> 1) & 1), wait_cycles);
      if (tl >= 1) ok = tc::mbar_wait_bounded(&bars[(tl - 1) & 1], (uint32_t)(((tl - 1) >> 1) & 1), wait_cycles) && ok;
    } else {
      tc::mbar_wait_bounded(&bars[tl & 1], (uint32_t)((tl >> 1) & 1), wait_cycles);
    }
    if (!ok) failed = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (failed) {
    if (tid == 0) atomicExch(err, (int)MLMC_ERR_TIMEOUT);
  } else {
    // warp w: lanes 32 (w % 4) of M tile w / 4, 16 output channels in two loads of 8
    const int mi = warp >> 2;
    const int r = mi * CT_M + 32 * (warp & 3) + lane;
    const int nw = cout * cin * 9;
    if (mi < mt) {
      float acc[16];
      const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(mi * CT_N);
      if (issued > 0) {
        tc::tmem_ld8(taddr, acc);
        tc::tmem_ld8(taddr + 8u, acc + 8);
      } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = 0.f;
      }
      if (r < rows) {
        const int tap = r / cip, ci = r - tap * cip;
        if (ci < cin) {
          float *dst = partial + (size_t)blockIdx.x * nw;
#pragma unroll
          for (int co = 0; co < 16; ++co)
            if (co < cout) dst[((size_t)co * cin + ci) * 9 + tap] = acc[co];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    tc::tmem_dealloc(tmem, 32);
  }
}

namespace {
std::once_flag g_conv_attr_once[64];
int g_conv_smem_max = 0;
}  // namespace

bool conv_tc_ok(int nx, int k, int cin, int cout) {
  if (cin < 1 || cout < 1 || cin > 16 || cout > CT_N) return false;
  if (k != 8 && k != 16 && k != 32 && k != 64 && k != 128) return false;
  return nx % (CT_M / k) == 0;
}

bool conv_wgrad_tc_ok(int k, int cin, int cout) {
  if (cin < 1 || cout < 1 || cin > 16 || cout > CT_N) return false;
  return k % 8 == 0 && (k <= WG_KC || k % WG_KC == 0);
}

int conv_wgrad_tc_blocks() { return 152; }

static void conv_attrs() {
  int dev = 0;
  MLMC_CUDA(cudaGetDevice(&dev));
  std::call_once(g_conv_attr_once[dev & 63], [] {
    const int a = (int)conv_tc_smem(128, 16), b = (int)wgrad_tc_smem(16, WG_KC);
#define MLMC_CONV_FNS(M)                                                                                      \
  (const void *)k_conv_tc<8, 8, M>, (const void *)k_conv_tc<8, 16, M>, (const void *)k_conv_tc<16, 8, M>,        \
      (const void *)k_conv_tc<16, 16, M>, (const void *)k_conv_tc<32, 8, M>, (const void *)k_conv_tc<32, 16, M>, \
      (const void *)k_conv_tc<64, 8, M>, (const void *)k_conv_tc<64, 16, M>, (const void *)k_conv_tc<128, 8, M>,  \
      (const void *)k_conv_tc<128, 16, M>
    const void *fs[] = {MLMC_CONV_FNS(0), MLMC_CONV_FNS(1)};
#undef MLMC_CONV_FNS
    for (const void *f : fs)
      check_cuda(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, a),
                 "cudaFuncSetAttribute(k_conv_tc)");
    check_cuda(cudaFuncSetAttribute(k_conv_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, b),
               "cudaFuncSetAttribute(k_conv_wgrad_tc)");
    g_conv_smem_max = a > b ? a : b;
  });
}

void launch_conv_tc(const float *in, const float *W, const float *act, float *out, int nx, int ny, int k, int cin,
                    int cout, int periodic, int mirror, int relu, int *err, cudaStream_t s) {
  if (!conv_tc_ok(nx, k, cin, cout)) throw cuda_error{cudaErrorInvalidValue, "k_conv_tc: unsupported shape"};
  conv_attrs();
  const int tiles = nx / (CT_M / k) * ny;
  const int cip = pad8(cin);
  // persistent CTAs: as many as fit on the GPU at once (shared memory bounds them)
  int dev = 0, sms = 0;
  MLMC_CUDA(cudaGetDevice(&dev));
  MLMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t smem = conv_tc_smem(k, cin);
  const int per_sm = (int)((227u * 1024u) / (smem + 2048u));
  const int grid = std::min(tiles, sms * std::max(1, std::min(per_sm, 4)));
#define MLMC_CONV_TC(KK, CC)                                                                                  \
  if (k == KK && cip == CC) {                                                                                 \
    if (mirror)                                                                                               \
      k_conv_tc<KK, CC, 1><<<grid, CT_THREADS, smem, s>>>(in, W, act, out, nx, ny, cin, cout, periodic, relu,   \
                                                          CT_WAIT_CYCLES, err);                                \
    else                                                                                                      \
      k_conv_tc<KK, CC, 0><<<grid, CT_THREADS, smem, s>>>(in, W, act, out, nx, ny, cin, cout, periodic, relu,   \
                                                          CT_WAIT_CYCLES, err);                                \
  } else
  MLMC_CONV_TC(8, 8) MLMC_CONV_TC(8, 16) MLMC_CONV_TC(16, 8) MLMC_CONV_TC(16, 16) MLMC_CONV_TC(32, 8)
  MLMC_CONV_TC(32, 16) MLMC_CONV_TC(64, 8) MLMC_CONV_TC(64, 16) MLMC_CONV_TC(128, 8) MLMC_CONV_TC(128, 16)
  throw cuda_error{cudaErrorInvalidValue, "k_conv_tc: unsupported shape"};
#undef MLMC_CONV_TC
  MLMC_LAUNCH_CHECK("k_conv_tc");
}

void launch_conv_wgrad_tc(const float *in, const float *gout, float *partial, int nx, int ny, int k, int cin,
                          int cout, int periodic, int *err, cudaStream_t s) {
  if (!conv_wgrad_tc_ok(k, cin, cout)) throw cuda_error{cudaErrorInvalidValue, "k_conv_wgrad_tc: unsupported shape"};
  if (((uintptr_t)in | (uintptr_t)gout) & 15) throw cuda_error{cudaErrorInvalidValue, "k_conv_wgrad_tc: alignment"};
  conv_attrs();
  const int kc = k < WG_KC ? k : WG_KC;
  k_conv_wgrad_tc<<<conv_wgrad_tc_blocks(), CT_THREADS, wgrad_tc_smem(cin, kc), s>>>(
      in, gout, partial, nx, ny, k, kc, cin, cout, periodic, CT_WAIT_CYCLES, err);
  MLMC_LAUNCH_CHECK("k_conv_wgrad_tc");
}

}  // namespace mlmc
