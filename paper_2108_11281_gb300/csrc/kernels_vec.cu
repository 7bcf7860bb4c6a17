// Vector-block kernels: noise generation, precision conversion, column-wise
// dot products (two-stage, fixed order), multi-AXPY (optionally summing the
// result's column norms) and column scaling.
// Vector blocks are [row][k] with the k columns (independent right-hand
// sides / samples) innermost, so a warp touches consecutive columns of one row.
#include <algorithm>
#include <atomic>

#include "mlmc_internal.cuh"

namespace mlmc {

void check_cuda(cudaError_t e, const char *where) {
  if (e != cudaSuccess) throw cuda_error{e, where};
}

unsigned resident_grid(size_t units, int per_sm) {
  static std::atomic<int> sms_of[64];              // SM count per device ordinal, 0 = not looked up
  int dev = 0;
  MLMC_CUDA(cudaGetDevice(&dev));
  int sms = dev < 64 ? sms_of[dev].load(std::memory_order_relaxed) : 0;
  if (sms == 0) {
    MLMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (dev < 64) sms_of[dev].store(sms, std::memory_order_relaxed);
  }
  const size_t g = std::min(units, (size_t)sms * (size_t)per_sm);
  return (unsigned)std::max<size_t>(g, 1);
}

// ------------------------------------------------------------------ Philox
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 64x64->128-bit products, key bumped by two Weyl constants between rounds.
struct u64x4 { uint64_t v[4]; };

__device__ inline u64x4 philox4x64_10(u64x4 c, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t lo0 = M0 * c.v[0], hi0 = __umul64hi(M0, c.v[0]);
    uint64_t lo1 = M1 * c.v[2], hi1 = __umul64hi(M1, c.v[2]);
    u64x4 o;
    o.v[0] = hi1 ^ c.v[1] ^ k0;
    o.v[1] = lo1;
    o.v[2] = hi0 ^ c.v[3] ^ k1;
    o.v[3] = lo0;
    c = o;
  }
  return c;
}

// kind 0 = Rademacher (256 rows per counter), 1 = Z4 (128 rows per counter).
// key = (seed, key_hi), counter = (row_block, first_sample + col, 0, 0).
template <class T>
__global__ void k_noise(int kind, uint64_t seed, uint64_t key_hi, uint64_t first_sample, size_t n,
                        int k, T *out) {
  const int rows_per = kind == 0 ? 256 : 128;
  size_t nblk = (n + rows_per - 1) / rows_per;
  size_t total = nblk * (size_t)k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int col = (int)(t % k);
    size_t blk = t / k;
    u64x4 c = {{(uint64_t)blk, first_sample + (uint64_t)col, 0ull, 0ull}};
    u64x4 w = philox4x64_10(c, seed, key_hi);
    size_t row0 = blk * rows_per;
    if (kind == 0) {
      for (int q = 0; q < 4; ++q)
        for (int b = 0; b < 64; ++b) {
          size_t row = row0 + q * 64 + b;
          if (row < n) {
            double v = ((w.v[q] >> b) & 1ull) ? -1.0 : 1.0;
            out[row * k + col] = make<T>(v, 0.0);
          }
        }
    } else {
      for (int q = 0; q < 4; ++q)
        for (int b = 0; b < 32; ++b) {
          size_t row = row0 + q * 32 + b;
          if (row < n) {
            int v = (int)((w.v[q] >> (2 * b)) & 3ull);   // x = i^v
            double r = v == 0 ? 1.0 : v == 2 ? -1.0 : 0.0;
            double i = v == 1 ? 1.0 : v == 3 ? -1.0 : 0.0;
            out[row * k + col] = make<T>(r, i);
          }
        }
    }
  }
}

void launch_noise(int kind, uint64_t seed, uint64_t key_hi, uint64_t first_sample, size_t n, int k,
                  DType t, void *out, cudaStream_t s) {
  size_t nblk = (n + (kind == 0 ? 255 : 127)) / (kind == 0 ? 256 : 128);
  unsigned g = grid_for(nblk * k, 128, 152 * 64);
  MLMC_DISPATCH(t, T, k_noise<T><<<g, 128, 0, s>>>(kind, seed, key_hi, first_sample, n, k, (T *)out));
  MLMC_LAUNCH_CHECK("k_noise");
}

// ------------------------------------------------------------------ convert / fill
template <class To, class From>
__global__ void k_convert(To *dst, const From *src, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = cvt<To, From>(src[i]);
}

void launch_convert(DType to, void *dst, DType from, const void *src, size_t count, cudaStream_t s) {
  unsigned g = grid_for(count, 256);
  if (to == F32 && from == F64) k_convert<float, double><<<g, 256, 0, s>>>((float *)dst, (const double *)src, count);
  else if (to == F64 && from == F32) k_convert<double, float><<<g, 256, 0, s>>>((double *)dst, (const float *)src, count);
  else if (to == C32 && from == C64) k_convert<cfloat, cdouble><<<g, 256, 0, s>>>((cfloat *)dst, (const cdouble *)src, count);
  else if (to == C64 && from == C32) k_convert<cdouble, cfloat><<<g, 256, 0, s>>>((cdouble *)dst, (const cfloat *)src, count);
  else if (to == from) {
    MLMC_CUDA(cudaMemcpyAsync(dst, src, count * dtype_size(to), cudaMemcpyDeviceToDevice, s));
    return;
  } else throw cuda_error{cudaErrorInvalidValue, "launch_convert: field mismatch"};
  MLMC_LAUNCH_CHECK("k_convert");
}

template <class T>
__global__ void k_fill_one(T *dst, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = make<T>(1.0, 0.0);
}

void launch_fill_one(DType t, void *dst, size_t count, cudaStream_t s) {
  MLMC_DISPATCH(t, T, k_fill_one<T><<<grid_for(count, 256), 256, 0, s>>>((T *)dst, count));
  MLMC_LAUNCH_CHECK("k_fill_one");
}

// out = a - b (elementwise)
template <class T>
__global__ void k_sub(T *out, const T *a, const T *b, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

void launch_sub(DType t, void *out, const void *a, const void *b, size_t count, cudaStream_t s) {
  MLMC_DISPATCH(t, T, k_sub<T><<<grid_for(count, 256), 256, 0, s>>>((T *)out, (const T *)a, (const T *)b, count));
  MLMC_LAUNCH_CHECK("k_sub");
}

void launch_fill_zero(DType t, void *dst, size_t count, cudaStream_t s) {
  MLMC_CUDA(cudaMemsetAsync(dst, 0, count * dtype_size(t), s));
}

// ------------------------------------------------------------------ column dots
// Accumulation is in FP64 (double or cdouble) for every storage type.
// Per-block partial sums are FP64 (double / cdouble) for every storage type;
// each thread's own running sum uses the storage precision's ALU (`lane_of`),
// since GB300's FP64 rate is a small fraction of its FP32 rate.
template <class T> struct acc_of { typedef double type; };
template <> struct acc_of<cdouble> { typedef cdouble type; };
template <> struct acc_of<cfloat> { typedef cdouble type; };
template <class T> struct lane_of { typedef T type; };
__device__ inline float dotc_l(float a, float b) { return a * b; }
__device__ inline double dotc_l(double a, double b) { return a * b; }
__device__ inline cfloat dotc_l(cfloat a, cfloat b) { return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re}; }
__device__ inline cdouble dotc_l(cdouble a, cdouble b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
__device__ inline double widen(float a) { return (double)a; }
__device__ inline double widen(double a) { return a; }
__device__ inline cdouble widen(cfloat a) { return {(double)a.re, (double)a.im}; }
__device__ inline cdouble widen(cdouble a) { return a; }

__device__ inline double dotc(double a, double b) { return a * b; }
__device__ inline double dotc(float a, float b) { return (double)a * (double)b; }
__device__ inline cdouble dotc(cdouble a, cdouble b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
__device__ inline cdouble dotc(cfloat a, cfloat b) {
  double ar = a.re, ai = a.im, br = b.re, bi = b.im;
  return {ar * br + ai * bi, ar * bi - ai * br};
}
__device__ inline double addd(double a, double b) { return a + b; }
__device__ inline cdouble addd(cdouble a, cdouble b) { return {a.re + b.re, a.im + b.im}; }

static const int DOT_THREADS = 256;
static const int DOT_MAXV = 8;          // basis vectors per pass over w
static const int DOT_PARTS = 152 * 4;   // fixed number of row chunks

int multidot_parts(size_t rows, int k) {
  (void)k;
  size_t p = rows < (size_t)DOT_PARTS ? rows : (size_t)DOT_PARTS;
  return (int)(p < 1 ? 1 : p);
}

// partial[part][v][c] = sum over rows of chunk `part` of conj(V_v[row][c]) * w[row][c].
// Each thread owns VEC consecutive columns (16-byte loads when k allows);
// the block covers 256 / (k / VEC) rows per step.
template <class T, int VEC> struct alignas(sizeof(T) * VEC) DPack { T v[VEC]; };

template <class T, int VEC>
__global__ void __launch_bounds__(DOT_THREADS, 4) k_multidot_partial(const T *V, size_t vstride, int nvec,
                                                                  const T *w, size_t rows, int k,
                                                                  typename acc_of<T>::type *partial) {
  typedef typename acc_of<T>::type A;
  typedef DPack<T, VEC> P;
  __shared__ A red[DOT_THREADS * VEC];
  const int kv = k / VEC;
  const int slots = DOT_THREADS / kv;          // rows handled per step
  const int tid = threadIdx.x;
  const int cv = tid % kv, slot = tid / kv;
  const bool live = slot < slots;
  const int part = blockIdx.x, nparts = gridDim.x;
  size_t chunk = (rows + nparts - 1) / nparts;
  size_t r0 = (size_t)part * chunk, r1 = r0 + chunk < rows ? r0 + chunk : rows;
  const P *Wp = (const P *)w;
  const P *Vp = (const P *)V;
  const size_t vs = vstride / VEC;
  constexpr int MV = (int)(64 / (sizeof(T) * VEC)) < DOT_MAXV ? (int)(64 / (sizeof(T) * VEC)) : DOT_MAXV;
  for (int v0 = 0; v0 < nvec; v0 += MV) {
    T acc[MV][VEC];
#pragma unroll
    for (int v = 0; v < MV; ++v)
#pragma unroll
      for (int u = 0; u < VEC; ++u) acc[v][u] = zero<T>();
    if (live) {
#pragma unroll 2
      for (size_t r = r0 + slot; r < r1; r += slots) {
        P wv = Wp[r * kv + cv];
#pragma unroll
        for (int v = 0; v < MV; ++v)
          if (v0 + v < nvec) {
            P xv = Vp[(size_t)(v0 + v) * vs + r * kv + cv];
#pragma unroll
            for (int u = 0; u < VEC; ++u) acc[v][u] = acc[v][u] + dotc_l(xv.v[u], wv.v[u]);
          }
      }
    }
#pragma unroll
    for (int v = 0; v < MV; ++v) {
      if (v0 + v >= nvec) break;
#pragma unroll
      for (int u = 0; u < VEC; ++u) red[tid * VEC + u] = live ? widen(acc[v][u]) : zero<A>();
      __syncthreads();
      // column c = cv * VEC + u lives at red[(slot * kv + cv) * VEC + u]
      for (int c = tid; c < k; c += DOT_THREADS) {
        const int cvv = c / VEC, u = c % VEC;
        A sum = red[cvv * VEC + u];
        for (int sl = 1; sl < slots; ++sl) sum = addd(sum, red[(sl * kv + cvv) * VEC + u]);
        partial[((size_t)part * nvec + v0 + v) * k + c] = sum;
      }
      __syncthreads();
    }
  }
}

// out[v][c] = sum_part partial[part][v][c]: one warp per output, lanes take
// parts lane, lane+32, ... in order, then a fixed shuffle tree (deterministic).
__device__ inline double shfl_add(double a, int o) { return a + __shfl_xor_sync(0xffffffffu, a, o); }
__device__ inline cdouble shfl_add(cdouble a, int o) {
  return {a.re + __shfl_xor_sync(0xffffffffu, a.re, o), a.im + __shfl_xor_sync(0xffffffffu, a.im, o)};
}

// Optional epilogue for the fixed-length FGMRES with unnormalised basis vectors
// u_i = s_i v_i (the scaling pass over each new basis vector is skipped; the cycle and the
// operator are linear, so z_j and w scale along).  With d_i = u_i^* w for w = A z_j and
// sc = s per (i, c), column j the new one: the Gram-Schmidt coefficient of u_i is
// coef = d_i / s_i^2 and the Hessenberg entry out = d_i / (s_i s_j), element by element.
template <class A>
__global__ void k_multidot_reduce(const A *partial, int nparts, int nvec, int k, A *out, const double *sc, A *coef,
                                  int j) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nvec * k) return;
  // each lane adds its parts in order; loads are independent, so four are in flight
  A s = zero<A>();
  const size_t stride = (size_t)nvec * k;
#pragma unroll 4
  for (int p = lane; p < nparts; p += 32) s = addd(s, partial[(size_t)p * stride + warp]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = shfl_add(s, o);
  if (lane == 0) {
    if (sc) {
      const int c = warp % k;
      const double si = sc[warp], sj = sc[(size_t)j * k + c];
      coef[warp] = s * make<A>(1.0 / (si * si), 0.0);
      out[warp] = s * make<A>(1.0 / (si * sj), 0.0);
    } else {
      out[warp] = s;
    }
  }
}

void launch_multidot(DType t, const void *V, size_t vstride, int nvec, const void *w, size_t rows,
                     int k, void *partials, int nparts, void *out, DType out_t, cudaStream_t s,
                     const double *lazy_sc, void *lazy_coef, int lazy_j) {
  (void)out_t;
  MLMC_DISPATCH(t, T, {
    typedef typename acc_of<T>::type A;
    constexpr int VW = sizeof(T) == 4 ? 2 : (16 / (int)sizeof(T) > 0 ? 16 / (int)sizeof(T) : 1);
    // one thread per column group of VW: at most DOT_THREADS groups (k <= 256, or 512 with packs)
    const bool packed = VW > 1 && k % VW == 0 && vstride % VW == 0;
    if ((packed ? k / VW : k) > DOT_THREADS)
      throw cuda_error{cudaErrorInvalidValue, "multidot: more column groups than threads"};
    if (packed)
      k_multidot_partial<T, VW><<<nparts, DOT_THREADS, 0, s>>>((const T *)V, vstride, nvec, (const T *)w, rows, k,
                                                               (A *)partials);
    else
      k_multidot_partial<T, 1><<<nparts, DOT_THREADS, 0, s>>>((const T *)V, vstride, nvec, (const T *)w, rows, k,
                                                              (A *)partials);
    MLMC_LAUNCH_CHECK("k_multidot_partial");
    int tot = nvec * k;
    k_multidot_reduce<A><<<(tot * 32 + 255) / 256, 256, 0, s>>>((const A *)partials, nparts, nvec, k, (A *)out,
                                                                lazy_sc, (A *)lazy_coef, lazy_j);
    MLMC_LAUNCH_CHECK("k_multidot_reduce");
  });
}

// ------------------------------------------------------------------ multi-AXPY
// w[r][c] += sign * sum_v V_v[r][c] * h[v*hstride + c]   (h is FP64 / complex FP64)
// The coefficients, rounded to the storage precision (FP32 lanes for FP32 blocks),
// sit in shared memory, so each thread keeps only its accumulator and 16-byte
// packs of w and V; all basis vectors that fit (32 KB of coefficients) are
// applied in one pass over w.  The grid is a multiple of k / VEC threads wide,
// so each thread keeps one column group for its whole grid-stride loop.
// (Measured on 1M rows x 64 FP32 columns: 6.1 TB/s against 4.3-4.9 TB/s with
// the coefficients in registers and 8-byte packs.)
static const int AXPY_SMEM = 32 * 1024;

__device__ inline float norm2_l(float a) { return a * a; }
__device__ inline double norm2_l(double a) { return a * a; }
__device__ inline float norm2_l(cfloat a) { return a.re * a.re + a.im * a.im; }
__device__ inline double norm2_l(cdouble a) { return a.re * a.re + a.im * a.im; }

// norm_part (optional): per block and column, sum over its rows of |w_new|^2 (the
// column norms of the result, for the Arnoldi step), summed per thread in row order
// and over the block's threads in thread order (deterministic), stored as the FP64
// accumulation type; k_multidot_reduce adds the blocks up.
template <class T, class H, int VEC>
__global__ void __launch_bounds__(256) k_multiaxpy(T *__restrict__ w, const T *__restrict__ V, size_t vstride, int nvec,
                                                   const H *__restrict__ h, size_t hstride, double sign, size_t total, int k,
                                                   int group, typename acc_of<T>::type *__restrict__ norm_part) {
  typedef DPack<T, VEC> P;
  typedef typename real_of<T>::type R;
  typedef typename acc_of<T>::type A;
  __shared__ double red[256 * VEC];
  R sq[VEC];
#pragma unroll
  for (int u = 0; u < VEC; ++u) sq[u] = R(0);
  extern __shared__ __align__(16) unsigned char axpy_smem[];
  T *hs = (T *)axpy_smem;
  const size_t stride = (size_t)gridDim.x * blockDim.x;       // in packs; a multiple of k / VEC
  const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const int kv = k / VEC;
  const int cv = (int)(t0 % kv);
  const size_t totv = total / VEC, vs = vstride / VEC;
  P *W = (P *)w;
  const P *Vp = (const P *)V;
  const P *Hp = (const P *)hs;
  for (int v0 = 0; v0 < nvec; v0 += group) {
    const int nv = nvec - v0 < group ? nvec - v0 : group;
    __syncthreads();
    for (int e = threadIdx.x; e < nv * k; e += blockDim.x)
      hs[e] = cvt<T, H>(rmul(sign, h[(size_t)(v0 + e / k) * hstride + e % k]));
    __syncthreads();
    const bool last = v0 + nv >= nvec;
    for (size_t i = t0; i < totv; i += stride) {
      P acc = W[i];
      for (int v = 0; v < nv; ++v) {
        const P x = Vp[(size_t)(v0 + v) * vs + i];
        const P hh = Hp[v * kv + cv];
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc.v[u] = acc.v[u] + x.v[u] * hh.v[u];
      }
      W[i] = acc;
      if (norm_part && last) {
#pragma unroll
        for (int u = 0; u < VEC; ++u) sq[u] += norm2_l(acc.v[u]);
      }
    }
  }
  if (norm_part) {
#pragma unroll
    for (int u = 0; u < VEC; ++u) red[threadIdx.x * VEC + u] = (double)sq[u];
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      const int cvv = c / VEC, u = c - (c / VEC) * VEC;
      double sum = 0.0;
      if ((int)blockDim.x % kv == 0) {
        // the block starts on a column-group boundary: its threads of group cvv are cvv + j kv
        for (int t = cvv; t < (int)blockDim.x; t += kv) sum += red[t * VEC + u];
      } else {
        for (int t = 0; t < (int)blockDim.x; ++t)
          if ((int)((blockIdx.x * blockDim.x + t) % kv) == cvv) sum += red[t * VEC + u];
      }
      norm_part[(size_t)blockIdx.x * k + c] = make<A>(sum, 0.0);
    }
  }
}

static unsigned column_grid(size_t total, int k) {
  // threads = a multiple of k, about 4 waves of 152 SMs x 2048 threads at most
  size_t want = (total + 255) / 256;
  size_t cap = 152 * 8;
  size_t g = want < cap ? want : cap;
  if (g < 1) g = 1;
  // round up so that g * 256 is a multiple of k
  size_t per = (size_t)k / std::__gcd((size_t)k, (size_t)256);
  g = ((g + per - 1) / per) * per;
  return (unsigned)g;
}

template <class T, class H>
static unsigned multiaxpy_go(void *w, const void *V, size_t vstride, int nvec, const void *h, size_t hstride,
                             double sign, size_t total, int k, void *norm_part, cudaStream_t s) {
  typedef typename acc_of<T>::type A;
  constexpr int VW = 16 / (int)sizeof(T) > 0 ? 16 / (int)sizeof(T) : 1;      // 16-byte packs
  int group = AXPY_SMEM / (k * (int)sizeof(T));
  if (group < 1) group = 1;
  if (group > nvec) group = nvec;
  const size_t smem = (size_t)group * k * sizeof(T);
  if (VW > 1 && k % VW == 0 && vstride % VW == 0) {
    unsigned g = column_grid(total / VW, k / VW);
    k_multiaxpy<T, H, VW><<<g, 256, smem, s>>>((T *)w, (const T *)V, vstride, nvec, (const H *)h, hstride, sign, total,
                                               k, group, (A *)norm_part);
    return g;
  }
  unsigned g = column_grid(total, k);
  k_multiaxpy<T, H, 1><<<g, 256, smem, s>>>((T *)w, (const T *)V, vstride, nvec, (const H *)h, hstride, sign, total,
                                            k, group, (A *)norm_part);
  return g;
}

int launch_multiaxpy(DType t, void *w, const void *V, size_t vstride, int nvec, const void *h,
                     DType h_t, size_t hstride, double sign, size_t rows, int k, cudaStream_t s, void *norm_part) {
  size_t total = rows * (size_t)k;
  (void)h_t;
  if (nvec <= 0) return 0;
  unsigned g = 0;
  switch (t) {
    case F64: g = multiaxpy_go<double, double>(w, V, vstride, nvec, h, hstride, sign, total, k, norm_part, s); break;
    case F32: g = multiaxpy_go<float, double>(w, V, vstride, nvec, h, hstride, sign, total, k, norm_part, s); break;
    case C64: g = multiaxpy_go<cdouble, cdouble>(w, V, vstride, nvec, h, hstride, sign, total, k, norm_part, s); break;
    case C32: g = multiaxpy_go<cfloat, cdouble>(w, V, vstride, nvec, h, hstride, sign, total, k, norm_part, s); break;
  }
  MLMC_LAUNCH_CHECK("k_multiaxpy");
  return (int)g;
}

int multiaxpy_norm_parts(size_t rows, int k) {
  // the largest grid multiaxpy_go can choose: column_grid caps at 152 * 8 blocks, then
  // rounds up to a multiple of k / gcd(k, 256)
  (void)rows;
  return 152 * 8 + k;
}

void launch_column_reduce(DType out_t, const void *partial, int nparts, int k, void *out, cudaStream_t s) {
  const int tot = k;
  if (out_t == C64)
    k_multidot_reduce<cdouble><<<(tot * 32 + 255) / 256, 256, 0, s>>>((const cdouble *)partial, nparts, 1, k,
                                                                        (cdouble *)out, nullptr, nullptr, 0);
  else
    k_multidot_reduce<double><<<(tot * 32 + 255) / 256, 256, 0, s>>>((const double *)partial, nparts, 1, k,
                                                                       (double *)out, nullptr, nullptr, 0);
  MLMC_LAUNCH_CHECK("k_multidot_reduce");
}

// ------------------------------------------------------------------ column scaling
// y[r][c] = x[r][c] * alpha[c]  (alpha real FP64)
template <class T>
__global__ void __launch_bounds__(256) k_scale_cols(T *y, const T *x, const double *alpha, size_t total, int k) {
  typedef typename real_of<T>::type R;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const R a = (R)alpha[t0 % k];
  for (size_t i = t0; i < total; i += stride) y[i] = rmul(a, x[i]);
}

void launch_scale_cols(DType t, void *y, const void *x, const void *alpha, int, size_t rows, int k,
                       cudaStream_t s) {
  size_t total = rows * (size_t)k;
  unsigned g = column_grid(total, k);
  MLMC_DISPATCH(t, T, k_scale_cols<T><<<g, 256, 0, s>>>((T *)y, (const T *)x, (const double *)alpha, total, k));
  MLMC_LAUNCH_CHECK("k_scale_cols");
}

// ------------------------------------------------------------------ arithmetic rate probe
// Eight independent FMA chains per thread (x <- x a + b; or additions x <- x + b),
// enough to keep the FP64 or FP32 pipes busy; the result is stored only under a condition that never
// holds, so the chains are not removed.  Measures the ALU ceiling that FP64
// kernels (apply, Arnoldi) meet on this GPU.
template <class T, bool ADD>
__global__ void __launch_bounds__(256) k_fma_rate(T *out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = (T)(threadIdx.x + q) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = ADD ? x[q] + b : fma(x[q], a, b);
  }
  T sum = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) sum += x[q];
  if (sum == (T)-1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

void launch_fma_rate(DType t, int add, void *out, int blocks, int iters, cudaStream_t s) {
  if (t == F64 && add)
    k_fma_rate<double, true><<<blocks, 256, 0, s>>>((double *)out, iters, 0.999999, 1e-7);
  else if (t == F64)
    k_fma_rate<double, false><<<blocks, 256, 0, s>>>((double *)out, iters, 0.999999, 1e-7);
  else
    k_fma_rate<float, false><<<blocks, 256, 0, s>>>((float *)out, iters, 0.999999f, 1e-7f);
  MLMC_LAUNCH_CHECK("k_fma_rate");
}

// Bandwidth probe: `passes` copies of n 16-byte packs between two buffers, a -> b, then
// b -> a, ... in one launch (every thread keeps its indices, so no pass reads what another
// thread writes); an L2-resident pair gives the L2 ceiling of the small coarse-level kernels
// without launch overhead in the measurement.
__global__ void __launch_bounds__(256) k_copy16(uint4 *a, uint4 *b, size_t n, int passes) {
  for (int p = 0; p < passes; ++p) {
    const uint4 *src = (p & 1) ? b : a;
    uint4 *dst = (p & 1) ? a : b;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
      dst[i] = src[i];
  }
}

void launch_copy16(void *a, void *b, size_t n16, int passes, int blocks, cudaStream_t s) {
  k_copy16<<<blocks, 256, 0, s>>>((uint4 *)a, (uint4 *)b, n16, passes);
  MLMC_LAUNCH_CHECK("k_copy16");
}

}  // namespace mlmc
