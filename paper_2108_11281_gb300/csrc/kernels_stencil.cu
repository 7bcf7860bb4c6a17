// Nearest-neighbour block-stencil kernels: operator apply / residual (the generic
// d x d block stencil, its row-split form for d = 8 and the constant-coefficient
// Example 5.1 operator) and red-black block Gauss-Seidel half-sweeps.  Transfers
// and the setup filter are in kernels_transfer.cu, the 9-point levels of the
// bilinear hierarchy in kernels_bilinear.cu.
//
// Layout: the operator of a level is coef[site][dir][r][c] (dir 0 self, 1 +x,
// 2 -x, 3 +y, 4 -y; periodic indexing, Dirichlet boundaries are zero blocks);
// vector blocks are [site][dof][k] with the k right-hand sides innermost, so
// the k threads of one site read consecutive addresses and share the
// coefficient loads through L1.
#include <cstring>
#include <type_traits>

#include "mlmc_internal.cuh"

namespace mlmc {

// ------------------------------------------------------------------ apply / residual
// One thread per (site, VEC consecutive columns): the d x d coefficient blocks
// are loaded once per VEC columns, the vector entries as 16-byte packs.
template <class T, int VEC> struct alignas(sizeof(T) * VEC) Pack { T v[VEC]; };

// Row r of a d x d coefficient block, with 16-byte loads when the row allows.
template <class T, int D>
__device__ inline void load_row(const T *__restrict__ p, T out[D]) {
  if constexpr ((D * sizeof(T)) % 16 == 0) {
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int i = 0; i < (int)(D * sizeof(T) / 16); ++i) {
      uint4 w = __ldg(q + i);
      memcpy(&out[i * (16 / sizeof(T))], &w, 16);
    }
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i) out[i] = p[i];
  }
}

template <class T, int D, int VEC>
__device__ __forceinline__ void stencil_body(const T *__restrict__ coef, const T *__restrict__ x,
                                             const T *__restrict__ b, T *__restrict__ y, int nx, int ny, int kv,
                                             int mode, int j, int t) {
  // j = lattice row; t = (site i of the row, pack c of VEC columns)
  typedef Pack<T, VEC> V;
  if (t < nx * kv) {
    const int i = t / kv, c = t - (t / kv) * kv;
    const int s = j * nx + i;
    int nb[5];
    nb[0] = s;
    nb[1] = j * nx + (i + 1 == nx ? 0 : i + 1);
    nb[2] = j * nx + (i == 0 ? nx - 1 : i - 1);
    nb[3] = (j + 1 == ny ? 0 : j + 1) * nx + i;
    nb[4] = (j == 0 ? ny - 1 : j - 1) * nx + i;
    T acc[D][VEC];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
      for (int u = 0; u < VEC; ++u) acc[r][u] = zero<T>();
#pragma unroll
    for (int dir = 0; dir < 5; ++dir) {
      const T *B = coef + ((size_t)s * 5 + dir) * D * D;
      const V *xs = (const V *)x + (size_t)nb[dir] * D * kv + c;
      V xq[D];
#pragma unroll
      for (int q = 0; q < D; ++q) xq[q] = xs[(size_t)q * kv];
#pragma unroll
      for (int r = 0; r < D; ++r) {
        T row[D];
        load_row<T, D>(B + r * D, row);
#pragma unroll
        for (int q = 0; q < D; ++q)
#pragma unroll
          for (int u = 0; u < VEC; ++u) acc[r][u] = acc[r][u] + row[q] * xq[q].v[u];
      }
    }
    size_t o = (size_t)s * D * kv + c;
#pragma unroll
    for (int r = 0; r < D; ++r) {
      V out;
      if (mode) {
        V bb = ((const V *)b)[o + (size_t)r * kv];
#pragma unroll
        for (int u = 0; u < VEC; ++u) out.v[u] = bb.v[u] - acc[r][u];
      } else {
#pragma unroll
        for (int u = 0; u < VEC; ++u) out.v[u] = acc[r][u];
      }
      ((V *)y)[o + (size_t)r * kv] = out;
    }
  }
}

// Resident grid striding over the units (row j, chunk of 256 threads of the row): the FP64
// block applies are bound by the FP64 pipe, which one block per unit leaves idle between
// blocks.
template <class T, int D, int VEC>
__global__ void __launch_bounds__(256) k_stencil(const T *__restrict__ coef, const T *__restrict__ x,
                                                 const T *__restrict__ b, T *__restrict__ y, int nx, int ny, int kv,
                                                 int mode, int bpr) {
  const int units = bpr * ny;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int j = u / bpr;
    stencil_body<T, D, VEC>(coef, x, b, y, nx, ny, kv, mode, j, (u - j * bpr) * 256 + threadIdx.x);
  }
}

// The same in blocks of 128 threads pinned at 8 per SM (<= 64 registers), for FP32
// blocks with d = 4 (the aggregation levels of the Laplace hierarchy), like the
// block smoother: both are load-latency bound.  The grid is resident (8 blocks per
// SM) and strides over the units (row j, chunk of 128 threads of the row), in
// row order, so the rows in flight stay a narrow band (vertical neighbours from L2).
// rev = 1 walks the rows from the last: the apply follows a smoothing half-sweep that
// ended there, whose last writes are then still in L2 when they are read.
template <class T, int D, int VEC>
__global__ void __launch_bounds__(128, 8) k_stencil_p(const T *__restrict__ coef, const T *__restrict__ x,
                                                      const T *__restrict__ b, T *__restrict__ y, int nx, int ny,
                                                      int kv, int mode, int bpr, int rev) {
  const int units = bpr * ny;
  for (int u0 = blockIdx.x; u0 < units; u0 += gridDim.x) {
    const int u = rev ? units - 1 - u0 : u0;
    const int j = u / bpr;
    stencil_body<T, D, VEC>(coef, x, b, y, nx, ny, kv, mode, j, (u - j * bpr) * 128 + threadIdx.x);
  }
}

// columns per thread for the generic kernels: 16-byte packs for FP32 data on
// small blocks; fewer columns per thread as d grows, to bound registers
template <class T, int D> struct gen_vec { static const int v = 1; };
template <int D> struct gen_vec<float, D> { static const int v = D <= 4 ? 4 : 2; };
template <int D> struct gen_vec<cfloat, D> { static const int v = D <= 2 ? 2 : 1; };

#define MLMC_DDISPATCH(d, DD, ...)                       \
  switch (d) {                                           \
    case 1: { const int DD = 1; __VA_ARGS__; } break;    \
    case 2: { const int DD = 2; __VA_ARGS__; } break;    \
    case 4: { const int DD = 4; __VA_ARGS__; } break;    \
    case 8: { const int DD = 8; __VA_ARGS__; } break;    \
    default: throw cuda_error{cudaErrorInvalidValue, "unsupported dofs per site"}; \
  }

// Row-split variant for large site blocks (d >= 8, the small coarse lattices of the
// Wilson hierarchy): one thread per (row r of a site, CV consecutive columns)
// accumulates that row over the 5 blocks; block = 32 x CV columns x D rows of one
// site.  CV = 2 (16-byte loads for complex FP32) halves the coefficient loads per
// column (Wilson 128^2, level 2, k = 128: apply 22.6 -> 18.8 us, smoother sweep
// 32.9 -> 26.9 us).  Each column takes the same operations in the same order in
// either form; the compiler's FMA contraction may differ in the last bit.
template <class T, int D, int CV>
__global__ void __launch_bounds__(256) k_stencil_rows(const T *__restrict__ coef, const T *__restrict__ x,
                                                      const T *__restrict__ b, T *__restrict__ y, int nx, int ny,
                                                      int k, int mode) {
  typedef Pack<T, CV> V;
  const int s = blockIdx.y;
  const int i = s % nx, j = s / nx;
  const int r = threadIdx.y;
  const int c = (blockIdx.x * 32 + threadIdx.x) * CV;   // k is a multiple of CV
  if (c >= k) return;
  int nb[5];
  nb[0] = s;
  nb[1] = j * nx + (i + 1 == nx ? 0 : i + 1);
  nb[2] = j * nx + (i == 0 ? nx - 1 : i - 1);
  nb[3] = (j + 1 == ny ? 0 : j + 1) * nx + i;
  nb[4] = (j == 0 ? ny - 1 : j - 1) * nx + i;
  const int kv = k / CV;
  T acc[CV];
#pragma unroll
  for (int u = 0; u < CV; ++u) acc[u] = zero<T>();
#pragma unroll
  for (int dir = 0; dir < 5; ++dir) {
    T row[D];                                      // row r of the block: 16-byte loads, warp-uniform
    load_row<T, D>(coef + (((size_t)s * 5 + dir) * D + r) * D, row);
    if constexpr (CV == 1) {
      const T *xs = x + (size_t)nb[dir] * D * k + c;
#pragma unroll
      for (int q = 0; q < D; ++q) acc[0] = acc[0] + row[q] * xs[(size_t)q * k];
    } else {
      const V *xs = reinterpret_cast<const V *>(x + (size_t)nb[dir] * D * k + c);
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const V xv = xs[(size_t)q * kv];
#pragma unroll
        for (int u = 0; u < CV; ++u) acc[u] = acc[u] + row[q] * xv.v[u];
      }
    }
  }
  const size_t o = ((size_t)s * D + r) * k + c;
  if constexpr (CV == 1) {
    y[o] = mode ? b[o] - acc[0] : acc[0];
  } else {
    V out;
    if (mode) {
      const V bb = *reinterpret_cast<const V *>(b + o);
#pragma unroll
      for (int u = 0; u < CV; ++u) out.v[u] = bb.v[u] - acc[u];
    } else {
#pragma unroll
      for (int u = 0; u < CV; ++u) out.v[u] = acc[u];
    }
    *reinterpret_cast<V *>(y + o) = out;
  }
}

// two columns per thread on blocks of at least 64 even columns
inline int rows_cv(int k) { return (k % 2 == 0 && k >= 64) ? 2 : 1; }

template <class T, int D>
static void stencil_go(const StencilView &A, const void *x, const void *b, void *y, int k, int mode, cudaStream_t s) {
  if constexpr (D >= 8) {
    if (A.nx * A.ny <= 65535) {
      if (rows_cv(k) == 2)
        k_stencil_rows<T, D, 2><<<dim3((k / 2 + 31) / 32, A.nx * A.ny), dim3(32, D), 0, s>>>(
            (const T *)A.coef, (const T *)x, (const T *)b, (T *)y, A.nx, A.ny, k, mode);
      else
        k_stencil_rows<T, D, 1><<<dim3((k + 31) / 32, A.nx * A.ny), dim3(32, D), 0, s>>>(
            (const T *)A.coef, (const T *)x, (const T *)b, (T *)y, A.nx, A.ny, k, mode);
      return;
    }
  }
  constexpr int VW = gen_vec<T, D>::v;
  if (VW > 1 && k % VW == 0) {
    int kv = k / VW;
    if constexpr (std::is_same<T, float>::value && D == 4)
    {
      const int bpr = (A.nx * kv + 127) / 128;
      k_stencil_p<T, D, VW><<<resident_grid(bpr * A.ny, 8), 128, 0, s>>>(
          (const T *)A.coef, (const T *)x, (const T *)b, (T *)y, A.nx, A.ny, kv, mode, bpr, 0);
    }
    else {
      const int bpr = (A.nx * kv + 255) / 256;
      static const int occ = blocks_per_sm(k_stencil<T, D, VW>, 256, 0);
      k_stencil<T, D, VW><<<resident_grid((size_t)bpr * A.ny, occ), 256, 0, s>>>(
          (const T *)A.coef, (const T *)x, (const T *)b, (T *)y, A.nx, A.ny, kv, mode, bpr);
    }
  } else {
    const int bpr = (A.nx * k + 255) / 256;
    static const int occ = blocks_per_sm(k_stencil<T, D, 1>, 256, 0);
    k_stencil<T, D, 1><<<resident_grid((size_t)bpr * A.ny, occ), 256, 0, s>>>(
        (const T *)A.coef, (const T *)x, (const T *)b, (T *)y, A.nx, A.ny, k, mode, bpr);
  }
}

// ------------------------------------------------------------------ Example 5.1, constant coefficients
// The four neighbours of site (i, j), each with a flag: present, or outside a
// Dirichlet lattice (periodic lattices wrap).  Straight-line code: no array
// indexed at run time, so nothing goes through local memory.
struct Nbrs {
  int s[4];
  bool on[4];
};

__device__ __forceinline__ Nbrs laplace_nbrs(int i, int j, int nx, int ny, int periodic) {
  Nbrs n;
  const int s = j * nx + i;
  n.on[0] = i + 1 < nx || periodic;
  n.s[0] = i + 1 < nx ? s + 1 : j * nx;
  n.on[1] = i > 0 || periodic;
  n.s[1] = i > 0 ? s - 1 : j * nx + nx - 1;
  n.on[2] = j + 1 < ny || periodic;
  n.s[2] = j + 1 < ny ? s + nx : i;
  n.on[3] = j > 0 || periodic;
  n.s[3] = j > 0 ? s - nx : (ny - 1) * nx + i;
  return n;
}

// Sum of the present neighbours' packs: (x_+x + x_-x) + (x_+y + x_-y), absent ones zero.
template <class T, int VEC>
__device__ __forceinline__ void laplace_nbr_sum(const Pack<T, VEC> *__restrict__ X, const Nbrs &n, int kv, int c,
                                                T sum[VEC]) {
  Pack<T, VEC> v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (n.on[q]) {
      v[q] = X[(size_t)n.s[q] * kv + c];
    } else {
#pragma unroll
      for (int u = 0; u < VEC; ++u) v[q].v[u] = zero<T>();
    }
  }
#pragma unroll
  for (int u = 0; u < VEC; ++u) sum[u] = (v[0].v[u] + v[1].v[u]) + (v[2].v[u] + v[3].v[u]);
}

// y = diag x - (sum of the in-grid neighbours) (mode 0) or r = b - that (mode 1),
// VEC columns per thread with 16-byte loads; grid.y = lattice row, so the +-y
// neighbours of a block are the rows just touched by the blocks before it (L2
// hits).  Per element: three additions and one fused multiply-add (FP64 lanes
// are the limit of the FP64 form on GB300).
template <class T, int VEC>
__device__ __forceinline__ void laplace_body(const T *__restrict__ x, const T *__restrict__ b, T *__restrict__ y,
                                             int nx, int ny, int kv, T diag, int periodic, int mode, int j, int t) {
  typedef Pack<T, VEC> V;
  if (t >= nx * kv) return;
  const int i = t / kv, c = t - (t / kv) * kv;
  const V *X = (const V *)x;
  const int s = j * nx + i;
  const Nbrs n = laplace_nbrs(i, j, nx, ny, periodic);
  V xc = X[(size_t)s * kv + c];
  T sum[VEC];
  laplace_nbr_sum<T, VEC>(X, n, kv, c, sum);
  V out;
  if (mode) {
    V bb = ((const V *)b)[(size_t)s * kv + c];
#pragma unroll
    for (int u = 0; u < VEC; ++u) out.v[u] = (bb.v[u] + sum[u]) - diag * xc.v[u];
  } else {
#pragma unroll
    for (int u = 0; u < VEC; ++u) out.v[u] = diag * xc.v[u] - sum[u];
  }
  ((V *)y)[(size_t)s * kv + c] = out;
}

// Resident grid striding over the units (row j, chunk of 256 threads of the row) in row
// order: the FP64 apply is bound by the FP64 pipe, which a grid of one block per unit
// leaves idle between blocks.
template <class T, int VEC>
__global__ void __launch_bounds__(256) k_laplace(const T *__restrict__ x, const T *__restrict__ b, T *__restrict__ y,
                                                 int nx, int ny, int kv, T diag, int periodic, int mode, int bpr) {
  const int units = bpr * ny;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int j = u / bpr;
    laplace_body<T, VEC>(x, b, y, nx, ny, kv, diag, periodic, mode, j, (u - j * bpr) * 256 + threadIdx.x);
  }
}

// Red-black Gauss-Seidel half-sweep for Example 5.1: x_s = (b_s + sum of neighbours) / diag
// on the sites of `colour`.  other_zero = 1: the other colour holds zeros (not read).
// Colour 1 takes the rows from the last: consecutive half-sweeps alternate direction, so
// each starts on the rows the previous one wrote last.
// The grid strides over the units (row, chunk of 256 threads of the row).
template <class T, int VEC>
__device__ __forceinline__ void laplace_rbgs_body(T *__restrict__ x, const T *__restrict__ b, int nx, int ny, int kv,
                                                  T dinv, int periodic, int colour, int other_zero, int j, int t) {
  typedef Pack<T, VEC> V;
  const int i0 = (j + colour) & 1;
  const int hx = (nx - i0 + 1) >> 1;      // sites of this colour in row j (odd nx too)
  if (t >= hx * kv) return;
  const int m = t / kv, c = t - (t / kv) * kv;
  const int i = 2 * m + i0;
  const int s = j * nx + i;
  V *X = (V *)x;
  V acc = ((const V *)b)[(size_t)s * kv + c];
  if (!other_zero) {
    const Nbrs n = laplace_nbrs(i, j, nx, ny, periodic);
    T sum[VEC];
    laplace_nbr_sum<T, VEC>(X, n, kv, c, sum);
#pragma unroll
    for (int u = 0; u < VEC; ++u) acc.v[u] = acc.v[u] + sum[u];
  }
#pragma unroll
  for (int u = 0; u < VEC; ++u) acc.v[u] = acc.v[u] * dinv;
  X[(size_t)s * kv + c] = acc;
}

template <class T, int VEC>
__global__ void __launch_bounds__(256) k_laplace_rbgs(T *__restrict__ x, const T *__restrict__ b, int nx, int ny,
                                                      int kv, T dinv, int periodic, int colour, int other_zero,
                                                      int bpr) {
  const int units = bpr * ny;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int jr = u / bpr;
    laplace_rbgs_body<T, VEC>(x, b, nx, ny, kv, dinv, periodic, colour, other_zero, colour ? ny - 1 - jr : jr,
                              (u - jr * bpr) * 256 + threadIdx.x);
  }
}

template <class T>
static int laplace_vec(int k) {
  const int v = 16 / (int)sizeof(T);
  return k % v == 0 ? v : 1;
}

// One damped-Jacobi sweep of the setup filter for Example 5.1 in one pass:
// out = x - omega D^-1 (A x) with A x = diag x - (sum of the in-grid neighbours), written
// as (1 - omega) x + (omega / diag) (sum of the neighbours): one multiply, one FMA and
// the three additions of the sum per element (out must not alias x).
template <class T, int VEC>
__device__ __forceinline__ void laplace_jacobi_body(const T *__restrict__ x, T *__restrict__ out, int nx, int ny,
                                                    int kv, T keep, T scale, int periodic, int j, int t) {
  typedef Pack<T, VEC> V;
  if (t >= nx * kv) return;
  const int i = t / kv, c = t - (t / kv) * kv;
  const V *X = (const V *)x;
  const int s = j * nx + i;
  const Nbrs n = laplace_nbrs(i, j, nx, ny, periodic);
  const V xc = X[(size_t)s * kv + c];
  T sum[VEC];
  laplace_nbr_sum<T, VEC>(X, n, kv, c, sum);
  V o;
#pragma unroll
  for (int u = 0; u < VEC; ++u) o.v[u] = keep * xc.v[u] + scale * sum[u];
  ((V *)out)[(size_t)s * kv + c] = o;
}

template <class T, int VEC>
__global__ void __launch_bounds__(256) k_laplace_jacobi(const T *__restrict__ x, T *__restrict__ out, int nx, int ny,
                                                        int kv, T keep, T scale, int periodic, int bpr) {
  const int units = bpr * ny;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int j = u / bpr;
    laplace_jacobi_body<T, VEC>(x, out, nx, ny, kv, keep, scale, periodic, j, (u - j * bpr) * 256 + threadIdx.x);
  }
}

void launch_laplace_jacobi(const StencilView &A, const void *x, void *out, int k, double omega, cudaStream_t s) {
  if (!A.const_laplace) throw cuda_error{cudaErrorInvalidValue, "laplace_jacobi: constant-coefficient Laplacian only"};
  auto go = [&](auto tag, auto vtag) {
    typedef decltype(tag) T;
    constexpr int VEC = decltype(vtag)::value;
    const int kv = k / VEC;
    const T keep = (T)(1.0 - omega), scale = (T)(omega / A.diag);
    const int bpr = (A.nx * kv + 255) / 256;
    static const int occ = blocks_per_sm(k_laplace_jacobi<T, VEC>, 256, 0);
    k_laplace_jacobi<T, VEC><<<resident_grid((size_t)bpr * A.ny, occ), 256, 0, s>>>(
        (const T *)x, (T *)out, A.nx, A.ny, kv, keep, scale, A.periodic, bpr);
  };
  if (A.t == F64) {
    if (laplace_vec<double>(k) == 2) go(double(), std::integral_constant<int, 2>());
    else go(double(), std::integral_constant<int, 1>());
  } else if (A.t == F32) {
    if (laplace_vec<float>(k) == 4) go(float(), std::integral_constant<int, 4>());
    else go(float(), std::integral_constant<int, 1>());
  } else {
    throw cuda_error{cudaErrorInvalidValue, "constant-coefficient Laplacian is real"};
  }
  MLMC_LAUNCH_CHECK("k_laplace_jacobi");
}

static void launch_laplace(const StencilView &A, const void *x, const void *b, void *y, int k, int mode,
                           cudaStream_t s) {
  auto go = [&](auto tag, auto vtag) {
    typedef decltype(tag) T;
    constexpr int VEC = decltype(vtag)::value;
    int kv = k / VEC;
    const int bpr = (A.nx * kv + 255) / 256;
    static const int occ = blocks_per_sm(k_laplace<T, VEC>, 256, 0);
    k_laplace<T, VEC><<<resident_grid((size_t)bpr * A.ny, occ), 256, 0, s>>>(
        (const T *)x, (const T *)b, (T *)y, A.nx, A.ny, kv, (T)A.diag, A.periodic, mode, bpr);
  };
  if (A.t == F64) {
    if (laplace_vec<double>(k) == 2) go(double(), std::integral_constant<int, 2>());
    else go(double(), std::integral_constant<int, 1>());
  } else if (A.t == F32) {
    if (laplace_vec<float>(k) == 4) go(float(), std::integral_constant<int, 4>());
    else go(float(), std::integral_constant<int, 1>());
  } else {
    throw cuda_error{cudaErrorInvalidValue, "constant-coefficient Laplacian is real"};
  }
  MLMC_LAUNCH_CHECK("k_laplace");
}

static void launch_laplace_rbgs(const StencilView &A, void *x, const void *b, int k, int colour, int other_zero,
                                cudaStream_t s) {
  auto go = [&](auto tag, auto vtag) {
    typedef decltype(tag) T;
    constexpr int VEC = decltype(vtag)::value;
    int kv = k / VEC;
    const int bpr = (((A.nx + 1) / 2) * kv + 255) / 256;
    static const int occ = blocks_per_sm(k_laplace_rbgs<T, VEC>, 256, 0);
    // FP64: a resident grid (FP64-pipe bound); FP32: one block per unit, measured faster
    // there (119 against 124 us per sweep on 1024^2 x 64)
    const unsigned grid = std::is_same<T, double>::value ? resident_grid((size_t)bpr * A.ny, occ)
                                                         : (unsigned)(bpr * A.ny);
    k_laplace_rbgs<T, VEC><<<grid, 256, 0, s>>>(
        (T *)x, (const T *)b, A.nx, A.ny, kv, (T)(1.0 / A.diag), A.periodic, colour, other_zero, bpr);
  };
  if (A.t == F64) {
    if (laplace_vec<double>(k) == 2) go(double(), std::integral_constant<int, 2>());
    else go(double(), std::integral_constant<int, 1>());
  } else if (A.t == F32) {
    if (laplace_vec<float>(k) == 4) go(float(), std::integral_constant<int, 4>());
    else go(float(), std::integral_constant<int, 1>());
  } else {
    throw cuda_error{cudaErrorInvalidValue, "constant-coefficient Laplacian is real"};
  }
  MLMC_LAUNCH_CHECK("k_laplace_rbgs");
}

void launch_stencil(const StencilView &A, const void *x, const void *b, void *y, int k, int mode,
                    cudaStream_t s) {
  if (A.const_laplace) {
    launch_laplace(A, x, b, y, k, mode, s);
    return;
  }
  if (A.taps == 9) {
    launch_stencil9(A, x, b, y, k, mode, s);
    return;
  }
  MLMC_DISPATCH(A.t, T, MLMC_DDISPATCH(A.d, D, stencil_go<T, D>(A, x, b, y, k, mode, s)));
  MLMC_LAUNCH_CHECK("k_stencil");
}

// ------------------------------------------------------------------ red-black block GS
// For every site s of colour `colour` ((i + j) % 2):
//   x_s = D_s^{-1} (b_s - sum over the 4 neighbour blocks A_{s,nb} x_nb),
// the exact solve of the site's row block given its neighbours, so the old x_s
// is not read.  Sites of one colour couple only to the other colour, so the
// half-sweep is an exact block Gauss-Seidel step in red-black order (needs nx,
// ny even).  other_zero = 1: the other colour holds zeros (not read), so the
// first half-sweep from x = 0 needs no initialised x.
// the smoother keeps 16-byte packs for complex FP32 blocks up to d = 8 (measured faster there)
// 16-byte packs where the block allows (measured on a level-2 shape, d = 4 FP32:
// 16-byte packs on a row-per-block grid 0.095 ms per sweep, 8-byte packs 0.107 ms)
template <class T, int D> struct rbgs_vec { static const int v = D <= 4 ? 16 / (int)sizeof(T) : 8 / (int)sizeof(T) > 0 ? 8 / (int)sizeof(T) : 1; };
template <int D> struct rbgs_vec<cfloat, D> { static const int v = D <= 8 ? 2 : 1; };
template <int D> struct rbgs_vec<cdouble, D> { static const int v = 1; };

// grid.y = lattice row j; threads of a row cover (site m of the colour, VEC columns).
template <class T, int D, int VEC>
__device__ __forceinline__ void rbgs_half_body(const T *__restrict__ coef, const T *__restrict__ dinv,
                                               T *__restrict__ x, const T *__restrict__ b, int nx, int ny, int kv,
                                               int colour, int other_zero, int j, int t) {
  // j = lattice row; t = (site m of the colour in the row, pack c of VEC columns)
  typedef Pack<T, VEC> V;
  const int hx = nx / 2;
  if (t < hx * kv) {
    const int m = t / kv, c = t - (t / kv) * kv;
    const int i = 2 * m + ((j + colour) & 1);
    const int s = j * nx + i;
    int nb[5];
    nb[0] = s;
    nb[1] = j * nx + (i + 1 == nx ? 0 : i + 1);
    nb[2] = j * nx + (i == 0 ? nx - 1 : i - 1);
    nb[3] = (j + 1 == ny ? 0 : j + 1) * nx + i;
    nb[4] = (j == 0 ? ny - 1 : j - 1) * nx + i;
    T res[D][VEC];
    size_t o = (size_t)s * D * kv + c;
#pragma unroll
    for (int r = 0; r < D; ++r) {
      V bb = ((const V *)b)[o + (size_t)r * kv];
#pragma unroll
      for (int u = 0; u < VEC; ++u) res[r][u] = bb.v[u];
    }
    if (!other_zero) {
#pragma unroll
      for (int dir = 1; dir < 5; ++dir) {
        const T *B = coef + ((size_t)s * 5 + dir) * D * D;
        const V *xs = (const V *)x + (size_t)nb[dir] * D * kv + c;
        V xq[D];
#pragma unroll
        for (int q = 0; q < D; ++q) xq[q] = xs[(size_t)q * kv];
#pragma unroll
        for (int r = 0; r < D; ++r) {
          T row[D];
          load_row<T, D>(B + r * D, row);
#pragma unroll
          for (int q = 0; q < D; ++q)
#pragma unroll
            for (int u = 0; u < VEC; ++u) res[r][u] = res[r][u] - row[q] * xq[q].v[u];
        }
      }
    }
    const T *Di = dinv + (size_t)s * D * D;
    V *X = (V *)x;
#pragma unroll
    for (int r = 0; r < D; ++r) {
      V out;
      T row[D];
      load_row<T, D>(Di + r * D, row);
#pragma unroll
      for (int u = 0; u < VEC; ++u) out.v[u] = zero<T>();
#pragma unroll
      for (int q = 0; q < D; ++q)
#pragma unroll
        for (int u = 0; u < VEC; ++u) out.v[u] = out.v[u] + row[q] * res[q][u];
      X[o + (size_t)r * kv] = out;
    }
  }
}

template <class T, int D, int VEC>
__global__ void __launch_bounds__(256) k_rbgs_half(const T *__restrict__ coef, const T *__restrict__ dinv,
                                                   T *__restrict__ x, const T *__restrict__ b, int nx, int ny, int kv,
                                                   int colour, int other_zero, int bpr) {
  // resident grid striding over the units (row j, chunk of 256 threads of the row)
  const int units = bpr * ny;
  for (int u = blockIdx.x; u < units; u += gridDim.x) {
    const int j = u / bpr;
    rbgs_half_body<T, D, VEC>(coef, dinv, x, b, nx, ny, kv, colour, other_zero, j, (u - j * bpr) * 256 + threadIdx.x);
  }
}

// The same half-sweep in blocks of 128 threads with residency pinned at 8 blocks
// per SM (<= 64 registers), for FP32 blocks with d = 4 (the aggregation levels of
// the Laplace hierarchy), on a resident grid striding over the units (row j, chunk of
// 128 threads of the row) in row order.  The kernel is load-latency bound; measured
// on the 256^2 x 4 level, k = 128, per sweep: 86.7-87.0 us here, 88.3 us with one
// block per unit (a grid of 8192 blocks), 90.6 us with 256 threads x 4
// blocks, 93.7 us unpinned (256 threads), 96-99 us with two or four neighbour
// blocks' loads issued together (80-128 registers, 2-3 blocks of 256 per SM) and
// 100-104 us with 5-8 blocks of 256 per SM (8-byte packs or spills).
template <class T, int D, int VEC>
__global__ void __launch_bounds__(128, 8) k_rbgs_half_p(const T *__restrict__ coef, const T *__restrict__ dinv,
                                                        T *__restrict__ x, const T *__restrict__ b, int nx, int ny,
                                                        int kv, int colour, int other_zero, int bpr) {
  // colour 1 walks the rows from the last: consecutive half-sweeps alternate direction,
  // so each starts on the rows the previous one wrote last (still in L2)
  const int units = bpr * ny;
  for (int u0 = blockIdx.x; u0 < units; u0 += gridDim.x) {
    const int u = colour ? units - 1 - u0 : u0;
    const int j = u / bpr;
    rbgs_half_body<T, D, VEC>(coef, dinv, x, b, nx, ny, kv, colour, other_zero, j, (u - j * bpr) * 128 + threadIdx.x);
  }
}

// Row-split variant for large site blocks (d >= 8, the coarse levels of the
// Wilson hierarchy, which are small lattices): one thread per (row r of a site,
// column c), so a site's block solve is spread over d x 32 threads instead of one
// thread per column.  Phase 1: res_r = b_r - sum over the 4 neighbour blocks of
// row r times their x (the 8 row threads of a column share the x loads in L1);
// phase 2, after the block barrier: x_r = sum_q Dinv[r][q] res_q from shared memory.
// Block = 32 x CV columns x D rows of one site; grid = (column chunks, sites of the
// colour).  CV = 2 as in k_stencil_rows.
template <class T, int D, int CV>
__global__ void __launch_bounds__(256) k_rbgs_half_rows(const T *__restrict__ coef, const T *__restrict__ dinv,
                                                        T *__restrict__ x, const T *__restrict__ b, int nx, int ny,
                                                        int k, int colour, int other_zero) {
  typedef Pack<T, CV> V;
  __shared__ T res[D][32 * CV];
  const int hx = nx / 2;
  const int idx = blockIdx.y;                       // site of this colour: row j, position m
  const int j = idx / hx, m = idx - (idx / hx) * hx;
  const int i = 2 * m + ((j + colour) & 1);
  const int s = j * nx + i;
  const int cl = threadIdx.x, r = threadIdx.y;
  const int c = (blockIdx.x * 32 + cl) * CV;        // k is a multiple of CV
  const bool live = c < k;
  const int kv = k / CV;
  if (live) {
    const V bb = *reinterpret_cast<const V *>(b + ((size_t)s * D + r) * k + c);
    T acc[CV];
#pragma unroll
    for (int u = 0; u < CV; ++u) acc[u] = bb.v[u];
    if (!other_zero) {
      int nb[4];
      nb[0] = j * nx + (i + 1 == nx ? 0 : i + 1);
      nb[1] = j * nx + (i == 0 ? nx - 1 : i - 1);
      nb[2] = (j + 1 == ny ? 0 : j + 1) * nx + i;
      nb[3] = (j == 0 ? ny - 1 : j - 1) * nx + i;
#pragma unroll
      for (int dir = 0; dir < 4; ++dir) {
        T row[D];                                    // row r of the block: 16-byte loads, warp-uniform
        load_row<T, D>(coef + (((size_t)s * 5 + dir + 1) * D + r) * D, row);
        const V *xs = reinterpret_cast<const V *>(x + (size_t)nb[dir] * D * k + c);
#pragma unroll
        for (int q = 0; q < D; ++q) {
          const V xv = xs[(size_t)q * kv];
#pragma unroll
          for (int u = 0; u < CV; ++u) acc[u] = acc[u] - row[q] * xv.v[u];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < CV; ++u) res[r][cl * CV + u] = acc[u];
  }
  __syncthreads();
  if (live) {
    T di[D];
    load_row<T, D>(dinv + ((size_t)s * D + r) * D, di);
    V out;
#pragma unroll
    for (int u = 0; u < CV; ++u) out.v[u] = zero<T>();
#pragma unroll
    for (int q = 0; q < D; ++q)
#pragma unroll
      for (int u = 0; u < CV; ++u) out.v[u] = out.v[u] + di[q] * res[q][cl * CV + u];
    *reinterpret_cast<V *>(x + ((size_t)s * D + r) * k + c) = out;
  }
}

template <class T, int D>
static void rbgs_go(const StencilView &A, void *x, const void *b, int k, int colour, int other_zero,
                    cudaStream_t s) {
  if constexpr (D >= 8) {
    if ((A.nx / 2) * A.ny <= 65535) {
      if (rows_cv(k) == 2)
        k_rbgs_half_rows<T, D, 2><<<dim3((k / 2 + 31) / 32, (A.nx / 2) * A.ny), dim3(32, D), 0, s>>>(
            (const T *)A.coef, (const T *)A.dinv, (T *)x, (const T *)b, A.nx, A.ny, k, colour, other_zero);
      else
        k_rbgs_half_rows<T, D, 1><<<dim3((k + 31) / 32, (A.nx / 2) * A.ny), dim3(32, D), 0, s>>>(
            (const T *)A.coef, (const T *)A.dinv, (T *)x, (const T *)b, A.nx, A.ny, k, colour, other_zero);
      return;
    }
  }
  constexpr int VW = rbgs_vec<T, D>::v;
  if (VW > 1 && k % VW == 0) {
    int kv = k / VW;
    if constexpr (std::is_same<T, float>::value && D == 4)
    {
      const int bpr = ((A.nx / 2) * kv + 127) / 128;
      k_rbgs_half_p<T, D, VW><<<resident_grid(bpr * A.ny, 8), 128, 0, s>>>(
          (const T *)A.coef, (const T *)A.dinv, (T *)x, (const T *)b, A.nx, A.ny, kv, colour, other_zero, bpr);
    }
    else {
      const int bpr = ((A.nx / 2) * kv + 255) / 256;
      static const int occ = blocks_per_sm(k_rbgs_half<T, D, VW>, 256, 0);
      k_rbgs_half<T, D, VW><<<resident_grid((size_t)bpr * A.ny, occ), 256, 0, s>>>(
          (const T *)A.coef, (const T *)A.dinv, (T *)x, (const T *)b, A.nx, A.ny, kv, colour, other_zero, bpr);
    }
  } else {
    const int bpr = ((A.nx / 2) * k + 255) / 256;
    static const int occ = blocks_per_sm(k_rbgs_half<T, D, 1>, 256, 0);
    k_rbgs_half<T, D, 1><<<resident_grid((size_t)bpr * A.ny, occ), 256, 0, s>>>(
        (const T *)A.coef, (const T *)A.dinv, (T *)x, (const T *)b, A.nx, A.ny, k, colour, other_zero, bpr);
  }
}

void launch_rbgs_half(const StencilView &A, void *x, const void *b, int k, int colour, cudaStream_t s) {
  if (A.const_laplace) {
    launch_laplace_rbgs(A, x, b, k, colour, 0, s);
    return;
  }
  if (A.taps == 9) throw cuda_error{cudaErrorInvalidValue, "9-point stencils are smoothed in four colours"};
  MLMC_DISPATCH(A.t, T, MLMC_DDISPATCH(A.d, D, rbgs_go<T, D>(A, x, b, k, colour, 0, s)));
  MLMC_LAUNCH_CHECK("k_rbgs_half");
}

void launch_rbgs_sweep(const StencilView &A, void *x, const void *b, int k, int order, int x_zero,
                       cudaStream_t s) {
  int first = order == 0 ? 0 : 1;
  if (A.const_laplace) {
    launch_laplace_rbgs(A, x, b, k, first, x_zero, s);
    launch_laplace_rbgs(A, x, b, k, 1 - first, 0, s);
    return;
  }
  if (A.taps == 9) {
    launch_gs9_sweep(A, x, b, k, order, x_zero, s);
    return;
  }
  // x_zero: the first half-sweep reads no neighbours and the second none of its own
  // old values, so x needs no initialisation
  MLMC_DISPATCH(A.t, T, MLMC_DDISPATCH(A.d, D, rbgs_go<T, D>(A, x, b, k, first, x_zero ? 1 : 0, s)));
  MLMC_LAUNCH_CHECK("k_rbgs_half");
  launch_rbgs_half(A, x, b, k, 1 - first, s);
}

}  // namespace mlmc
