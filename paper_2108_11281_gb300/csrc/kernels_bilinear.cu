// The paper's hierarchy for Example 5.1 (Sec. 5): bilinear interpolation
// between grids N_l = 2 N_{l+1} + 1 (coarse point I on fine point 2I + 1,
// Dirichlet), its adjoint as restriction (full weighting without the 1/4),
// and the 9-point Galerkin operators of the coarse levels with their
// 4-colour Gauss-Seidel smoother.
//
// Layout: a 9-point operator is coef[site][9] with taps 0 self, 1 +x, 2 -x,
// 3 +y, 4 -y, 5 (+x,+y), 6 (-x,+y), 7 (+x,-y), 8 (-x,-y); taps that leave the
// grid are zero and never followed.  Vector blocks are [site][k] (d = 1) with
// the k right-hand sides innermost; one thread handles VEC consecutive
// columns of one site with 16-byte loads, grid.y is the lattice row.
#include <type_traits>

#include "mlmc_internal.cuh"

namespace mlmc {

namespace {

template <class T, int VEC> struct alignas(sizeof(T) * VEC) PackB { T v[VEC]; };

__device__ __constant__ int c_tap_dx[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
__device__ __constant__ int c_tap_dy[9] = {0, 0, 0, 1, -1, 1, 1, -1, -1};

template <class T>
int vec_of(int k) {
  const int v = 16 / (int)sizeof(T);
  return k % v == 0 ? v : 1;
}

}  // namespace

// y = A x (mode 0) or y = b - A x (mode 1).
template <class T, int VEC>
__global__ void __launch_bounds__(256) k_stencil9(const T *__restrict__ coef, const T *__restrict__ x,
                                                  const T *__restrict__ b, T *__restrict__ y, int nx, int ny, int kv,
                                                  int mode) {
  typedef PackB<T, VEC> V;
  const int j = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nx * kv) return;
  const int i = t / kv, c = t - (t / kv) * kv;
  const int s = j * nx + i;
  const V *X = (const V *)x;
  const T *a = coef + (size_t)s * 9;
  T acc[VEC];
#pragma unroll
  for (int u = 0; u < VEC; ++u) acc[u] = T(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const int ii = i + c_tap_dx[q], jj = j + c_tap_dy[q];
    if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
    const T w = __ldg(a + q);
    const V xn = X[(size_t)(jj * nx + ii) * kv + c];
#pragma unroll
    for (int u = 0; u < VEC; ++u) acc[u] += w * xn.v[u];
  }
  V out;
  if (mode) {
    const V bb = ((const V *)b)[(size_t)s * kv + c];
#pragma unroll
    for (int u = 0; u < VEC; ++u) out.v[u] = bb.v[u] - acc[u];
  } else {
#pragma unroll
    for (int u = 0; u < VEC; ++u) out.v[u] = acc[u];
  }
  ((V *)y)[(size_t)s * kv + c] = out;
}

// One colour of a 4-colour Gauss-Seidel sweep: for the sites with
// (i mod 2) + 2 (j mod 2) == colour, x_s = dinv_s (b_s - sum_{q != 0} a_q x_nb(q)).
// Sites of one colour do not couple in a 9-point stencil, so this is exact
// Gauss-Seidel in colour order.  grid.y runs over the rows of that parity.
template <class T, int VEC>
__global__ void __launch_bounds__(256) k_gs9_colour(const T *__restrict__ coef, const T *__restrict__ dinv,
                                                    T *__restrict__ x, const T *__restrict__ b, int nx, int ny, int kv,
                                                    int colour) {
  typedef PackB<T, VEC> V;
  const int j = 2 * blockIdx.y + (colour >> 1);
  const int i0 = colour & 1;
  const int hx = (nx - i0 + 1) >> 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ny || t >= hx * kv) return;
  const int m = t / kv, c = t - (t / kv) * kv;
  const int i = 2 * m + i0;
  const int s = j * nx + i;
  V *X = (V *)x;
  const T *a = coef + (size_t)s * 9;
  V acc = ((const V *)b)[(size_t)s * kv + c];
#pragma unroll
  for (int q = 1; q < 9; ++q) {
    const int ii = i + c_tap_dx[q], jj = j + c_tap_dy[q];
    if (ii < 0 || ii >= nx || jj < 0 || jj >= ny) continue;
    const T w = __ldg(a + q);
    const V xn = X[(size_t)(jj * nx + ii) * kv + c];
#pragma unroll
    for (int u = 0; u < VEC; ++u) acc.v[u] -= w * xn.v[u];
  }
  const T di = __ldg(dinv + s);
#pragma unroll
  for (int u = 0; u < VEC; ++u) acc.v[u] *= di;
  X[(size_t)s * kv + c] = acc;
}

// rc[I, J] = sum_{a, b in {-1, 0, 1}} w_a w_b r[2I+1+a, 2J+1+b], w_0 = 1, w_{+-1} = 1/2
// (R = P^T of bilinear interpolation); every fine index is inside the grid.
template <class T, int VEC>
__global__ void __launch_bounds__(256) k_restrict_bilinear(const T *__restrict__ r, T *__restrict__ rc, int nxc,
                                                           int nyc, int kv) {
  typedef PackB<T, VEC> V;
  const int J = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nxc * kv) return;
  const int I = t / kv, c = t - (t / kv) * kv;
  const int nx = 2 * nxc + 1;
  const V *R = (const V *)r;
  T acc[VEC];
#pragma unroll
  for (int u = 0; u < VEC; ++u) acc[u] = T(0);
#pragma unroll
  for (int bb = -1; bb <= 1; ++bb) {
#pragma unroll
    for (int aa = -1; aa <= 1; ++aa) {
      const T w = T((aa == 0 ? 1.0 : 0.5) * (bb == 0 ? 1.0 : 0.5));
      const V v = R[(size_t)((2 * J + 1 + bb) * nx + 2 * I + 1 + aa) * kv + c];
#pragma unroll
      for (int u = 0; u < VEC; ++u) acc[u] += w * v.v[u];
    }
  }
  V out;
#pragma unroll
  for (int u = 0; u < VEC; ++u) out.v[u] = acc[u];
  ((V *)rc)[(size_t)(J * nxc + I) * kv + c] = out;
}

// x[i, j] += (P ec)[i, j]: odd i takes coarse column (i-1)/2 with weight 1, even i
// the columns i/2 - 1 and i/2 with weight 1/2 each (those inside the coarse grid);
// the same in y.
template <class T, int VEC>
__global__ void __launch_bounds__(256) k_prolong_bilinear(const T *__restrict__ ec, T *__restrict__ x, int nx, int ny,
                                                          int kv) {
  typedef PackB<T, VEC> V;
  const int j = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nx * kv) return;
  const int i = t / kv, c = t - (t / kv) * kv;
  const int nxc = (nx - 1) / 2, nyc = (ny - 1) / 2;
  // two candidate coarse columns / rows each, weight 0 where one does not exist
  // (its index clamped into the grid, so every load stays in bounds)
  int ia, ib, ja, jb;
  T wa, wb, va, vb;
  if (i & 1) { ia = ib = (i - 1) >> 1; wa = T(1); wb = T(0); }
  else {
    ia = i / 2 - 1; ib = i / 2;
    wa = ia >= 0 ? T(0.5) : T(0); wb = ib < nxc ? T(0.5) : T(0);
    ia = ia < 0 ? 0 : ia; ib = ib >= nxc ? nxc - 1 : ib;
  }
  if (j & 1) { ja = jb = (j - 1) >> 1; va = T(1); vb = T(0); }
  else {
    ja = j / 2 - 1; jb = j / 2;
    va = ja >= 0 ? T(0.5) : T(0); vb = jb < nyc ? T(0.5) : T(0);
    ja = ja < 0 ? 0 : ja; jb = jb >= nyc ? nyc - 1 : jb;
  }
  const V *E = (const V *)ec;
  V *X = (V *)x;
  V acc = X[(size_t)(j * nx + i) * kv + c];
  const V e00 = E[(size_t)(ja * nxc + ia) * kv + c], e01 = E[(size_t)(ja * nxc + ib) * kv + c];
  const V e10 = E[(size_t)(jb * nxc + ia) * kv + c], e11 = E[(size_t)(jb * nxc + ib) * kv + c];
#pragma unroll
  for (int u = 0; u < VEC; ++u)
    acc.v[u] += va * (wa * e00.v[u] + wb * e01.v[u]) + vb * (wa * e10.v[u] + wb * e11.v[u]);
  X[(size_t)(j * nx + i) * kv + c] = acc;
}

namespace {

template <class F>
void real_dispatch(DType t, int k, F &&f) {
  if (t == F64) {
    if (vec_of<double>(k) == 2) f(double(), std::integral_constant<int, 2>());
    else f(double(), std::integral_constant<int, 1>());
  } else if (t == F32) {
    if (vec_of<float>(k) == 4) f(float(), std::integral_constant<int, 4>());
    else f(float(), std::integral_constant<int, 1>());
  } else {
    throw cuda_error{cudaErrorInvalidValue, "the bilinear hierarchy is real (Example 5.1)"};
  }
}

}  // namespace

void launch_stencil9(const StencilView &A, const void *x, const void *b, void *y, int k, int mode, cudaStream_t s) {
  real_dispatch(A.t, k, [&](auto tag, auto vtag) {
    typedef decltype(tag) T;
    constexpr int VEC = decltype(vtag)::value;
    const int kv = k / VEC;
    dim3 g((A.nx * kv + 255) / 256, A.ny);
    k_stencil9<T, VEC><<<g, 256, 0, s>>>((const T *)A.coef, (const T *)x, (const T *)b, (T *)y, A.nx, A.ny, kv, mode);
  });
  MLMC_LAUNCH_CHECK("k_stencil9");
}

void launch_gs9_sweep(const StencilView &A, void *x, const void *b, int k, int order, int x_zero, cudaStream_t s) {
  if (x_zero) MLMC_CUDA(cudaMemsetAsync(x, 0, (size_t)A.nx * A.ny * k * dtype_size(A.t), s));
  real_dispatch(A.t, k, [&](auto tag, auto vtag) {
    typedef decltype(tag) T;
    constexpr int VEC = decltype(vtag)::value;
    const int kv = k / VEC;
    for (int q = 0; q < 4; ++q) {
      const int colour = order == 0 ? q : 3 - q;
      const int hx = (A.nx - (colour & 1) + 1) >> 1;
      const int rows = (A.ny - (colour >> 1) + 1) >> 1;
      if (hx <= 0 || rows <= 0) continue;
      dim3 g((hx * kv + 255) / 256, rows);
      k_gs9_colour<T, VEC><<<g, 256, 0, s>>>((const T *)A.coef, (const T *)A.dinv, (T *)x, (const T *)b, A.nx, A.ny,
                                             kv, colour);
    }
  });
  MLMC_LAUNCH_CHECK("k_gs9_colour");
}

void launch_restrict_bilinear(DType t, const void *r, void *rc, int nxc, int nyc, int k, cudaStream_t s) {
  real_dispatch(t, k, [&](auto tag, auto vtag) {
    typedef decltype(tag) T;
    constexpr int VEC = decltype(vtag)::value;
    const int kv = k / VEC;
    dim3 g((nxc * kv + 255) / 256, nyc);
    k_restrict_bilinear<T, VEC><<<g, 256, 0, s>>>((const T *)r, (T *)rc, nxc, nyc, kv);
  });
  MLMC_LAUNCH_CHECK("k_restrict_bilinear");
}

void launch_prolong_bilinear(DType t, const void *ec, void *x, int nx, int ny, int k, cudaStream_t s) {
  real_dispatch(t, k, [&](auto tag, auto vtag) {
    typedef decltype(tag) T;
    constexpr int VEC = decltype(vtag)::value;
    const int kv = k / VEC;
    dim3 g((nx * kv + 255) / 256, ny);
    k_prolong_bilinear<T, VEC><<<g, 256, 0, s>>>((const T *)ec, (T *)x, nx, ny, kv);
  });
  MLMC_LAUNCH_CHECK("k_prolong_bilinear");
}

}  // namespace mlmc
