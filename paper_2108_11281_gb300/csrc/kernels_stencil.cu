// Nearest-neighbour block-stencil kernels: operator apply / residual, red-black
// block Gauss-Seidel half-sweeps, aggregation restriction and prolongation,
// and the damped-Jacobi update used by the setup filter.
//
// Layout: the operator of a level is coef[site][dir][r][c] (dir 0 self, 1 +x,
// 2 -x, 3 +y, 4 -y; periodic indexing, Dirichlet boundaries are zero blocks);
// vector blocks are [site][dof][k] with the k right-hand sides innermost, so
// the k threads of one site read consecutive addresses and share the
// coefficient loads through L1.
#include "mlmc_internal.cuh"

namespace mlmc {

__device__ inline void neighbours(int s, int nx, int ny, int nb[5]) {
  int i = s % nx, j = s / nx;
  nb[0] = s;
  nb[1] = j * nx + (i + 1 == nx ? 0 : i + 1);
  nb[2] = j * nx + (i == 0 ? nx - 1 : i - 1);
  nb[3] = (j + 1 == ny ? 0 : j + 1) * nx + i;
  nb[4] = (j == 0 ? ny - 1 : j - 1) * nx + i;
}

// ------------------------------------------------------------------ apply / residual
template <class T, int D>
__global__ void k_stencil(const T *__restrict__ coef, const T *__restrict__ x, const T *__restrict__ b,
                          T *__restrict__ y, int nx, int ny, int k, int mode) {
  size_t total = (size_t)nx * ny * k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int c = (int)(t % k);
    int s = (int)(t / k);
    int nb[5];
    neighbours(s, nx, ny, nb);
    T acc[D];
#pragma unroll
    for (int r = 0; r < D; ++r) acc[r] = zero<T>();
#pragma unroll
    for (int dir = 0; dir < 5; ++dir) {
      const T *B = coef + ((size_t)s * 5 + dir) * D * D;
      const T *xs = x + (size_t)nb[dir] * D * k + c;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        T xv = xs[(size_t)q * k];
#pragma unroll
        for (int r = 0; r < D; ++r) acc[r] = acc[r] + B[r * D + q] * xv;
      }
    }
    size_t o = (size_t)s * D * k + c;
#pragma unroll
    for (int r = 0; r < D; ++r) y[o + (size_t)r * k] = mode ? b[o + (size_t)r * k] - acc[r] : acc[r];
  }
}

#define MLMC_DDISPATCH(d, DD, ...)                       \
  switch (d) {                                           \
    case 1: { const int DD = 1; __VA_ARGS__; } break;    \
    case 2: { const int DD = 2; __VA_ARGS__; } break;    \
    case 4: { const int DD = 4; __VA_ARGS__; } break;    \
    case 8: { const int DD = 8; __VA_ARGS__; } break;    \
    case 16: { const int DD = 16; __VA_ARGS__; } break;  \
    default: throw cuda_error{cudaErrorInvalidValue, "unsupported dofs per site"}; \
  }

void launch_stencil(const StencilView &A, const void *x, const void *b, void *y, int k, int mode,
                    cudaStream_t s) {
  size_t total = (size_t)A.nx * A.ny * k;
  unsigned g = grid_for(total, 256, (size_t)1 << 20);
  MLMC_DISPATCH(A.t, T, MLMC_DDISPATCH(A.d, D,
    k_stencil<T, D><<<g, 256, 0, s>>>((const T *)A.coef, (const T *)x, (const T *)b, (T *)y, A.nx, A.ny, k, mode)));
  MLMC_LAUNCH_CHECK("k_stencil");
}

// ------------------------------------------------------------------ red-black block GS
// For every site s of colour `colour` ((i + j) % 2): x_s += D_s^{-1} (b - A x)_s.
// Sites of one colour couple only to the other colour, so the half-sweep is
// an exact block Gauss-Seidel step in red-black order (needs nx, ny even).
template <class T, int D>
__global__ void k_rbgs_half(const T *__restrict__ coef, const T *__restrict__ dinv, T *__restrict__ x,
                            const T *__restrict__ b, int nx, int ny, int k, int colour) {
  int hx = nx / 2;
  size_t total = (size_t)hx * ny * k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int c = (int)(t % k);
    int idx = (int)(t / k);
    int j = idx / hx, m = idx % hx;
    int i = 2 * m + ((j + colour) & 1);
    int s = j * nx + i;
    int nb[5];
    neighbours(s, nx, ny, nb);
    T res[D];
    size_t o = (size_t)s * D * k + c;
#pragma unroll
    for (int r = 0; r < D; ++r) res[r] = b[o + (size_t)r * k];
#pragma unroll
    for (int dir = 0; dir < 5; ++dir) {
      const T *B = coef + ((size_t)s * 5 + dir) * D * D;
      const T *xs = x + (size_t)nb[dir] * D * k + c;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        T xv = xs[(size_t)q * k];
#pragma unroll
        for (int r = 0; r < D; ++r) res[r] = res[r] - B[r * D + q] * xv;
      }
    }
    const T *Di = dinv + (size_t)s * D * D;
#pragma unroll
    for (int r = 0; r < D; ++r) {
      T upd = zero<T>();
#pragma unroll
      for (int q = 0; q < D; ++q) upd = upd + Di[r * D + q] * res[q];
      x[o + (size_t)r * k] = x[o + (size_t)r * k] + upd;
    }
  }
}

void launch_rbgs_half(const StencilView &A, void *x, const void *b, int k, int colour, cudaStream_t s) {
  size_t total = (size_t)(A.nx / 2) * A.ny * k;
  unsigned g = grid_for(total, 256, (size_t)1 << 20);
  MLMC_DISPATCH(A.t, T, MLMC_DDISPATCH(A.d, D,
    k_rbgs_half<T, D><<<g, 256, 0, s>>>((const T *)A.coef, (const T *)A.dinv, (T *)x, (const T *)b, A.nx, A.ny, k, colour)));
  MLMC_LAUNCH_CHECK("k_rbgs_half");
}

// ------------------------------------------------------------------ restriction / prolongation
// rc[I][q][c] = sum_{loc,a} conj(P[I][loc*d + a][q]) r[site(I,loc)][a][c]
template <class T, int DC>
__global__ void k_restrict(const T *__restrict__ P, const T *__restrict__ r, T *__restrict__ rc, int nx,
                           int ny, int d, int ax, int ay, int k) {
  int ncx = nx / ax, ncy = ny / ay;
  size_t total = (size_t)ncx * ncy * k;
  int m = ax * ay * d;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int c = (int)(t % k);
    int I = (int)(t / k);
    int bi = I % ncx, bj = I / ncx;
    T acc[DC];
#pragma unroll
    for (int q = 0; q < DC; ++q) acc[q] = zero<T>();
    const T *PI = P + (size_t)I * m * DC;
    for (int jj = 0; jj < ay; ++jj)
      for (int ii = 0; ii < ax; ++ii) {
        int s = (bj * ay + jj) * nx + bi * ax + ii;
        int loc = jj * ax + ii;
        for (int a = 0; a < d; ++a) {
          T xv = r[((size_t)s * d + a) * k + c];
          const T *Pr = PI + (size_t)(loc * d + a) * DC;
#pragma unroll
          for (int q = 0; q < DC; ++q) acc[q] = acc[q] + conj(Pr[q]) * xv;
        }
      }
#pragma unroll
    for (int q = 0; q < DC; ++q) rc[((size_t)I * DC + q) * k + c] = acc[q];
  }
}

// x[s][a][c] += sum_q P[I(s)][loc(s)*d + a][q] ec[I][q][c]
template <class T, int DC>
__global__ void k_prolong_add(const T *__restrict__ P, const T *__restrict__ ec, T *__restrict__ x, int nx,
                              int ny, int d, int ax, int ay, int k) {
  int ncx = nx / ax;
  size_t total = (size_t)nx * ny * k;
  int m = ax * ay * d;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    int c = (int)(t % k);
    int s = (int)(t / k);
    int i = s % nx, j = s / nx;
    int I = (j / ay) * ncx + i / ax;
    int loc = (j % ay) * ax + (i % ax);
    T e[DC];
#pragma unroll
    for (int q = 0; q < DC; ++q) e[q] = ec[((size_t)I * DC + q) * k + c];
    const T *PI = P + (size_t)I * m * DC;
    for (int a = 0; a < d; ++a) {
      const T *Pr = PI + (size_t)(loc * d + a) * DC;
      T acc = zero<T>();
#pragma unroll
      for (int q = 0; q < DC; ++q) acc = acc + Pr[q] * e[q];
      size_t o = ((size_t)s * d + a) * k + c;
      x[o] = x[o] + acc;
    }
  }
}

void launch_restrict(const ProlongView &P, const void *r, void *rc, int k, cudaStream_t s) {
  size_t total = (size_t)(P.nx / P.ax) * (P.ny / P.ay) * k;
  unsigned g = grid_for(total, 128, (size_t)1 << 20);
  MLMC_DISPATCH(P.t, T, MLMC_DDISPATCH(P.dc, DC,
    k_restrict<T, DC><<<g, 128, 0, s>>>((const T *)P.P, (const T *)r, (T *)rc, P.nx, P.ny, P.d, P.ax, P.ay, k)));
  MLMC_LAUNCH_CHECK("k_restrict");
}

void launch_prolong_add(const ProlongView &P, const void *ec, void *x, int k, cudaStream_t s) {
  size_t total = (size_t)P.nx * P.ny * k;
  unsigned g = grid_for(total, 256, (size_t)1 << 20);
  MLMC_DISPATCH(P.t, T, MLMC_DDISPATCH(P.dc, DC,
    k_prolong_add<T, DC><<<g, 256, 0, s>>>((const T *)P.P, (const T *)ec, (T *)x, P.nx, P.ny, P.d, P.ax, P.ay, k)));
  MLMC_LAUNCH_CHECK("k_prolong_add");
}

// ------------------------------------------------------------------ damped Jacobi update
// out = base + omega * D^{-1} (rhs - y); D = diagonal entries of the self block.
template <class T>
__global__ void k_jacobi_update(const T *__restrict__ coef, T *out, const T *base, const T *rhs,
                                const T *__restrict__ y, double omega, int nsite, int d, int k) {
  size_t total = (size_t)nsite * d * k;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    size_t row = t / k;
    int s = (int)(row / d), a = (int)(row % d);
    T diag = coef[((size_t)s * 5) * d * d + a * d + a];
    T yy = y ? y[t] : zero<T>();
    T v = rhs ? rhs[t] - yy : -yy;
    // v / diag = v * conj(diag) / |diag|^2
    typedef typename real_of<T>::type R;
    T q = rmul((R)(omega / (double)abs2(diag)), conj(diag) * v);
    out[t] = base ? base[t] + q : q;
  }
}

void launch_jacobi_update(const StencilView &A, void *out, const void *base, const void *rhs,
                          const void *y, double omega, int k, cudaStream_t s) {
  int nsite = A.nx * A.ny;
  unsigned g = grid_for((size_t)nsite * A.d * k, 256, (size_t)1 << 20);
  MLMC_DISPATCH(A.t, T, k_jacobi_update<T><<<g, 256, 0, s>>>((const T *)A.coef, (T *)out, (const T *)base,
                                                             (const T *)rhs, (const T *)y, omega, nsite, A.d, k));
  MLMC_LAUNCH_CHECK("k_jacobi_update");
}

}  // namespace mlmc
