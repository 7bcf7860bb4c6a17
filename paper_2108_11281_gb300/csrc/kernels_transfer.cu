// Aggregation transfers (restriction P^* r and prolongation x += P e, with
// dense per-aggregate blocks) and the damped-Jacobi update of the setup filter.
#include "mlmc_internal.cuh"

namespace mlmc {

#define MLMC_DDISPATCH(d, DD, ...)                       \
  switch (d) {                                           \
    case 1: { const int DD = 1; __VA_ARGS__; } break;    \
    case 2: { const int DD = 2; __VA_ARGS__; } break;    \
    case 4: { const int DD = 4; __VA_ARGS__; } break;    \
    case 8: { const int DD = 8; __VA_ARGS__; } break;    \
    default: throw cuda_error{cudaErrorInvalidValue, "unsupported dofs per site"}; \
  }

// ------------------------------------------------------------------ restriction / prolongation
// rc[I][q][c] = sum_{loc,a} conj(P[I][loc*d + a][q]) r[site(I,loc)][a][c]
// One thread per (aggregate, VEC consecutive columns), 16-byte packs when k allows.
template <class T, int VEC> struct alignas(sizeof(T) * VEC) TPack { T v[VEC]; };

// One thread per (aggregate, group of QG coarse dofs, VEC columns): with many
// coarse dofs per aggregate the groups keep enough threads in flight.
template <class T, int DC, int VEC, int QG>
__global__ void __launch_bounds__(128) k_restrict(const T *__restrict__ P, const T *__restrict__ r, T *__restrict__ rc,
                                                  int nx, int ny, int d, int ax, int ay, int kv) {
  typedef TPack<T, VEC> V;
  constexpr int NG = DC / QG;
  int ncx = nx / ax, ncy = ny / ay;
  const unsigned total = (unsigned)ncx * ncy * NG * kv;
  int m = ax * ay * d;
  const V *R = (const V *)r;
  V *RC = (V *)rc;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int c = (int)(t % (unsigned)kv);
    const unsigned ig = t / (unsigned)kv;
    const int g = (int)(ig % NG);
    const int I = (int)(ig / NG);
    int bi = I % ncx, bj = I / ncx;
    T acc[QG][VEC];
#pragma unroll
    for (int q = 0; q < QG; ++q)
#pragma unroll
      for (int u = 0; u < VEC; ++u) acc[q][u] = zero<T>();
    const T *PI = P + (size_t)I * m * DC + g * QG;
    // the aggregate's m = ax * ay * d fine entries, e = loc * d + a (the row of P), in
    // batches of 8 loads issued before their products (the loads are independent;
    // one load at a time left the small coarse-level launches latency-bound)
    for (int e0 = 0; e0 < m; e0 += 8) {
      V xv[8];
#pragma unroll
      for (int b8 = 0; b8 < 8; ++b8) {
        const int e = e0 + b8;
        if (e < m) {
          const int loc = e / d, a = e - (e / d) * d;
          const int jj = loc / ax, ii = loc - (loc / ax) * ax;
          const int s = (bj * ay + jj) * nx + bi * ax + ii;
          xv[b8] = R[((size_t)s * d + a) * kv + c];
        }
      }
#pragma unroll
      for (int b8 = 0; b8 < 8; ++b8) {
        const int e = e0 + b8;
        if (e < m) {
          const T *Pr = PI + (size_t)e * DC;
#pragma unroll
          for (int q = 0; q < QG; ++q) {
            T pq = conj(Pr[q]);
#pragma unroll
            for (int u = 0; u < VEC; ++u) acc[q][u] = acc[q][u] + pq * xv[b8].v[u];
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < QG; ++q) {
      V o;
#pragma unroll
      for (int u = 0; u < VEC; ++u) o.v[u] = acc[q][u];
      RC[((size_t)I * DC + g * QG + q) * kv + c] = o;
    }
  }
}

// Split variant for small coarse levels: the S threads of an item (aggregate I,
// coarse-dof group g, columns c) each sum a contiguous S-th of the aggregate's
// m fine entries, and thread split 0 adds the S partials in split order
// (deterministic).  Block = S x W threads, W = 256 / S items.
template <class T, int DC, int VEC, int QG, int S>
__global__ void __launch_bounds__(256) k_restrict_split(const T *__restrict__ P, const T *__restrict__ r,
                                                        T *__restrict__ rc, int nx, int ny, int d, int ax, int ay,
                                                        int kv) {
  typedef TPack<T, VEC> V;
  constexpr int NG = DC / QG, W = 256 / S;
  __shared__ T red[S][W][QG][VEC];
  const int split = threadIdx.x / W, w = threadIdx.x - (threadIdx.x / W) * W;
  const int ncx = nx / ax, ncy = ny / ay;
  const unsigned total = (unsigned)ncx * ncy * NG * kv;
  const unsigned t = blockIdx.x * W + w;
  const int m = ax * ay * d;
  const V *R = (const V *)r;
  T acc[QG][VEC];
#pragma unroll
  for (int q = 0; q < QG; ++q)
#pragma unroll
    for (int u = 0; u < VEC; ++u) acc[q][u] = zero<T>();
  int c = 0, g = 0, I = 0;
  if (t < total) {
    c = (int)(t % (unsigned)kv);
    const unsigned ig = t / (unsigned)kv;
    g = (int)(ig % NG);
    I = (int)(ig / NG);
    const int bi = I % ncx, bj = I / ncx;
    const T *PI = P + (size_t)I * m * DC + g * QG;
    const int per = (m + S - 1) / S;
    const int e0 = split * per, e1 = min(m, e0 + per);
    for (int e = e0; e < e1; ++e) {
      const int loc = e / d, a = e - (e / d) * d;
      const int jj = loc / ax, ii = loc - (loc / ax) * ax;
      const int s = (bj * ay + jj) * nx + bi * ax + ii;
      const V xv = R[((size_t)s * d + a) * kv + c];
      const T *Pr = PI + (size_t)e * DC;
#pragma unroll
      for (int q = 0; q < QG; ++q) {
        const T pq = conj(Pr[q]);
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[q][u] = acc[q][u] + pq * xv.v[u];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < QG; ++q)
#pragma unroll
    for (int u = 0; u < VEC; ++u) red[split][w][q][u] = acc[q][u];
  __syncthreads();
  if (split == 0 && t < total) {
    V *RC = (V *)rc;
#pragma unroll
    for (int q = 0; q < QG; ++q) {
      V o;
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        T sum = red[0][w][q][u];
        for (int sp = 1; sp < S; ++sp) sum = sum + red[sp][w][q][u];
        o.v[u] = sum;
      }
      RC[((size_t)I * DC + g * QG + q) * kv + c] = o;
    }
  }
}

// x[s][a][c] += sum_q P[I(s)][loc(s)*d + a][q] ec[I][q][c]
template <class T, int DC, int VEC>
__global__ void __launch_bounds__(256) k_prolong_add(const T *__restrict__ P, const T *__restrict__ ec, T *__restrict__ x,
                                                     int nx, int ny, int d, int ax, int ay, int kv) {
  typedef TPack<T, VEC> V;
  int ncx = nx / ax;
  const unsigned total = (unsigned)nx * ny * kv;
  int m = ax * ay * d;
  const V *E = (const V *)ec;
  V *X = (V *)x;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int s = (int)(t / (unsigned)kv);
    const int c = (int)(t - (unsigned)s * kv);
    int i = s % nx, j = s / nx;
    int I = (j / ay) * ncx + i / ax;
    int loc = (j % ay) * ax + (i % ax);
    V e[DC];
#pragma unroll
    for (int q = 0; q < DC; ++q) e[q] = E[((size_t)I * DC + q) * kv + c];
    const T *PI = P + (size_t)I * m * DC;
    for (int a = 0; a < d; ++a) {
      const T *Pr = PI + (size_t)(loc * d + a) * DC;
      size_t o = ((size_t)s * d + a) * kv + c;
      V xv = X[o];
#pragma unroll
      for (int q = 0; q < DC; ++q) {
        T pq = Pr[q];
#pragma unroll
        for (int u = 0; u < VEC; ++u) xv.v[u] = xv.v[u] + pq * e[q].v[u];
      }
      X[o] = xv;
    }
  }
}

template <class T> struct tr_vec { static const int v = 1; };
template <> struct tr_vec<float> { static const int v = 4; };
template <> struct tr_vec<double> { static const int v = 2; };
template <> struct tr_vec<cfloat> { static const int v = 2; };

template <class T, int DC>
static void restrict_go(const ProlongView &P, const void *r, void *rc, int k, cudaStream_t s) {
  constexpr int VW = tr_vec<T>::v;
  constexpr int QG = DC <= 4 ? DC : 2;
  const int vec = (VW > 1 && k % VW == 0) ? VW : 1;
  const int kv = k / vec;
  const size_t items = (size_t)(P.nx / P.ax) * (P.ny / P.ay) * (DC / QG) * kv;
  const int m = P.ax * P.ay * P.d;
  if (items < 32768 && m >= 32) {
    // few items: spread each aggregate's sum over 8 threads
    constexpr int S = 8;
    unsigned gs = (unsigned)((items + 256 / S - 1) / (256 / S));
    if (vec == VW && VW > 1)
      k_restrict_split<T, DC, VW, QG, S><<<gs, 256, 0, s>>>((const T *)P.P, (const T *)r, (T *)rc, P.nx, P.ny, P.d,
                                                             P.ax, P.ay, kv);
    else
      k_restrict_split<T, DC, 1, QG, S><<<gs, 256, 0, s>>>((const T *)P.P, (const T *)r, (T *)rc, P.nx, P.ny, P.d,
                                                            P.ax, P.ay, kv);
    return;
  }
  unsigned g = grid_for(items, 128, (size_t)1 << 20);
  if (vec == VW && VW > 1)
    k_restrict<T, DC, VW, QG><<<g, 128, 0, s>>>((const T *)P.P, (const T *)r, (T *)rc, P.nx, P.ny, P.d, P.ax, P.ay, kv);
  else
    k_restrict<T, DC, 1, QG><<<g, 128, 0, s>>>((const T *)P.P, (const T *)r, (T *)rc, P.nx, P.ny, P.d, P.ax, P.ay, kv);
}

template <class T, int DC>
static void prolong_go(const ProlongView &P, const void *ec, void *x, int k, cudaStream_t s) {
  constexpr int VW = tr_vec<T>::v;
  const int vec = (VW > 1 && k % VW == 0) ? VW : 1;
  const int kv = k / vec;
  unsigned g = grid_for((size_t)P.nx * P.ny * kv, 256, (size_t)1 << 20);
  if (vec == VW && VW > 1)
    k_prolong_add<T, DC, VW><<<g, 256, 0, s>>>((const T *)P.P, (const T *)ec, (T *)x, P.nx, P.ny, P.d, P.ax, P.ay, kv);
  else
    k_prolong_add<T, DC, 1><<<g, 256, 0, s>>>((const T *)P.P, (const T *)ec, (T *)x, P.nx, P.ny, P.d, P.ax, P.ay, kv);
}

void launch_restrict(const ProlongView &P, const void *r, void *rc, int k, cudaStream_t s) {
  if (P.bilinear) {
    launch_restrict_bilinear(P.t, r, rc, (P.nx - 1) / 2, (P.ny - 1) / 2, k, s);
    return;
  }
  MLMC_DISPATCH(P.t, T, MLMC_DDISPATCH(P.dc, DC, restrict_go<T, DC>(P, r, rc, k, s)));
  MLMC_LAUNCH_CHECK("k_restrict");
}

void launch_prolong_add(const ProlongView &P, const void *ec, void *x, int k, cudaStream_t s) {
  if (P.bilinear) {
    launch_prolong_bilinear(P.t, ec, x, P.nx, P.ny, k, s);
    return;
  }
  MLMC_DISPATCH(P.t, T, MLMC_DDISPATCH(P.dc, DC, prolong_go<T, DC>(P, ec, x, k, s)));
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
