// Aggregation transfers (restriction P^* r and prolongation x += P e, with
// dense per-aggregate blocks) and the damped-Jacobi update of the setup filter.
#include <type_traits>

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

// x[s][a][c] += sum_q P[I(s)][loc(s)*d + a][q] ec[I][q][c], on every site (colour < 0)
// or on the sites of one red-black colour only (the cycle's post-smoothing overwrites the
// other colour first without reading it, so its prolongation would be dead work).
template <class T, int DC, int VEC>
__global__ void __launch_bounds__(256) k_prolong_add(const T *__restrict__ P, const T *__restrict__ ec, T *__restrict__ x,
                                                     int nx, int ny, int d, int ax, int ay, int kv, int colour) {
  typedef TPack<T, VEC> V;
  int ncx = nx / ax;
  const unsigned total = (unsigned)(colour < 0 ? nx : nx / 2) * ny * kv;
  int m = ax * ay * d;
  const V *E = (const V *)ec;
  V *X = (V *)x;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int ts = (int)(t / (unsigned)kv);
    const int c = (int)(t - (unsigned)ts * kv);
    int s = ts;
    if (colour >= 0) {
      const int hj = ts / (nx / 2), hm = ts - hj * (nx / 2);
      s = hj * nx + 2 * hm + ((hj + colour) & 1);
    }
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
  // resident grid striding over the items (block scheduling costs more than the tail)
  const size_t blocks = (items + 127) / 128;
  if (vec == VW && VW > 1) {
    static const int occ = blocks_per_sm(k_restrict<T, DC, VW, QG>, 128, 0);
    k_restrict<T, DC, VW, QG><<<resident_grid(blocks, occ), 128, 0, s>>>((const T *)P.P, (const T *)r, (T *)rc, P.nx,
                                                                         P.ny, P.d, P.ax, P.ay, kv);
  } else {
    static const int occ = blocks_per_sm(k_restrict<T, DC, 1, QG>, 128, 0);
    k_restrict<T, DC, 1, QG><<<resident_grid(blocks, occ), 128, 0, s>>>((const T *)P.P, (const T *)r, (T *)rc, P.nx,
                                                                        P.ny, P.d, P.ax, P.ay, kv);
  }
}

template <class T, int DC>
static void prolong_go(const ProlongView &P, const void *ec, void *x, int k, int colour, cudaStream_t s) {
  constexpr int VW = tr_vec<T>::v;
  const int vec = (VW > 1 && k % VW == 0) ? VW : 1;
  const int kv = k / vec;
  const size_t sites = colour < 0 ? (size_t)P.nx * P.ny : (size_t)(P.nx / 2) * P.ny;
  const size_t blocks = (sites * kv + 255) / 256;
  if (vec == VW && VW > 1) {
    static const int occ = blocks_per_sm(k_prolong_add<T, DC, VW>, 256, 0);
    k_prolong_add<T, DC, VW><<<resident_grid(blocks, occ), 256, 0, s>>>((const T *)P.P, (const T *)ec, (T *)x, P.nx,
                                                                        P.ny, P.d, P.ax, P.ay, kv, colour);
  } else {
    static const int occ = blocks_per_sm(k_prolong_add<T, DC, 1>, 256, 0);
    k_prolong_add<T, DC, 1><<<resident_grid(blocks, occ), 256, 0, s>>>((const T *)P.P, (const T *)ec, (T *)x, P.nx,
                                                                       P.ny, P.d, P.ax, P.ay, kv, colour);
  }
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
  MLMC_DISPATCH(P.t, T, MLMC_DDISPATCH(P.dc, DC, prolong_go<T, DC>(P, ec, x, k, -1, s)));
  MLMC_LAUNCH_CHECK("k_prolong_add");
}

void launch_prolong_add_colour(const ProlongView &P, const void *ec, void *x, int k, int colour, cudaStream_t s) {
  if (P.bilinear || P.nx % 2) {
    launch_prolong_add(P, ec, x, k, s);
    return;
  }
  MLMC_DISPATCH(P.t, T, MLMC_DDISPATCH(P.dc, DC, prolong_go<T, DC>(P, ec, x, k, colour, s)));
  MLMC_LAUNCH_CHECK("k_prolong_add");
}

// ------------------------------------------------------------------ residual and restriction, fused
// After a red-black (block) Gauss-Seidel sweep that updated colour 1 - `colour` last,
// the residual b - A x vanishes on that colour: each of its site blocks was solved
// exactly given its neighbours (up to rounding).  The restricted residual of the cycle
// (Remark 4.1) therefore only needs the residual on the sites of `colour`, computed on
// the fly: rc[I][q][c] = sum over the aggregate's sites s of that colour of
// sum_a conj(P[I][loc*d + a][q]) (b - A x)_s[a][c].  Against a residual kernel and a
// restriction kernel this saves writing and re-reading r and half of the residual work.
// The colour sites of an aggregate are spread over RR_SLOTS threads (slot n takes the
// colour sites n, n + RR_SLOTS, ... in site order; odd aggregate sides: the sites
// n, n + RR_SLOTS, ... of either colour, the other colour skipped), each for VEC
// columns; the block is
// (KC column packs) x (RR_SLOTS slots) of one aggregate, and the slots' partial sums meet
// in shared memory, added in slot order (deterministic).
constexpr int RR_SLOTS = 8;

template <class T, int D, int DC, int VEC, int KC>
__global__ void __launch_bounds__(KC * RR_SLOTS, 256 / (KC * RR_SLOTS) * 4) k_residual_restrict(const T *__restrict__ coef,
                                                                     const T *__restrict__ x,
                                                                     const T *__restrict__ b,
                                                                     const T *__restrict__ P, T *__restrict__ rc,
                                                                     int nx, int ny, int ax, int ay, int kv,
                                                                     int colour) {
  typedef TPack<T, VEC> V;
  __shared__ V red[RR_SLOTS][DC][KC];
  const int ncx = nx / ax;
  const int I = blockIdx.x;
  const int cc = threadIdx.x, slot = threadIdx.y;
  const int c = blockIdx.y * KC + cc;
  const int bi = I % ncx, bj = I / ncx;
  const int m = ax * ay * D;
  const V *X = (const V *)x;
  const V *B = (const V *)b;
  T acc[DC][VEC];
#pragma unroll
  for (int q = 0; q < DC; ++q)
#pragma unroll
    for (int u = 0; u < VEC; ++u) acc[q][u] = zero<T>();
  if (c < kv) {
    const T *PI = P + (size_t)I * m * DC;
    // with ax and ay even every aggregate row holds ax / 2 sites of each colour: the n-th
    // colour site is row n / (ax / 2), column 2 (n mod ax / 2) + ((colour + row) mod 2)
    const bool even = ((ax | ay) & 1) == 0;
    const int hax = ax >> 1, ncol = even ? hax * ay : ax * ay;
    for (int n = slot; n < ncol; n += RR_SLOTS) {
      int ii, jj;
      if (even) {
        jj = n / hax;
        ii = 2 * (n - jj * hax) + ((colour + jj) & 1);
      } else {
        jj = n / ax;
        ii = n - jj * ax;
      }
      const int loc = jj * ax + ii;
      const int i = bi * ax + ii, j = bj * ay + jj;
      if (((i + j) & 1) != colour) continue;            // the residual is zero there
      const int s = j * nx + i;
      int nb[5];
      nb[0] = s;
      nb[1] = j * nx + (i + 1 == nx ? 0 : i + 1);
      nb[2] = j * nx + (i == 0 ? nx - 1 : i - 1);
      nb[3] = (j + 1 == ny ? 0 : j + 1) * nx + i;
      nb[4] = (j == 0 ? ny - 1 : j - 1) * nx + i;
      T r[D][VEC];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const V bb = B[((size_t)s * D + a) * kv + c];
#pragma unroll
        for (int u = 0; u < VEC; ++u) r[a][u] = bb.v[u];
      }
#pragma unroll
      for (int dir = 0; dir < 5; ++dir) {
        const T *Bd = coef + ((size_t)s * 5 + dir) * D * D;
        V xq[D];
#pragma unroll
        for (int q = 0; q < D; ++q) xq[q] = X[((size_t)nb[dir] * D + q) * kv + c];
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int q = 0; q < D; ++q) {
            const T w = Bd[a * D + q];
#pragma unroll
            for (int u = 0; u < VEC; ++u) r[a][u] = r[a][u] - w * xq[q].v[u];
          }
      }
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const T *Pr = PI + (size_t)(loc * D + a) * DC;
#pragma unroll
        for (int q = 0; q < DC; ++q) {
          const T pq = conj(Pr[q]);
#pragma unroll
          for (int u = 0; u < VEC; ++u) acc[q][u] = acc[q][u] + pq * r[a][u];
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < DC; ++q)
#pragma unroll
    for (int u = 0; u < VEC; ++u) red[slot][q][cc].v[u] = acc[q][u];
  __syncthreads();
  // DC x KC output packs, one per thread, the slots added in order
  const int tid = slot * KC + cc;
  if (tid < DC * KC) {
    const int q = tid / KC, c2 = tid - (tid / KC) * KC;
    const int co = blockIdx.y * KC + c2;
    if (co < kv) {
      V o = red[0][q][c2];
#pragma unroll
      for (int sl = 1; sl < RR_SLOTS; ++sl)
#pragma unroll
        for (int u = 0; u < VEC; ++u) o.v[u] = o.v[u] + red[sl][q][c2].v[u];
      ((V *)rc)[((size_t)I * DC + q) * kv + co] = o;
    }
  }
}

// The same for the constant-coefficient Example 5.1 operator (d = 1, no matrix read):
// r_s = b_s - (diag x_s - sum of the in-grid neighbours).
template <class T, int DC, int VEC>
__global__ void __launch_bounds__(128) k_laplace_residual_restrict(const T *__restrict__ x, const T *__restrict__ b,
                                                                   const T *__restrict__ P, T *__restrict__ rc,
                                                                   int nx, int ny, int ax, int ay, int kv, T diag,
                                                                   int periodic, int colour) {
  typedef TPack<T, VEC> V;
  const int ncx = nx / ax, ncy = ny / ay;
  const unsigned total = (unsigned)ncx * ncy * kv;
  const int m = ax * ay;
  const V *X = (const V *)x;
  const V *B = (const V *)b;
  V *RC = (V *)rc;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int c = (int)(t % (unsigned)kv);
    const int I = (int)(t / (unsigned)kv);
    const int bi = I % ncx, bj = I / ncx;
    T acc[DC][VEC];
#pragma unroll
    for (int q = 0; q < DC; ++q)
#pragma unroll
      for (int u = 0; u < VEC; ++u) acc[q][u] = zero<T>();
    const T *PI = P + (size_t)I * m * DC;
    for (int loc = 0; loc < m; ++loc) {
      const int jj = loc / ax, ii = loc - jj * ax;
      const int i = bi * ax + ii, j = bj * ay + jj;
      if (((i + j) & 1) != colour) continue;
      const int s = j * nx + i;
      const bool on0 = i + 1 < nx || periodic, on1 = i > 0 || periodic;
      const bool on2 = j + 1 < ny || periodic, on3 = j > 0 || periodic;
      const int s0 = i + 1 < nx ? s + 1 : j * nx, s1 = i > 0 ? s - 1 : j * nx + nx - 1;
      const int s2 = j + 1 < ny ? s + nx : i, s3 = j > 0 ? s - nx : (ny - 1) * nx + i;
      V x0, x1, x2, x3;
#pragma unroll
      for (int u = 0; u < VEC; ++u) x0.v[u] = x1.v[u] = x2.v[u] = x3.v[u] = zero<T>();
      if (on0) x0 = X[(size_t)s0 * kv + c];
      if (on1) x1 = X[(size_t)s1 * kv + c];
      if (on2) x2 = X[(size_t)s2 * kv + c];
      if (on3) x3 = X[(size_t)s3 * kv + c];
      const V xs = X[(size_t)s * kv + c];
      const V bb = B[(size_t)s * kv + c];
      const T *Pr = PI + (size_t)loc * DC;
      T r[VEC];
#pragma unroll
      for (int u = 0; u < VEC; ++u) r[u] = (bb.v[u] + ((x0.v[u] + x1.v[u]) + (x2.v[u] + x3.v[u]))) - diag * xs.v[u];
#pragma unroll
      for (int q = 0; q < DC; ++q) {
        const T pq = Pr[q];
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[q][u] = acc[q][u] + pq * r[u];
      }
    }
#pragma unroll
    for (int q = 0; q < DC; ++q) {
      V o;
#pragma unroll
      for (int u = 0; u < VEC; ++u) o.v[u] = acc[q][u];
      RC[((size_t)I * DC + q) * kv + c] = o;
    }
  }
}

bool residual_restrict_ok(const StencilView &A, const ProlongView &P) {
  if (P.bilinear || A.taps == 9 || A.nx % 2 || A.ny % 2) return false;
  if (A.const_laplace) return A.t == F32 || A.t == F64;
  return A.d <= 4 && P.dc <= 4 && A.d == P.d;
}


template <class T, int D, int DC>
static void residual_restrict_go(const StencilView &A, const ProlongView &P, const void *x, const void *b, void *rc,
                                 int k, int colour, cudaStream_t s) {
  constexpr int VW = tr_vec<T>::v;
  const int vec = (VW > 1 && k % VW == 0) ? VW : 1;
  const int kv = k / vec;
  const unsigned aggs = (unsigned)(P.nx / P.ax) * (P.ny / P.ay);
  // column packs per block: 32, or fewer for narrow blocks (16 on the 256^2 x 4 level at
  // k = 128: 62.2 against 59.5 us)
  auto go = [&](auto vtag, auto ktag) {
    constexpr int V = decltype(vtag)::value, KC = decltype(ktag)::value;
    k_residual_restrict<T, D, DC, V, KC><<<dim3(aggs, (kv + KC - 1) / KC), dim3(KC, RR_SLOTS), 0, s>>>(
        (const T *)A.coef, (const T *)x, (const T *)b, (const T *)P.P, (T *)rc, A.nx, A.ny, P.ax, P.ay, kv, colour);
  };
  if (vec == VW && VW > 1) {
    if (kv >= 32) go(std::integral_constant<int, VW>(), std::integral_constant<int, 32>());
    else if (kv >= 16) go(std::integral_constant<int, VW>(), std::integral_constant<int, 16>());
    else go(std::integral_constant<int, VW>(), std::integral_constant<int, 8>());
  } else {
    if (kv >= 32) go(std::integral_constant<int, 1>(), std::integral_constant<int, 32>());
    else if (kv >= 16) go(std::integral_constant<int, 1>(), std::integral_constant<int, 16>());
    else go(std::integral_constant<int, 1>(), std::integral_constant<int, 8>());
  }
}

template <class T, int DC>
static void laplace_residual_restrict_go(const StencilView &A, const ProlongView &P, const void *x, const void *b,
                                         void *rc, int k, int colour, cudaStream_t s) {
  constexpr int VW = tr_vec<T>::v;
  const int vec = (VW > 1 && k % VW == 0) ? VW : 1;
  const int kv = k / vec;
  const size_t items = (size_t)(P.nx / P.ax) * (P.ny / P.ay) * kv;
  const size_t blocks = (items + 127) / 128;
  static const int occ_v = blocks_per_sm(k_laplace_residual_restrict<T, DC, VW>, 128, 0);
  static const int occ_1 = blocks_per_sm(k_laplace_residual_restrict<T, DC, 1>, 128, 0);
  const unsigned g = resident_grid(blocks, vec == VW && VW > 1 ? occ_v : occ_1);
  if (vec == VW && VW > 1)
    k_laplace_residual_restrict<T, DC, VW><<<g, 128, 0, s>>>((const T *)x, (const T *)b, (const T *)P.P, (T *)rc,
                                                             A.nx, A.ny, P.ax, P.ay, kv, (T)A.diag, A.periodic,
                                                             colour);
  else
    k_laplace_residual_restrict<T, DC, 1><<<g, 128, 0, s>>>((const T *)x, (const T *)b, (const T *)P.P, (T *)rc,
                                                            A.nx, A.ny, P.ax, P.ay, kv, (T)A.diag, A.periodic,
                                                            colour);
}

void launch_residual_restrict(const StencilView &A, const ProlongView &P, const void *x, const void *b, void *rc,
                              int k, int colour, cudaStream_t s) {
  if (!residual_restrict_ok(A, P)) throw cuda_error{cudaErrorInvalidValue, "residual_restrict: unsupported level"};
  if (A.const_laplace) {
    if (A.t == F32) {
      MLMC_DDISPATCH(P.dc, DC, laplace_residual_restrict_go<float, DC>(A, P, x, b, rc, k, colour, s));
    } else {
      MLMC_DDISPATCH(P.dc, DC, laplace_residual_restrict_go<double, DC>(A, P, x, b, rc, k, colour, s));
    }
  } else {
    switch (A.d * 16 + P.dc) {
#define MLMC_RR(DD, CC)                                                                                       \
  case DD * 16 + CC:                                                                                          \
    MLMC_DISPATCH(A.t, T, (residual_restrict_go<T, DD, CC>(A, P, x, b, rc, k, colour, s)));                  \
    break;
      MLMC_RR(1, 1) MLMC_RR(1, 2) MLMC_RR(1, 4) MLMC_RR(2, 2) MLMC_RR(2, 4) MLMC_RR(4, 4)
#undef MLMC_RR
      default:
        throw cuda_error{cudaErrorInvalidValue, "residual_restrict: unsupported dofs"};
    }
  }
  MLMC_LAUNCH_CHECK("k_residual_restrict");
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
