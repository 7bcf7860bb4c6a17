// Setup-time kernels: inverse self blocks for the smoother, per-aggregate
// modified Gram-Schmidt (P blocks), Galerkin coarse stencils P^* A P, dense
// Gauss-Jordan inverse and trace of the coarsest operator, and the dense
// coarsest-level apply used inside every multigrid cycle.
#include <algorithm>
#include <mutex>

#include "mlmc.h"
#include "mlmc_internal.cuh"

namespace mlmc {

__device__ inline double mag(double a) { return fabs(a); }
__device__ inline double mag(float a) { return fabs((double)a); }
__device__ inline double mag(cdouble a) { return sqrt(abs2(a)); }
__device__ inline double mag(cfloat a) { return sqrt((double)abs2(a)); }

// a / b for a field element b (used only off the hot path)
template <class T> __device__ inline T divide(T a, T b) {
  typedef typename real_of<T>::type R;
  return rmul((R)(1.0 / (double)abs2(b)), a * conj(b));
}

// ------------------------------------------------------------------ self-block inverses
// One thread per site; Gauss-Jordan with partial pivoting on the d x d block.
template <class T, int D>
__global__ void k_block_inverse(const T *coef, T *dinv, int nsite, int *err) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsite) return;
  T a[D][D], inv[D][D];
  const T *B = coef + (size_t)s * 5 * D * D;   // dir 0 = self
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      a[r][c] = B[r * D + c];
      inv[r][c] = r == c ? make<T>(1.0, 0.0) : zero<T>();
    }
  for (int p = 0; p < D; ++p) {
    int piv = p;
    double best = mag(a[p][p]);
    for (int r = p + 1; r < D; ++r)
      if (mag(a[r][p]) > best) { best = mag(a[r][p]); piv = r; }
    if (best == 0.0) { atomicExch(err, 1); return; }
    if (piv != p)
      for (int c = 0; c < D; ++c) {
        T t = a[p][c]; a[p][c] = a[piv][c]; a[piv][c] = t;
        t = inv[p][c]; inv[p][c] = inv[piv][c]; inv[piv][c] = t;
      }
    T pv = a[p][p];
    for (int c = 0; c < D; ++c) { a[p][c] = divide(a[p][c], pv); inv[p][c] = divide(inv[p][c], pv); }
    for (int r = 0; r < D; ++r) {
      if (r == p) continue;
      T f = a[r][p];
      for (int c = 0; c < D; ++c) { a[r][c] = a[r][c] - f * a[p][c]; inv[r][c] = inv[r][c] - f * inv[p][c]; }
    }
  }
  T *O = dinv + (size_t)s * D * D;
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) O[r * D + c] = inv[r][c];
}

void launch_block_inverse(DType t, const void *coef, void *dinv, int nsite, int d, int *err, cudaStream_t s) {
  unsigned g = (nsite + 63) / 64;
#define MLMC_BI_CASE(DD) case DD: MLMC_DISPATCH(t, T, k_block_inverse<T, DD><<<g, 64, 0, s>>>((const T *)coef, (T *)dinv, nsite, err)); break;
  switch (d) {
    MLMC_BI_CASE(1) MLMC_BI_CASE(2) MLMC_BI_CASE(4) MLMC_BI_CASE(8)
    default: throw cuda_error{cudaErrorInvalidValue, "block inverse: unsupported d"};
  }
#undef MLMC_BI_CASE
  MLMC_LAUNCH_CHECK("k_block_inverse");
}

// ------------------------------------------------------------------ per-aggregate MGS
// One warp per aggregate.  V holds the test vectors as a block [site][dof][ntv].
// Column q = h*ntv + t keeps test vector t on the dofs of spin half h (first /
// second half of each site's dofs) when spin_split, else q = t.  Columns are
// orthonormalised in order by modified Gram-Schmidt into P[I][loc*d + a][q].
__device__ inline cdouble warp_sum_c(cdouble v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
    v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
  }
  return v;
}
__device__ inline double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline cdouble to_cd(double a) { return {a, 0.0}; }
__device__ inline cdouble to_cd(cdouble a) { return a; }
template <class T> __device__ inline T from_cd(cdouble a);
template <> __device__ inline double from_cd<double>(cdouble a) { return a.re; }
template <> __device__ inline cdouble from_cd<cdouble>(cdouble a) { return a; }

template <class T>
__global__ void k_mgs(const T *V, T *P, int nx, int ny, int d, int ax, int ay, int ntv, int spin_split,
                      int *err) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
  int lane = threadIdx.x % 32;
  int ncx = nx / ax, ncy = ny / ay;
  if (warp >= ncx * ncy) return;
  int I = warp, bi = I % ncx, bj = I / ncx;
  int m = ax * ay * d;
  int dc = spin_split ? 2 * ntv : ntv;
  T *PI = P + (size_t)I * m * dc;
  for (int q = 0; q < dc; ++q) {
    int h = spin_split ? q / ntv : 0, tv = spin_split ? q % ntv : q;
    // load column q into P[:, q]
    for (int row = lane; row < m; row += 32) {
      int loc = row / d, a = row % d;
      int s = (bj * ay + loc / ax) * nx + bi * ax + loc % ax;
      bool keep = !spin_split || ((a < d / 2) == (h == 0));
      PI[(size_t)row * dc + q] = keep ? V[((size_t)s * d + a) * ntv + tv] : zero<T>();
    }
    __syncwarp();
    // modified Gram-Schmidt, each column twice (one pass loses orthogonality on
    // nearly dependent smooth test vectors; R P = I is what Remark 4.3 needs)
    for (int pass = 0; pass < 2; ++pass)
    for (int p = 0; p < q; ++p) {
      cdouble acc = {0.0, 0.0};
      for (int row = lane; row < m; row += 32) {
        cdouble pp = to_cd(PI[(size_t)row * dc + p]), vv = to_cd(PI[(size_t)row * dc + q]);
        acc.re += pp.re * vv.re + pp.im * vv.im;
        acc.im += pp.re * vv.im - pp.im * vv.re;
      }
      acc = warp_sum_c(acc);
      T coef = from_cd<T>(acc);
      for (int row = lane; row < m; row += 32)
        PI[(size_t)row * dc + q] = PI[(size_t)row * dc + q] - coef * PI[(size_t)row * dc + p];
      __syncwarp();
    }
    double nrm2 = 0.0;
    for (int row = lane; row < m; row += 32) nrm2 += (double)abs2(PI[(size_t)row * dc + q]);
    nrm2 = warp_sum_d(nrm2);
    if (nrm2 == 0.0) { if (lane == 0) atomicExch(err, 2); return; }
    double inv = 1.0 / sqrt(nrm2);
    for (int row = lane; row < m; row += 32)
      PI[(size_t)row * dc + q] = rmul(inv, PI[(size_t)row * dc + q]);
    __syncwarp();
  }
}

void launch_mgs(DType t, const void *V, void *P, int nx, int ny, int d, int ax, int ay, int ntv,
                int spin_split, int *err, cudaStream_t s) {
  int nagg = (nx / ax) * (ny / ay);
  unsigned g = (nagg * 32 + 127) / 128;
  if (t == F64) k_mgs<double><<<g, 128, 0, s>>>((const double *)V, (double *)P, nx, ny, d, ax, ay, ntv, spin_split, err);
  else if (t == C64) k_mgs<cdouble><<<g, 128, 0, s>>>((const cdouble *)V, (cdouble *)P, nx, ny, d, ax, ay, ntv, spin_split, err);
  else throw cuda_error{cudaErrorInvalidValue, "mgs: FP64 only"};
  MLMC_LAUNCH_CHECK("k_mgs");
}

// ------------------------------------------------------------------ Galerkin coarse stencil
// Coarse block (cdir, p, q) of coarse site I:
//   sum over fine sites s in I, fine directions fd whose link leaves I towards cdir
//   (interior links and the self block go to cdir 0) of
//   sum_{a,b} conj(P_I[loc(s) d + a][p]) A_s[fd][a][b] P_J[loc(t) d + b][q],  t = nb(s, fd), J = agg(t).
template <class T>
__global__ void k_galerkin(const T *coef, const T *P, T *cc, int nx, int ny, int d, int ax, int ay, int dc) {
  int I = blockIdx.x;
  int ncx = nx / ax;
  int bi = I % ncx, bj = I / ncx;
  int m = ax * ay * d;
  int entries = 5 * dc * dc;
  for (int e = threadIdx.x; e < entries; e += blockDim.x) {
    int cdir = e / (dc * dc), p = (e / dc) % dc, q = e % dc;
    T acc = zero<T>();
    for (int loc = 0; loc < ax * ay; ++loc) {
      int ii = loc % ax, jj = loc / ax;
      int i = bi * ax + ii, j = bj * ay + jj;
      int s = j * nx + i;
      for (int fd = 0; fd < 5; ++fd) {
        int target;
        int ti = i, tj = j;
        switch (fd) {
          case 0: target = 0; break;
          case 1: target = ii == ax - 1 ? 1 : 0; ti = i + 1 == nx ? 0 : i + 1; break;
          case 2: target = ii == 0 ? 2 : 0; ti = i == 0 ? nx - 1 : i - 1; break;
          case 3: target = jj == ay - 1 ? 3 : 0; tj = j + 1 == ny ? 0 : j + 1; break;
          default: target = jj == 0 ? 4 : 0; tj = j == 0 ? ny - 1 : j - 1; break;
        }
        if (target != cdir) continue;
        int J = (tj / ay) * ncx + ti / ax;
        int locj = (tj % ay) * ax + (ti % ax);
        const T *B = coef + ((size_t)s * 5 + fd) * d * d;
        const T *PI = P + (size_t)I * m * dc;
        const T *PJ = P + (size_t)J * m * dc;
        for (int a = 0; a < d; ++a) {
          T left = conj(PI[(size_t)(loc * d + a) * dc + p]);
          T inner = zero<T>();
          for (int b = 0; b < d; ++b) inner = inner + B[a * d + b] * PJ[(size_t)(locj * d + b) * dc + q];
          acc = acc + left * inner;
        }
      }
    }
    cc[(((size_t)I * 5 + cdir) * dc + p) * dc + q] = acc;
  }
}

void launch_galerkin(const StencilView &fine, const ProlongView &P, void *coarse_coef, cudaStream_t s) {
  int nagg = (fine.nx / P.ax) * (fine.ny / P.ay);
  if (fine.t == F64) k_galerkin<double><<<nagg, 128, 0, s>>>((const double *)fine.coef, (const double *)P.P, (double *)coarse_coef, fine.nx, fine.ny, fine.d, P.ax, P.ay, P.dc);
  else if (fine.t == C64) k_galerkin<cdouble><<<nagg, 128, 0, s>>>((const cdouble *)fine.coef, (const cdouble *)P.P, (cdouble *)coarse_coef, fine.nx, fine.ny, fine.d, P.ax, P.ay, P.dc);
  else throw cuda_error{cudaErrorInvalidValue, "galerkin: FP64 only"};
  MLMC_LAUNCH_CHECK("k_galerkin");
}

// ------------------------------------------------------------------ dense Gauss-Jordan inverse
// Both kernels run the elimination in one cooperative launch (every block resident);
// block b owns rows [b R, (b + 1) R).  Rows are never swapped: at step q the pivot is the
// unused row with the largest |M[r][q]| (ties: the smaller r); after each step every
// block publishes its best candidate for the next column and a grid barrier (an atomic
// counter) separates the steps.  Every barrier wait is bounded (about a second): on
// timeout the block records MLMC_ERR_TIMEOUT and returns, and the others time out at their
// next wait.  Data written by other blocks is read through L2 (__ldcg).
//
// k_gj_inplace (n <= 4096; own rows in shared memory where they fit, else in place in M):
// in-place Gauss-Jordan on M = A (n x n).  Step q with pivot row p, a = M[p][q]: every
// other row i takes g = M[i][q] / a, M[i][c] -= g M[p][c] (c != q), M[i][q] = -g; row p is
// scaled (M[p][c] /= a, M[p][q] = 1 / a) by its owner at the start of the next step, so
// during a step all blocks read the unchanged pivot row while each writes only its own
// rows (kept in shared memory; a block publishes to M only its candidate for the next
// pivot, and all its rows at the end).  At the end M[piv_q][pos(c)] =
// A^-1[q][c] with pos(piv_q) = q (k_gj_extract_inplace).
//
// k_gj_coop (n > 4096): the same pivoting on work = [A | I] (n x 2n) in global memory,
// rows never scaled: every other row takes work[r][c] -= (work[r][q] / work[piv][q])
// work[piv][c] for c > q; row piv_q ends as work[piv_q][q] x [e_q | row q of A^-1]
// (k_gj_extract).
template <class T>
__global__ void k_gj_init(const T *A, T *work, int n) {
  size_t total = (size_t)n * 2 * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(t / (2 * n)), c = (int)(t % (2 * n));
    work[t] = c < n ? A[(size_t)r * n + c] : (c - n == r ? make<T>(1.0, 0.0) : zero<T>());
  }
}

constexpr int GJ_THREADS = 256;
constexpr int GJ_MAX_ROWS = 64;                 // rows per block (n <= 64 x blocks)
constexpr int GJ_COLS = 16;                     // k_gj_inplace: columns per thread (n <= 4096)
constexpr int GJ_ROWB = 8;                      // k_gj_inplace: rows updated together
constexpr long long GJ_WAIT_CYCLES = 2000000000LL;

__device__ inline double ldcg_d(const double *p) { return __ldcg(p); }
__device__ inline cdouble ldcg_d(const cdouble *p) {
  const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
  return {v.x, v.y};
}
__device__ inline float ldcg_d(const float *p) { return __ldcg(p); }
__device__ inline cfloat ldcg_d(const cfloat *p) {
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
  return {v.x, v.y};
}

// largest (mag, smaller row on ties) over the block; returns it in every thread
__device__ inline void gj_block_best(double &m, int &r, double *sm, int *sr) {
  sm[threadIdx.x] = m;
  sr[threadIdx.x] = r;
  __syncthreads();
  for (int o = GJ_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double m2 = sm[threadIdx.x + o];
      const int r2 = sr[threadIdx.x + o];
      if (m2 > sm[threadIdx.x] || (m2 == sm[threadIdx.x] && r2 < sr[threadIdx.x])) {
        sm[threadIdx.x] = m2;
        sr[threadIdx.x] = r2;
      }
    }
    __syncthreads();
  }
  m = sm[0];
  r = sr[0];
  __syncthreads();
}

// The same on an integer key: a magnitude m >= 0 orders like its bit pattern, so
// (key, row) = (bits(m), r) compares on the integer units (0 = none or zero); warp shuffles,
// then the warps' winners through shared memory.  Returns the winner in every thread.
__device__ inline unsigned long long gj_key(double m) {
  return m > 0.0 ? (unsigned long long)__double_as_longlong(m) : 0ull;
}
__device__ inline bool gj_better(unsigned long long k2, int r2, unsigned long long k1, int r1) {
  return k2 > k1 || (k2 == k1 && r2 < r1);
}
__device__ inline void gj_block_best_key(unsigned long long &key, int &row, unsigned long long *wk, int *wr) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
    const int r2 = __shfl_xor_sync(0xffffffffu, row, o);
    if (gj_better(k2, r2, key, row)) { key = k2; row = r2; }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { wk[warp] = key; wr[warp] = row; }
  __syncthreads();
  key = lane < (GJ_THREADS >> 5) ? wk[lane] : 0ull;
  row = lane < (GJ_THREADS >> 5) ? wr[lane] : 0x7fffffff;
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
    const int r2 = __shfl_xor_sync(0xffffffffu, row, o);
    if (gj_better(k2, r2, key, row)) { key = k2; row = r2; }
  }
  key = __shfl_sync(0xffffffffu, key, 0);
  row = __shfl_sync(0xffffffffu, row, 0);
  __syncthreads();                 // wk / wr free for the next call
}

// bounded grid barrier number `round` (1, 2, ...): false when the wait gave up
__device__ inline bool gj_grid_barrier(unsigned *bar, unsigned round, long long wait_cycles, int *err, int *fail_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    // release: the block's writes (ordered before this thread by the barrier above) are
    // visible to whoever acquires the count
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    const unsigned target = round * gridDim.x;
    const long long t0 = clock64();
    unsigned seen = 0;
    int failed = 0;
    for (unsigned it = 0;; ++it) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(bar) : "memory");
      if (seen >= target) break;
      if (clock64() - t0 > wait_cycles) {
        failed = 1;
        atomicExch(err, (int)MLMC_ERR_TIMEOUT);
        break;
      }
      if (it > 32) __nanosleep(32);
    }
    *fail_sh = failed;
  }
  __syncthreads();
  return *fail_sh == 0;
}

template <class T>
__global__ void __launch_bounds__(GJ_THREADS) k_gj_coop(T *work, int n, int rows, int *pivrow, int *used,
                                                      double *cand_mag, int *cand_row, unsigned *bar, int *err,
                                                      long long wait_cycles) {
  __shared__ double sm[GJ_THREADS];
  __shared__ int sr[GJ_THREADS];
  __shared__ T fr[GJ_MAX_ROWS];
  __shared__ int fail_sh;
  const int tid = threadIdx.x, G = gridDim.x;
  const int r0 = blockIdx.x * rows, r1 = min(n, r0 + rows);
  const size_t ld = (size_t)2 * n;
  unsigned round = 0;
  // candidates for column 0
  {
    double m = -1.0;
    int r = n;
    for (int rr = r0 + tid; rr < r1; rr += GJ_THREADS) {
      const double v = mag(ldcg_d(work + (size_t)rr * ld));
      if (v > m || (v == m && rr < r)) { m = v; r = rr; }
    }
    gj_block_best(m, r, sm, sr);
    if (tid == 0) { cand_mag[blockIdx.x] = m; cand_row[blockIdx.x] = r; }
    if (!gj_grid_barrier(bar, ++round, wait_cycles, err, &fail_sh)) return;
  }
  for (int q = 0; q < n; ++q) {
    const int par = q & 1;
    // the pivot: best of the blocks' candidates
    double m = -1.0;
    int piv = n;
    for (int b = tid; b < G; b += GJ_THREADS) {
      const double v = __ldcg(cand_mag + par * G + b);
      const int r = __ldcg(cand_row + par * G + b);
      if (v > m || (v == m && r < piv)) { m = v; piv = r; }
    }
    gj_block_best(m, piv, sm, sr);
    if (!(m > 0.0) || piv >= n) {
      if (blockIdx.x == 0 && tid == 0) atomicExch(err, 3);
      return;
    }
    if (blockIdx.x == 0 && tid == 0) pivrow[q] = piv;
    if (piv >= r0 && piv < r1 && tid == 0) used[piv] = 1;
    const T pv = ldcg_d(work + (size_t)piv * ld + q);
    // factors of the own rows (zero for the pivot row)
    for (int rr = r0 + tid; rr < r1; rr += GJ_THREADS)
      fr[rr - r0] = rr == piv ? zero<T>() : divide(ldcg_d(work + (size_t)rr * ld + q), pv);
    __syncthreads();
    for (int c = q + 1 + tid; c < 2 * n; c += GJ_THREADS) {
      const T pc = ldcg_d(work + (size_t)piv * ld + c);
      for (int rr = r0; rr < r1; ++rr) {
        if (rr == piv) continue;
        T *w = work + (size_t)rr * ld + c;
        *w = *w - fr[rr - r0] * pc;
      }
    }
    if (q + 1 == n) break;
    __syncthreads();
    // own candidate for column q + 1 (unused rows)
    m = -1.0;
    int cr = n;
    for (int rr = r0 + tid; rr < r1; rr += GJ_THREADS) {
      if (rr == piv || used[rr]) continue;
      const double v = mag(ldcg_d(work + (size_t)rr * ld + q + 1));
      if (v > m || (v == m && rr < cr)) { m = v; cr = rr; }
    }
    gj_block_best(m, cr, sm, sr);
    if (tid == 0) { cand_mag[(1 - par) * G + blockIdx.x] = m; cand_row[(1 - par) * G + blockIdx.x] = cr; }
    if (!gj_grid_barrier(bar, ++round, wait_cycles, err, &fail_sh)) return;
  }
}

// SMEM = false: the own rows are updated in place in M (initialised from A by the caller);
// nothing to publish or write back.
template <class T, bool SMEM>
__global__ void __launch_bounds__(GJ_THREADS) k_gj_inplace(const T *A, T *M, int n, int rows, int *pivrow,
                                                         double *cand_mag, int *cand_row, unsigned *bar, int *err,
                                                         long long wait_cycles) {
  extern __shared__ __align__(16) unsigned char gj_smem[];
  const int r0_ = blockIdx.x * rows;
  T *Ms = SMEM ? reinterpret_cast<T *>(gj_smem) : M + (size_t)r0_ * n;   // own rows, rows x n
  __shared__ unsigned long long wk[GJ_THREADS / 32];
  __shared__ int wr[GJ_THREADS / 32];
  __shared__ T fr[GJ_MAX_ROWS];
  __shared__ unsigned char used[GJ_MAX_ROWS];
  __shared__ int fail_sh;
  const int tid = threadIdx.x, G = gridDim.x;
  const int r0 = blockIdx.x * rows, nr = max(0, min(n, r0 + rows) - r0);
  unsigned long long *ckey = reinterpret_cast<unsigned long long *>(cand_mag);
  if (SMEM)
    for (int e = tid; e < nr * n; e += GJ_THREADS) Ms[e] = A[(size_t)r0 * n + e];
  for (int i = tid; i < GJ_MAX_ROWS; i += GJ_THREADS) used[i] = 0;
  __syncthreads();
  // this block's candidate for column q (unused own rows), published with its row, which
  // is the only row of the block that can become the next pivot
  auto candidate = [&](int col, int slot) {
    unsigned long long key = 0ull;
    int r = 0x7fffffff;
    for (int i = tid; i < nr; i += GJ_THREADS) {
      if (used[i]) continue;
      const unsigned long long k2 = gj_key(mag(Ms[(size_t)i * n + col]));
      if (gj_better(k2, r0 + i, key, r)) { key = k2; r = r0 + i; }
    }
    gj_block_best_key(key, r, wk, wr);
    if (tid == 0) { ckey[slot * G + blockIdx.x] = key; cand_row[slot * G + blockIdx.x] = r; }
    if (SMEM && r < n)
      for (int c = tid; c < n; c += GJ_THREADS) M[(size_t)r * n + c] = Ms[(size_t)(r - r0) * n + c];
  };
  unsigned round = 0;
  candidate(0, 0);
  if (!gj_grid_barrier(bar, ++round, wait_cycles, err, &fail_sh)) return;
  int prev = -1;
  for (int q = 0; q < n; ++q) {
    const int par = q & 1;
    unsigned long long key = 0ull;
    int p = 0x7fffffff;
    for (int b = tid; b < G; b += GJ_THREADS) {
      const unsigned long long k2 = __ldcg(ckey + par * G + b);
      const int r2 = __ldcg(cand_row + par * G + b);
      if (gj_better(k2, r2, key, p)) { key = k2; p = r2; }
    }
    gj_block_best_key(key, p, wk, wr);
    if (key == 0ull || p >= n) {
      if (blockIdx.x == 0 && tid == 0) atomicExch(err, 3);
      return;
    }
    if (blockIdx.x == 0 && tid == 0) pivrow[q] = p;
    // the previous pivot row, if it is ours: its deferred scaling
    if (prev >= r0 && prev < r0 + nr) {
      T *row = Ms + (size_t)(prev - r0) * n;
      const T ra = divide(make<T>(1.0, 0.0), row[q - 1]);     // one FP64 division per row
      __syncthreads();
      for (int c = tid; c < n; c += GJ_THREADS) row[c] = c == q - 1 ? ra : row[c] * ra;
      __syncthreads();
    }
    if (p >= r0 && p < r0 + nr && tid == 0) used[p - r0] = 1;
    // the pivot row: this thread's columns and the pivot, loaded together (one L2 latency)
    T pcs[GJ_COLS];
#pragma unroll
    for (int u = 0; u < GJ_COLS; ++u) {
      const int c = tid + u * GJ_THREADS;
      pcs[u] = c < n ? ldcg_d(M + (size_t)p * n + c) : zero<T>();
    }
    const T ra = divide(make<T>(1.0, 0.0), ldcg_d(M + (size_t)p * n + q));
    for (int i = tid; i < nr; i += GJ_THREADS) fr[i] = r0 + i == p ? zero<T>() : Ms[(size_t)i * n + q] * ra;
    __syncthreads();
    // own rows, up to GJ_ROWB at a time: all loads, then the FMAs, then the stores
#pragma unroll
    for (int u = 0; u < GJ_COLS; ++u) {
      const int c = tid + u * GJ_THREADS;
      if (c >= n) break;
      for (int i0 = 0; i0 < nr; i0 += GJ_ROWB) {
        T v[GJ_ROWB];
#pragma unroll
        for (int w = 0; w < GJ_ROWB; ++w)
          if (i0 + w < nr) v[w] = Ms[(size_t)(i0 + w) * n + c];
#pragma unroll
        for (int w = 0; w < GJ_ROWB; ++w) {
          const int i = i0 + w;
          if (i < nr && r0 + i != p) {
            v[w] = c == q ? zero<T>() - fr[i] : v[w] - fr[i] * pcs[u];
            Ms[(size_t)i * n + c] = v[w];
          }
        }
      }
    }
    prev = p;
    __syncthreads();
    if (q + 1 == n) break;
    candidate(q + 1, 1 - par);
    if (!gj_grid_barrier(bar, ++round, wait_cycles, err, &fail_sh)) return;
  }
  // every block has read the last pivot row: scale it, then publish all own rows
  if (!gj_grid_barrier(bar, ++round, wait_cycles, err, &fail_sh)) return;
  if (prev >= r0 && prev < r0 + nr) {
    T *row = Ms + (size_t)(prev - r0) * n;
    const T ra = divide(make<T>(1.0, 0.0), row[n - 1]);
    __syncthreads();
    for (int c = tid; c < n; c += GJ_THREADS) row[c] = c == n - 1 ? ra : row[c] * ra;
    __syncthreads();
  }
  if (SMEM)
    for (int e = tid; e < nr * n; e += GJ_THREADS) M[(size_t)r0 * n + e] = Ms[e];
}

// A^-1[q][c] = M[piv_q][pos(c)], pos(piv_j) = j
template <class T>
__global__ void k_gj_extract_inplace(const T *M, const int *pivrow, T *Ainv, int n) {
  size_t total = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / n), j = (int)(t % n);
    Ainv[(size_t)q * n + pivrow[j]] = M[(size_t)pivrow[q] * n + j];
  }
}

template <class T>
__global__ void k_gj_extract(const T *work, const int *pivrow, T *Ainv, int n) {
  size_t total = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / n), c = (int)(t % n);
    const int pr = pivrow[q];
    Ainv[t] = divide(work[(size_t)pr * 2 * n + n + c], work[(size_t)pr * 2 * n + q]);
  }
}

namespace {
struct GjScratch {
  size_t pivrow, used, cmag, crow, bar, total;
};
GjScratch gj_layout(int n, int G) {
  GjScratch L{};
  size_t o = 0;
  auto take = [&o](size_t bytes) { size_t at = o; o = (o + bytes + 255) / 256 * 256; return at; };
  L.pivrow = take((size_t)n * 4);
  L.used = take((size_t)n * 4);
  L.cmag = take((size_t)2 * G * 8);
  L.crow = take((size_t)2 * G * 4);
  L.bar = take(16);
  L.total = o;
  return L;
}
int gj_blocks(int n) {
  int dev = 0, sms = 0;
  MLMC_CUDA(cudaGetDevice(&dev));
  MLMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int G = std::min(sms, n);
  while ((n + G - 1) / G > GJ_MAX_ROWS) G *= 2;     // more blocks than SMs only for n > 64 x SMs
  return std::max(G, 1);
}
}  // namespace

size_t gauss_jordan_scratch_bytes(int n) { return gj_layout(n, gj_blocks(n)).total; }

constexpr size_t GJ_SMEM_MAX = 200 * 1024;      // own rows of k_gj_inplace in shared memory

// The dynamic shared-memory limit of k_gj_inplace, raised once per device to GJ_SMEM_MAX
// (a per-call value would race between host threads building hierarchies concurrently).
template <class T>
void gj_inplace_attrs() {
  static std::once_flag once[64];
  int dev = 0;
  MLMC_CUDA(cudaGetDevice(&dev));
  std::call_once(once[dev & 63], [] {
    check_cuda(cudaFuncSetAttribute(k_gj_inplace<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)GJ_SMEM_MAX),
               "cudaFuncSetAttribute(k_gj_inplace)");
  });
}

void launch_gauss_jordan(DType t, const void *A, void *Ainv, void *work, int n, int *err, void *scratch,
                         size_t scratch_bytes, cudaStream_t s) {
  const int G = gj_blocks(n);
  const GjScratch L = gj_layout(n, G);
  if (scratch_bytes < L.total) throw cuda_error{cudaErrorInvalidValue, "gauss_jordan: scratch too small"};
  int dev = 0, sms = 0;
  MLMC_CUDA(cudaGetDevice(&dev));
  MLMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  char *sc = (char *)scratch;
  MLMC_CUDA(cudaMemsetAsync(sc, 0, L.total, s));
  int *pivrow = (int *)(sc + L.pivrow), *used = (int *)(sc + L.used), *crow = (int *)(sc + L.crow);
  double *cmag = (double *)(sc + L.cmag);
  unsigned *bar = (unsigned *)(sc + L.bar);
  long long wait = GJ_WAIT_CYCLES;
  int rows = (n + G - 1) / G;
  MLMC_DISPATCH(t, T, {
    const unsigned g = grid_for((size_t)n * n, 256);
    T *wk = (T *)work;
    const size_t smem = (size_t)rows * n * sizeof(T);
    int per_sm = 0;
    const T *a = (const T *)A;
    if (smem <= GJ_SMEM_MAX && n <= GJ_COLS * GJ_THREADS) {
      gj_inplace_attrs<T>();
      MLMC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_inplace<T, true>, GJ_THREADS, smem));
      if ((long long)per_sm * sms < G) throw cuda_error{cudaErrorInvalidValue, "gauss_jordan: blocks cannot be resident"};
      void *args[] = {&a, &wk, &n, &rows, &pivrow, &cmag, &crow, &bar, &err, &wait};
      MLMC_CUDA(cudaLaunchCooperativeKernel((const void *)k_gj_inplace<T, true>, dim3(G), dim3(GJ_THREADS), args,
                                            smem, s));
      k_gj_extract_inplace<T><<<g, 256, 0, s>>>((const T *)work, pivrow, (T *)Ainv, n);
    } else if (n <= GJ_COLS * GJ_THREADS) {
      // the same elimination on the rows in place in global memory (n x n, L2-resident for
      // the coarsest sizes of the hierarchies)
      MLMC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_inplace<T, false>, GJ_THREADS, 0));
      if ((long long)per_sm * sms < G) throw cuda_error{cudaErrorInvalidValue, "gauss_jordan: blocks cannot be resident"};
      MLMC_CUDA(cudaMemcpyAsync(wk, a, (size_t)n * n * sizeof(T), cudaMemcpyDeviceToDevice, s));
      void *args[] = {&a, &wk, &n, &rows, &pivrow, &cmag, &crow, &bar, &err, &wait};
      MLMC_CUDA(cudaLaunchCooperativeKernel((const void *)k_gj_inplace<T, false>, dim3(G), dim3(GJ_THREADS), args,
                                            0, s));
      k_gj_extract_inplace<T><<<g, 256, 0, s>>>((const T *)work, pivrow, (T *)Ainv, n);
    } else {
      MLMC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_coop<T>, GJ_THREADS, 0));
      if ((long long)per_sm * sms < G) throw cuda_error{cudaErrorInvalidValue, "gauss_jordan: blocks cannot be resident"};
      const unsigned g2 = grid_for((size_t)n * 2 * n, 256);
      k_gj_init<T><<<g2, 256, 0, s>>>((const T *)A, wk, n);
      void *args[] = {&wk, &n, &rows, &pivrow, &used, &cmag, &crow, &bar, &err, &wait};
      MLMC_CUDA(cudaLaunchCooperativeKernel((const void *)k_gj_coop<T>, dim3(G), dim3(GJ_THREADS), args, 0, s));
      k_gj_extract<T><<<g, 256, 0, s>>>((const T *)work, pivrow, (T *)Ainv, n);
    }
  });
  MLMC_LAUNCH_CHECK("gauss_jordan");
}

// sum of the diagonal in index order, into FP64 (complex)
template <class T>
__global__ void k_trace(const T *A, int n, double *out) {
  if (threadIdx.x || blockIdx.x) return;
  double r = 0.0, i = 0.0;
  for (int k = 0; k < n; ++k) { r += (double)re(A[(size_t)k * n + k]); i += (double)im(A[(size_t)k * n + k]); }
  out[0] = r;
  out[1] = i;
}

void launch_trace(DType t, const void *A, int n, void *out, cudaStream_t s) {
  MLMC_DISPATCH(t, T, k_trace<T><<<1, 32, 0, s>>>((const T *)A, n, (double *)out));
  MLMC_LAUNCH_CHECK("k_trace");
}

// ------------------------------------------------------------------ dense coarsest apply
// Y[i][c] = sum_j Ainv[i][j] B[j][c].  64 x 32 output tiles, 128 threads with
// a 4 x 4 register tile each, j in steps of 16 through shared memory; the j
// range is split over `splits` blocks (grid.z) writing partial tiles that a
// second kernel adds in split order.
constexpr int DA_BM = 64, DA_BN = 32, DA_BK = 16;

template <class T>
__global__ void __launch_bounds__(128) k_dense_apply(const T *__restrict__ A, const T *__restrict__ B, T *__restrict__ Y,
                                                     int n, int k, int jchunk) {
  __shared__ T As[DA_BK][DA_BM + 1];
  __shared__ T Bs[DA_BK][DA_BN];
  const int tx = threadIdx.x % 8, ty = threadIdx.x / 8;        // 8 x 16 threads, 4 x 4 outputs each
  const int row0 = blockIdx.y * DA_BM, col0 = blockIdx.x * DA_BN;
  const int j_begin = blockIdx.z * jchunk, j_end = min(n, j_begin + jchunk);
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = zero<T>();
  for (int j0 = j_begin; j0 < j_end; j0 += DA_BK) {
    for (int e = threadIdx.x; e < DA_BK * DA_BM; e += 128) {
      int r = e / DA_BK, jj = e % DA_BK;
      int gi = row0 + r, gj = j0 + jj;
      As[jj][r] = (gi < n && gj < j_end) ? A[(size_t)gi * n + gj] : zero<T>();
    }
    for (int e = threadIdx.x; e < DA_BK * DA_BN; e += 128) {
      int jj = e / DA_BN, c = e % DA_BN;
      int gj = j0 + jj, gc = col0 + c;
      Bs[jj][c] = (gj < j_end && gc < k) ? B[(size_t)gj * k + gc] : zero<T>();
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < DA_BK; ++jj) {
      T av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[jj][ty * 4 + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[jj][tx * 4 + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = acc[a][b] + av[a] * bv[b];
    }
    __syncthreads();
  }
  T *Yz = Y + (size_t)blockIdx.z * n * k;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int r = row0 + ty * 4 + a, c = col0 + tx * 4 + b;
      if (r < n && c < k) Yz[(size_t)r * k + c] = acc[a][b];
    }
}

// Narrow blocks (k <= 8, e.g. the test vectors of the setup's bootstrap cycles): one warp
// per row of Ainv, the lanes take j = lane, lane + 32, ... for all k columns, then a
// fixed shuffle tree per column (deterministic).  Reads Ainv once; no padded columns.
template <class T>
__device__ inline T shfl_xor_t(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
template <>
__device__ inline cdouble shfl_xor_t(cdouble v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.re, o), __shfl_xor_sync(0xffffffffu, v.im, o)};
}
template <>
__device__ inline cfloat shfl_xor_t(cfloat v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.re, o), __shfl_xor_sync(0xffffffffu, v.im, o)};
}

template <class T, int KN>
__global__ void __launch_bounds__(256) k_dense_apply_narrow(const T *__restrict__ A, const T *__restrict__ B,
                                                            T *__restrict__ Y, int n, int k) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    T acc[KN];
#pragma unroll
    for (int c = 0; c < KN; ++c) acc[c] = zero<T>();
    const T *Ai = A + (size_t)i * n;
    for (int j = lane; j < n; j += 32) {
      const T a = Ai[j];
      const T *Bj = B + (size_t)j * k;
#pragma unroll
      for (int c = 0; c < KN; ++c)
        if (c < k) acc[c] = acc[c] + a * Bj[c];
    }
#pragma unroll
    for (int c = 0; c < KN; ++c) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[c] = acc[c] + shfl_xor_t(acc[c], o);
    }
    if (lane < k) {
      T out = acc[0];
#pragma unroll
      for (int c = 1; c < KN; ++c)
        if (c == lane) out = acc[c];
      Y[(size_t)i * k + lane] = out;
    }
  }
}

template <class T>
__global__ void k_dense_sum(const T *part, int splits, size_t count, T *Y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    T s = part[i];
    for (int z = 1; z < splits; ++z) s = s + part[(size_t)z * count + i];
    Y[i] = s;
  }
}

int dense_apply_splits(int n, int k) {
  int tiles = ((k + DA_BN - 1) / DA_BN) * ((n + DA_BM - 1) / DA_BM);
  int s = 152 / (tiles > 0 ? tiles : 1);
  if (s > 8) s = 8;
  if (s < 1) s = 1;
  while (s > 1 && n / s < 4 * DA_BK) --s;
  return s;
}

void launch_dense_apply(DType t, const void *Ainv, const void *B, void *Y, int n, int k, void *part, cudaStream_t s) {
  if (k <= 8) {
    const unsigned g = resident_grid(((size_t)n * 32 + 255) / 256, 8);
    MLMC_DISPATCH(t, T, {
      if (k <= 4)
        k_dense_apply_narrow<T, 4><<<g, 256, 0, s>>>((const T *)Ainv, (const T *)B, (T *)Y, n, k);
      else
        k_dense_apply_narrow<T, 8><<<g, 256, 0, s>>>((const T *)Ainv, (const T *)B, (T *)Y, n, k);
    });
    MLMC_LAUNCH_CHECK("k_dense_apply_narrow");
    return;
  }
  int splits = part ? dense_apply_splits(n, k) : 1;
  int jchunk = (n + splits - 1) / splits;
  jchunk = (jchunk + DA_BK - 1) / DA_BK * DA_BK;
  dim3 g((k + DA_BN - 1) / DA_BN, (n + DA_BM - 1) / DA_BM, splits);
  MLMC_DISPATCH(t, T, {
    if (splits == 1) {
      k_dense_apply<T><<<g, 128, 0, s>>>((const T *)Ainv, (const T *)B, (T *)Y, n, k, jchunk);
    } else {
      k_dense_apply<T><<<g, 128, 0, s>>>((const T *)Ainv, (const T *)B, (T *)part, n, k, jchunk);
      size_t cnt = (size_t)n * k;
      k_dense_sum<T><<<grid_for(cnt, 256), 256, 0, s>>>((const T *)part, splits, cnt, (T *)Y);
    }
  });
  MLMC_LAUNCH_CHECK("k_dense_apply");
}

}  // namespace mlmc
