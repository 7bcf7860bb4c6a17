// Setup-time kernels: inverse self blocks for the smoother, per-aggregate
// modified Gram-Schmidt (P blocks), Galerkin coarse stencils P^* A P, dense
// Gauss-Jordan inverse and trace of the coarsest operator, and the dense
// coarsest-level apply used inside every multigrid cycle.
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
// work = [A | I] (n x 2n, row-major).  Per pivot column p: pick the largest
// |entry| in rows >= p, swap it to row p, scale row p, save column p, then
// eliminate column p from every other row.
template <class T>
__global__ void k_gj_init(const T *A, T *work, int n) {
  size_t total = (size_t)n * 2 * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(t / (2 * n)), c = (int)(t % (2 * n));
    work[t] = c < n ? A[(size_t)r * n + c] : (c - n == r ? make<T>(1.0, 0.0) : zero<T>());
  }
}

template <class T>
__global__ void k_gj_pivot(T *work, int n, int p, int *err, T *col) {
  __shared__ double best[256];
  __shared__ int where[256];
  double b = -1.0;
  int w = p;
  for (int r = p + threadIdx.x; r < n; r += blockDim.x) {
    double m = mag(work[(size_t)r * 2 * n + p]);
    if (m > b) { b = m; w = r; }
  }
  best[threadIdx.x] = b;
  where[threadIdx.x] = w;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      if (best[threadIdx.x + o] > best[threadIdx.x] ||
          (best[threadIdx.x + o] == best[threadIdx.x] && where[threadIdx.x + o] < where[threadIdx.x])) {
        best[threadIdx.x] = best[threadIdx.x + o];
        where[threadIdx.x] = where[threadIdx.x + o];
      }
    }
    __syncthreads();
  }
  int piv = where[0];
  if (best[0] <= 0.0) { if (threadIdx.x == 0) atomicExch(err, 3); return; }
  // swap rows p and piv, then scale row p by 1 / pivot
  T pv = work[(size_t)piv * 2 * n + p];
  __syncthreads();
  for (int c = threadIdx.x; c < 2 * n; c += blockDim.x) {
    T a = work[(size_t)p * 2 * n + c], bb = work[(size_t)piv * 2 * n + c];
    work[(size_t)piv * 2 * n + c] = a;
    work[(size_t)p * 2 * n + c] = divide(bb, pv);
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) col[r] = work[(size_t)r * 2 * n + p];
}

template <class T>
__global__ void k_gj_eliminate(T *work, int n, int p, const T *col) {
  size_t width = (size_t)2 * n - p;
  size_t total = (size_t)n * width;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(t / width);
    int c = p + (int)(t % width);
    if (r == p) continue;
    T f = col[r];
    work[(size_t)r * 2 * n + c] = work[(size_t)r * 2 * n + c] - f * work[(size_t)p * 2 * n + c];
  }
}

template <class T>
__global__ void k_gj_extract(const T *work, T *Ainv, int n) {
  size_t total = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(t / n), c = (int)(t % n);
    Ainv[t] = work[(size_t)r * 2 * n + n + c];
  }
}

void launch_gauss_jordan(DType t, const void *A, void *Ainv, void *work, int n, int *err, void *colbuf,
                         cudaStream_t s) {
  MLMC_DISPATCH(t, T, {
    unsigned g = grid_for((size_t)n * 2 * n, 256);
    k_gj_init<T><<<g, 256, 0, s>>>((const T *)A, (T *)work, n);
    for (int p = 0; p < n; ++p) {
      k_gj_pivot<T><<<1, 256, 0, s>>>((T *)work, n, p, err, (T *)colbuf);
      k_gj_eliminate<T><<<g, 256, 0, s>>>((T *)work, n, p, (const T *)colbuf);
    }
    k_gj_extract<T><<<g, 256, 0, s>>>((const T *)work, (T *)Ainv, n);
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
