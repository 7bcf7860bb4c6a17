// Per-column kernels of the batched flexible GMRES (Saad, Alg. 9.6): every
// column of a vector block is an independent system, and its small Hessenberg
// least-squares problem (Givens rotations, triangular solve) is handled by one
// thread in FP64, as are the coefficient rescalings of the fixed-length FGMRES that
// keeps its basis unnormalised.  Also: sample combination and accumulation (Secs. 2-3), the
// fine-operator builders (Examples 5.1 and 5.3) and a dense scatter of the
// coarsest operator.
#include "mlmc_internal.cuh"

namespace mlmc {

__device__ inline double cabs_(double a) { return fabs(a); }
__device__ inline double cabs_(cdouble a) { return sqrt(a.re * a.re + a.im * a.im); }
__device__ inline double creal_(double a) { return a; }
__device__ inline double creal_(cdouble a) { return a.re; }
template <class H> __device__ inline H hdiv(H a, H b);
template <> __device__ inline double hdiv<double>(double a, double b) { return a / b; }
template <> __device__ inline cdouble hdiv<cdouble>(cdouble a, cdouble b) {
  double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
template <class H> __device__ inline H hreal(double v) { return make<H>(v, 0.0); }

// sc (optional): norms s_i of the unnormalised basis vectors of the fixed-length
// variant (see k_multidot_reduce); s_0 = |b|.
template <class H>
__global__ void k_arnoldi_init(H *g, double *bnorm, double *invnrm, int *active, int *jdone, int k,
                               double tol, int first, int *nactive, double *sc) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const double g0 = creal_(g[c]);
  const bool finite = isfinite(g0);
  double beta = finite ? sqrt(fmax(g0, 0.0)) : 0.0;
  if (first) bnorm[c] = beta;
  g[c] = hreal<H>(beta);
  jdone[c] = 0;
  int a = finite && beta > 0.0 && beta > tol * bnorm[c];
  active[c] = a;
  invnrm[c] = a ? 1.0 / beta : 0.0;
  if (sc) sc[c] = beta > 0.0 ? beta : 1.0;
  if (a) atomicAdd(nactive, 1);
  else if (!finite) atomicAdd(nactive, NONFINITE_COLUMN);    // a residual that is NaN or infinite
}

// y_i /= s_i for the computed rows: x = sum_i z_i y_i with z_i built from u_i.
template <class H>
__global__ void k_lazy_y(H *y, const double *sc, const int *jdone, int m, int k) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * k) return;
  const int i = t / k, c = t - (t / k) * k;
  if (i < jdone[c]) y[t] = y[t] * hreal<H>(1.0 / sc[t]);
}

// Hessenberg column j of column c lives at H[(j*(m+1) + i)*k + c], i = 0..j+1.
// On entry H[j][j+1] holds |w|^2 from a column dot.
// sc (optional, the unnormalised variant): the new basis vector keeps its norm,
// s_{j+1} = |u_{j+1}|, and the Hessenberg entry is |u_{j+1}| / s_j.
template <class H>
__global__ void k_arnoldi_step(H *Hm, H *cs, H *sn, H *g, int j, int m, int k, int *active, int *jdone,
                               const double *bnorm, double tol, double *invnrm, double *resid, int *nactive,
                               int fixed, double *sc) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  H *h = Hm + (size_t)j * (m + 1) * k + c;
  if (!active[c]) {
    invnrm[c] = 0.0;
    if (sc) sc[(size_t)(j + 1) * k + c] = 1.0;   // its vectors are zero: any finite scale
    return;
  }
  double nrm = sqrt(fmax(creal_(h[(size_t)(j + 1) * k]), 0.0));
  invnrm[c] = nrm > 0.0 ? 1.0 / nrm : 0.0;
  if (sc) {
    sc[(size_t)(j + 1) * k + c] = nrm > 0.0 ? nrm : 1.0;
    nrm = nrm / sc[(size_t)j * k + c];
  }
  h[(size_t)(j + 1) * k] = hreal<H>(nrm);
  for (int i = 0; i < j; ++i) {
    H a = h[(size_t)i * k], b = h[(size_t)(i + 1) * k];
    H ci = cs[(size_t)i * k + c], si = sn[(size_t)i * k + c];
    h[(size_t)i * k] = conj(ci) * a + conj(si) * b;
    h[(size_t)(i + 1) * k] = -(si * a) + ci * b;
  }
  H a = h[(size_t)j * k], b = h[(size_t)(j + 1) * k];
  double den = sqrt(cabs_(a) * cabs_(a) + cabs_(b) * cabs_(b));
  H cj, sj;
  if (den > 0.0) {
    cj = hdiv(a, hreal<H>(den));
    sj = hdiv(b, hreal<H>(den));
  } else {
    cj = hreal<H>(1.0);
    sj = hreal<H>(0.0);
  }
  cs[(size_t)j * k + c] = cj;
  sn[(size_t)j * k + c] = sj;
  h[(size_t)j * k] = hreal<H>(den);
  h[(size_t)(j + 1) * k] = hreal<H>(0.0);
  H gj = g[(size_t)j * k + c];
  g[(size_t)(j + 1) * k + c] = -(sj * gj);
  g[(size_t)j * k + c] = conj(cj) * gj;
  jdone[c] = j + 1;
  double r = cabs_(g[(size_t)(j + 1) * k + c]);
  resid[c] = r;
  bool still = fixed ? (nrm > 0.0 && den > 0.0) : (r > tol * bnorm[c] && den > 0.0 && nrm > 0.0);
  if (!still) {
    active[c] = 0;
    invnrm[c] = 0.0;
  } else {
    atomicAdd(nactive, 1);
  }
}

// y = R^{-1} g over the first jdone[c] rows; y_i = 0 beyond.
template <class H>
__global__ void k_trisolve(const H *Hm, const H *g, H *y, const int *jdone, int m, int k) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  int J = jdone[c];
  for (int i = m - 1; i >= 0; --i) {
    if (i >= J) {
      y[(size_t)i * k + c] = hreal<H>(0.0);
      continue;
    }
    H s = g[(size_t)i * k + c];
    for (int l = i + 1; l < J; ++l) s = s - Hm[((size_t)l * (m + 1) + i) * k + c] * y[(size_t)l * k + c];
    y[(size_t)i * k + c] = hdiv(s, Hm[((size_t)i * (m + 1) + i) * k + c]);
  }
}

template <class H>
__global__ void k_add_acc(H *dst, const H *src, int count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = dst[i] + src[i];
}

void launch_arnoldi_init(int hc, void *g, double *bnorm, double *invnrm, int *active, int *jdone, int k,
                         double tol, int first, int *nactive, cudaStream_t s, double *sc) {
  unsigned gr = (k + 63) / 64;
  if (hc) k_arnoldi_init<cdouble><<<gr, 64, 0, s>>>((cdouble *)g, bnorm, invnrm, active, jdone, k, tol, first, nactive,
                                                     sc);
  else k_arnoldi_init<double><<<gr, 64, 0, s>>>((double *)g, bnorm, invnrm, active, jdone, k, tol, first, nactive, sc);
  MLMC_LAUNCH_CHECK("k_arnoldi_init");
}


void launch_lazy_y(int hc, void *y, const double *sc, const int *jdone, int m, int k, cudaStream_t s) {
  unsigned gr = (m * k + 127) / 128;
  if (hc) k_lazy_y<cdouble><<<gr, 128, 0, s>>>((cdouble *)y, sc, jdone, m, k);
  else k_lazy_y<double><<<gr, 128, 0, s>>>((double *)y, sc, jdone, m, k);
  MLMC_LAUNCH_CHECK("k_lazy_y");
}

void launch_arnoldi_step(int hc, void *H, void *cs, void *sn, void *g, int j, int m, int k, int *active,
                         int *jdone, const double *bnorm, double tol, double *invnrm, double *resid,
                         int *nactive, int fixed, cudaStream_t s, double *sc) {
  unsigned gr = (k + 63) / 64;
  if (hc) k_arnoldi_step<cdouble><<<gr, 64, 0, s>>>((cdouble *)H, (cdouble *)cs, (cdouble *)sn, (cdouble *)g, j, m, k,
                                                     active, jdone, bnorm, tol, invnrm, resid, nactive, fixed, sc);
  else k_arnoldi_step<double><<<gr, 64, 0, s>>>((double *)H, (double *)cs, (double *)sn, (double *)g, j, m, k,
                                                 active, jdone, bnorm, tol, invnrm, resid, nactive, fixed, sc);
  MLMC_LAUNCH_CHECK("k_arnoldi_step");
}

void launch_trisolve(int hc, const void *H, const void *g, void *y, const int *jdone, int m, int k, cudaStream_t s) {
  unsigned gr = (k + 63) / 64;
  if (hc) k_trisolve<cdouble><<<gr, 64, 0, s>>>((const cdouble *)H, (const cdouble *)g, (cdouble *)y, jdone, m, k);
  else k_trisolve<double><<<gr, 64, 0, s>>>((const double *)H, (const double *)g, (double *)y, jdone, m, k);
  MLMC_LAUNCH_CHECK("k_trisolve");
}

void launch_add_acc(int hc, void *dst, const void *src, int count, cudaStream_t s) {
  unsigned gr = (count + 127) / 128;
  if (hc) k_add_acc<cdouble><<<gr, 128, 0, s>>>((cdouble *)dst, (const cdouble *)src, count);
  else k_add_acc<double><<<gr, 128, 0, s>>>((double *)dst, (const double *)src, count);
  MLMC_LAUNCH_CHECK("k_add_acc");
}

template <class H>
__global__ void k_col_factor(const H *dot, double *alpha, double scale, int k) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  double v = fabs(creal_(dot[c]));
  alpha[c] = v > 0.0 ? scale / v : 0.0;
}

void launch_col_factor(int hc, const void *dot, double *alpha, double scale, int k, cudaStream_t s) {
  unsigned gr = (k + 63) / 64;
  if (hc) k_col_factor<cdouble><<<gr, 64, 0, s>>>((const cdouble *)dot, alpha, scale, k);
  else k_col_factor<double><<<gr, 64, 0, s>>>((const double *)dot, alpha, scale, k);
  MLMC_LAUNCH_CHECK("k_col_factor");
}

// ------------------------------------------------------------------ samples
template <class H>
__global__ void k_sample_combine(const H *a, const H *b, cdouble *out, int k) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  H v = b ? a[c] - b[c] : a[c];
  out[c] = cdouble{creal_(v), (double)im(v)};
}

void launch_sample_combine(int hc, const void *a, const void *b, void *out, int k, cudaStream_t s) {
  unsigned gr = (k + 63) / 64;
  if (hc) k_sample_combine<cdouble><<<gr, 64, 0, s>>>((const cdouble *)a, (const cdouble *)b, (cdouble *)out, k);
  else k_sample_combine<double><<<gr, 64, 0, s>>>((const double *)a, (const double *)b, (cdouble *)out, k);
  MLMC_LAUNCH_CHECK("k_sample_combine");
}

// Running (N, mean, M2) of the level's samples, updated with one block of k samples: the block's own mean and M2 = sum |s - mean_b|^2 by a fixed-order tree
// (deterministic), then the pairwise merge of Chan, Golub and LeVeque:
//   N = Na + Nb,  d = mean_b - mean_a,  mean = mean_a + d Nb / N,
//   M2 = M2_a + M2_b + |d|^2 Na Nb / N.
// M2 / (N - 1) is the unbiased complex variance E|s - E s|^2.
__device__ inline void block_tree_sum(double *a, double *b) {
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      a[threadIdx.x] += a[threadIdx.x + o];
      b[threadIdx.x] += b[threadIdx.x + o];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_accumulate(const cdouble *smp, int k, double *acc) {
  __shared__ double sr[256], si[256];
  const int t = threadIdx.x;
  // thread t holds samples t, t + 256, ... (summed in that order), then a fixed tree
  double re = 0.0, im = 0.0;
  for (int i = t; i < k; i += 256) {
    re += smp[i].re;
    im += smp[i].im;
  }
  sr[t] = re;
  si[t] = im;
  __syncthreads();
  block_tree_sum(sr, si);
  const double mbr = sr[0] / k, mbi = si[0] / k;
  __syncthreads();
  double q = 0.0;
  for (int i = t; i < k; i += 256) {
    const double dr = smp[i].re - mbr, di = smp[i].im - mbi;
    q += dr * dr + di * di;
  }
  sr[t] = q;
  si[t] = 0.0;
  __syncthreads();
  block_tree_sum(sr, si);
  if (t == 0) {
    const double na = acc[0], nb = (double)k, n = na + nb;
    const double er = mbr - acc[1], ei = mbi - acc[2];
    acc[1] += er * nb / n;
    acc[2] += ei * nb / n;
    acc[3] += sr[0] + (er * er + ei * ei) * na * nb / n;
    acc[0] = n;
  }
}

void launch_accumulate(const void *samples, int k, double *acc, cudaStream_t s) {
  if (k < 1 || k > 4096) throw cuda_error{cudaErrorInvalidValue, "k_accumulate: 1 <= k <= 4096"};
  k_accumulate<<<1, 256, 0, s>>>((const cdouble *)samples, k, acc);
  MLMC_LAUNCH_CHECK("k_accumulate");
}

// ------------------------------------------------------------------ fine operators
// Example 5.1: diagonal 4 + shift, -1 to each neighbour; Dirichlet drops links leaving the grid.
__global__ void k_build_laplace(double *coef, int nx, int ny, double shift, int periodic) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nx * ny) return;
  int i = s % nx, j = s / nx;
  double *B = coef + (size_t)s * 5;
  B[0] = 4.0 + shift;
  B[1] = (periodic || i + 1 < nx) ? -1.0 : 0.0;
  B[2] = (periodic || i > 0) ? -1.0 : 0.0;
  B[3] = (periodic || j + 1 < ny) ? -1.0 : 0.0;
  B[4] = (periodic || j > 0) ? -1.0 : 0.0;
}

void launch_build_laplace(double *coef, int nx, int ny, double shift, int periodic, cudaStream_t s) {
  k_build_laplace<<<(nx * ny + 255) / 256, 256, 0, s>>>(coef, nx, ny, shift, periodic);
  MLMC_LAUNCH_CHECK("k_build_laplace");
}

// Example 5.3, Eq. schwinger_coupling with s1 = [[0,1],[1,0]], s2 = [[0,i],[-i,0]]:
//   +x: -U_x(s) (I - s1), -x: -conj(U_x(s-x)) (I + s1), +y: -U_y(s) (I - s2), -y: -conj(U_y(s-y)) (I + s2).
__global__ void k_build_wilson(cdouble *coef, const cdouble *links, int nx, int ny, double mass) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  int n = nx * ny;
  if (s >= n) return;
  int i = s % nx, j = s / nx;
  int xm = j * nx + (i == 0 ? nx - 1 : i - 1);
  int ym = (j == 0 ? ny - 1 : j - 1) * nx + i;
  cdouble ux = links[s], uy = links[n + s];
  cdouble uxm = conj(links[xm]), uym = conj(links[n + ym]);
  // 2x2 spin matrices, row-major
  const cdouble one = {1, 0}, zer = {0, 0}, I = {0, 1};
  cdouble s1[4] = {zer, one, one, zer};
  cdouble s2[4] = {zer, I, -I, zer};
  cdouble id[4] = {one, zer, zer, one};
  cdouble *B = coef + (size_t)s * 5 * 4;
  for (int e = 0; e < 4; ++e) {
    B[0 * 4 + e] = (e == 0 || e == 3) ? cdouble{4.0 + mass, 0.0} : zer;
    B[1 * 4 + e] = -(ux * (id[e] - s1[e]));
    B[2 * 4 + e] = -(uxm * (id[e] + s1[e]));
    B[3 * 4 + e] = -(uy * (id[e] - s2[e]));
    B[4 * 4 + e] = -(uym * (id[e] + s2[e]));
  }
}

void launch_build_wilson(cdouble *coef, const cdouble *links, int nx, int ny, double mass, cudaStream_t s) {
  k_build_wilson<<<(nx * ny + 127) / 128, 128, 0, s>>>(coef, links, nx, ny, mass);
  MLMC_LAUNCH_CHECK("k_build_wilson");
}

// ------------------------------------------------------------------ dense scatter
template <class T>
__global__ void k_stencil_to_dense_add(const T *coef, T *dense, int nx, int ny, int d, int dir) {
  int nsite = nx * ny;
  int n = nsite * d;
  size_t total = (size_t)nsite * d * d;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    int s = (int)(t / (d * d));
    int r = (int)(t / d) % d, c = (int)(t % d);
    int i = s % nx, j = s / nx;
    int nb = s;
    if (dir == 1) nb = j * nx + (i + 1) % nx;
    if (dir == 2) nb = j * nx + (i + nx - 1) % nx;
    if (dir == 3) nb = ((j + 1) % ny) * nx + i;
    if (dir == 4) nb = ((j + ny - 1) % ny) * nx + i;
    T *dst = dense + (size_t)(s * d + r) * n + nb * d + c;
    *dst = *dst + coef[((size_t)s * 5 + dir) * d * d + r * d + c];
  }
}

void launch_stencil_to_dense(const StencilView &A, void *dense, cudaStream_t s) {
  size_t n = (size_t)A.nx * A.ny * A.d;
  MLMC_CUDA(cudaMemsetAsync(dense, 0, n * n * dtype_size(A.t), s));
  MLMC_DISPATCH(A.t, T, {
    // one launch per direction: directions that meet on the same entry add in order
    for (int dir = 0; dir < 5; ++dir)
      k_stencil_to_dense_add<T><<<grid_for((size_t)A.nx * A.ny * A.d * A.d, 256), 256, 0, s>>>(
          (const T *)A.coef, (T *)dense, A.nx, A.ny, A.d, dir);
  });
  MLMC_LAUNCH_CHECK("k_stencil_to_dense");
}

}  // namespace mlmc
