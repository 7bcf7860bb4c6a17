// Internal header of libmlmc: scalar types, dtype dispatch and the launcher
// declarations shared by the translation units.  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

namespace mlmc {

// ----------------------------------------------------------------- scalars
struct __align__(16) cdouble { double re, im; };
struct __align__(8) cfloat { float re, im; };

// element type of a vector block / operator storage
enum DType : int { F64 = 0, F32 = 1, C64 = 2, C32 = 3 };
inline bool dtype_complex(DType t) { return t == C64 || t == C32; }
inline size_t dtype_size(DType t) { return t == F64 ? 8 : t == F32 ? 4 : t == C64 ? 16 : 8; }
inline DType dtype_lower(DType t) { return t == F64 ? F32 : t == C64 ? C32 : t; }

template <class T> struct real_of { typedef T type; };
template <> struct real_of<cdouble> { typedef double type; };
template <> struct real_of<cfloat> { typedef float type; };

__host__ __device__ inline double re(double a) { return a; }
__host__ __device__ inline float re(float a) { return a; }
__host__ __device__ inline double re(cdouble a) { return a.re; }
__host__ __device__ inline float re(cfloat a) { return a.re; }
__host__ __device__ inline double im(double) { return 0.0; }
__host__ __device__ inline float im(float) { return 0.0f; }
__host__ __device__ inline double im(cdouble a) { return a.im; }
__host__ __device__ inline float im(cfloat a) { return a.im; }

template <class T> __host__ __device__ inline T zero() { return T(0); }
template <> __host__ __device__ inline cdouble zero<cdouble>() { return cdouble{0.0, 0.0}; }
template <> __host__ __device__ inline cfloat zero<cfloat>() { return cfloat{0.0f, 0.0f}; }

template <class T> __host__ __device__ inline T make(double r, double i);
template <> __host__ __device__ inline double make<double>(double r, double) { return r; }
template <> __host__ __device__ inline float make<float>(double r, double) { return (float)r; }
template <> __host__ __device__ inline cdouble make<cdouble>(double r, double i) { return cdouble{r, i}; }
template <> __host__ __device__ inline cfloat make<cfloat>(double r, double i) { return cfloat{(float)r, (float)i}; }

__host__ __device__ inline cdouble operator+(cdouble a, cdouble b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ inline cdouble operator-(cdouble a, cdouble b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ inline cdouble operator-(cdouble a) { return {-a.re, -a.im}; }
__host__ __device__ inline cdouble operator*(cdouble a, cdouble b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ inline cdouble operator*(double s, cdouble a) { return {s * a.re, s * a.im}; }
__host__ __device__ inline cfloat operator+(cfloat a, cfloat b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ inline cfloat operator-(cfloat a, cfloat b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ inline cfloat operator-(cfloat a) { return {-a.re, -a.im}; }
__host__ __device__ inline cfloat operator*(cfloat a, cfloat b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ inline cfloat operator*(float s, cfloat a) { return {s * a.re, s * a.im}; }

__host__ __device__ inline double conj(double a) { return a; }
__host__ __device__ inline float conj(float a) { return a; }
__host__ __device__ inline cdouble conj(cdouble a) { return {a.re, -a.im}; }
__host__ __device__ inline cfloat conj(cfloat a) { return {a.re, -a.im}; }
__host__ __device__ inline double abs2(double a) { return a * a; }
__host__ __device__ inline float abs2(float a) { return a * a; }
__host__ __device__ inline double abs2(cdouble a) { return a.re * a.re + a.im * a.im; }
__host__ __device__ inline float abs2(cfloat a) { return a.re * a.re + a.im * a.im; }
// a * b with a real scalar
__host__ __device__ inline double rmul(double s, double a) { return s * a; }
__host__ __device__ inline float rmul(float s, float a) { return s * a; }
__host__ __device__ inline cdouble rmul(double s, cdouble a) { return {s * a.re, s * a.im}; }
__host__ __device__ inline cfloat rmul(float s, cfloat a) { return {s * a.re, s * a.im}; }

// conversions between precisions of the same field
template <class To, class From> __host__ __device__ inline To cvt(From a);
template <> __host__ __device__ inline double cvt<double, double>(double a) { return a; }
template <> __host__ __device__ inline float cvt<float, float>(float a) { return a; }
template <> __host__ __device__ inline double cvt<double, float>(float a) { return (double)a; }
template <> __host__ __device__ inline float cvt<float, double>(double a) { return (float)a; }
template <> __host__ __device__ inline cdouble cvt<cdouble, cdouble>(cdouble a) { return a; }
template <> __host__ __device__ inline cfloat cvt<cfloat, cfloat>(cfloat a) { return a; }
template <> __host__ __device__ inline cdouble cvt<cdouble, cfloat>(cfloat a) { return {(double)a.re, (double)a.im}; }
template <> __host__ __device__ inline cfloat cvt<cfloat, cdouble>(cdouble a) { return {(float)a.re, (float)a.im}; }
template <> __host__ __device__ inline float cvt<float, cfloat>(cfloat a) { return a.re; }

template <class T> struct dtype_of;
template <> struct dtype_of<double> { static const DType v = F64; };
template <> struct dtype_of<float> { static const DType v = F32; };
template <> struct dtype_of<cdouble> { static const DType v = C64; };
template <> struct dtype_of<cfloat> { static const DType v = C32; };

// run `body` with T bound to the element type of `t`
#define MLMC_DISPATCH(t, T, ...)                                 \
  switch (t) {                                                   \
    case ::mlmc::F64: { typedef double T; __VA_ARGS__; } break;  \
    case ::mlmc::F32: { typedef float T; __VA_ARGS__; } break;   \
    case ::mlmc::C64: { typedef ::mlmc::cdouble T; __VA_ARGS__; } break; \
    case ::mlmc::C32: { typedef ::mlmc::cfloat T; __VA_ARGS__; } break;  \
  }

// ----------------------------------------------------------------- errors
struct cuda_error {
  cudaError_t code;
  std::string where;
};
void check_cuda(cudaError_t e, const char *where);
#define MLMC_CUDA(call) ::mlmc::check_cuda((call), #call)
#define MLMC_LAUNCH_CHECK(name) ::mlmc::check_cuda(cudaGetLastError(), name)

inline unsigned grid_for(size_t work, int block, size_t cap = 152 * 32) {
  size_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// Grid of a kernel whose blocks stride over `units` work units: `per_sm` blocks per
// SM of the current device (all resident at once when the kernel's resources allow),
// at most `units`, at least 1.
unsigned resident_grid(size_t units, int per_sm);

// Blocks of `kernel` that fit on one SM at once (launch block size, dynamic shared
// memory), at least 1.
template <class F>
int blocks_per_sm(F kernel, int block, size_t smem) {
  int n = 0;
  check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem), "occupancy");
  return n > 0 ? n : 1;
}

// ----------------------------------------------------------------- views
// Nearest-neighbour block stencil on an nx x ny periodic lattice with d dofs
// per site: coef[site][dir][r][c], dir = 0 self, 1 +x, 2 -x, 3 +y, 4 -y.
// Dirichlet boundaries are zero blocks.  Vector blocks are [site][dof][k].
struct StencilView {
  int nx, ny, d;
  DType t;            // element type of coef / dinv
  const void *coef;   // [nsite][5][d][d]
  const void *dinv;   // [nsite][d][d] inverse of the self block (smoother), may be null
  int const_laplace;  // 1: Example 5.1 operator, applied without reading coef
  double diag;        //    its diagonal 4 + shift
  int periodic;       //    0: Dirichlet
  int taps;           // 5: the nearest-neighbour block stencil above; 9: a 9-point scalar
                      //    stencil coef[site][9] (bilinear coarse levels, Dirichlet, d = 1)
};

// Per-aggregate prolongation blocks P[agg][loc*d + a][q] with loc = jj*ax + ii.
struct ProlongView {
  int nx, ny, d;      // fine lattice
  int ax, ay, dc;     // aggregate shape and coarse dofs
  DType t;
  const void *P;
  int bilinear;       // 1: bilinear interpolation from the (nx-1)/2 x (ny-1)/2 grid (no P array)
};

// ----------------------------------------------------------------- launchers
// vector kernels (kernels_vec.cu)
void launch_noise(int kind, uint64_t seed, uint64_t key_hi, uint64_t first_sample, size_t n, int k,
                  DType t, void *out, cudaStream_t s);
void launch_convert(DType to, void *dst, DType from, const void *src, size_t count, cudaStream_t s);
void launch_fill_zero(DType t, void *dst, size_t count, cudaStream_t s);
// blocks x 256 threads, each running 8 FMA (add = 1: addition) chains of `iters` steps (F64 or F32);
// out (blocks x 256 entries) is written only under a condition that never holds
void launch_fma_rate(DType t, int add, void *out, int blocks, int iters, cudaStream_t s);
// `passes` copies a -> b -> a ... of n16 16-byte packs in one launch (bandwidth probe)
void launch_copy16(void *a, void *b, size_t n16, int passes, int blocks, cudaStream_t s);
void launch_fill_one(DType t, void *dst, size_t count, cudaStream_t s);
void launch_sub(DType t, void *out, const void *a, const void *b, size_t count, cudaStream_t s);
// y[i][c] = alpha[c] * x[i][c] (+ y if accumulate)
void launch_scale_cols(DType t, void *y, const void *x, const void *alpha, int alpha_is_inverse_norm,
                       size_t rows, int k, cudaStream_t s);
// partial[b][v][c] of sum_i conj(V_v[i][c]) * w[i][c], v < nvec; then out[v][c] (fixed order)
// lazy_sc (optional): the unnormalised-basis epilogue of k_multidot_reduce (out = d / (s_i s_j),
// lazy_coef = d / s_i^2 with s from lazy_sc, column lazy_j the new one)
void launch_multidot(DType t, const void *V, size_t vstride, int nvec, const void *w, size_t rows,
                     int k, void *partials, int nparts, void *out, DType out_t, cudaStream_t s,
                     const double *lazy_sc = nullptr, void *lazy_coef = nullptr, int lazy_j = 0);
// w[i][c] -= sum_v V_v[i][c] * h[v][c]  (h in out precision), optional column mask
// norm_part (optional): per-block column sums of |w_new|^2 in the FP64 accumulation
// type (multiaxpy_norm_parts(rows, k) x k entries at most); returns the block count
// to pass to launch_column_reduce.
int launch_multiaxpy(DType t, void *w, const void *V, size_t vstride, int nvec, const void *h,
                     DType h_t, size_t hstride, double sign, size_t rows, int k, cudaStream_t s,
                     void *norm_part = nullptr);
int multiaxpy_norm_parts(size_t rows, int k);
// out[c] = sum_p partial[p][c] (fixed order), FP64 or complex FP64
void launch_column_reduce(DType out_t, const void *partial, int nparts, int k, void *out, cudaStream_t s);
int multidot_parts(size_t rows, int k);

}  // namespace mlmc

namespace mlmc {
// stencil kernels (kernels_stencil.cu)
// mode 0: y = A x;  mode 1: y = b - A x
void launch_stencil(const StencilView &A, const void *x, const void *b, void *y, int k, int mode,
                    cudaStream_t s);
// one red-black block Gauss-Seidel half-sweep over sites of `colour`
void launch_rbgs_half(const StencilView &A, void *x, const void *b, int k, int colour, cudaStream_t s);
// one full red-black sweep (order 0: red then black, 1: black then red).  x_zero = 1
// means x holds zeros on entry (x need not be initialised: the kernels skip it).
void launch_rbgs_sweep(const StencilView &A, void *x, const void *b, int k, int order, int x_zero,
                       cudaStream_t s);
// rc = P^* r
void launch_restrict(const ProlongView &P, const void *r, void *rc, int k, cudaStream_t s);
// x += P ec
void launch_prolong_add(const ProlongView &P, const void *ec, void *x, int k, cudaStream_t s);
// x += P ec on the sites of one red-black colour only (aggregation levels; all sites otherwise)
void launch_prolong_add_colour(const ProlongView &P, const void *ec, void *x, int k, int colour, cudaStream_t s);
// rc = P^* (b - A x) with the residual taken on the sites of `colour` only (zero on the
// other colour after a red-black Gauss-Seidel sweep that updated it last); aggregation
// levels with d, dc <= 4 and the Example 5.1 fine level
bool residual_restrict_ok(const StencilView &A, const ProlongView &P);
void launch_residual_restrict(const StencilView &A, const ProlongView &P, const void *x, const void *b, void *rc,
                              int k, int colour, cudaStream_t s);
// out = base + omega * D^{-1} (rhs - y), D = diagonal entries of the self blocks; base/rhs may be null
// one damped-Jacobi sweep out = x - omega D^-1 A x of the constant-coefficient Laplacian
void launch_laplace_jacobi(const StencilView &A, const void *x, void *out, int k, double omega, cudaStream_t s);
void launch_jacobi_update(const StencilView &A, void *out, const void *base, const void *rhs,
                          const void *y, double omega, int k, cudaStream_t s);
// bilinear hierarchy of Example 5.1 (kernels_bilinear.cu), real data, d = 1
void launch_stencil9(const StencilView &A, const void *x, const void *b, void *y, int k, int mode, cudaStream_t s);
// one 4-colour Gauss-Seidel sweep (order 0: colours 0..3, 1: 3..0); x_zero: x is zeroed first
void launch_gs9_sweep(const StencilView &A, void *x, const void *b, int k, int order, int x_zero, cudaStream_t s);
// rc = P^T r from the fine (2 nxc + 1) x (2 nyc + 1) grid
void launch_restrict_bilinear(DType t, const void *r, void *rc, int nxc, int nyc, int k, cudaStream_t s);
// x += P ec on the fine nx x ny grid
void launch_prolong_bilinear(DType t, const void *ec, void *x, int nx, int ny, int k, cudaStream_t s);
// setup kernels (kernels_setup.cu)
void launch_block_inverse(DType t, const void *coef, void *dinv, int nsite, int d, int *err,
                          cudaStream_t s);
void launch_mgs(DType t, const void *V, void *P, int nx, int ny, int d, int ax, int ay, int ntv,
                int spin_split, int *err, cudaStream_t s);
void launch_galerkin(const StencilView &fine, const ProlongView &P, void *coarse_coef, cudaStream_t s);
// dense inverse of an n x n matrix (row-major), work = n x 2n elements, scratch of
// gauss_jordan_scratch_bytes(n) bytes; *err = 3 for a singular matrix, MLMC_ERR_TIMEOUT
// when a bounded grid-barrier wait gave up
size_t gauss_jordan_scratch_bytes(int n);
void launch_gauss_jordan(DType t, const void *A, void *Ainv, void *work, int n, int *err, void *scratch,
                         size_t scratch_bytes, cudaStream_t s);
void launch_trace(DType t, const void *A, int n, void *out /* FP64 (complex) */, cudaStream_t s);
// Y = Ainv * B  (n x n times n x k, row-major / [row][k])
// part: scratch of dense_apply_splits(n, k) * n * k elements (or null: no split of j)
void launch_dense_apply(DType t, const void *Ainv, const void *B, void *Y, int n, int k, void *part, cudaStream_t s);
int dense_apply_splits(int n, int k);
// Tensor-core (tcgen05, 3xTF32) variant for FP32 / complex-FP32 data, any n, k >= 1.
// part: dense_apply_tc_part_bytes(t, n, k) bytes of K-slice partials (none needed
// when that is 0); err: device int that receives MLMC_ERR_TIMEOUT if a bounded
// wait gives up.  Pointers 16-byte aligned.  withhold != 0: test mode that
// issues no MMA, so the first bounded wait runs out (about 1 ms).
bool dense_apply_tc_ok(DType t, int n, int k);
size_t dense_apply_tc_part_bytes(DType t, int n, int k);
void launch_dense_apply_tc(DType t, const void *Ainv, const void *B, void *Y, int n, int k, void *part,
                           size_t part_bytes, int *err, cudaStream_t s, int withhold = 0);
}  // namespace mlmc

namespace mlmc {
// per-column Krylov kernels (kernels_krylov.cu).  `hc` = 1 for complex Hessenberg data.
// g0[c] holds |r|^2 on entry (from a column dot); sets beta, active, invnrm.
// sc (optional): per-column norms of the unnormalised basis vectors of the
// fixed-length FGMRES (s_0 = |b| here; s_{j+1} set by the step)
// Added to the active-column count by launch_arnoldi_init for every column whose
// residual norm is not finite (such a column can never converge).
constexpr int NONFINITE_COLUMN = 1 << 20;
void launch_arnoldi_init(int hc, void *g, double *bnorm, double *invnrm, int *active, int *jdone,
                         int k, double tol, int first, int *nactive, cudaStream_t s, double *sc = nullptr);
// unnormalised basis: Gram-Schmidt coefficients d_i / s_i^2 into coef, Hessenberg
// entries d_i / (s_i s_j) in place; and y_i /= s_i before the solution update
void launch_lazy_y(int hc, void *y, const double *sc, const int *jdone, int m, int k, cudaStream_t s);
void launch_arnoldi_step(int hc, void *H, void *cs, void *sn, void *g, int j, int m, int k, int *active,
                         int *jdone, const double *bnorm, double tol, double *invnrm, double *resid,
                         int *nactive, int fixed, cudaStream_t s, double *sc = nullptr);
void launch_trisolve(int hc, const void *H, const void *g, void *y, const int *jdone, int m, int k,
                     cudaStream_t s);
void launch_add_acc(int hc, void *dst, const void *src, int count, cudaStream_t s);
// out[c] = a[c] - b[c] (complex FP64 samples from two column dots)
void launch_sample_combine(int hc, const void *a, const void *b, void *out, int k, cudaStream_t s);
// Welford accumulation of k complex samples into acc = {N, mean.re, mean.im, M2}
void launch_accumulate(const void *samples, int k, double *acc, cudaStream_t s);
// fine block stencils from the operator descriptor
void launch_build_laplace(double *coef, int nx, int ny, double shift, int periodic, cudaStream_t s);
void launch_build_wilson(cdouble *coef, const cdouble *links, int nx, int ny, double mass, cudaStream_t s);
// dense n x n matrix of a block stencil level (row-major)
void launch_stencil_to_dense(const StencilView &A, void *dense, cudaStream_t s);
}  // namespace mlmc

namespace mlmc {
// learned correction (kernels_learned.cu)
void launch_to_channels(DType t, const void *x, float *a, int nsite, int d, int k, cudaStream_t s);
void launch_add_from_channels(DType t, void *x, const float *a, int nsite, int d, int k, cudaStream_t s);
void launch_conv_fwd(int ci, int co, bool relu, const float *in, const float *W, float *out, int nx, int ny, int k,
                     int periodic, cudaStream_t s);
void launch_conv_bwd_data(int ci, int co, const float *gout, const float *W, const float *act, float *gin, int nx,
                          int ny, int k, int periodic, cudaStream_t s);
int conv_weight_blocks();
void launch_conv_bwd_weight(int ci, int co, const float *in, const float *gout, float *partial, float *grad,
                            float scale, int nx, int ny, int k, int periodic, cudaStream_t s);
// tensor-core convolutions (kernels_conv_tc.cu): forward (mirror = 0; W [cout][cin][9]) or
// backward-data (mirror = 1; W [cin][cout][9]), output masked by act > 0 when act is given
bool conv_tc_ok(int nx, int k, int cin, int cout);
void launch_conv_tc(const float *in, const float *W, const float *act, float *out, int nx, int ny, int k, int cin,
                    int cout, int periodic, int mirror, int relu, int *err, cudaStream_t s);
// per-CTA partial weight gradients [conv_wgrad_tc_blocks()][cout][cin][9]; k_weight_reduce adds them
bool conv_wgrad_tc_ok(int k, int cin, int cout);
int conv_wgrad_tc_blocks();
void launch_conv_wgrad_tc(const float *in, const float *gout, float *partial, int nx, int ny, int k, int cin,
                          int cout, int periodic, int *err, cudaStream_t s);
// grad[w] = scale * sum over blocks of partial[block][w], blocks in order
void launch_weight_reduce(const float *partial, int nblocks, int nw, float *grad, float scale, cudaStream_t s);
void launch_adam(float *W, const float *g, float *m, float *v, int n, float lr, int step, cudaStream_t s);
void launch_spin_flip(DType t, void *x, int nsite, int d, int k, cudaStream_t s);
// alpha[c] = scale / |dot[c]| (real part), FP64 per-column factors from a column dot
void launch_col_factor(int hc, const void *dot, double *alpha, double scale, int k, cudaStream_t s);
}  // namespace mlmc
