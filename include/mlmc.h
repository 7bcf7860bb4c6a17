/*
 * libmlmc: multilevel Monte-Carlo estimation of tr(A^{-1}) on one GB300 GPU.
 *
 * The method is that of Frommer, Nasr Khalil and Ramirez-Hidalgo, "A
 * multilevel approach to variance reduction in the stochastic estimation of
 * the trace of a matrix" (arXiv 2108.11281).  A is given indirectly (Sec. 3):
 * here as a lattice operator descriptor (Example 5.1 Laplacian, Example 5.3
 * 2-spin Wilson/Schwinger operator).  An aggregation multigrid hierarchy with
 * orthonormal prolongations P_l and Galerkin operators A_{l+1} = P_l^* A_l P_l
 * (Sec. 4.1) gives the telescoping sum of Remark 4.3,
 *   tr(A^{-1}) = sum_{l<L} [tr(A_l^{-1}) - tr(P_l A_{l+1}^{-1} P_l^*)] + tr(A_L^{-1}),
 * whose level differences are estimated by Hutchinson samples (Sec. 3) and
 * whose last term is computed exactly (Remark 4.2).  Samples need solves with
 * A_l and A_{l+1}, done by flexible GMRES preconditioned by a multigrid cycle
 * over the levels below (Remark 4.1, Example 5.3).
 *
 * Conventions for every entry point:
 *  - The return value is an mlmc_status; 0 is success.  No exception and no
 *    abort crosses this interface.  mlmc_last_error() describes the last
 *    failure of the calling thread.
 *  - "host" pointers are ordinary CPU memory, read or written only during
 *    the call.  "device" pointers are CUDA global memory of the current
 *    device, owned by the caller.
 *  - All GPU work is issued on the stream given at setup (NULL: a private
 *    blocking stream of the handle, ordered with the legacy default stream).
 *    Calls return after their work has completed.
 *  - A hierarchy handle owns all device memory it allocates and must be used
 *    by one host thread at a time.
 *  - Vector blocks on the device are laid out [site][dof][k]: the k columns
 *    (independent right-hand sides or samples) are innermost.  Real operators
 *    use double, complex operators interleaved (re, im) double pairs.
 *  - Noise: sample j of level l is column (j - first) of a block and depends
 *    only on (seed, l, j): Philox4x64-10 with key (seed, (purpose << 8) | l)
 *    and counter (row_block, j, 0, 0); Rademacher rows take one bit each
 *    (256 rows per counter), Z4 rows two bits (128 rows per counter).
 */
#ifndef MLMC_H
#define MLMC_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } mlmc_c64;

typedef enum {
  MLMC_OK = 0,
  MLMC_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of range */
  MLMC_ERR_UNSUPPORTED = 2,   /* a valid request the library does not implement */
  MLMC_ERR_CUDA = 3,          /* a CUDA call failed; see mlmc_last_error() */
  MLMC_ERR_OOM = 4,           /* device allocation failed */
  MLMC_ERR_NOT_CONVERGED = 5, /* a solve hit max_iter before reaching tol */
  MLMC_ERR_SINGULAR = 6,      /* zero pivot / dependent test vectors in setup */
  MLMC_ERR_TIMEOUT = 7,       /* a bounded device wait gave up */
  MLMC_ERR_REJECTED = 8       /* a result failed its FP64 acceptance check */
} mlmc_status;

enum { MLMC_OP_LAPLACE2D = 1, MLMC_OP_WILSON2D = 2 };
enum { MLMC_NOISE_RADEMACHER = 0, MLMC_NOISE_Z4 = 1 };
enum { MLMC_PURPOSE_NOISE = 0, MLMC_PURPOSE_WARMUP = 1, MLMC_PURPOSE_SETUP = 2, MLMC_PURPOSE_TRAIN = 3 };
enum { MLMC_SETUP_SMOOTH = 0, MLMC_SETUP_INVERSE = 1, MLMC_SETUP_CONSTANT = 2 };
enum { MLMC_PREC_FP64 = 0, MLMC_PREC_MIXED_FP32 = 1 };
enum { MLMC_FORM_SIMPLIFIED = 0, MLMC_FORM_HAT = 1, MLMC_FORM_PLAIN = 2 };
enum { MLMC_CYCLE_V = 0, MLMC_CYCLE_K = 1 };
enum { MLMC_ALLOC_RHO = 0, MLMC_ALLOC_OPTIMAL = 1, MLMC_ALLOC_FIXED = 2 };
enum { MLMC_COST_COUNTED = 0, MLMC_COST_NOMINAL = 1 };
enum { MLMC_TRANSFER_AGGREGATION = 0, MLMC_TRANSFER_BILINEAR = 1 };

/* Fine operator A = A_1 (Examples 5.1 and 5.3).  Sites s = j*nx + i. */
typedef struct {
  int kind;          /* MLMC_OP_LAPLACE2D: (4 + shift) u_ij - sum of the 4 neighbours, real, d = 1.
                        MLMC_OP_WILSON2D: Eq. schwinger_coupling, complex, d = 2, periodic.     */
  int nx, ny;        /* lattice; multiples of agg_x^(L-1), agg_y^(L-1)                            */
  int periodic;      /* Laplace only: 0 Dirichlet (Example 5.1), 1 periodic                     */
  double shift;      /* Laplace: sigma in A + sigma I                                           */
  double mass;       /* Wilson: m in (4 + m)                                                    */
  const mlmc_c64 *links; /* Wilson, host, [2][ny][nx]: [0] = exp(i Theta) on (i,j)->(i+1,j),
                            [1] = exp(i Phi) on (i,j)->(i,j+1).  NULL for Laplace.            */
} mlmc_operator_desc;

/* Hierarchy and solver parameters (Secs. 4.1, 5; Example 5.3). */
typedef struct {
  int levels;          /* L >= 2                                                              */
  int agg_x, agg_y;    /* aggregate shape (Example 5.3: 4 x 4)                                */
  int n_tv;            /* test vectors per aggregate (same count on every level)              */
  int spin_split;      /* 1: split each test vector into the two spin halves of a site's
                          dofs, doubling the coarse dofs and keeping J A = A^* J (Ex. 5.3)    */
  int setup_kind;      /* MLMC_SETUP_SMOOTH: v <- v - omega D^{-1} A v, `setup_sweeps` times;
                          MLMC_SETUP_INVERSE: v <- two damped-Jacobi steps on A x = v;
                          MLMC_SETUP_CONSTANT: one constant test vector (n_tv = 1)            */
  int setup_sweeps;    /* filter sweeps on level 1                                            */
  int coarse_sweeps;   /* filter sweeps on levels >= 2, applied to R_{l-1} V_{l-1}            */
  double setup_omega;  /* damping of the filter                                               */
  uint64_t setup_seed; /* Philox seed of the test vectors (purpose SETUP, level 1)           */
  int bootstrap;       /* rounds of v <- v - M(A v) with M one FP64 cycle, then rebuild       */
  int boot_iters;      /* applications per round                                              */
  int smooth_pre, smooth_post; /* red-black block Gauss-Seidel sweeps per cycle                */
  int cycle;           /* MLMC_CYCLE_V or MLMC_CYCLE_K (Krylov-accelerated coarse correction) */
  int kcycle_its;      /* FGMRES steps per coarse correction in a K-cycle                     */
  int fgmres_restart;  /* outer FGMRES restart length m                                       */
  int max_iter;        /* outer FGMRES iteration cap per solve                                */
  int precision;       /* MLMC_PREC_FP64 or MLMC_PREC_MIXED_FP32 (FP32 cycle under FP64 FGMRES)*/
  int block;           /* largest vector-block width k (columns per solve), 1..256            */
  int reorth;          /* 1: classical Gram-Schmidt twice in the outer Arnoldi                */
  int inner_its;       /* > 0: the outer FP64 FGMRES is preconditioned by this many FGMRES
                          steps in the cycle precision (each preconditioned by one cycle);
                          0: by one cycle                                                      */
  int graphs;          /* 1: replay each inner solve as a captured CUDA graph                   */
  int coarse_smooth;   /* > 0: pre- and post-smoothing sweeps on levels >= 2 (else as level 1) */
  int coarse_block;    /* > 0: vector-block width of samples on level differences >= 2 (their
                          solves are small, so wider blocks fill the GPU); 0 = block          */
  const void *const *user_P; /* optional, host: user_P[l-1] = P_l as blocks [agg][ax*ay*d][dc]
                          (double, or mlmc_c64 for complex operators); columns must be
                          orthonormal.  Replaces the test-vector setup.  NULL = build P.      */
  int transfer;        /* MLMC_TRANSFER_AGGREGATION (above), or MLMC_TRANSFER_BILINEAR: the
                          paper's hierarchy for Example 5.1 (Sec. 5): Dirichlet Laplacian with
                          N_l = 2 N_{l+1} + 1 (every side above the coarsest odd), P_l bilinear
                          interpolation, R_l = P_l^T, Galerkin 9-point coarse operators
                          smoothed by 4-colour Gauss-Seidel.  R P != I, so samples and
                          estimates need MLMC_FORM_HAT (or MLMC_FORM_PLAIN); agg_*, n_tv,
                          spin_split, setup_*, bootstrap and user_P are ignored.           */
  int coarse_growth;   /* g > 0: the block width grows by 2^g per level difference beyond the
                          second (coarse_block on difference 2, then 2^g x, 4^g x, ... up to
                          512 columns for real operators, 256 for complex ones): coarser
                          levels are cheaper per column and draw more samples, so wider
                          blocks amortise their latency-bound launches.  0 = coarse_block
                          on every difference >= 2.  Samples do not depend on widths.       */
} mlmc_hierarchy_params;

typedef struct mlmc_hierarchy mlmc_hierarchy;

/* Sec. 5 estimate parameters. */
typedef struct {
  double eps;          /* relative accuracy target (paper: 1e-3)                             */
  double weights[16];  /* w_l, sum 1, rho_l = sqrt(w_l) eps |tau|; all 0 = 1/(L-1) each     */
  int noise;           /* MLMC_NOISE_RADEMACHER or MLMC_NOISE_Z4                             */
  uint64_t seed;
  double tol;          /* relative residual of every level solve                             */
  int min_samples;     /* floor on N_l (paper: 5)                                            */
  int max_samples;     /* cap on N_l                                                          */
  int form;            /* MLMC_FORM_SIMPLIFIED (Remark 4.3, noise on each level's space),
                          MLMC_FORM_HAT (Eq. tr_ml_dec: noise on the fine space restricted by
                          R^_l; same exact term since R^_L P^_L = I), or MLMC_FORM_PLAIN
                          (Eq. plain_tr_estimate: Hutchinson on A_1 alone, one "level",
                          no coarse term: the comparison the paper makes in Sec. 5)          */
  int allocation;      /* MLMC_ALLOC_RHO: Sec. 5 per-level targets rho_l from `weights`;
                          MLMC_ALLOC_OPTIMAL: Sec. 2 N_l proportional to sqrt(V_l / C_l) with
                          V_l, C_l (cost model per sample) estimated as samples arrive, until
                          sum V_l / N_l <= (eps tau)^2;
                          MLMC_ALLOC_FIXED: exactly n_fixed[l] samples on level difference l
                          (serving requests with a fixed sample budget; eps unused)            */
  int n_fixed[16];
  int cost_model;      /* per-sample cost C_l of MLMC_ALLOC_OPTIMAL (Sec. 5 cost model, nnz(B)
                          per product B x): MLMC_COST_COUNTED (0) = the products the samples'
                          solves actually performed (iteration counts included), averaged
                          over the samples drawn; MLMC_COST_NOMINAL (1) = a fixed figure per
                          level difference that does not depend on the solver: the
                          restrictions the noise needs (nnz(P_j) each) plus one product with
                          each operator solved with (nnz(A_l), nnz(A_{l+1}); n_L^2 for the
                          coarsest dense inverse).  N_l then depends on the samples alone.   */
  int tau_separate;    /* 0 (default): tau's five full estimates (Sec. 5) are samples 0..4 of
                          every level's noise stream, which also count in the level means (so
                          rho_l and N_l correlate with the means they control); 1: they come
                          from five separate samples per level (Philox purpose
                          MLMC_PURPOSE_WARMUP) that do not enter the means (their solves are
                          not in cost_nnz)                                                     */
} mlmc_estimate_params;

typedef struct {
  mlmc_c64 trace;        /* sum of level means + exact coarsest term                         */
  double std_err;        /* sqrt(sum_l V_l / N_l)                                            */
  double tau;            /* mean - rms deviation of the 5 warm-up estimates                  */
  mlmc_c64 coarse_term;  /* tr(A_L^{-1}) (Remark 4.2)                                        */
  int levels;
  int n_samples[16];     /* N_l per level difference                                         */
  mlmc_c64 mean[16];
  double variance[16];   /* unbiased sample variance, complex convention of Sec. 3           */
  double iters[16];      /* mean outer FGMRES iterations per solve on level l                */
  double seconds[16];    /* wall time spent on level difference l                            */
  double cost_nnz[16];   /* Sec. 5 cost model: sum of nnz(B) over products B x, per level
                            difference (both solves, transfers, smoothing sweeps, coarsest
                            products); entry L-1: n_L^3 for the exact coarsest term          */
  double weights_used[16]; /* w_l with rho_l^2 = w_l (eps tau)^2 (optimal: sqrt(V_l C_l) share) */
  double seconds_total;
} mlmc_estimate_result;

/* Build the hierarchy on the GPU (Sec. 4.1; Example 5.3): fine operator,
 * test vectors, per-aggregate orthonormalisation, Galerkin coarse operators,
 * smoother blocks, dense inverse of A_L (Gauss-Jordan with partial pivoting in
 * one cooperative launch whose grid-barrier waits are bounded: a wait that
 * gives up returns MLMC_ERR_TIMEOUT; a zero pivot MLMC_ERR_SINGULAR).
 * `stream` is a cudaStream_t or NULL
 * (NULL: the handle creates and owns a private stream).  On success *out owns
 * the device memory until mlmc_destroy_hierarchy.  Device buffers are
 * stream-ordered on that stream (no device-wide synchronisation when a handle
 * allocates or frees, so handles on different streams run concurrently); a
 * caller's stream must stay valid until mlmc_destroy_hierarchy returns.     */
int mlmc_setup_hierarchy(const mlmc_operator_desc *op, const mlmc_hierarchy_params *params,
                         void *stream, mlmc_hierarchy **out);
void mlmc_destroy_hierarchy(mlmc_hierarchy *h);

/* Level sizes: lattice nx, ny and dofs per site d of level l (1-based). */
int mlmc_level_info(const mlmc_hierarchy *h, int level, int *nx, int *ny, int *d);
/* Stencil taps of level l's operator as returned by mlmc_get_operator: 5
 * (nearest-neighbour blocks) or 9 (the 9-point coarse levels of the bilinear
 * hierarchy: taps 0 self, 1 +x, 2 -x, 3 +y, 4 -y, 5 (+x,+y), 6 (-x,+y),
 * 7 (+x,-y), 8 (-x,-y)). */
int mlmc_level_taps(const mlmc_hierarchy *h, int level, int *taps);

/* Copy P_l (level l < L) to host as blocks [agg][ax*ay*d][dc] (FP64 / c64).
 * MLMC_ERR_UNSUPPORTED for the bilinear hierarchy (P is applied, not stored). */
int mlmc_get_prolongation(const mlmc_hierarchy *h, int level, void *host_out);
/* Copy the block stencil of A_l to host as [site][taps][d][d] (FP64 / c64);
 * 5 taps: directions 0 self, 1 +x, 2 -x, 3 +y, 4 -y (periodic indexing);
 * 9 taps: see mlmc_level_taps (Dirichlet). */
int mlmc_get_operator(const mlmc_hierarchy *h, int level, void *host_out);

/* y = A_l x for a device block of k columns (FP64 / c64). */
int mlmc_apply(mlmc_hierarchy *h, int level, const void *x, void *y, int k);
/* Solve A_l x = b for a device block of k columns to relative residual tol
 * (Remark 4.1).  iters (host, optional) receives the outer iteration count. */
int mlmc_solve(mlmc_hierarchy *h, int level, const void *b, void *x, int k, double tol, int *iters);
/* Noise block (Eqs. iid_components1 / iid_components2) into a device buffer
 * [n][k]: column c is sample first + c of (seed, level, purpose). */
int mlmc_noise(int noise, uint64_t seed, int level, int purpose, uint64_t first, int n, int k,
               int complex_out, void *out, void *stream);

/* Level-difference samples (Remark 4.3): for j in [first, first + n_samples),
 *   s_j = x_j^* A_l^{-1} x_j - (P_l^* x_j)^* A_{l+1}^{-1} (P_l^* x_j),  x_j = noise(seed, l, j),
 * for 1 <= level < L; level == L gives x^* A_L^{-1} x.  out_samples is host
 * memory of n_samples entries.  out_iters (host, optional) receives the
 * outer iteration count of each block's two solves (one entry per block of
 * the level's block width: at most n_samples entries). */
int mlmc_sample_level(mlmc_hierarchy *h, int level, int noise, uint64_t seed, uint64_t first,
                      int n_samples, double tol, mlmc_c64 *out_samples, int *out_iters);

/* One block of level-difference samples for a caller-driven estimate, e.g. one
 * estimate whose blocks are spread over several GPUs (Sec. 2 estimator; the
 * per-level statistics of Sec. 5 are merged block by block): samples
 * first .. first + k - 1 of level difference `level` (1 <= level < L) in the
 * given form (as mlmc_sample_level_form), 1 <= k <= that level difference's
 * block width.  out_samples (host, optional): the k samples.  out_stats (host,
 * optional, 4 doubles): the block's N, mean (re, im) and sum of |s - mean|^2,
 * from the device's fixed-order reduction.  out_cost (host, optional): the
 * Sec. 5 cost model of the block's products.  Synchronous on return. */
int mlmc_sample_block(mlmc_hierarchy *h, int level, int form, int noise, uint64_t seed, uint64_t first, int k,
                      double tol, mlmc_c64 *out_samples, double *out_stats, double *out_cost);
/* The cycle's restricted residual (Remark 4.1) in one pass: rc = P_l^* m (b - A_l x)
 * with m the indicator of the sites of `colour` ((i + j) mod 2): after a red-black
 * Gauss-Seidel sweep the residual vanishes on the colour updated last, so the cycle
 * passes the other one.  Device blocks x, b [n_l][k], rc [n_{l+1}][k] in FP64
 * (precision MLMC_PREC_FP64) or FP32 (MLMC_PREC_MIXED_FP32, mixed form only);
 * aggregation levels with at most 4 dofs per site and coarse site; 1 <= k <= 65536
 * (the caller's blocks, independent of the hierarchy's block widths).  Synchronous. */
int mlmc_residual_restrict(mlmc_hierarchy *h, int level, int precision, const void *x, const void *b, void *rc,
                           int k, int colour);
/* Samples per block on level difference `level` (1 <= level < L): the widths the
 * estimate draws (block, coarse_block, coarse_growth, mlmc_set_block_width). */
int mlmc_block_width(const mlmc_hierarchy *h, int level, int *k);
/* The nominal per-sample cost of level difference `level` (MLMC_COST_NOMINAL). */
int mlmc_nominal_sample_cost(const mlmc_hierarchy *h, int level, int form, double *out);

/* Column dots out[c] = sum_i conj(x[i][c]) y[i][c] of two device blocks [n][k]
 * (the x_j^* y_j products of the difference samples, Remark 4.3), in FP64:
 * double (complex = 0) or interleaved complex double (complex = 1) inputs; out
 * is device memory of k doubles or k complex doubles.  Summation order is
 * fixed (per-column partial sums over 608 row chunks, then a fixed tree).
 * Allocates and frees its scratch (608 x k partial sums) on every call; k <= 256. */
int mlmc_column_dots(int complex_data, const void *x, const void *y, int n, int k, void *out, void *stream);

/* mlmc_column_dots without any allocation (the paper has no counterpart).  It
 * serves callers that cannot let a library allocate device memory:
 * applications whose own memory manager owns every byte of device memory (a
 * pool sized up front, a fixed budget per process), and latency-critical loops
 * that must not pay an allocator's synchronisation or its failure modes in the
 * middle of a run.  Same arguments and result as mlmc_column_dots, and like it
 * the call returns once `out` has been written.  Its scratch is a fixed array
 * of 2,490,368 bytes inside the library (608 row chunks x 256 columns x 16
 * bytes), present on every GPU that loads the library until the process
 * exits; k > 256 is rejected with MLMC_ERR_INVALID_ARG.  The first call on a
 * device (and the first after its context was replaced, e.g. by
 * cudaDeviceReset) looks up the array's device address with
 * cudaGetSymbolAddress, with that device current; make that first call before
 * any stream capture.  All calls share the one array and it keeps the last
 * call's partial sums, which every call overwrites before reading; calls that
 * overlap on the GPU (other streams, other threads) race, so issue them one
 * after another.  Errors are described by mlmc_noalloc_last_error(). */
int mlmc_column_dots_noalloc(int complex_data, const void *x, const void *y, int n, int k, void *out,
                             void *stream);
const char *mlmc_noalloc_last_error(void);

/* mlmc_sample_level for a chosen form (see mlmc_estimate_params.form); the
 * plain form is only defined on level 1. */
int mlmc_sample_level_form(mlmc_hierarchy *h, int level, int form, int noise, uint64_t seed, uint64_t first,
                           int n_samples, double tol, mlmc_c64 *out_samples);

/* ---- Coarsest-level dense apply (Sec. 4: the coarsest system is solved
 * directly; the FP32 cycle applies the inverse A_L^-1 computed at setup) ---
 * Y = A B for FP32 data on the device: A n x n row-major, B and Y n x k with
 * the k columns innermost (complex_data: complex64 interleaved (re, im)).
 * which = MLMC_DENSE_TC runs the tcgen05 tensor-core kernel (three TF32
 * products per term, FP32 accuracy; every mbarrier wait bounded, a wait that
 * gives up returns MLMC_ERR_TIMEOUT and leaves Y unspecified); MLMC_DENSE_SIMT
 * the CUDA-core kernel.  MLMC_DENSE_TC_WITHHOLD exercises the timeout path:
 * the tensor-core kernel issues no MMA, its first wait runs out after about
 * 1 ms, and the call returns MLMC_ERR_TIMEOUT with the context intact.
 * Any n >= 1, 1 <= k <= 4096; pointers 16-byte aligned (else
 * MLMC_ERR_INVALID_ARG).  The call allocates its scratch, runs on `stream`
 * and is synchronous on return. */
enum { MLMC_DENSE_SIMT = 0, MLMC_DENSE_TC = 1, MLMC_DENSE_TC_WITHHOLD = 2, MLMC_DENSE_AUTO = 3 };
int mlmc_dense_apply(int complex_data, const void *A, const void *B, void *Y, int n, int k, int which, void *stream);
/* Kernel of the FP32 cycle's coarsest apply for this handle: MLMC_DENSE_TC,
 * MLMC_DENSE_SIMT, or MLMC_DENSE_AUTO (the default): the tensor cores when the
 * real contraction length (n_L, or 2 n_L for complex operators) is at least
 * 512, else the CUDA cores (measured: n_L = 1024 real 20.6 vs 55.4 us,
 * 512 complex 24.3 vs 30.8 us, 225 real 20.7 vs 14.5 us at k = 128).  The
 * FP64 cycle always uses the CUDA-core kernel, GB300's FP64 tensor rate being
 * far below its FP32 one.  A change of kernel synchronises the handle's stream
 * and drops the CUDA graphs captured for the inner solves (they are captured
 * again on next use). */
int mlmc_set_dense_kernel(mlmc_hierarchy *h, int which);

/* Kernels of the learned correction's 3x3 convolutions (forward, backward-data,
 * weight gradient) for this handle.  MLMC_CONV_TC: on the tensor cores
 * (tcgen05 implicit GEMMs, three TF32 products per term for FP32 accuracy,
 * accumulators in tensor memory, every wait bounded) whenever the block width
 * k is 8, 16, 32, 64 or 128 and the fine lattice's rows hold whole tiles of
 * 128 / k sites (weight gradient: k a multiple of 8, at most 32 or a multiple
 * of 32), else on the CUDA cores; MLMC_CONV_SIMT: always on the CUDA cores;
 * MLMC_CONV_AUTO (the default): whichever of the two ran the network faster
 * on a fine-level block of the sample width, timed once when the network is
 * first installed or trained (or when AUTO is set again).  A change drops the
 * CUDA graphs captured for the inner solves. */
enum { MLMC_CONV_SIMT = 0, MLMC_CONV_AUTO = 1, MLMC_CONV_TC = 2 };
int mlmc_set_conv_kernel(mlmc_hierarchy *h, int which);

/* The exact coarsest term of the estimator (Remark 4.2), tr(A_L^{-1} R^_L P^_L)
 * from the FP64 dense inverse: tr(A_L^{-1}) when R^_L P^_L = I (aggregation). */
int mlmc_coarse_trace_exact(mlmc_hierarchy *h, mlmc_c64 *out);

/* The Sec. 5 procedure: exact coarse term; the first block of every level
 * difference, whose samples 0..4 (plus the exact term) are the five full
 * estimates that give tau = mean - rms deviation; then sampling in blocks
 * until every level meets its target (rho_l split, Sec. 2 optimal allocation,
 * or a fixed budget), with N_l >= min_samples. */
int mlmc_trace_estimate(mlmc_hierarchy *h, const mlmc_estimate_params *p, mlmc_estimate_result *r);

/* ---- Batched, uneven serving (many instances) ---------------------------- */
/* Active vector-block width (columns per solve) of this handle's estimates
 * and sample calls, 1 <= k <= block.  Samples do not depend on k. */
int mlmc_set_block_width(mlmc_hierarchy *h, int k);
/* Autotuner: time one block of level-`level` samples for k = 16, 32, ...,
 * block (each twice; the second, warm run counts) and keep the k with the
 * lowest time per sample as the active width.  Uses the setup noise stream,
 * so no estimate sample is consumed.  Wall-clock based: the choice may vary
 * between runs. */
int mlmc_autotune_block(mlmc_hierarchy *h, int level, int noise, double tol, int *k_out, double *seconds_per_sample);
/* Run mlmc_trace_estimate on `count` independent hierarchies with `workers`
 * host threads.  Each hierarchy works on its own stream, so instances of
 * uneven size overlap on the GPU.  status[i] receives each instance's status;
 * the return value is the first failing one (or MLMC_OK). */
int mlmc_trace_estimate_batch(mlmc_hierarchy *const *hs, int count, const mlmc_estimate_params *params, int workers,
                              mlmc_estimate_result *results, int *status);

/* Measured arithmetic ceiling (the paper has no counterpart; a roofline
 * denominator): operations per second of the whole GPU, fused multiply-adds
 * in FP64 (fp64 = 1) or FP32 (fp64 = 0), or FP64 additions (fp64 = 2), from 8
 * independent chains per thread on 8 blocks of 256 threads per SM; or
 * (fp64 = 3) the L2 bandwidth in bytes per second, from a copy between two
 * 16 MB buffers that stay in L2 (the ceiling of the small coarse-level
 * kernels).  Timed with CUDA events on `stream`; allocates its buffers;
 * synchronous on return. */
int mlmc_measure_fma_rate(int fp64, void *stream, double *fma_per_s);

/* Time one kernel family on level l with CUDA events on the hierarchy's
 * stream: which = 0 operator apply (FP64), 1 operator apply (FP32),
 * 2 red-black GS sweep, 3 column multi-dot of 4 basis blocks against w,
 * 4 multi-AXPY of 4 basis blocks into w, 5 coarsest dense apply
 * Y = A_L^-1 B (level = L; the kernel chosen by mlmc_set_dense_kernel),
 * 6 restriction R_l = P_l^* from level l to l+1, 7 prolongation x += P_l e
 * from level l+1, 8 the learned correction's network on a level-1 block (mixed
 * form; the convolutions chosen by mlmc_set_conv_kernel; its FLOPs are
 * 2 x 9 x (16 c0 + 256 + 16 c0) per site and column, c0 its input channels),
 * 9 the cycle's fused residual and restriction from level l to l+1 (after
 * red-black pre-smoothing the residual lives on one colour)
 * (2-9 in the cycle precision).  k <= block on level 1,
 * k <= max(block, coarse_block) on the coarser levels (6, 7: also within
 * level l+1's buffers).
 * Reports the average launch time and the algorithmic bytes one launch must
 * move (for 5: the dense inverse once plus B and Y; its FLOPs are
 * 2 n_L^2 k real, 8 n_L^2 k complex). */
int mlmc_profile_kernel(mlmc_hierarchy *h, int which, int level, int k, int reps,
                        double *ms_per_launch, double *bytes_per_launch);

/* ---- Learned correction (not in the paper; the project's smoother) --------
 * A bias-free 3-layer 3x3 convolutional network c0 -> 16 -> 16 -> c0 (ReLU
 * after layers 1 and 2; c0 = real channels per fine site: 1 Laplace, 4
 * Wilson) applied in the FP32 cycle on the fine level after the coarse-grid
 * correction: x += net(b - A x), then the red-black post-smoothing.  Weights
 * are FP32, concatenated [W1 | W2 | W3], each [c_out][c_in][3][3] with tap
 * (ty, tx) reading site (i + tx - 1, j + ty - 1).  Needs the mixed form.
 * Acceptance stays with the FP64 outer FGMRES true residual; a solve that
 * does not converge with the net is repeated without it.                    */
typedef struct {
  int n_pairs;               /* fine-level residuals to capture from plain solves (rounded up to blocks) */
  int epochs;                /* passes of Adam over the training blocks                                  */
  double lr;                 /* Adam step size                                                           */
  double tol;                /* relative tolerance of the plain solves that generate the residuals     */
  uint64_t seed;             /* right-hand sides of those solves: Philox purpose 3, level 1              */
  const float *init_weights; /* host, optional: initial weights (else a seeded Rademacher initialisation) */
  int enable;                /* 1: switch the net on if its validation loss is below 1                  */
} mlmc_train_params;

typedef struct {
  int pairs, blocks, epochs, enabled, n_weights;
  double loss_first, loss_last;   /* mean training loss of the first / last epoch                       */
  double val_loss;                /* mean ||A net(r) - r||^2 / ||r||^2 on held-out residuals           */
  double seconds_capture, seconds_train;
} mlmc_train_report;

/* State of the learned correction: *enabled (1 when the network acts in the
 * FP32 cycle) and *fallbacks (level solves that did not converge with it and
 * were repeated without it, since the handle was created).  Either pointer may
 * be NULL. */
int mlmc_learned_stats(const mlmc_hierarchy *h, int *enabled, int *fallbacks);

/* Capture residual/error pairs from plain multigrid solves (the error enters
 * through A e = r), train the network on the GPU (forward, backward, Adam),
 * validate, and install it.  weights_out (host, optional) receives n_weights floats. */
int mlmc_learned_train(mlmc_hierarchy *h, const mlmc_train_params *p, float *weights_out, mlmc_train_report *rep);
/* Install weights (host, n_weights floats) and switch the net on (enable = 1) or off. */
int mlmc_learned_set(mlmc_hierarchy *h, const float *weights, int enable);
/* e = net(r) for a device block of k columns in the FP32 field of the fine level. */
int mlmc_learned_apply(mlmc_hierarchy *h, const void *r, void *e, int k);
/* Loss of a device block r (FP32 field of the fine level, k columns) and its
 * weight gradient (host, n_weights floats). */
int mlmc_learned_grad(mlmc_hierarchy *h, const void *r, int k, double *loss, float *grad_out);

/* Number of kernel launches issued by this handle since setup (for reports). */
int mlmc_launch_count(const mlmc_hierarchy *h, uint64_t *count);

const char *mlmc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
