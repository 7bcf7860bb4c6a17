// Host side of libmlmc: the C ABI of include/mlmc.h, hierarchy setup on the
// GPU (Sec. 4.1, Example 5.3), the batched flexible GMRES driver with its
// multigrid-cycle preconditioner (Remark 4.1), level-difference samples
// (Remark 4.3), the exact coarsest term (Remark 4.2) and the Sec. 5 estimate.
// Every numerical step runs in the kernels of the other translation units;
// this file only sequences launches and owns device memory.
#include <algorithm>
#include <atomic>
#include <thread>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "mlmc.h"
#include "mlmc_internal.cuh"

using namespace mlmc;

namespace {

thread_local std::string g_last_error;

struct mlmc_fail {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg) { throw mlmc_fail{code, msg}; }

// Stream of the current entry point's device allocations (set by need() /
// need_level() to the hierarchy's stream, or to the call's stream).  Buffers are
// stream-ordered (cudaMallocAsync / cudaFreeAsync): a hierarchy that allocates or
// frees does not synchronise the device, so instances on other streams keep running.
thread_local cudaStream_t g_alloc_stream = nullptr;

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;   // the stream it was allocated on, and is freed on
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes), s(o.s) { o.p = nullptr; o.bytes = 0; }
  DevBuf &operator=(DevBuf &&o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; s = o.s; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t nbytes) {
    release();
    if (nbytes == 0) nbytes = 16;
    s = g_alloc_stream;
    cudaError_t e = cudaMallocAsync(&p, nbytes, s);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      p = nullptr;
      fail(MLMC_ERR_OOM, "device allocation of " + std::to_string(nbytes) + " bytes failed");
    }
    check_cuda(e, "cudaMallocAsync");
    bytes = nbytes;
  }
  template <class T> T *as() const { return (T *)p; }
};

struct Level {
  int nx = 0, ny = 0, d = 0;
  size_t nsite = 0, n = 0;
  DevBuf coef64, dinv64, coef32, dinv32;   // block stencil and inverse self blocks
  int ax = 0, ay = 0, dc = 0;              // aggregation towards the next level
  DevBuf P64, P32;
  int taps = 5;                            // 5: block stencil; 9: 9-point scalar stencil (bilinear levels >= 2)
  DevBuf Ainv64, Ainv32;                   // coarsest level only
  DevBuf dense_part;                       // split-j partial products of the coarsest apply
};

// Workspace of one batched FGMRES (one level, one element type).
struct Krylov {
  DType t = F64;
  int hc = 0;               // complex Hessenberg data
  size_t n = 0;
  int k = 0, m = 0;
  DevBuf V, Z, partials, H, cs, sn, g, y, h2, bnorm, invnrm, resid, active, jdone, nactive;
  DevBuf sc, hco;           // fixed-length variant: basis-vector norms, Gram-Schmidt coefficients
  int h_nactive = 0;         // host copy of the active-column count (pageable: the copy waits for it)
};

struct CycleBufs {
  DevBuf b, x, r;
  std::unique_ptr<Krylov> kcyc;   // K-cycle FGMRES on this level
};

// An instantiated CUDA graph of one fixed-length inner solve (level, width k,
// network state), with the cost-model and launch counts it represents.
struct GraphEntry {
  int level = -1, k = 0, net = 0;
  cudaGraphExec_t exec = nullptr;
  double cost = 0.0;
  uint64_t launches = 0;
};

}  // namespace

// A private stream, destroyed after every member buffer was freed on it (it is
// the first member, so the last one destroyed).
struct OwnedStream {
  cudaStream_t s = nullptr;
  ~OwnedStream() {
    if (s) cudaStreamDestroy(s);
  }
};

struct mlmc_hierarchy {
  OwnedStream own;     // set when the caller passes the legacy stream
  cudaStream_t stream = nullptr;
  int complex_op = 0;
  DType t64 = F64, t32 = F32;
  mlmc_hierarchy_params prm{};
  int L = 0, kmax = 0;
  int kact = 0;        // active vector-block width of estimates and sample calls (<= kmax)
  int kwide = 0;       // vector-block width of samples drawn on level difference 2 (coarse levels)
  int kgrow = 0;       // g > 0: the width grows by 2^g per further level difference (up to 512; 256 complex)
  int kbig = 0;        // the largest block width of any level difference: sizes the per-column scratch
  std::vector<int> wl; // per level: the widest block its buffers serve
  // block width of level difference l0 (0-based; l0 = 0 is the fine difference)
  int kdiff(int l0) const {
    if (l0 == 0) return kact;
    long k = kwide;
    const long cap = complex_op ? 256L : 512L;     // column groups of the Arnoldi dot products
    for (int i = 1; i < l0 && kgrow; ++i) k = std::min(k << std::min(kgrow, 4), cap);
    return (int)k;
  }
  std::vector<Level> lv;
  std::vector<CycleBufs> cyc[2];                  // [0] FP64 cycle, [1] FP32 cycle
  std::vector<std::unique_ptr<Krylov>> outer;     // FP64 outer FGMRES per level
  std::vector<std::unique_ptr<Krylov>> inner[2];  // fixed-length inner FGMRES per level, [0] FP64 [1] FP32
  int const_laplace = 0, periodic = 0;
  int dense_kernel = MLMC_DENSE_AUTO;   // coarsest apply of the FP32 cycle: tensor cores, CUDA cores, or by size
  int conv_kernel = MLMC_CONV_AUTO;     // learned correction's convolutions: CUDA cores, tensor cores, or by timing
  int conv_auto_tc = 0;                 // MLMC_CONV_AUTO: 1 when the tensor-core kernels timed faster
  double conv_tuned_ms[2] = {0.0, 0.0}; // that timing: network forward, CUDA cores / tensor cores
  int conv_tuned = 0;
  int bilinear = 0;    // the Example 5.1 hierarchy of Sec. 5: bilinear P, Galerkin 9-point levels
  double coarse_term_hat = 0.0;   // bilinear: tr(A_L^{-1} R^_L P^_L) (Remark 4.2), computed at setup
  double laplace_diag = 4.0;
  // learned correction on the fine level (FP32 cycle only)
  int net_on = 0, net_c0 = 0, net_nw = 0, net_alloc_k = 0, net_step = 0, net_fallbacks = 0;
  DevBuf netW, netG, netM, netV, netPart, act0, act1, act2, act3, g1, g2, lcol, lalpha;
  DevBuf capture;
  size_t capture_blocks = 0, capture_n = 0;
  int capturing = 0;
  // CUDA graphs of the inner solves
  std::vector<GraphEntry> graphs;
  ~mlmc_hierarchy() {
    for (auto &g : graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
  }
  std::vector<DevBuf> xs, ys;                     // sample blocks per level (FP64)
  DevBuf dots, dots_part, samples, acc, err, trace;
  DevBuf coarse_r;     // FP64 residual of the mixed form's refined coarsest solve (n_L x widest block)
  uint64_t launches = 0;
  double iters_accum[16] = {0}, solves_accum[16] = {0};
  double cost = 0.0;   // Sec. 5 cost model: running sum of nnz(B) over products B x (per column)
};

namespace {

using H_t = mlmc_hierarchy;

size_t acc_size(const H_t &h) { return h.complex_op ? 16 : 8; }

StencilView view(const H_t &h, int l, int lo) {
  const Level &L = h.lv[l];
  StencilView v;
  v.nx = L.nx;
  v.ny = L.ny;
  v.d = L.d;
  v.t = lo ? h.t32 : h.t64;
  v.coef = lo ? L.coef32.p : L.coef64.p;
  v.dinv = lo ? L.dinv32.p : L.dinv64.p;
  v.const_laplace = (l == 0 && h.const_laplace) ? 1 : 0;
  v.diag = h.laplace_diag;
  v.periodic = h.periodic;
  v.taps = L.taps;
  return v;
}

ProlongView pview(const H_t &h, int l, int lo) {
  const Level &L = h.lv[l];
  ProlongView v;
  v.nx = L.nx;
  v.ny = L.ny;
  v.d = L.d;
  v.ax = L.ax;
  v.ay = L.ay;
  v.dc = L.dc;
  v.t = lo ? h.t32 : h.t64;
  v.P = lo ? L.P32.p : L.P64.p;
  v.bilinear = h.bilinear;
  return v;
}

void alloc_krylov(H_t &h, Krylov &K, DType t, size_t n, int k, int m) {
  K.t = t;
  K.hc = dtype_complex(t);
  K.n = n;
  K.k = k;
  K.m = m;
  size_t blk = n * (size_t)k * dtype_size(t);
  size_t as = acc_size(h);
  K.V.alloc(blk * (m + 1));
  K.Z.alloc(blk * m);
  // multi-dot partials of up to m + 1 vectors, or the multi-AXPY's fused column norms
  K.partials.alloc(std::max((size_t)multidot_parts(n, k) * (m + 1), (size_t)multiaxpy_norm_parts(n, k)) * k * as);
  K.H.alloc((size_t)m * (m + 1) * k * as);
  K.cs.alloc((size_t)m * k * as);
  K.sn.alloc((size_t)m * k * as);
  K.g.alloc((size_t)(m + 1) * k * as);
  K.y.alloc((size_t)m * k * as);
  K.h2.alloc((size_t)(m + 1) * k * as);
  K.bnorm.alloc(k * sizeof(double));
  K.invnrm.alloc(k * sizeof(double));
  K.resid.alloc(k * sizeof(double));
  K.active.alloc(k * sizeof(int));
  K.jdone.alloc(k * sizeof(int));
  K.nactive.alloc(sizeof(int));
  K.sc.alloc((size_t)(m + 1) * k * sizeof(double));
  K.hco.alloc((size_t)(m + 1) * k * as);
}

int read_nactive(H_t &h, Krylov &K) {
  check_cuda(cudaMemcpyAsync(&K.h_nactive, K.nactive.p, sizeof(int), cudaMemcpyDeviceToHost, h.stream), "D2H nactive");
  check_cuda(cudaStreamSynchronize(h.stream), "sync");
  return K.h_nactive;
}

// Number of (site, coupled site) pairs of a nearest-neighbour stencil on an
// nx x ny lattice: the site itself and its distinct +-x, +-y neighbours
// (Dirichlet: neighbours off the lattice are absent; periodic: on sides of 1
// or 2 sites the neighbours coincide with the site or with each other).
double site_pairs(int nx, int ny, int periodic) {
  auto axis = [&](int n) {               // distinct neighbours other than the site, summed over a line
    if (!periodic) return 2.0 * n - 2.0;
    return n >= 3 ? 2.0 * n : n == 2 ? 2.0 : 0.0;
  };
  return (double)nx * ny + axis(nx) * ny + axis(ny) * nx;
}

// nnz of A_l: Example 5.1 (5n - 2nx - 2ny with Dirichlet), Example 5.3 (9 per row:
// a diagonal self block and four full 2 x 2 hopping blocks), Table 1's 9-point
// levels, and full d x d blocks for every coupled site pair on coarse levels
double nnz_of(const H_t &h, int l) {
  const Level &L = h.lv[l];
  if (l == 0 && h.const_laplace) return site_pairs(L.nx, L.ny, h.periodic);
  if (l == 0 && h.complex_op) return 2.0 * L.nsite + 4.0 * (site_pairs(L.nx, L.ny, 1) - L.nsite);
  if (L.taps == 9) return (3.0 * L.nx - 2.0) * (3.0 * L.ny - 2.0);      // Table 1: (3 N_l - 2)^2
  return site_pairs(L.nx, L.ny, h.periodic || h.complex_op) * L.d * L.d;   // Wilson lattices are periodic
}

// nnz(P_l): the cost-model weight of one restriction or prolongation per column.
// Aggregation: every fine dof row holds the dc columns of its aggregate, or
// half of them with the spin split (each column lives on one spin half).
double nnz_P(const H_t &h, int l) {
  if (h.bilinear) return 9.0 * (double)h.lv[l + 1].n;     // three 1-D weights per coarse point and direction
  return (double)h.lv[l].n * h.lv[l].dc / (h.prm.spin_split ? 2.0 : 1.0);
}

// Nominal cost of one sample of level difference l (0-based) in the Sec. 5
// cost model, independent of how many iterations the solves take: the
// restrictions the sample's noise needs, then one product with each operator
// it solves with (the multigrid solve costs a level-independent multiple of
// that for an optimal solver), the dense inverse of the coarsest level
// counting n_L^2.
double nominal_sample_cost(const H_t &h, int l, int form) {
  auto solve_cost = [&](int lev) {
    return lev == h.L - 1 ? (double)h.lv[lev].n * h.lv[lev].n : nnz_of(h, lev);
  };
  if (form == MLMC_FORM_PLAIN) return solve_cost(0);
  double c = solve_cost(l);
  if (l + 1 < h.L) c += solve_cost(l + 1);
  const int restrictions = form == MLMC_FORM_HAT ? l + 1 : 1;   // R^_l x, R^_{l+1} x  /  R_l x
  for (int j = (form == MLMC_FORM_HAT ? 0 : l); j < (form == MLMC_FORM_HAT ? restrictions : l + 1); ++j)
    if (j + 1 < h.L) c += nnz_P(h, j);
  return c;
}

void apply_op(H_t &h, int l, int lo, const void *x, void *y, int k) {
  launch_stencil(view(h, l, lo), x, nullptr, y, k, 0, h.stream);
  h.launches++;
  h.cost += nnz_of(h, l) * k;
}

void residual_op(H_t &h, int l, int lo, const void *x, const void *b, void *r, int k) {
  launch_stencil(view(h, l, lo), x, b, r, k, 1, h.stream);
  h.launches++;
  h.cost += nnz_of(h, l) * k;
}

void dense_apply(H_t &h, int lo, const void *b, void *x, int k) {
  const Level &C = h.lv[h.L - 1];
  const int kdim = (int)C.n * (h.complex_op ? 2 : 1);
  const bool tc = h.dense_kernel == MLMC_DENSE_TC || (h.dense_kernel == MLMC_DENSE_AUTO && kdim >= 512);
  if (lo && tc && dense_apply_tc_ok(h.t32, (int)C.n, k)) {
    launch_dense_apply_tc(h.t32, C.Ainv32.p, b, x, (int)C.n, k, C.dense_part.p, C.dense_part.bytes, h.err.as<int>(),
                          h.stream);
    h.launches += dense_apply_tc_part_bytes(h.t32, (int)C.n, k) ? 2 : 1;
  } else {
    launch_dense_apply(lo ? h.t32 : h.t64, lo ? C.Ainv32.p : C.Ainv64.p, b, x, (int)C.n, k, C.dense_part.p,
                       h.stream);
    h.launches++;
  }
  h.cost += (double)C.n * C.n * k;
}

void multidot(H_t &h, Krylov &K, const void *V, int nvec, const void *w, int k, void *out,
              const double *lazy_sc = nullptr, void *lazy_coef = nullptr, int lazy_j = 0) {
  launch_multidot(K.t, V, K.n * (size_t)k, nvec, w, K.n, k, K.partials.p, multidot_parts(K.n, k), out,
                  K.hc ? C64 : F64, h.stream, lazy_sc, lazy_coef, lazy_j);
  h.launches += 2;
}

using Precond = std::function<void(const void *, void *)>;

// Batched flexible GMRES(m) (Saad, Alg. 9.6) on level l with element type K.t.
// fixed_its > 0: exactly that many steps from x0 = 0, no host synchronisation
// (K-cycle coarse correction).  Otherwise restarts from the true residual
// until every column meets ||b - A x|| <= tol ||b|| or max_iter is reached.
// Returns the number of iterations.
int fgmres(H_t &h, Krylov &K, int l, int lo, const void *b, void *x, int k, double tol, int fixed_its,
           int maxit, const Precond &M, bool reorth, bool *converged) {
  const size_t es = dtype_size(K.t), as = acc_size(h);
  const size_t blk = K.n * (size_t)k;
  const int m = K.m;
  auto Vj = [&](int j) { return (char *)K.V.p + (size_t)j * blk * es; };
  auto Zj = [&](int j) { return (char *)K.Z.p + (size_t)j * blk * es; };
  auto Hcol = [&](int j) { return (char *)K.H.p + (size_t)j * (m + 1) * k * as; };
  const bool fixed = fixed_its > 0;
  // fixed length (inner solves, K-cycle): the basis vectors stay unnormalised (no
  // scaling pass over each new vector; see k_multidot_reduce)
  const bool lazy = fixed && !reorth;
  double *sc = lazy ? K.sc.as<double>() : nullptr;
  cudaStream_t s = h.stream;

  check_cuda(cudaMemcpyAsync(Vj(0), b, blk * es, cudaMemcpyDeviceToDevice, s), "copy b");
  multidot(h, K, Vj(0), 1, Vj(0), k, K.g.p);
  check_cuda(cudaMemsetAsync(K.nactive.p, 0, sizeof(int), s), "memset");
  launch_arnoldi_init(K.hc, K.g.p, K.bnorm.as<double>(), K.invnrm.as<double>(), K.active.as<int>(),
                      K.jdone.as<int>(), k, fixed ? 0.0 : tol, 1, K.nactive.as<int>(), s, sc);
  h.launches++;
  check_cuda(cudaMemsetAsync(x, 0, blk * es, s), "memset x");
  if (converged) *converged = true;
  if (!fixed) {
    const int na = read_nactive(h, K);
    if (na >= NONFINITE_COLUMN) {            // b is not finite: no iteration can help
      if (converged) *converged = false;
      return 0;
    }
    if (na == 0) return 0;
  }
  int its = 0;
  for (;;) {
    if (!lazy) {
      launch_scale_cols(K.t, Vj(0), Vj(0), K.invnrm.p, 0, K.n, k, s);
      h.launches++;
    }
    int jlast = 0;
    for (int j = 0; j < m; ++j) {
      M(Vj(j), Zj(j));
      apply_op(h, l, lo, Zj(j), Vj(j + 1), k);
      // unnormalised basis: the reduction also forms the Hessenberg entries and the
      // multi-AXPY's coefficients (see k_multidot_reduce)
      multidot(h, K, K.V.p, j + 1, Vj(j + 1), k, Hcol(j), lazy ? sc : nullptr, lazy ? K.hco.p : nullptr, j);
      // fixed length: the multi-AXPY also sums |u_{j+1}|^2 per column (no separate norm pass)
      const int nparts = launch_multiaxpy(K.t, Vj(j + 1), K.V.p, blk, j + 1, lazy ? K.hco.p : Hcol(j),
                                          K.hc ? C64 : F64, k, -1.0, K.n, k, s, lazy ? K.partials.p : nullptr);
      h.launches++;
      if (reorth) {
        multidot(h, K, K.V.p, j + 1, Vj(j + 1), k, K.h2.p);
        launch_multiaxpy(K.t, Vj(j + 1), K.V.p, blk, j + 1, K.h2.p, K.hc ? C64 : F64, k, -1.0, K.n, k, s);
        launch_add_acc(K.hc, Hcol(j), K.h2.p, (j + 1) * k, s);
        h.launches += 2;
      }
      if (lazy) {
        launch_column_reduce(K.hc ? C64 : F64, K.partials.p, nparts, k, (char *)Hcol(j) + (size_t)(j + 1) * k * as, s);
        h.launches++;
      } else {
        multidot(h, K, Vj(j + 1), 1, Vj(j + 1), k, (char *)Hcol(j) + (size_t)(j + 1) * k * as);
      }
      check_cuda(cudaMemsetAsync(K.nactive.p, 0, sizeof(int), s), "memset");
      launch_arnoldi_step(K.hc, K.H.p, K.cs.p, K.sn.p, K.g.p, j, m, k, K.active.as<int>(), K.jdone.as<int>(),
                          K.bnorm.as<double>(), tol, K.invnrm.as<double>(), K.resid.as<double>(),
                          K.nactive.as<int>(), fixed ? 1 : 0, s, sc);
      h.launches++;
      if (!lazy) {
        launch_scale_cols(K.t, Vj(j + 1), Vj(j + 1), K.invnrm.p, 0, K.n, k, s);
        h.launches++;
      }
      ++its;
      jlast = j + 1;
      if (fixed) {
        if (its >= fixed_its) break;
        continue;
      }
      if (read_nactive(h, K) == 0 || its >= maxit) break;
    }
    launch_trisolve(K.hc, K.H.p, K.g.p, K.y.p, K.jdone.as<int>(), m, k, s);
    if (lazy) {
      launch_lazy_y(K.hc, K.y.p, sc, K.jdone.as<int>(), m, k, s);
      h.launches++;
    }
    launch_multiaxpy(K.t, x, K.Z.p, blk, jlast, K.y.p, K.hc ? C64 : F64, k, 1.0, K.n, k, s);
    h.launches += 2;
    if (fixed) return its;
    // FP64 true residual: restart, or stop when every column meets tol
    residual_op(h, l, lo, x, b, Vj(0), k);
    multidot(h, K, Vj(0), 1, Vj(0), k, K.g.p);
    check_cuda(cudaMemsetAsync(K.nactive.p, 0, sizeof(int), s), "memset");
    launch_arnoldi_init(K.hc, K.g.p, K.bnorm.as<double>(), K.invnrm.as<double>(), K.active.as<int>(),
                        K.jdone.as<int>(), k, tol, 0, K.nactive.as<int>(), s);
    h.launches++;
    const int na = read_nactive(h, K);
    if (na >= NONFINITE_COLUMN) {            // the iterate went NaN / infinite: stop, not converged
      if (converged) *converged = false;
      return its;
    }
    if (na == 0) return its;
    if (its >= maxit) {
      if (converged) *converged = false;
      return its;
    }
  }
}

void fine_hooks(H_t &h, void *x, const void *b, int k);

// One multigrid cycle (Remark 4.1) on levels l..L in FP64 (lo = 0) or FP32 (lo = 1):
// red-black block GS pre-smoothing from x = 0, residual, restriction, coarse
// correction (dense inverse on level L, recursion for a V-cycle, or kcycle_its
// FGMRES steps preconditioned by the next cycle for a K-cycle), prolongation,
// post-smoothing in reverse colour order.
void cycle(H_t &h, int lo, int l, const void *b, void *x, int k) {
  const int last = h.L - 1;
  cudaStream_t s = h.stream;
  if (l == last) {
    dense_apply(h, lo, b, x, k);
    return;
  }
  Level &Lv = h.lv[l];
  DType t = lo ? h.t32 : h.t64;
  size_t blk = Lv.n * (size_t)k;
  (void)blk;
  (void)t;
  CycleBufs &cb = h.cyc[lo][l];
  CycleBufs &cn = h.cyc[lo][l + 1];
  StencilView A = view(h, l, lo);
  const int npre = (l > 0 && h.prm.coarse_smooth > 0) ? h.prm.coarse_smooth : h.prm.smooth_pre;
  const int npost = (l > 0 && h.prm.coarse_smooth > 0) ? h.prm.coarse_smooth : h.prm.smooth_post;
  if (npre < 1) launch_fill_zero(t, x, blk, s);
  for (int it = 0; it < npre; ++it) {
    launch_rbgs_sweep(A, x, b, k, 0, it == 0, s);
    h.launches += 2;
    h.cost += nnz_of(h, l) * k;
  }
  const ProlongView Pv = pview(h, l, lo);
  if (npre >= 1 && residual_restrict_ok(A, Pv)) {
    // the pre-smoothing sweeps end on colour 1, so the residual lives on colour 0 only:
    // residual and restriction in one pass, r never stored
    launch_residual_restrict(A, Pv, x, b, cn.b.p, k, 0, s);
    h.launches++;
    h.cost += nnz_of(h, l) * k;                 // the residual's product, as counted before
  } else {
    residual_op(h, l, lo, x, b, cb.r.p, k);
    launch_restrict(Pv, cb.r.p, cn.b.p, k, s);
    h.launches++;
  }
  h.cost += 2.0 * nnz_P(h, l) * k;              // restriction and the prolongation below: nnz(P) each
  if (l + 1 == last) {
    dense_apply(h, lo, cn.b.p, cn.x.p, k);
  } else if (h.prm.cycle == MLMC_CYCLE_V) {
    cycle(h, lo, l + 1, cn.b.p, cn.x.p, k);
  } else {
    Precond M = [&h, lo, l, k](const void *v, void *z) { cycle(h, lo, l + 1, v, z, k); };
    fgmres(h, *cn.kcyc, l + 1, lo, cn.b.p, cn.x.p, k, 0.0, h.prm.kcycle_its, h.prm.kcycle_its, M, false, nullptr);
  }
  // the post-smoothing starts with colour 1 and does not read x there, so colour 1 needs no
  // prolongation, unless the fine-level hooks (learned correction, capture) read all of x
  const bool hooks = l == 0 && lo == 1 && (h.net_on || h.capturing);
  if (npost >= 1 && !hooks && A.taps == 5)
    launch_prolong_add_colour(Pv, cn.x.p, x, k, 0, s);
  else
    launch_prolong_add(Pv, cn.x.p, x, k, s);
  h.launches++;
  if (l == 0 && lo == 1) fine_hooks(h, x, b, k);
  for (int it = 0; it < npost; ++it) {
    launch_rbgs_sweep(A, x, b, k, 1, 0, s);
    h.launches += 2;
    h.cost += nnz_of(h, l) * k;
  }
}

// FP64 preconditioner of the outer solve on level l.  With inner_its > 0 it
// is `inner_its` steps of FGMRES in the cycle precision preconditioned by the
// cycle (no host synchronisation); else one cycle.  In the mixed form the
// input is rounded to FP32 and the result widened back to FP64; the outer
// FP64 FGMRES with its FP64 true residual recovers full accuracy.
// Replays (capturing on first use) the inner solve on the fixed buffers
// cyc[lo][l].b -> cyc[lo][l].x as one CUDA graph: it has no host
// synchronisation, so the whole fixed-length FGMRES with its cycles is one launch.
void inner_graph(H_t &h, int lo, int l, int k, const std::function<void()> &body) {
  GraphEntry *ge = nullptr;
  for (auto &g : h.graphs)
    if (g.level == l && g.k == k && g.net == h.net_on && g.exec) ge = &g;
  if (!ge) {
    GraphEntry g;
    g.level = l;
    g.k = k;
    g.net = h.net_on;
    double c0 = h.cost;
    uint64_t n0 = h.launches;
    cudaGraph_t graph = nullptr;
    check_cuda(cudaStreamBeginCapture(h.stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    try {
      body();
    } catch (...) {
      cudaStreamEndCapture(h.stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    check_cuda(cudaStreamEndCapture(h.stream, &graph), "end capture");
    cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    check_cuda(e, "graph instantiate");
    g.cost = h.cost - c0;
    g.launches = h.launches - n0;
    h.cost = c0;
    h.launches = n0;
    h.graphs.push_back(g);
    ge = &h.graphs.back();
  }
  check_cuda(cudaGraphLaunch(ge->exec, h.stream), "graph launch");
  h.cost += ge->cost;
  h.launches += ge->launches;
}

// FP64 preconditioner of the outer solve on level l.  With inner_its > 0 it
// is `inner_its` steps of FGMRES in the cycle precision preconditioned by the
// cycle (no host synchronisation, replayed as a CUDA graph); else one cycle.
// In the mixed form the input is rounded to FP32 and the result widened back
// to FP64; the outer FP64 FGMRES with its FP64 true residual recovers full
// accuracy.
Precond outer_precond(H_t &h, int l, int k) {
  const int lo = h.prm.precision == MLMC_PREC_MIXED_FP32 ? 1 : 0;
  const int nin = h.prm.inner_its;
  auto inner = [&h, l, k, lo, nin](const void *b, void *x) {
    if (nin > 0) {
      Precond M = [&h, l, k, lo](const void *v, void *z) { cycle(h, lo, l, v, z, k); };
      fgmres(h, *h.inner[lo][l], l, lo, b, x, k, 0.0, nin, nin, M, false, nullptr);
    } else {
      cycle(h, lo, l, b, x, k);
    }
  };
  return [&h, l, k, lo, inner](const void *v, void *z) {
    CycleBufs &cb = h.cyc[lo][l];
    size_t cnt = h.lv[l].n * (size_t)k;
    DType t = lo ? h.t32 : h.t64;
    launch_convert(t, cb.b.p, h.t64, v, cnt, h.stream);
    if (h.prm.graphs && !h.capturing) inner_graph(h, lo, l, k, [&] { inner(cb.b.p, cb.x.p); });
    else inner(cb.b.p, cb.x.p);
    launch_convert(h.t64, z, t, cb.x.p, cnt, h.stream);
    h.launches += 2;
  };
}

// x = A_L^{-1} b on the coarsest level in FP64 accuracy.  FP64 form: the FP64 dense
// inverse.  Mixed form: the FP32 inverse (tensor cores where the cycle uses them) with
// two steps of iterative refinement against the FP64 operator, x <- x + A32^{-1}(b - A x):
// each step multiplies the relative error by about cond(A_L) x 2^-24, so two steps leave
// it far below the FP64 form's tolerances, at three FP32 products instead of one FP64
// product (FP64 arithmetic is the GB300's slow path).
void coarse_solve(H_t &h, const void *b, void *x, int k) {
  const int Lc = h.L - 1;
  if (h.prm.precision != MLMC_PREC_MIXED_FP32) {
    dense_apply(h, 0, b, x, k);
    return;
  }
  const Level &C = h.lv[Lc];
  const size_t cnt = C.n * (size_t)k;
  CycleBufs &cb = h.cyc[1][Lc];
  void *r = h.coarse_r.p;
  cudaStream_t s = h.stream;
  launch_convert(h.t32, cb.b.p, h.t64, b, cnt, s);
  dense_apply(h, 1, cb.b.p, cb.x.p, k);
  launch_convert(h.t64, x, h.t32, cb.x.p, cnt, s);
  h.launches += 2;
  for (int it = 0; it < 2; ++it) {
    residual_op(h, Lc, 0, x, b, r, k);
    launch_convert(h.t32, cb.b.p, h.t64, r, cnt, s);
    dense_apply(h, 1, cb.b.p, cb.x.p, k);
    launch_convert(h.t64, r, h.t32, cb.x.p, cnt, s);
    launch_add_acc(h.complex_op, x, r, (int)cnt, s);
    h.launches += 3;
  }
}

// x = A_l^{-1} b in FP64 (dense inverse on the coarsest level).
int solve_level(H_t &h, int l, const void *b, void *x, int k, double tol, bool *conv) {
  if (conv) *conv = true;
  if (l == h.L - 1) {
    coarse_solve(h, b, x, k);
    return 0;
  }
  int its = fgmres(h, *h.outer[l], l, 0, b, x, k, tol, 0, h.prm.max_iter, outer_precond(h, l, k),
                   h.prm.reorth != 0, conv);
  if (conv && !*conv && h.net_on) {
    // the plain smoother is the fallback: repeat the solve without the network
    h.net_on = 0;
    its += fgmres(h, *h.outer[l], l, 0, b, x, k, tol, 0, h.prm.max_iter, outer_precond(h, l, k),
                  h.prm.reorth != 0, conv);
    h.net_on = 1;
    h.net_fallbacks++;
  }
  if (l < 16) {
    h.iters_accum[l] += its;
    h.solves_accum[l] += 1;
  }
  return its;
}

uint64_t key_hi(int purpose, int level) { return ((uint64_t)purpose << 8) | (uint64_t)level; }

// ----------------------------------------------------------------- learned correction
// Network c0 -> 16 -> 16 -> c0 (3x3 taps, ReLU, no bias) on the fine lattice,
// FP32; weights concatenated [W1 | W2 | W3], each [c_out][c_in][3][3].
const int NET_CH = 16;

int net_weights(int c0) { return 9 * (NET_CH * c0 + NET_CH * NET_CH + c0 * NET_CH); }

void net_alloc(H_t &h) {
  const Level &F = h.lv[0];
  if (h.net_c0 == 0) {
    h.net_c0 = F.d * (h.complex_op ? 2 : 1);
    h.net_nw = net_weights(h.net_c0);
    h.netW.alloc(h.net_nw * sizeof(float));
    h.netG.alloc(h.net_nw * sizeof(float));
    h.netM.alloc(h.net_nw * sizeof(float));
    h.netV.alloc(h.net_nw * sizeof(float));
    h.netPart.alloc((size_t)conv_weight_blocks() * NET_CH * NET_CH * 9 * sizeof(float));
    h.lcol.alloc(2 * (size_t)h.kmax * 16);
    h.lalpha.alloc((size_t)h.kmax * sizeof(double));
  }
  if (h.net_alloc_k < h.kmax) {
    size_t big = F.nsite * (size_t)NET_CH * h.kmax * sizeof(float);
    size_t small = F.nsite * (size_t)h.net_c0 * h.kmax * sizeof(float);
    h.act0.alloc(small);
    h.act1.alloc(big);
    h.act2.alloc(big);
    h.act3.alloc(small);
    h.g1.alloc(big);
    h.g2.alloc(big);
    h.net_alloc_k = h.kmax;
  }
}

const float *netW1(H_t &h) { return h.netW.as<float>(); }
const float *netW2(H_t &h) { return h.netW.as<float>() + 9 * NET_CH * h.net_c0; }
const float *netW3(H_t &h) { return h.netW.as<float>() + 9 * (NET_CH * h.net_c0 + NET_CH * NET_CH); }

// One convolution layer: the tensor-core implicit GEMM (kernels_conv_tc.cu) when the
// handle allows it and the shape fits (k in {8, 16, 32, 64, 128}, whole tiles of 128 / k
// sites per lattice row), else the CUDA-core kernel (kernels_learned.cu).
bool conv_on_tc(const H_t &h, int nx, int k, int cin, int cout) {
  const bool want = h.conv_kernel == MLMC_CONV_TC || (h.conv_kernel == MLMC_CONV_AUTO && h.conv_auto_tc);
  return want && conv_tc_ok(nx, k, cin, cout);
}

void conv_forward(H_t &h, int ci, int co, bool relu, const float *in, const float *W, float *out, int k) {
  const Level &F = h.lv[0];
  const int per = h.periodic || h.complex_op;
  if (conv_on_tc(h, F.nx, k, ci, co))
    launch_conv_tc(in, W, nullptr, out, F.nx, F.ny, k, ci, co, per, 0, relu ? 1 : 0, h.err.as<int>(), h.stream);
  else
    launch_conv_fwd(ci, co, relu, in, W, out, F.nx, F.ny, k, per, h.stream);
  h.launches++;
}

// gradient wrt the input of a layer ci -> co, masked by act > 0 (the ReLU below it)
void conv_backward_data(H_t &h, int ci, int co, const float *gout, const float *W, const float *act, float *gin,
                        int k) {
  const Level &F = h.lv[0];
  const int per = h.periodic || h.complex_op;
  if (conv_on_tc(h, F.nx, k, co, ci))
    launch_conv_tc(gout, W, act, gin, F.nx, F.ny, k, co, ci, per, 1, 0, h.err.as<int>(), h.stream);
  else
    launch_conv_bwd_data(ci, co, gout, W, act, gin, F.nx, F.ny, k, per, h.stream);
  h.launches++;
}

void conv_backward_weight(H_t &h, int ci, int co, const float *in, const float *gout, float *G, int k) {
  const Level &F = h.lv[0];
  const int per = h.periodic || h.complex_op;
  const bool want = h.conv_kernel == MLMC_CONV_TC || (h.conv_kernel == MLMC_CONV_AUTO && h.conv_auto_tc);
  if (want && conv_wgrad_tc_ok(k, ci, co)) {
    launch_conv_wgrad_tc(in, gout, h.netPart.as<float>(), F.nx, F.ny, k, ci, co, per, h.err.as<int>(), h.stream);
    launch_weight_reduce(h.netPart.as<float>(), conv_wgrad_tc_blocks(), ci * co * 9, G, 1.f, h.stream);
  } else {
    launch_conv_bwd_weight(ci, co, in, gout, h.netPart.as<float>(), G, 1.f, F.nx, F.ny, k, per, h.stream);
  }
  h.launches += 2;
}

// act3 = net(r) in channel layout; act0..act2 keep the activations
void net_forward(H_t &h, const void *r, int k) {
  const Level &F = h.lv[0];
  cudaStream_t s = h.stream;
  launch_to_channels(h.t32, r, h.act0.as<float>(), (int)F.nsite, F.d, k, s);
  h.launches++;
  conv_forward(h, h.net_c0, NET_CH, true, h.act0.as<float>(), netW1(h), h.act1.as<float>(), k);
  conv_forward(h, NET_CH, NET_CH, true, h.act1.as<float>(), netW2(h), h.act2.as<float>(), k);
  conv_forward(h, NET_CH, h.net_c0, false, h.act2.as<float>(), netW3(h), h.act3.as<float>(), k);
}

// MLMC_CONV_AUTO: time the network on a fine-level block of the sample width with the
// tensor-core and with the CUDA-core convolutions (CUDA events, after a warm-up) and keep
// the faster; the captured inner solves are dropped, since they bake the choice in.
// Runs outside any stream capture (when the network is installed or trained).
// Captured inner solves bake in the kernel choices: drop them when a choice changes.
void drop_graphs(mlmc_hierarchy &h) {
  check_cuda(cudaStreamSynchronize(h.stream), "sync");
  for (auto &g : h.graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h.graphs.clear();
}

void tune_conv(H_t &h) {
  if (h.conv_kernel != MLMC_CONV_AUTO) return;
  const Level &F = h.lv[0];
  const int k = h.kdiff(0);
  if (!conv_tc_ok(F.nx, k, h.net_c0, NET_CH)) {
    h.conv_auto_tc = 0;
    return;
  }
  void *x = h.cyc[1][0].b.p;
  launch_noise(h.complex_op, 9, 0, 0, F.n, k, h.t32, x, h.stream);
  cudaEvent_t e0, e1;
  check_cuda(cudaEventCreate(&e0), "event");
  check_cuda(cudaEventCreate(&e1), "event");
  float ms[2] = {0.f, 0.f};
  for (int tc = 0; tc < 2; ++tc) {
    h.conv_auto_tc = tc;
    net_forward(h, x, k);
    check_cuda(cudaEventRecord(e0, h.stream), "record");
    for (int r = 0; r < 3; ++r) net_forward(h, x, k);
    check_cuda(cudaEventRecord(e1, h.stream), "record");
    check_cuda(cudaEventSynchronize(e1), "sync");
    check_cuda(cudaEventElapsedTime(&ms[tc], e0, e1), "elapsed");
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h.conv_auto_tc = ms[1] < ms[0] ? 1 : 0;
  h.conv_tuned = 1;
  h.conv_tuned_ms[0] = ms[0] / 3.0;
  h.conv_tuned_ms[1] = ms[1] / 3.0;
  drop_graphs(h);
}

// Loss mean_c ||A net(r_c) - r_c||^2 / ||r_c||^2 over the block and (grad = 1)
// its weight gradients in netG.  Uses the FP32 cycle buffers of level 0 as scratch.
double net_loss_grad(H_t &h, const void *r, int k, bool grad, bool read_loss) {
  const Level &F = h.lv[0];
  cudaStream_t s = h.stream;
  size_t cnt = F.n * (size_t)k;
  void *E = h.cyc[1][0].x.p, *Tt = h.cyc[1][0].b.p;
  net_forward(h, r, k);
  launch_fill_zero(h.t32, E, cnt, s);
  launch_add_from_channels(h.t32, E, h.act3.as<float>(), (int)F.nsite, F.d, k, s);
  residual_op(h, 0, 1, E, r, Tt, k);                             // t = r - A e
  Krylov &K = *h.outer[0];
  const size_t as = acc_size(h);
  char *nr2 = h.lcol.as<char>(), *nt2 = nr2 + (size_t)k * as;
  launch_multidot(h.t32, r, cnt, 1, r, F.n, k, K.partials.p, multidot_parts(F.n, k), nr2, C64, s);
  launch_multidot(h.t32, Tt, cnt, 1, Tt, F.n, k, K.partials.p, multidot_parts(F.n, k), nt2, C64, s);
  h.launches += 6;
  double loss = 0.0;
  if (read_loss) {
    std::vector<char> buf(2 * (size_t)k * as);
    check_cuda(cudaMemcpyAsync(buf.data(), nr2, 2 * (size_t)k * as, cudaMemcpyDeviceToHost, s), "D2H loss");
    check_cuda(cudaStreamSynchronize(s), "sync");
    for (int c = 0; c < k; ++c) {
      double a2 = *(double *)(buf.data() + c * as), t2 = *(double *)(buf.data() + (k + c) * as);
      if (a2 > 0) loss += t2 / a2 / k;
    }
  }
  if (!grad) return loss;
  // g = -2 A^H t / (||r||^2 k);  A^H = J A J for the Wilson operator (J A = A^* J), A for the Laplacian
  if (h.complex_op) launch_spin_flip(h.t32, Tt, (int)F.nsite, F.d, k, s);
  apply_op(h, 0, 1, Tt, E, k);
  if (h.complex_op) launch_spin_flip(h.t32, E, (int)F.nsite, F.d, k, s);
  launch_col_factor(h.complex_op, nr2, h.lalpha.as<double>(), -2.0 / k, k, s);
  launch_scale_cols(h.t32, E, E, h.lalpha.p, 0, F.n, k, s);
  float *g3 = h.act3.as<float>();     // reuse: the output activations are no longer needed
  launch_to_channels(h.t32, E, g3, (int)F.nsite, F.d, k, s);
  float *G = h.netG.as<float>();
  float *G1 = G, *G2 = G + 9 * NET_CH * h.net_c0, *G3 = G2 + 9 * NET_CH * NET_CH;
  conv_backward_weight(h, NET_CH, h.net_c0, h.act2.as<float>(), g3, G3, k);
  conv_backward_data(h, NET_CH, h.net_c0, g3, netW3(h), h.act2.as<float>(), h.g2.as<float>(), k);
  conv_backward_weight(h, NET_CH, NET_CH, h.act1.as<float>(), h.g2.as<float>(), G2, k);
  conv_backward_data(h, NET_CH, NET_CH, h.g2.as<float>(), netW2(h), h.act1.as<float>(), h.g1.as<float>(), k);
  conv_backward_weight(h, h.net_c0, NET_CH, h.act0.as<float>(), h.g1.as<float>(), G1, k);
  h.launches += h.complex_op ? 5 : 3;   // spin flips, column factors, scaling, channel layout
  return loss;
}

// Fine-level hooks of the FP32 cycle, after the coarse-grid correction:
// capture the residual (training data) and/or apply x += net(b - A x).
void fine_hooks(H_t &h, void *x, const void *b, int k) {
  if (h.capturing && h.capture_n < h.capture_blocks && k == h.kmax) {
    const Level &F = h.lv[0];
    char *slot = h.capture.as<char>() + h.capture_n * F.n * (size_t)k * dtype_size(h.t32);
    residual_op(h, 0, 1, x, b, slot, k);
    h.capture_n++;
  }
  if (h.net_on) {
    const Level &F = h.lv[0];
    void *r = h.cyc[1][0].r.p;
    residual_op(h, 0, 1, x, b, r, k);
    net_forward(h, r, k);
    launch_add_from_channels(h.t32, x, h.act3.as<float>(), (int)F.nsite, F.d, k, h.stream);
    h.launches++;
  }
}

// ----------------------------------------------------------------- setup
void filter(H_t &h, int l, void *V, void *tmp, void *tmp2, int ntv, int kind, int sweeps, double omega) {
  StencilView A = view(h, l, 0);
  if (kind == MLMC_SETUP_SMOOTH && A.const_laplace) {
    // Example 5.1: apply and update in one pass, alternating between V and tmp
    void *src = V, *dst = tmp;
    for (int it = 0; it < sweeps; ++it) {
      launch_laplace_jacobi(A, src, dst, ntv, omega, h.stream);
      h.launches++;
      std::swap(src, dst);
    }
    if (src != V)
      check_cuda(cudaMemcpyAsync(V, src, h.lv[l].n * (size_t)ntv * dtype_size(h.t64), cudaMemcpyDeviceToDevice,
                                 h.stream), "copy filtered V");
    return;
  }
  for (int it = 0; it < sweeps; ++it) {
    if (kind == MLMC_SETUP_SMOOTH) {
      apply_op(h, l, 0, V, tmp, ntv);
      launch_jacobi_update(A, V, V, nullptr, tmp, omega, ntv, h.stream);
      h.launches++;
    } else if (kind == MLMC_SETUP_INVERSE) {
      launch_jacobi_update(A, tmp2, nullptr, V, nullptr, omega, ntv, h.stream);   // x1 = w D^-1 v
      apply_op(h, l, 0, tmp2, tmp, ntv);                                          // A x1
      launch_jacobi_update(A, V, tmp2, V, tmp, omega, ntv, h.stream);             // x1 + w D^-1 (v - A x1)
      h.launches += 2;
    }
  }
}

void check_err(H_t &h, const char *what) {
  int e = 0;
  check_cuda(cudaMemcpyAsync(&e, h.err.p, sizeof(int), cudaMemcpyDeviceToHost, h.stream), "D2H err");
  check_cuda(cudaStreamSynchronize(h.stream), "sync");
  if (e == MLMC_ERR_TIMEOUT) fail(MLMC_ERR_TIMEOUT, std::string(what) + ": a bounded wait gave up");
  if (e) fail(MLMC_ERR_SINGULAR, std::string(what) + ": singular block or dependent test vectors (code " +
                                      std::to_string(e) + ")");
}

// The tensor-core coarsest apply records MLMC_ERR_TIMEOUT in h.err when one of
// its bounded waits gives up; the entry points that run solves report it.
void check_timeout(H_t &h) {
  int e = 0;
  check_cuda(cudaMemcpyAsync(&e, h.err.p, sizeof(int), cudaMemcpyDeviceToHost, h.stream), "D2H err");
  check_cuda(cudaStreamSynchronize(h.stream), "sync");
  if (e == MLMC_ERR_TIMEOUT) {
    check_cuda(cudaMemsetAsync(h.err.p, 0, sizeof(int), h.stream), "memset err");
    fail(MLMC_ERR_TIMEOUT, "a bounded tensor-core wait in the coarsest apply gave up");
  }
}

// Levels 2..L from the level-1 test vectors (or from user-supplied P).
void build_levels(H_t &h, const void *V1, const void *const *user_P) {
  const int ntv = h.prm.n_tv;
  const size_t es = dtype_size(h.t64);
  DevBuf Va, Vb, T1, T2;
  size_t maxn = h.lv[0].n;
  Va.alloc(maxn * ntv * es);
  Vb.alloc(maxn * ntv * es);
  T1.alloc(maxn * ntv * es);
  T2.alloc(maxn * ntv * es);
  if (!user_P) check_cuda(cudaMemcpyAsync(Va.p, V1, h.lv[0].n * ntv * es, cudaMemcpyDeviceToDevice, h.stream), "copy V");
  void *V = Va.p, *Vn = Vb.p;
  for (int l = 0; l + 1 < h.L; ++l) {
    Level &F = h.lv[l];
    Level &C = h.lv[l + 1];
    size_t pbytes = (size_t)(F.nx / F.ax) * (F.ny / F.ay) * F.ax * F.ay * F.d * F.dc * es;
    if (user_P) {
      check_cuda(cudaMemcpyAsync(F.P64.p, user_P[l], pbytes, cudaMemcpyHostToDevice, h.stream), "H2D P");
    } else {
      if (l > 0) filter(h, l, V, T1.p, T2.p, ntv, h.prm.setup_kind, h.prm.coarse_sweeps, h.prm.setup_omega);
      launch_mgs(h.t64, V, F.P64.p, F.nx, F.ny, F.d, F.ax, F.ay, ntv, h.prm.spin_split, h.err.as<int>(), h.stream);
      h.launches++;
    }
    launch_galerkin(view(h, l, 0), pview(h, l, 0), C.coef64.p, h.stream);
    h.launches++;
    if (!user_P && l + 2 < h.L) {
      launch_restrict(pview(h, l, 0), V, Vn, ntv, h.stream);
      h.launches++;
      std::swap(V, Vn);
    }
  }
  check_err(h, "setup (MGS)");
  for (int l = 0; l + 1 < h.L; ++l) {
    launch_block_inverse(h.t64, h.lv[l].coef64.p, h.lv[l].dinv64.p, (int)h.lv[l].nsite, h.lv[l].d,
                         h.err.as<int>(), h.stream);
    h.launches++;
  }
  check_err(h, "setup (smoother blocks)");
  Level &C = h.lv[h.L - 1];
  {
    DevBuf dense, work, col;
    dense.alloc(C.n * C.n * es);
    work.alloc(C.n * 2 * C.n * es);
    const size_t gjb = gauss_jordan_scratch_bytes((int)C.n);
    col.alloc(gjb);
    launch_stencil_to_dense(view(h, h.L - 1, 0), dense.p, h.stream);
    launch_gauss_jordan(h.t64, dense.p, C.Ainv64.p, work.p, (int)C.n, h.err.as<int>(), col.p, gjb, h.stream);
    h.launches += 5 + 3;
    check_err(h, "coarsest inverse");
  }
  if (h.prm.precision == MLMC_PREC_MIXED_FP32) {
    for (int l = 0; l < h.L; ++l) {
      Level &Lv = h.lv[l];
      launch_convert(h.t32, Lv.coef32.p, h.t64, Lv.coef64.p, Lv.nsite * Lv.taps * Lv.d * Lv.d, h.stream);
      if (l + 1 < h.L) {
        launch_convert(h.t32, Lv.dinv32.p, h.t64, Lv.dinv64.p, Lv.nsite * Lv.d * Lv.d, h.stream);
        size_t pc = (size_t)(Lv.nx / Lv.ax) * (Lv.ny / Lv.ay) * Lv.ax * Lv.ay * Lv.d * Lv.dc;
        launch_convert(h.t32, Lv.P32.p, h.t64, Lv.P64.p, pc, h.stream);
      }
      h.launches += 3;
    }
    launch_convert(h.t32, C.Ainv32.p, h.t64, C.Ainv64.p, C.n * C.n, h.stream);
    h.launches++;
  }
}

// ----------------------------------------------------------------- bilinear hierarchy (Sec. 5, Example 5.1)
// 9-point stencils on the host, taps 0 self, 1 +x, 2 -x, 3 +y, 4 -y, 5 (+x,+y),
// 6 (-x,+y), 7 (+x,-y), 8 (-x,-y), row-major over sites s = j*nx + i.
const int kTapDx[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
const int kTapDy[9] = {0, 0, 0, 1, -1, 1, 1, -1, -1};

int tap_of(int dx, int dy) {
  for (int q = 0; q < 9; ++q)
    if (kTapDx[q] == dx && kTapDy[q] == dy) return q;
  return -1;
}

// A_c = P^T A P for bilinear P from the ((nx-1)/2) x ((ny-1)/2) grid: coarse
// point (I, J) sits on fine (2I+1, 2J+1) with 1-D weights 1 (centre), 1/2 (+-1).
std::vector<double> galerkin9(const std::vector<double> &Af, int nx, int ny) {
  const int ncx = (nx - 1) / 2, ncy = (ny - 1) / 2;
  std::vector<double> Ac((size_t)ncx * ncy * 9, 0.0);
  auto w1 = [](int a) { return a == 0 ? 1.0 : 0.5; };
  for (int J = 0; J < ncy; ++J)
    for (int I = 0; I < ncx; ++I) {
      double *row = &Ac[((size_t)J * ncx + I) * 9];
      for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
          const int px = 2 * I + 1 + a, py = 2 * J + 1 + b;
          const double wp = w1(a) * w1(b);
          const double *ap = &Af[((size_t)py * nx + px) * 9];
          for (int q = 0; q < 9; ++q) {
            const int qx = px + kTapDx[q], qy = py + kTapDy[q];
            if (qx < 0 || qx >= nx || qy < 0 || qy >= ny || ap[q] == 0.0) continue;
            for (int J2 = J - 1; J2 <= J + 1; ++J2)
              for (int I2 = I - 1; I2 <= I + 1; ++I2) {
                if (I2 < 0 || I2 >= ncx || J2 < 0 || J2 >= ncy) continue;
                const int ex = qx - (2 * I2 + 1), ey = qy - (2 * J2 + 1);
                if (ex < -1 || ex > 1 || ey < -1 || ey > 1) continue;
                row[tap_of(I2 - I, J2 - J)] += wp * ap[q] * w1(ex) * w1(ey);
              }
          }
        }
    }
  return Ac;
}

// Levels 2..L by Galerkin coarsening with bilinear P (host, FP64), their smoother
// diagonals, the coarsest inverse, and the exact term of the hat form,
// tr(A_L^{-1} R^_L P^_L) = sum_ij (A_L^{-1})_ij M_ji with M = R^_L P^_L obtained by
// coarsening the identity the same way (M is symmetric: R = P^T).
void build_bilinear(H_t &h, const mlmc_operator_desc *op) {
  const int L = h.L;
  std::vector<double> A, M;
  {
    const int nx = h.lv[0].nx, ny = h.lv[0].ny;
    A.assign((size_t)nx * ny * 9, 0.0);
    M.assign((size_t)nx * ny * 9, 0.0);
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double *a = &A[((size_t)j * nx + i) * 9];
        a[0] = 4.0 + op->shift;
        for (int q = 1; q <= 4; ++q) {
          const int ii = i + kTapDx[q], jj = j + kTapDy[q];
          if (ii >= 0 && ii < nx && jj >= 0 && jj < ny) a[q] = -1.0;
        }
        M[((size_t)j * nx + i) * 9] = 1.0;
      }
  }
  const size_t es = sizeof(double);
  for (int l = 0; l + 1 < L; ++l) {
    A = galerkin9(A, h.lv[l].nx, h.lv[l].ny);
    M = galerkin9(M, h.lv[l].nx, h.lv[l].ny);
    Level &C = h.lv[l + 1];
    check_cuda(cudaMemcpyAsync(C.coef64.p, A.data(), A.size() * es, cudaMemcpyHostToDevice, h.stream), "H2D coef");
    if (l + 2 < L) {
      std::vector<double> dinv(C.nsite);
      for (size_t s = 0; s < C.nsite; ++s) {
        if (A[s * 9] == 0.0) fail(MLMC_ERR_SINGULAR, "zero diagonal in a Galerkin level");
        dinv[s] = 1.0 / A[s * 9];
      }
      check_cuda(cudaMemcpyAsync(C.dinv64.p, dinv.data(), dinv.size() * es, cudaMemcpyHostToDevice, h.stream),
                 "H2D dinv");
      check_cuda(cudaStreamSynchronize(h.stream), "sync");   // dinv leaves scope
    }
    check_cuda(cudaStreamSynchronize(h.stream), "sync");     // A and M are reassigned next
  }
  launch_block_inverse(h.t64, h.lv[0].coef64.p, h.lv[0].dinv64.p, (int)h.lv[0].nsite, 1, h.err.as<int>(), h.stream);
  h.launches++;
  check_err(h, "setup (smoother diagonal)");
  // coarsest: dense matrix from the 9-point stencil, Gauss-Jordan inverse (Remark 4.2)
  Level &C = h.lv[L - 1];
  const int nxL = C.nx, nyL = C.ny, n = (int)C.n;
  {
    std::vector<double> dense((size_t)n * n, 0.0);
    for (int j = 0; j < nyL; ++j)
      for (int i = 0; i < nxL; ++i)
        for (int q = 0; q < 9; ++q) {
          const int ii = i + kTapDx[q], jj = j + kTapDy[q];
          if (ii < 0 || ii >= nxL || jj < 0 || jj >= nyL) continue;
          dense[((size_t)j * nxL + i) * n + (size_t)jj * nxL + ii] = A[((size_t)j * nxL + i) * 9 + q];
        }
    DevBuf dd, work, col;
    dd.alloc(dense.size() * es);
    work.alloc((size_t)n * 2 * n * es);
    const size_t gjb = gauss_jordan_scratch_bytes(n);
    col.alloc(gjb);
    check_cuda(cudaMemcpyAsync(dd.p, dense.data(), dense.size() * es, cudaMemcpyHostToDevice, h.stream), "H2D dense");
    launch_gauss_jordan(h.t64, dd.p, C.Ainv64.p, work.p, n, h.err.as<int>(), col.p, gjb, h.stream);
    h.launches += 3;
    check_err(h, "coarsest inverse");
    std::vector<double> Ainv((size_t)n * n);
    check_cuda(cudaMemcpyAsync(Ainv.data(), C.Ainv64.p, Ainv.size() * es, cudaMemcpyDeviceToHost, h.stream), "D2H Ainv");
    check_cuda(cudaStreamSynchronize(h.stream), "sync");
    double tr = 0.0;
    for (int j = 0; j < nyL; ++j)
      for (int i = 0; i < nxL; ++i)
        for (int q = 0; q < 9; ++q) {
          const int ii = i + kTapDx[q], jj = j + kTapDy[q];
          if (ii < 0 || ii >= nxL || jj < 0 || jj >= nyL) continue;
          const size_t r = (size_t)j * nxL + i, c = (size_t)jj * nxL + ii;
          tr += Ainv[r * n + c] * M[r * 9 + q];
        }
    h.coarse_term_hat = tr;
  }
  if (h.prm.precision == MLMC_PREC_MIXED_FP32) {
    for (int l = 0; l < L; ++l) {
      Level &Lv = h.lv[l];
      launch_convert(h.t32, Lv.coef32.p, h.t64, Lv.coef64.p, Lv.nsite * Lv.taps, h.stream);
      if (l + 1 < L) launch_convert(h.t32, Lv.dinv32.p, h.t64, Lv.dinv64.p, Lv.nsite, h.stream);
      h.launches += 2;
    }
    launch_convert(h.t32, C.Ainv32.p, h.t64, C.Ainv64.p, C.n * C.n, h.stream);
    h.launches++;
  }
}

void validate(const mlmc_operator_desc *op, const mlmc_hierarchy_params *p) {
  if (!op || !p) fail(MLMC_ERR_INVALID_ARG, "null descriptor or parameters");
  if (op->kind != MLMC_OP_LAPLACE2D && op->kind != MLMC_OP_WILSON2D) fail(MLMC_ERR_INVALID_ARG, "unknown operator kind");
  if (op->nx < 2 || op->ny < 2) fail(MLMC_ERR_INVALID_ARG, "lattice too small");
  if (op->kind == MLMC_OP_WILSON2D && !op->links) fail(MLMC_ERR_INVALID_ARG, "Wilson operator needs links");
  if (p->levels < 2 || p->levels > 16) fail(MLMC_ERR_INVALID_ARG, "levels must be in 2..16");
  if (p->transfer != MLMC_TRANSFER_AGGREGATION && p->transfer != MLMC_TRANSFER_BILINEAR)
    fail(MLMC_ERR_INVALID_ARG, "unknown transfer");
  if (p->transfer == MLMC_TRANSFER_BILINEAR) {
    // Sec. 5, Example 5.1: Dirichlet Laplacian, N_{l+1} = (N_l - 1) / 2 with N_l odd
    if (op->kind != MLMC_OP_LAPLACE2D || op->periodic)
      fail(MLMC_ERR_UNSUPPORTED, "the bilinear hierarchy is built for the Dirichlet Laplacian (Example 5.1)");
    if (p->block < 1 || p->block > 256) fail(MLMC_ERR_INVALID_ARG, "block must be in 1..256");
    if (p->coarse_block < 0 || p->coarse_block > 256) fail(MLMC_ERR_INVALID_ARG, "coarse_block must be in 0..256");
    if (p->fgmres_restart < 1 || p->fgmres_restart > 64) fail(MLMC_ERR_INVALID_ARG, "fgmres_restart must be in 1..64");
    if (p->max_iter < 1) fail(MLMC_ERR_INVALID_ARG, "max_iter must be positive");
    if (p->cycle == MLMC_CYCLE_K && (p->kcycle_its < 1 || p->kcycle_its > 8))
      fail(MLMC_ERR_INVALID_ARG, "kcycle_its must be in 1..8");
    if (p->inner_its < 0 || p->inner_its > 32) fail(MLMC_ERR_INVALID_ARG, "inner_its must be in 0..32");
    if (p->precision != MLMC_PREC_FP64 && p->precision != MLMC_PREC_MIXED_FP32)
      fail(MLMC_ERR_INVALID_ARG, "unknown precision");
    if ((double)op->nx * op->ny * (p->coarse_growth > 0 ? 512 : std::max(p->block, p->coarse_block)) >= 2147483648.0)
      fail(MLMC_ERR_UNSUPPORTED, "n * block must stay below 2^31 (32-bit kernel indexing)");
    long nx = op->nx, ny = op->ny;
    for (int l = 0; l + 1 < p->levels; ++l) {
      if (nx % 2 == 0 || ny % 2 == 0 || nx < 3 || ny < 3)
        fail(MLMC_ERR_INVALID_ARG, "bilinear coarsening needs odd sides >= 3 on every level above the coarsest");
      nx = (nx - 1) / 2;
      ny = (ny - 1) / 2;
    }
    if (nx * ny > 8192) fail(MLMC_ERR_INVALID_ARG, "coarsest level larger than 8192 unknowns");
    return;
  }
  if (p->agg_x < 1 || p->agg_y < 1) fail(MLMC_ERR_INVALID_ARG, "bad aggregate shape");
  if (p->block < 1 || p->block > 256) fail(MLMC_ERR_INVALID_ARG, "block must be in 1..256");
  if (p->coarse_block < 0 || p->coarse_block > 256) fail(MLMC_ERR_INVALID_ARG, "coarse_block must be in 0..256");
  if (p->n_tv < 1 || p->n_tv > 16) fail(MLMC_ERR_INVALID_ARG, "n_tv must be in 1..16");
  if (p->setup_kind == MLMC_SETUP_CONSTANT && (p->n_tv != 1 || p->spin_split))
    fail(MLMC_ERR_INVALID_ARG, "constant setup needs n_tv = 1 and no spin split");
  if (p->fgmres_restart < 1 || p->fgmres_restart > 64) fail(MLMC_ERR_INVALID_ARG, "fgmres_restart must be in 1..64");
  if (p->max_iter < 1) fail(MLMC_ERR_INVALID_ARG, "max_iter must be positive");
  if (p->cycle == MLMC_CYCLE_K && (p->kcycle_its < 1 || p->kcycle_its > 8))
    fail(MLMC_ERR_INVALID_ARG, "kcycle_its must be in 1..8");
  if (p->inner_its < 0 || p->inner_its > 32) fail(MLMC_ERR_INVALID_ARG, "inner_its must be in 0..32");
  if (p->precision != MLMC_PREC_FP64 && p->precision != MLMC_PREC_MIXED_FP32)
    fail(MLMC_ERR_INVALID_ARG, "unknown precision");
  if ((double)op->nx * op->ny * (op->kind == MLMC_OP_WILSON2D ? 2 : 1) *
          (p->coarse_growth > 0 ? 512 : std::max(p->block, p->coarse_block)) >=
      2147483648.0)
    fail(MLMC_ERR_UNSUPPORTED, "n * block must stay below 2^31 (32-bit kernel indexing)");
  long nx = op->nx, ny = op->ny;
  for (int l = 0; l + 1 < p->levels; ++l) {
    if (nx % p->agg_x || ny % p->agg_y) fail(MLMC_ERR_INVALID_ARG, "lattice not divisible by the aggregates");
    if (nx % 2 || ny % 2) fail(MLMC_ERR_INVALID_ARG, "smoothed levels need even lattice sizes");
    nx /= p->agg_x;
    ny /= p->agg_y;
  }
  int dc = p->n_tv * (p->spin_split ? 2 : 1);
  if (dc != 1 && dc != 2 && dc != 4 && dc != 8)
    fail(MLMC_ERR_UNSUPPORTED, "coarse dofs per site must be 1, 2, 4 or 8");
  if (nx * ny * dc > 8192) fail(MLMC_ERR_INVALID_ARG, "coarsest level larger than 8192 unknowns");
}

void setup(H_t &h, const mlmc_operator_desc *op, const mlmc_hierarchy_params *p, cudaStream_t stream) {
  validate(op, p);
  if (!stream) {
    // stream capture is not allowed on the legacy default stream: use a private
    // blocking stream (ordered with the legacy stream; every call synchronises it)
    check_cuda(cudaStreamCreate(&h.own.s), "stream create");
    stream = h.own.s;
  }
  h.stream = stream;
  g_alloc_stream = stream;
  h.prm = *p;
  h.complex_op = op->kind == MLMC_OP_WILSON2D;
  h.const_laplace = op->kind == MLMC_OP_LAPLACE2D;
  h.periodic = op->periodic ? 1 : 0;
  h.laplace_diag = 4.0 + op->shift;
  h.t64 = h.complex_op ? C64 : F64;
  h.t32 = h.complex_op ? C32 : F32;
  h.L = p->levels;
  h.bilinear = p->transfer == MLMC_TRANSFER_BILINEAR;
  h.kmax = p->block;
  h.kact = p->block;
  h.kwide = p->coarse_block > 0 ? p->coarse_block : p->block;
  h.kgrow = p->coarse_growth > 0 ? std::min(p->coarse_growth, 4) : 0;
  h.kbig = h.kmax;
  for (int l0 = 1; l0 + 1 < h.L; ++l0) h.kbig = std::max(h.kbig, h.kdiff(l0));
  // level l serves the solves of differences l (its fine side) and l - 1 (its coarse side)
  h.wl.assign(h.L, 0);
  for (int l = 0; l < h.L; ++l) {
    int w = l == 0 ? h.kmax : 0;
    if (l >= 1 && l + 1 < h.L) w = std::max(w, h.kdiff(l));
    if (l >= 1) w = std::max(w, l - 1 == 0 ? h.kmax : h.kdiff(l - 1));
    h.wl[l] = w;
  }
  const bool mixed = p->precision == MLMC_PREC_MIXED_FP32;
  const int dc = p->n_tv * (p->spin_split ? 2 : 1);
  const size_t es = dtype_size(h.t64), es32 = dtype_size(h.t32);
  h.lv.resize(h.L);
  for (int l = 0; l < h.L; ++l) {
    Level &Lv = h.lv[l];
    if (h.bilinear) {
      Lv.nx = l == 0 ? op->nx : (h.lv[l - 1].nx - 1) / 2;
      Lv.ny = l == 0 ? op->ny : (h.lv[l - 1].ny - 1) / 2;
      Lv.d = 1;
      Lv.taps = l == 0 ? 5 : 9;
    } else {
      Lv.nx = l == 0 ? op->nx : h.lv[l - 1].nx / p->agg_x;
      Lv.ny = l == 0 ? op->ny : h.lv[l - 1].ny / p->agg_y;
      Lv.d = l == 0 ? (h.complex_op ? 2 : 1) : dc;
    }
    Lv.nsite = (size_t)Lv.nx * Lv.ny;
    Lv.n = Lv.nsite * Lv.d;
    Lv.coef64.alloc(Lv.nsite * Lv.taps * Lv.d * Lv.d * es);
    if (mixed) Lv.coef32.alloc(Lv.nsite * Lv.taps * Lv.d * Lv.d * es32);
    if (l + 1 < h.L) {
      Lv.ax = h.bilinear ? 2 : p->agg_x;
      Lv.ay = h.bilinear ? 2 : p->agg_y;
      Lv.dc = h.bilinear ? 1 : dc;
      Lv.dinv64.alloc(Lv.nsite * Lv.d * Lv.d * es);
      Lv.P64.alloc(h.bilinear ? 0 : Lv.n * dc * es);      // bilinear P has no stored entries
      if (mixed) {
        Lv.dinv32.alloc(Lv.nsite * Lv.d * Lv.d * es32);
        Lv.P32.alloc(h.bilinear ? 0 : Lv.n * dc * es32);
      }
    } else {
      Lv.Ainv64.alloc(Lv.n * Lv.n * es);
      size_t most = 0;     // the split count depends on the column count of a call
      for (int kk = 1; kk <= std::max(h.kbig, p->n_tv); ++kk)
        most = std::max(most, (size_t)dense_apply_splits((int)Lv.n, kk) * kk);
      size_t part_bytes = most * Lv.n * es;
      if (mixed)
        for (int kk = 1; kk <= std::max(h.kbig, p->n_tv); ++kk)
          part_bytes = std::max(part_bytes, dense_apply_tc_part_bytes(dtype_lower(h.t64), (int)Lv.n, kk));
      Lv.dense_part.alloc(part_bytes);
      if (mixed) Lv.Ainv32.alloc(Lv.n * Lv.n * es32);
    }
  }
  // workspaces.  The FP64 cycle serves the solves in the FP64 form; in the
  // mixed form it only serves the setup bootstrap (n_tv columns) and the
  // FP32 cycle serves the solves.
  // Level 0 holds blocks of `block` columns; levels >= 1 also serve the wider
  // coarse-level samples (`coarse_block` columns).
  const int k = h.kmax;
  auto width = [&](int l) { return h.wl[l]; };
  for (int lo = 0; lo < (mixed ? 2 : 1); ++lo) {
    DType t = lo ? h.t32 : h.t64;
    h.cyc[lo].resize(h.L);
    for (int l = 0; l < h.L; ++l) {
      int kc = (lo == 0 && mixed) ? p->n_tv : std::max(width(l), p->n_tv);
      CycleBufs &cb = h.cyc[lo][l];
      size_t bytes = h.lv[l].n * (size_t)kc * dtype_size(t);
      cb.b.alloc(bytes);
      cb.x.alloc(bytes);
      if (l + 1 < h.L) cb.r.alloc(bytes);
      if (p->cycle == MLMC_CYCLE_K && l >= 1 && l + 1 < h.L) {
        cb.kcyc.reset(new Krylov());
        alloc_krylov(h, *cb.kcyc, t, h.lv[l].n, kc, p->kcycle_its);
      }
    }
  }
  h.outer.resize(h.L);
  h.xs.resize(h.L);
  h.ys.resize(h.L);
  for (int l = 0; l < h.L; ++l) {
    // the hat form draws every level difference's noise on the fine level, so the
    // fine noise block also takes the coarse-level width
    h.xs[l].alloc(h.lv[l].n * (size_t)(l == 0 ? h.kbig : width(l)) * es);
    h.ys[l].alloc(h.lv[l].n * (size_t)width(l) * es);
    if (l + 1 < h.L) {
      h.outer[l].reset(new Krylov());
      alloc_krylov(h, *h.outer[l], h.t64, h.lv[l].n, width(l), p->fgmres_restart);
      if (p->inner_its > 0) {
        int lo = mixed ? 1 : 0;
        h.inner[lo].resize(h.L);
        h.inner[lo][l].reset(new Krylov());
        alloc_krylov(h, *h.inner[lo][l], lo ? h.t32 : h.t64, h.lv[l].n, width(l), p->inner_its);
      }
    }
  }
  (void)k;
  h.dots.alloc(2 * (size_t)h.kbig * 16);
  if (mixed) h.coarse_r.alloc(h.lv[h.L - 1].n * (size_t)std::max(h.kbig, h.wl[h.L - 1]) * dtype_size(h.t64));
  h.dots_part.alloc((size_t)multidot_parts(h.lv[0].n, h.kbig) * h.kbig * 16);   // sample-dot partial sums
  h.samples.alloc((size_t)h.kbig * 16);
  h.acc.alloc(4 * sizeof(double));
  h.err.alloc(sizeof(int));
  h.trace.alloc(2 * sizeof(double));
  check_cuda(cudaMemsetAsync(h.err.p, 0, sizeof(int), h.stream), "memset err");

  // fine operator (Examples 5.1 / 5.3)
  Level &F = h.lv[0];
  if (h.complex_op) {
    DevBuf links;
    links.alloc(2 * F.nsite * sizeof(cdouble));
    check_cuda(cudaMemcpyAsync(links.p, op->links, 2 * F.nsite * sizeof(cdouble), cudaMemcpyHostToDevice, h.stream), "H2D links");
    launch_build_wilson(F.coef64.as<cdouble>(), links.as<cdouble>(), F.nx, F.ny, op->mass, h.stream);
    check_cuda(cudaStreamSynchronize(h.stream), "sync");
  } else {
    launch_build_laplace(F.coef64.as<double>(), F.nx, F.ny, op->shift, op->periodic, h.stream);
  }
  h.launches++;

  if (h.bilinear) {
    build_bilinear(h, op);
    check_cuda(cudaStreamSynchronize(h.stream), "sync");
    return;
  }
  if (p->user_P) {
    build_levels(h, nullptr, p->user_P);
    check_cuda(cudaStreamSynchronize(h.stream), "sync");
    return;
  }
  // level-1 test vectors, filtered
  const int ntv = p->n_tv;
  DevBuf V1, T1, T2;
  V1.alloc(F.n * ntv * es);
  T1.alloc(F.n * ntv * es);
  T2.alloc(F.n * ntv * es);
  if (p->setup_kind == MLMC_SETUP_CONSTANT) {
    launch_fill_one(h.t64, V1.p, F.n, h.stream);
  } else {
    launch_noise(h.complex_op ? 1 : 0, p->setup_seed, key_hi(MLMC_PURPOSE_SETUP, 1), 0, F.n, ntv, h.t64, V1.p, h.stream);
    filter(h, 0, V1.p, T1.p, T2.p, ntv, p->setup_kind, p->setup_sweeps, p->setup_omega);
  }
  h.launches++;
  build_levels(h, V1.p, nullptr);
  if (p->setup_kind != MLMC_SETUP_CONSTANT) {
    for (int round = 0; round < p->bootstrap; ++round) {
      // v <- v - M(A v), M one FP64 cycle of the current hierarchy
      for (int it = 0; it < p->boot_iters; ++it) {
        apply_op(h, 0, 0, V1.p, T1.p, ntv);
        cycle(h, 0, 0, T1.p, T2.p, ntv);
        launch_sub(h.t64, V1.p, V1.p, T2.p, F.n * ntv, h.stream);
        h.launches++;
      }
      build_levels(h, V1.p, nullptr);
    }
  }
  check_cuda(cudaStreamSynchronize(h.stream), "sync");
}

// Samples first..first+k-1 of level l (0-based) into h.samples (complex FP64).
// Returns the summed outer iterations of the two solves.
// Samples first..first+k-1 of level l (0-based) into h.samples (complex FP64).
//   simplified (Remark 4.3): x in F^{n_l};  s = x^* A_l^{-1} x - (R_l x)^* A_{l+1}^{-1} (R_l x)
//   hat (Eq. tr_ml_dec):     x in F^{n_1}, z_l = R^_l x = R_{l-1} ... R_1 x; then as above with z_l for x
//   plain (Eq. plain_tr_estimate): l = 0 only, s = x^* A_1^{-1} x (no coarse solve)
// Returns the summed outer iterations of the solves.
int sample_block(H_t &h, int l, int noise, uint64_t seed, uint64_t first, int k, double tol, int purpose,
                 bool *conv, int form = MLMC_FORM_SIMPLIFIED) {
  const int kind = noise == MLMC_NOISE_Z4 ? 1 : 0;
  cudaStream_t s = h.stream;
  if (form == MLMC_FORM_HAT) {
    launch_noise(kind, seed, key_hi(purpose, l + 1), first, h.lv[0].n, k, h.t64, h.xs[0].p, s);
    h.launches++;
    for (int j = 0; j < l; ++j) {                // R^_l x: restrict down to level l
      launch_restrict(pview(h, j, 0), h.xs[j].p, h.xs[j + 1].p, k, s);
      h.launches++;
      h.cost += nnz_P(h, j) * k;
    }
  } else {
    launch_noise(kind, seed, key_hi(purpose, l + 1), first, h.lv[l].n, k, h.t64, h.xs[l].p, s);
    h.launches++;
  }
  bool c1 = true, c2 = true;
  int its = solve_level(h, l, h.xs[l].p, h.ys[l].p, k, tol, &c1);
  char *dxy = h.dots.as<char>(), *dzw = dxy + (size_t)k * 16;
  auto coldot = [&](int lev, const void *a, const void *b, void *out) {
    launch_multidot(h.t64, a, h.lv[lev].n * (size_t)k, 1, b, h.lv[lev].n, k,
                    h.dots_part.p, multidot_parts(h.lv[lev].n, k), out, h.complex_op ? C64 : F64, s);
    h.launches += 2;
  };
  coldot(l, h.xs[l].p, h.ys[l].p, dxy);
  if (l + 1 < h.L && form != MLMC_FORM_PLAIN) {
    launch_restrict(pview(h, l, 0), h.xs[l].p, h.xs[l + 1].p, k, s);
    h.launches++;
    its += solve_level(h, l + 1, h.xs[l + 1].p, h.ys[l + 1].p, k, tol, &c2);
    coldot(l + 1, h.xs[l + 1].p, h.ys[l + 1].p, dzw);
    launch_sample_combine(h.complex_op, dxy, dzw, h.samples.p, k, s);
  } else {
    launch_sample_combine(h.complex_op, dxy, nullptr, h.samples.p, k, s);
  }
  h.launches++;
  if (conv) *conv = c1 && c2;
  return its;
}

void copy_samples_out(H_t &h, int k, mlmc_c64 *out) {
  check_cuda(cudaMemcpyAsync(out, h.samples.p, (size_t)k * sizeof(mlmc_c64), cudaMemcpyDeviceToHost, h.stream), "D2H samples");
  check_cuda(cudaStreamSynchronize(h.stream), "sync");
}

int translate(const std::function<void()> &fn) {
  struct AllocReset {
    AllocReset() { g_alloc_stream = nullptr; }
    ~AllocReset() { g_alloc_stream = nullptr; }
  } reset;
  try {
    fn();
    return MLMC_OK;
  } catch (const mlmc_fail &f) {
    g_last_error = f.msg;
    return f.code;
  } catch (const cuda_error &e) {
    g_last_error = std::string(e.where) + ": " + cudaGetErrorString(e.code);
    if (e.code == cudaErrorMemoryAllocation) return MLMC_ERR_OOM;
    return MLMC_ERR_CUDA;
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return MLMC_ERR_OOM;
  } catch (...) {
    g_last_error = "unknown failure";
    return MLMC_ERR_CUDA;
  }
}

void need(H_t *h) {
  if (!h) fail(MLMC_ERR_INVALID_ARG, "null hierarchy");
  g_alloc_stream = h->stream;
}

void need_level(const H_t *h, int level, int lo, int hi) {
  if (!h) fail(MLMC_ERR_INVALID_ARG, "null hierarchy");
  g_alloc_stream = h->stream;
  if (level < lo || level > hi) fail(MLMC_ERR_INVALID_ARG, "level out of range");
}

}  // namespace

extern "C" {

int mlmc_setup_hierarchy(const mlmc_operator_desc *op, const mlmc_hierarchy_params *params, void *stream,
                         mlmc_hierarchy **out) {
  return translate([&] {
    if (!out) fail(MLMC_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    std::unique_ptr<H_t> h(new H_t());
    setup(*h, op, params, (cudaStream_t)stream);
    *out = h.release();
  });
}

void mlmc_destroy_hierarchy(mlmc_hierarchy *h) {
  if (!h) return;
  cudaStream_t s = h->stream;
  const bool own = h->own.s != nullptr;
  cudaStreamSynchronize(s);
  delete h;                              // queues the frees of its buffers on s
  if (!own) cudaStreamSynchronize(s);    // a caller's stream: the frees are done on return
}

int mlmc_level_info(const mlmc_hierarchy *h, int level, int *nx, int *ny, int *d) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L : 0);
    const Level &Lv = h->lv[level - 1];
    if (nx) *nx = Lv.nx;
    if (ny) *ny = Lv.ny;
    if (d) *d = Lv.d;
  });
}

int mlmc_level_taps(const mlmc_hierarchy *h, int level, int *taps) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L : 0);
    if (!taps) fail(MLMC_ERR_INVALID_ARG, "null output");
    *taps = h->lv[level - 1].taps;
  });
}

int mlmc_get_prolongation(const mlmc_hierarchy *h, int level, void *host_out) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L - 1 : 0);
    if (!host_out) fail(MLMC_ERR_INVALID_ARG, "null output");
    if (h->bilinear) fail(MLMC_ERR_UNSUPPORTED, "bilinear P is not stored (it is applied by its stencil)");
    const Level &Lv = h->lv[level - 1];
    check_cuda(cudaMemcpyAsync(host_out, Lv.P64.p, Lv.n * Lv.dc * dtype_size(h->t64), cudaMemcpyDeviceToHost, h->stream), "D2H P");
    check_cuda(cudaStreamSynchronize(h->stream), "sync");
  });
}

int mlmc_get_operator(const mlmc_hierarchy *h, int level, void *host_out) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L : 0);
    if (!host_out) fail(MLMC_ERR_INVALID_ARG, "null output");
    const Level &Lv = h->lv[level - 1];
    check_cuda(cudaMemcpyAsync(host_out, Lv.coef64.p, Lv.nsite * Lv.taps * Lv.d * Lv.d * dtype_size(h->t64),
                               cudaMemcpyDeviceToHost, h->stream), "D2H coef");
    check_cuda(cudaStreamSynchronize(h->stream), "sync");
  });
}

int mlmc_apply(mlmc_hierarchy *h, int level, const void *x, void *y, int k) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L : 0);
    if (!x || !y || k < 1 || k > 256) fail(MLMC_ERR_INVALID_ARG, "bad vector block");
    apply_op(*h, level - 1, 0, x, y, k);
    check_cuda(cudaStreamSynchronize(h->stream), "sync");
  });
}

int mlmc_solve(mlmc_hierarchy *h, int level, const void *b, void *x, int k, double tol, int *iters) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L : 0);
    if (!b || !x || k < 1 || k > h->kmax) fail(MLMC_ERR_INVALID_ARG, "bad vector block (k must be <= block)");
    if (!(tol > 0.0)) fail(MLMC_ERR_INVALID_ARG, "tol must be positive");
    bool conv = true;
    int its = solve_level(*h, level - 1, b, x, k, tol, &conv);
    check_cuda(cudaStreamSynchronize(h->stream), "sync");
    if (iters) *iters = its;
    check_timeout(*h);
    if (!conv) fail(MLMC_ERR_NOT_CONVERGED, "solve did not reach tol within max_iter");
  });
}

int mlmc_noise(int noise, uint64_t seed, int level, int purpose, uint64_t first, int n, int k, int complex_out,
               void *out, void *stream) {
  return translate([&] {
    if (!out || n < 1 || k < 1 || k > 4096) fail(MLMC_ERR_INVALID_ARG, "bad noise block");
    if (noise != MLMC_NOISE_RADEMACHER && noise != MLMC_NOISE_Z4) fail(MLMC_ERR_INVALID_ARG, "unknown noise");
    if (noise == MLMC_NOISE_Z4 && !complex_out) fail(MLMC_ERR_INVALID_ARG, "Z4 noise needs complex output");
    launch_noise(noise == MLMC_NOISE_Z4 ? 1 : 0, seed, key_hi(purpose, level), first, (size_t)n, k,
                 complex_out ? C64 : F64, out, (cudaStream_t)stream);
    check_cuda(cudaStreamSynchronize((cudaStream_t)stream), "sync");
  });
}

int mlmc_sample_level(mlmc_hierarchy *h, int level, int noise, uint64_t seed, uint64_t first, int n_samples,
                      double tol, mlmc_c64 *out_samples, int *out_iters) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L : 0);
    if (n_samples < 0 || (n_samples > 0 && !out_samples)) fail(MLMC_ERR_INVALID_ARG, "bad sample output");
    if (noise == MLMC_NOISE_Z4 && !h->complex_op) fail(MLMC_ERR_INVALID_ARG, "Z4 noise needs a complex operator");
    if (!(tol > 0.0)) fail(MLMC_ERR_INVALID_ARG, "tol must be positive");
    if (h->bilinear && level < h->L)
      fail(MLMC_ERR_INVALID_ARG, "the simplified form needs R P = I; use the hat form with a bilinear hierarchy");
    bool all_conv = true;
    const int kl = h->kdiff(std::min(level - 1, h->L - 2));   // level L: the coarsest buffers' width
    for (int done = 0, b = 0; done < n_samples; ++b) {
      int k = std::min(kl, n_samples - done);
      bool conv = true;
      int its = sample_block(*h, level - 1, noise, seed, first + done, k, tol, MLMC_PURPOSE_NOISE, &conv);
      copy_samples_out(*h, k, out_samples + done);
      if (out_iters) out_iters[b] = its;
      all_conv = all_conv && conv;
      done += k;
    }
    check_timeout(*h);
    if (!all_conv) fail(MLMC_ERR_NOT_CONVERGED, "a level solve did not reach tol within max_iter");
  });
}

int mlmc_sample_block(mlmc_hierarchy *h, int level, int form, int noise, uint64_t seed, uint64_t first, int k,
                      double tol, mlmc_c64 *out_samples, double *out_stats, double *out_cost) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L - 1 : 0);
    if (form != MLMC_FORM_SIMPLIFIED && form != MLMC_FORM_HAT && form != MLMC_FORM_PLAIN)
      fail(MLMC_ERR_INVALID_ARG, "unknown form");
    if (form == MLMC_FORM_PLAIN && level != 1) fail(MLMC_ERR_INVALID_ARG, "plain samples live on level 1");
    if (form == MLMC_FORM_SIMPLIFIED && h->bilinear)
      fail(MLMC_ERR_INVALID_ARG, "the simplified form needs R P = I; use the hat form with a bilinear hierarchy");
    if (noise == MLMC_NOISE_Z4 && !h->complex_op) fail(MLMC_ERR_INVALID_ARG, "Z4 noise needs a complex operator");
    if (!(tol > 0.0)) fail(MLMC_ERR_INVALID_ARG, "tol must be positive");
    if (k < 1 || k > h->kdiff(level - 1)) fail(MLMC_ERR_INVALID_ARG, "k must be within the level's block width");
    H_t &H = *h;
    bool conv = true;
    const double c0 = H.cost;
    sample_block(H, level - 1, noise, seed, first, k, tol, MLMC_PURPOSE_NOISE, &conv, form);
    if (out_cost) *out_cost = H.cost - c0;
    if (out_stats) {
      // the block's own (N, mean, M2) by the device's fixed-order reduction
      check_cuda(cudaMemsetAsync(H.acc.p, 0, 4 * sizeof(double), H.stream), "memset acc");
      launch_accumulate(H.samples.p, k, H.acc.as<double>(), H.stream);
      H.launches++;
      check_cuda(cudaMemcpyAsync(out_stats, H.acc.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, H.stream),
                 "D2H stats");
    }
    if (out_samples) copy_samples_out(H, k, out_samples);
    check_cuda(cudaStreamSynchronize(H.stream), "sync");
    check_timeout(H);
    if (!conv) fail(MLMC_ERR_NOT_CONVERGED, "a level solve did not reach tol within max_iter");
  });
}

int mlmc_residual_restrict(mlmc_hierarchy *h, int level, int precision, const void *x, const void *b, void *rc,
                           int k, int colour) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L - 1 : 0);
    const int lo = precision == MLMC_PREC_MIXED_FP32 ? 1 : 0;
    if (lo && h->prm.precision != MLMC_PREC_MIXED_FP32) fail(MLMC_ERR_INVALID_ARG, "FP32 data needs the mixed form");
    if (!x || !b || !rc || k < 1 || k > 65536 || (colour != 0 && colour != 1))
      fail(MLMC_ERR_INVALID_ARG, "bad arguments");
    const StencilView A = view(*h, level - 1, lo);
    const ProlongView P = pview(*h, level - 1, lo);
    if (!residual_restrict_ok(A, P)) fail(MLMC_ERR_UNSUPPORTED, "not an aggregation level with d, dc <= 4");
    launch_residual_restrict(A, P, x, b, rc, k, colour, h->stream);
    check_cuda(cudaStreamSynchronize(h->stream), "sync");
  });
}

int mlmc_block_width(const mlmc_hierarchy *h, int level, int *k) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L - 1 : 0);
    if (!k) fail(MLMC_ERR_INVALID_ARG, "null output");
    *k = h->kdiff(level - 1);
  });
}

int mlmc_nominal_sample_cost(const mlmc_hierarchy *h, int level, int form, double *out) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L - 1 : 0);
    if (!out) fail(MLMC_ERR_INVALID_ARG, "null output");
    *out = nominal_sample_cost(*h, level - 1, form);
  });
}

int mlmc_column_dots(int complex_data, const void *x, const void *y, int n, int k, void *out, void *stream) {
  return translate([&] {
    if (!x || !y || !out || n < 1 || k < 1 || k > 256) fail(MLMC_ERR_INVALID_ARG, "bad column-dot arguments (k must be in 1..256)");
    cudaStream_t s = (cudaStream_t)stream;
    g_alloc_stream = s;
    DType t = complex_data ? C64 : F64;
    int parts = multidot_parts((size_t)n, k);
    DevBuf part;
    part.alloc((size_t)parts * k * (complex_data ? 16 : 8));
    launch_multidot(t, x, (size_t)n * k, 1, y, (size_t)n, k, part.p, parts, out, t, s);
    check_cuda(cudaStreamSynchronize(s), "sync");
  });
}

int mlmc_sample_level_form(mlmc_hierarchy *h, int level, int form, int noise, uint64_t seed, uint64_t first,
                           int n_samples, double tol, mlmc_c64 *out_samples) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L : 0);
    if (form != MLMC_FORM_SIMPLIFIED && form != MLMC_FORM_HAT && form != MLMC_FORM_PLAIN)
      fail(MLMC_ERR_INVALID_ARG, "unknown form");
    if (form == MLMC_FORM_PLAIN && level != 1) fail(MLMC_ERR_INVALID_ARG, "plain samples live on level 1");
    if (form == MLMC_FORM_SIMPLIFIED && h->bilinear && level < h->L)
      fail(MLMC_ERR_INVALID_ARG, "the simplified form needs R P = I; use the hat form with a bilinear hierarchy");
    if (n_samples < 0 || (n_samples > 0 && !out_samples)) fail(MLMC_ERR_INVALID_ARG, "bad sample output");
    if (noise == MLMC_NOISE_Z4 && !h->complex_op) fail(MLMC_ERR_INVALID_ARG, "Z4 noise needs a complex operator");
    if (!(tol > 0.0)) fail(MLMC_ERR_INVALID_ARG, "tol must be positive");
    bool all_conv = true;
    const int kl = h->kdiff(std::min(level - 1, h->L - 2));   // level L: the coarsest buffers' width
    for (int done = 0; done < n_samples;) {
      int k = std::min(kl, n_samples - done);
      bool conv = true;
      sample_block(*h, level - 1, noise, seed, first + done, k, tol, MLMC_PURPOSE_NOISE, &conv, form);
      copy_samples_out(*h, k, out_samples + done);
      all_conv = all_conv && conv;
      done += k;
    }
    check_timeout(*h);
    if (!all_conv) fail(MLMC_ERR_NOT_CONVERGED, "a level solve did not reach tol within max_iter");
  });
}

int mlmc_dense_apply(int complex_data, const void *A, const void *B, void *Y, int n, int k, int which,
                     void *stream) {
  return translate([&] {
    if (!A || !B || !Y || n < 1 || k < 1 || k > 4096) fail(MLMC_ERR_INVALID_ARG, "bad dense apply arguments");
    if (which != MLMC_DENSE_SIMT && which != MLMC_DENSE_TC && which != MLMC_DENSE_TC_WITHHOLD)
      fail(MLMC_ERR_INVALID_ARG, "unknown dense kernel");
    if ((((uintptr_t)A) | ((uintptr_t)B) | ((uintptr_t)Y)) & 15)
      fail(MLMC_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    const DType t = complex_data ? C32 : F32;
    cudaStream_t s = (cudaStream_t)stream;
    g_alloc_stream = s;
    DevBuf part, err;
    err.alloc(sizeof(int));
    check_cuda(cudaMemsetAsync(err.p, 0, sizeof(int), s), "memset err");
    if (which != MLMC_DENSE_SIMT) {
      part.alloc(dense_apply_tc_part_bytes(t, n, k));
      launch_dense_apply_tc(t, A, B, Y, n, k, part.p, part.bytes, err.as<int>(), s, which == MLMC_DENSE_TC_WITHHOLD);
    } else {
      part.alloc((size_t)dense_apply_splits(n, k) * n * k * dtype_size(t));
      launch_dense_apply(t, A, B, Y, n, k, part.p, s);
    }
    int e = 0;
    check_cuda(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H err");
    check_cuda(cudaStreamSynchronize(s), "sync");
    if (e == MLMC_ERR_TIMEOUT) fail(MLMC_ERR_TIMEOUT, "a bounded tensor-core wait gave up");
  });
}

int mlmc_set_dense_kernel(mlmc_hierarchy *h, int which) {
  return translate([&] {
    need(h);
    if (which != MLMC_DENSE_SIMT && which != MLMC_DENSE_TC && which != MLMC_DENSE_AUTO)
      fail(MLMC_ERR_INVALID_ARG, "unknown dense kernel");
    if (h->dense_kernel != which) drop_graphs(*h);
    h->dense_kernel = which;
  });
}

int mlmc_set_conv_kernel(mlmc_hierarchy *h, int which) {
  return translate([&] {
    need(h);
    if (which != MLMC_CONV_SIMT && which != MLMC_CONV_AUTO && which != MLMC_CONV_TC)
      fail(MLMC_ERR_INVALID_ARG, "unknown conv kernel");
    if (h->conv_kernel != which) drop_graphs(*h);
    h->conv_kernel = which;
    if (which == MLMC_CONV_AUTO && h->net_c0) tune_conv(*h);
  });
}

int mlmc_coarse_trace_exact(mlmc_hierarchy *h, mlmc_c64 *out) {
  return translate([&] {
    need(h);
    if (!out) fail(MLMC_ERR_INVALID_ARG, "null output");
    if (h->bilinear) {
      out->re = h->coarse_term_hat;
      out->im = 0.0;
      return;
    }
    const Level &C = h->lv[h->L - 1];
    launch_trace(h->t64, C.Ainv64.p, (int)C.n, h->trace.p, h->stream);
    h->launches++;
    check_cuda(cudaMemcpyAsync(out, h->trace.p, sizeof(mlmc_c64), cudaMemcpyDeviceToHost, h->stream), "D2H trace");
    check_cuda(cudaStreamSynchronize(h->stream), "sync");
  });
}

int mlmc_trace_estimate(mlmc_hierarchy *h, const mlmc_estimate_params *p, mlmc_estimate_result *r) {
  return translate([&] {
    need(h);
    if (!p || !r) fail(MLMC_ERR_INVALID_ARG, "null parameters or result");
    if (!(p->eps > 0.0) || !(p->tol > 0.0)) fail(MLMC_ERR_INVALID_ARG, "eps and tol must be positive");
    if (p->form != MLMC_FORM_SIMPLIFIED && p->form != MLMC_FORM_HAT && p->form != MLMC_FORM_PLAIN)
      fail(MLMC_ERR_INVALID_ARG, "unknown form");
    const bool plain = p->form == MLMC_FORM_PLAIN;
    if (p->form == MLMC_FORM_SIMPLIFIED && h->bilinear)
      fail(MLMC_ERR_INVALID_ARG, "the simplified form needs R P = I; use the hat form with a bilinear hierarchy");
    if (p->noise == MLMC_NOISE_Z4 && !h->complex_op) fail(MLMC_ERR_INVALID_ARG, "Z4 noise needs a complex operator");
    if (p->allocation != MLMC_ALLOC_RHO && p->allocation != MLMC_ALLOC_OPTIMAL && p->allocation != MLMC_ALLOC_FIXED)
      fail(MLMC_ERR_INVALID_ARG, "unknown allocation");
    if (p->allocation == MLMC_ALLOC_FIXED)
      for (int l = 0; l < h->L - 1; ++l)
        if (p->n_fixed[l] < 5) fail(MLMC_ERR_INVALID_ARG, "n_fixed must be >= 5 on every level difference");
    if (p->cost_model != MLMC_COST_COUNTED && p->cost_model != MLMC_COST_NOMINAL)
      fail(MLMC_ERR_INVALID_ARG, "unknown cost model");
    H_t &H = *h;
    const int L = H.L, nd = plain ? 1 : L - 1;
    std::memset(r, 0, sizeof(*r));
    r->levels = plain ? 2 : L;
    for (int l = 0; l < 16; ++l) H.iters_accum[l] = H.solves_accum[l] = 0.0;
    auto t0 = std::chrono::steady_clock::now();
    mlmc_c64 TL = {0.0, 0.0};
    if (!plain) {
      // Remark 4.2: tr(P^_L A_L^{-1} R^_L) = tr(A_L^{-1} R^_L P^_L); = tr(A_L^{-1}) when R^_L P^_L = I
      // (aggregation), else the setup's value (bilinear)
      const Level &C = H.lv[L - 1];
      if (H.bilinear) {
        TL.re = H.coarse_term_hat;
        TL.im = 0.0;
      } else {
        launch_trace(H.t64, C.Ainv64.p, (int)C.n, H.trace.p, H.stream);
        H.launches++;
        check_cuda(cudaMemcpyAsync(&TL, H.trace.p, sizeof(TL), cudaMemcpyDeviceToHost, H.stream), "D2H trace");
        check_cuda(cudaStreamSynchronize(H.stream), "sync");
      }
      // Remark 4.2 cost of the exact term: inversion of A_L (n_L^3)
      r->cost_nnz[nd] = std::pow((double)H.lv[L - 1].n, 3.0);
    }
    r->coarse_term = TL;
    const int minN = p->min_samples > 0 ? p->min_samples : 5;
    const int maxN = p->max_samples > 0 ? p->max_samples : (1 << 24);
    auto cap = [&](int l) { return p->allocation == MLMC_ALLOC_FIXED ? p->n_fixed[l] : maxN; };
    // per-level state: accumulators live on the device ({N, mean re, mean im, M2} x levels)
    DevBuf accs;
    accs.alloc((size_t)nd * 4 * sizeof(double));
    check_cuda(cudaMemsetAsync(accs.p, 0, (size_t)nd * 4 * sizeof(double), H.stream), "memset acc");
    std::vector<double> st((size_t)nd * 4, 0.0), cost(nd, 0.0), secs(nd, 0.0), nominal(nd, 0.0);
    for (int l = 0; l < nd; ++l) nominal[l] = nominal_sample_cost(H, l, p->form);
    const bool nominal_cost = p->cost_model == MLMC_COST_NOMINAL;
    std::vector<mlmc_c64> tmp(std::max(5, H.kbig));
    double warm[5];
    for (int i = 0; i < 5; ++i) warm[i] = TL.re;
    auto width = [&](int l) { return H.kdiff(l); };
    // one block of samples on level difference l; samples 0..4 also enter the five
    // full estimates that define tau
    auto draw = [&](int l) {
      auto tl = std::chrono::steady_clock::now();
      double c0 = H.cost;
      int N0 = (int)st[4 * l];
      int k = std::min(width(l), cap(l) - N0);
      if (k <= 0) return false;
      bool conv = true;
      sample_block(H, l, p->noise, p->seed, (uint64_t)N0, k, p->tol, MLMC_PURPOSE_NOISE, &conv, p->form);
      if (!conv) fail(MLMC_ERR_NOT_CONVERGED, "level solve did not converge");
      if (N0 < 5 && !p->tau_separate) {
        copy_samples_out(H, k, tmp.data());
        for (int i = N0; i < std::min(5, N0 + k); ++i) warm[i] += tmp[i - N0].re;
      }
      launch_accumulate(H.samples.p, k, accs.as<double>() + 4 * l, H.stream);
      H.launches++;
      check_cuda(cudaMemcpyAsync(&st[4 * l], accs.as<double>() + 4 * l, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                                 H.stream), "D2H acc");
      check_cuda(cudaStreamSynchronize(H.stream), "sync");
      cost[l] += nominal_cost ? nominal[l] * k : H.cost - c0;
      secs[l] += std::chrono::duration<double>(std::chrono::steady_clock::now() - tl).count();
      return true;
    };
    auto var = [&](int l) { double N = st[4 * l]; return N > 1 ? st[4 * l + 3] / (N - 1) : INFINITY; };
    // Sec. 5: five full estimates (one sample per level difference plus the exact term);
    // they are samples 0..4 of every level's stream, drawn with each level's first block,
    // or (tau_separate) five samples of the warm-up stream that do not enter the means
    if (p->tau_separate) {
      for (int l = 0; l < nd; ++l)
        for (int done = 0; done < 5;) {
          const int k = std::min(5 - done, width(l));
          bool conv = true;
          const double c0 = H.cost;
          sample_block(H, l, p->noise, p->seed, (uint64_t)done, k, p->tol, MLMC_PURPOSE_WARMUP, &conv, p->form);
          H.cost = c0;
          if (!conv) fail(MLMC_ERR_NOT_CONVERGED, "level solve did not converge");
          copy_samples_out(H, k, tmp.data());
          for (int i = 0; i < k; ++i) warm[done + i] += tmp[i].re;
          done += k;
        }
    }
    for (int l = 0; l < nd; ++l)
      while (st[4 * l] < 5)
        if (!draw(l)) fail(MLMC_ERR_INVALID_ARG, "fewer than five samples allowed on a level");
    double mean = 0.0;
    for (double v : warm) mean += v / 5.0;
    double ms = 0.0;
    for (double v : warm) ms += (v - mean) * (v - mean) / 5.0;
    double tau = mean - std::sqrt(ms);
    r->tau = tau;
    const double target = p->eps * std::fabs(tau);            // standard error of the estimate
    std::vector<double> w(nd, 0.0);
    if (p->allocation == MLMC_ALLOC_FIXED) {
      for (int l = 0; l < nd; ++l)
        while (st[4 * l] < p->n_fixed[l]) draw(l);
    } else if (p->allocation == MLMC_ALLOC_RHO) {
      // Sec. 5: rho_l = sqrt(w_l) eps |tau|; sample each level until its standard error meets rho_l
      double wsum = 0.0;
      for (int l = 0; l < nd; ++l) wsum += p->weights[l];
      for (int l = 0; l < nd; ++l) {
        w[l] = wsum > 0.0 ? p->weights[l] / wsum : 1.0 / nd;
        double rho = std::sqrt(w[l]) * target;
        for (;;) {
          double N = st[4 * l];
          if (N >= minN && std::sqrt(var(l) / N) <= rho) break;
          if (!draw(l)) break;
        }
      }
    } else {
      // Sec. 2: minimise sum N_l C_l subject to sum V_l / N_l = (eps tau)^2, i.e.
      // N_l = (eps tau)^-2 sqrt(V_l / C_l) sum_j sqrt(V_j C_j), with V_l and C_l (cost
      // model per sample) estimated from the samples drawn so far (the first block of
      // every level is the pilot).
      for (int round = 0; round < 100000; ++round) {
        double S = 0.0;
        for (int l = 0; l < nd; ++l) S += std::sqrt(var(l) * cost[l] / st[4 * l]);
        bool more = false;
        double tot = 0.0;
        for (int l = 0; l < nd; ++l) {
          double Cl = cost[l] / st[4 * l];
          double want = std::max((double)minN, std::ceil(std::sqrt(var(l) / Cl) * S / (target * target)));
          w[l] = std::sqrt(var(l) * Cl) / S;
          tot += var(l) / st[4 * l];
          if (st[4 * l] < want && st[4 * l] < maxN) {
            more = true;
            draw(l);
          }
        }
        if (!more && tot <= target * target) break;
        if (!more) {             // variances grew: add a block where it reduces the variance most per cost
          int best = 0;
          double gain = -1.0;
          for (int l = 0; l < nd; ++l) {
            double N = st[4 * l], k = std::min(width(l), maxN - (int)N);
            if (k <= 0) continue;
            double g = (var(l) / N - var(l) / (N + k)) / (cost[l] / N * k);
            if (g > gain) { gain = g; best = l; }
          }
          if (gain < 0.0) break;
          draw(best);
        }
      }
    }
    check_timeout(H);
    double var_sum = 0.0;
    mlmc_c64 total = TL;
    for (int l = 0; l < nd; ++l) {
      double N = st[4 * l];
      double v = N > 1 ? st[4 * l + 3] / (N - 1) : 0.0;
      r->n_samples[l] = (int)N;
      r->mean[l].re = st[4 * l + 1];
      r->mean[l].im = st[4 * l + 2];
      r->variance[l] = v;
      r->seconds[l] = secs[l];
      r->cost_nnz[l] = cost[l];
      r->weights_used[l] = w[l];
      total.re += st[4 * l + 1];
      total.im += st[4 * l + 2];
      if (N > 0) var_sum += v / N;
      double solves = H.solves_accum[l];
      r->iters[l] = solves > 0 ? H.iters_accum[l] / solves : 0.0;
    }
    r->trace = total;
    r->std_err = std::sqrt(var_sum);
    r->seconds_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  });
}

int mlmc_profile_kernel(mlmc_hierarchy *h, int which, int level, int k, int reps, double *ms_per_launch,
                        double *bytes_per_launch) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L : 0);
    // level 1 holds blocks of `block` columns, the coarser levels also the coarse-level blocks
    if (k < 1 || k > h->wl[level - 1] || reps < 1) fail(MLMC_ERR_INVALID_ARG, "bad k or reps");
    H_t &H = *h;
    int l = level - 1;
    int lo = which == 0 ? 0 : (H.prm.precision == MLMC_PREC_MIXED_FP32 ? 1 : 0);
    if (which == 1 && !lo) fail(MLMC_ERR_INVALID_ARG, "FP32 kernels need the mixed form");
    if (which < 0 || which > 9) fail(MLMC_ERR_INVALID_ARG, "unknown kernel family");
    if (which == 9 && (l == H.L - 1 || k > H.wl[l + 1] || !residual_restrict_ok(view(H, l, lo), pview(H, l, lo))))
      fail(MLMC_ERR_INVALID_ARG, "the fused residual restriction needs an aggregation level above the coarsest");
    if (which == 8 && (l != 0 || H.prm.precision != MLMC_PREC_MIXED_FP32))
      fail(MLMC_ERR_INVALID_ARG, "the learned correction acts on level 1 in the mixed form");
    if (which == 8) net_alloc(H);
    if (which == 5 && l != H.L - 1) fail(MLMC_ERR_INVALID_ARG, "the dense apply lives on the coarsest level");
    if ((which == 6 || which == 7) && (l == H.L - 1 || k > H.wl[l + 1]))
      fail(MLMC_ERR_INVALID_ARG, "transfers run from a level above the coarsest, k within the coarse buffers");
    if (which == 2 && l == H.L - 1) fail(MLMC_ERR_INVALID_ARG, "no smoother on the coarsest level");
    const Level &Lv = H.lv[l];
    DType t = lo ? H.t32 : H.t64;
    size_t es = dtype_size(t);
    void *x = lo ? H.cyc[1][l].b.p : H.xs[l].p;
    void *y = lo ? H.cyc[1][l].x.p : H.ys[l].p;
    launch_noise(H.complex_op, 1, 0, 0, Lv.n, k, t, x, H.stream);
    launch_fill_zero(t, y, Lv.n * (size_t)k, H.stream);
    cudaEvent_t e0, e1;
    check_cuda(cudaEventCreate(&e0), "event");
    check_cuda(cudaEventCreate(&e1), "event");
    const int nvec = 4;      // which 3 / 4: basis vectors of a mid-length inner Arnoldi step
    DevBuf Vb, part, outb;
    if (which >= 3) {
      Vb.alloc((size_t)nvec * Lv.n * k * es);
      for (int v = 0; v < nvec; ++v)
        launch_noise(H.complex_op, 2 + v, 0, 0, Lv.n, k, t, Vb.as<char>() + (size_t)v * Lv.n * k * es, H.stream);
      part.alloc((size_t)multidot_parts(Lv.n, k) * nvec * k * 16);
      outb.alloc((size_t)nvec * k * 16);
      launch_fill_zero(F64, outb.p, (size_t)nvec * k * (H.complex_op ? 2 : 1), H.stream);
    }
    auto body = [&] {
      if (which == 2) {
        launch_rbgs_sweep(view(H, l, lo), y, x, k, 0, 0, H.stream);
      } else if (which == 3) {
        launch_multidot(t, Vb.p, Lv.n * (size_t)k, nvec, x, Lv.n, k, part.p, multidot_parts(Lv.n, k), outb.p,
                        H.complex_op ? C64 : F64, H.stream);
      } else if (which == 5) {
        dense_apply(H, lo, x, y, k);
      } else if (which == 4) {
        launch_multiaxpy(t, y, Vb.p, Lv.n * (size_t)k, nvec, outb.p, H.complex_op ? C64 : F64, k, -1e-30, Lv.n, k,
                         H.stream);
      } else if (which == 8) {
        net_forward(H, x, k);
      } else if (which == 9) {
        launch_residual_restrict(view(H, l, lo), pview(H, l, lo), y, x, H.cyc[lo][l + 1].b.p, k, 0, H.stream);
      } else if (which == 6) {
        launch_restrict(pview(H, l, lo), x, H.cyc[lo][l + 1].b.p, k, H.stream);
      } else if (which == 7) {
        launch_prolong_add(pview(H, l, lo), H.cyc[lo][l + 1].b.p, y, k, H.stream);
      } else {
        launch_stencil(view(H, l, lo), x, nullptr, y, k, 0, H.stream);
      }
    };
    for (int i = 0; i < 3; ++i) body();
    check_cuda(cudaEventRecord(e0, H.stream), "record");
    for (int i = 0; i < reps; ++i) body();
    check_cuda(cudaEventRecord(e1, H.stream), "record");
    check_cuda(cudaEventSynchronize(e1), "sync");
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    double vec = (double)Lv.n * k * es;
    bool const_coef = l == 0 && !H.complex_op;      // Example 5.1 stencil has no matrix to read
    double coefb = const_coef ? 0.0 : (double)Lv.nsite * Lv.taps * Lv.d * Lv.d * es;
    double bytes;
    if (which == 9) {
      // b on one colour, x everywhere (the colour's own and its neighbours), the colour's
      // coefficient blocks, P, the coarse block out
      const Level &C = H.lv[l + 1];
      bytes = 0.5 * vec + vec + 0.5 * coefb + (double)Lv.n * Lv.dc * es + (double)C.n * k * es;
      if (ms_per_launch) *ms_per_launch = ms / reps;
    } else if (which == 8) {
      // the network's activations: the block in (to channels), then per layer its input
      // channels read and output channels written (c0 -> 16 -> 16 -> c0), FP32
      const double pairs = (double)Lv.nsite * k, c0 = H.net_c0;
      bytes = vec + pairs * 4.0 * (c0 + (c0 + 16) + 32 + (16 + c0));
      if (ms_per_launch) *ms_per_launch = ms / reps;
    } else if (which == 6 || which == 7) {
      // restriction: the fine block in, the coarse block out; prolongation: the coarse block
      // in, the fine block read and written; both read the P blocks once (none for bilinear P)
      const Level &C = H.lv[l + 1];
      double cvec = (double)C.n * k * es;
      double pb = H.bilinear ? 0.0 : (double)Lv.n * Lv.dc * es;
      bytes = (which == 6 ? vec : 2.0 * vec) + cvec + pb;
      if (ms_per_launch) *ms_per_launch = ms / reps;
    } else if (which == 5) {
      // the dense inverse once, the block in, the block out
      bytes = (double)Lv.n * Lv.n * es + 2.0 * vec;
      if (ms_per_launch) *ms_per_launch = ms / reps;
    } else if (which == 3 || which == 4) {
      // multi-dot reads nvec basis blocks and w; multi-AXPY also writes w
      bytes = (which == 3 ? nvec + 1.0 : nvec + 2.0) * vec;
      if (ms_per_launch) *ms_per_launch = ms / reps;
    } else if (which == 2) {
      // one sweep = two half-sweeps: each reads b on its colour and the other
      // colour's x as neighbours and writes x on its colour (3 passes in all),
      // plus the off-diagonal coefficient blocks and the inverse self blocks
      double dinvb = (double)Lv.nsite * Lv.d * Lv.d * es;
      double offb = Lv.taps == 9 ? coefb * 8.0 / 9.0 : coefb * 4.0 / 5.0;
      bytes = 3.0 * vec + (const_coef ? 0.0 : offb + dinvb);
      if (ms_per_launch) *ms_per_launch = ms / reps;
    } else {
      bytes = 2.0 * vec + coefb;
      if (ms_per_launch) *ms_per_launch = ms / reps;
    }
    if (bytes_per_launch) *bytes_per_launch = bytes;
  });
}

int mlmc_measure_fma_rate(int fp64, void *stream, double *fma_per_s) {
  return translate([&] {
    if (!fma_per_s) fail(MLMC_ERR_INVALID_ARG, "null output");
    cudaStream_t s = (cudaStream_t)stream;
    g_alloc_stream = s;
    int dev = 0, sms = 0;
    check_cuda(cudaGetDevice(&dev), "device");
    check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attribute");
    if (fp64 < 0 || fp64 > 3) fail(MLMC_ERR_INVALID_ARG, "unknown operation");
    if (fp64 == 3) {
      // L2 bandwidth: a 16 MB to 16 MB copy (32 MB in L2), bytes read + written per second
      const size_t bytes = (size_t)16 << 20;
      DevBuf a, b;
      a.alloc(bytes);
      b.alloc(bytes);
      check_cuda(cudaMemsetAsync(a.p, 0, bytes, s), "memset");
      cudaEvent_t e0, e1;
      check_cuda(cudaEventCreate(&e0), "event");
      check_cuda(cudaEventCreate(&e1), "event");
      const int passes = 64;
      launch_copy16(a.p, b.p, bytes / 16, 4, sms * 8, s);
      check_cuda(cudaEventRecord(e0, s), "record");
      const int reps = 4;
      for (int i = 0; i < reps; ++i) launch_copy16(a.p, b.p, bytes / 16, passes, sms * 8, s);
      check_cuda(cudaEventRecord(e1, s), "record");
      check_cuda(cudaEventSynchronize(e1), "sync");
      float ms = 0.f;
      check_cuda(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      *fma_per_s = (double)reps * passes * 2.0 * bytes / (ms * 1e-3);
      return;
    }
    const int blocks = sms * 8, iters = fp64 ? 4096 : 65536;
    DevBuf out;
    out.alloc((size_t)blocks * 256 * 8);
    DType t = fp64 ? F64 : F32;
    const int add = fp64 == 2;
    cudaEvent_t e0, e1;
    check_cuda(cudaEventCreate(&e0), "event");
    check_cuda(cudaEventCreate(&e1), "event");
    launch_fma_rate(t, add, out.p, blocks, iters, s);            // warm-up
    check_cuda(cudaEventRecord(e0, s), "record");
    const int reps = 5;
    for (int i = 0; i < reps; ++i) launch_fma_rate(t, add, out.p, blocks, iters, s);
    check_cuda(cudaEventRecord(e1, s), "record");
    check_cuda(cudaEventSynchronize(e1), "sync");
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *fma_per_s = (double)reps * blocks * 256.0 * iters * 8.0 / (ms * 1e-3);
  });
}

int mlmc_learned_set(mlmc_hierarchy *h, const float *weights, int enable) {
  return translate([&] {
    need(h);
    if (h->prm.precision != MLMC_PREC_MIXED_FP32) fail(MLMC_ERR_UNSUPPORTED, "the learned correction runs in the mixed form");
    net_alloc(*h);
    if (weights)
      check_cuda(cudaMemcpyAsync(h->netW.p, weights, h->net_nw * sizeof(float), cudaMemcpyHostToDevice, h->stream), "H2D W");
    check_cuda(cudaStreamSynchronize(h->stream), "sync");
    if (enable && !h->conv_tuned) tune_conv(*h);
    h->net_on = enable ? 1 : 0;
  });
}

int mlmc_learned_stats(const mlmc_hierarchy *h, int *enabled, int *fallbacks) {
  return translate([&] {
    if (!h) fail(MLMC_ERR_INVALID_ARG, "null handle");
    if (enabled) *enabled = h->net_on;
    if (fallbacks) *fallbacks = h->net_fallbacks;
  });
}

int mlmc_learned_apply(mlmc_hierarchy *h, const void *r, void *e, int k) {
  return translate([&] {
    need(h);
    if (h->prm.precision != MLMC_PREC_MIXED_FP32) fail(MLMC_ERR_UNSUPPORTED, "the learned correction runs in the mixed form");
    if (!r || !e || k < 1 || k > h->kmax) fail(MLMC_ERR_INVALID_ARG, "bad block");
    net_alloc(*h);
    const Level &F = h->lv[0];
    net_forward(*h, r, k);
    launch_fill_zero(h->t32, e, F.n * (size_t)k, h->stream);
    launch_add_from_channels(h->t32, e, h->act3.as<float>(), (int)F.nsite, F.d, k, h->stream);
    check_cuda(cudaStreamSynchronize(h->stream), "sync");
  });
}

int mlmc_learned_grad(mlmc_hierarchy *h, const void *r, int k, double *loss, float *grad_out) {
  return translate([&] {
    need(h);
    if (h->prm.precision != MLMC_PREC_MIXED_FP32) fail(MLMC_ERR_UNSUPPORTED, "the learned correction runs in the mixed form");
    if (!r || k < 1 || k > h->kmax) fail(MLMC_ERR_INVALID_ARG, "bad block");
    net_alloc(*h);
    double l = net_loss_grad(*h, r, k, true, true);
    if (loss) *loss = l;
    if (grad_out)
      check_cuda(cudaMemcpyAsync(grad_out, h->netG.p, h->net_nw * sizeof(float), cudaMemcpyDeviceToHost, h->stream), "D2H G");
    check_cuda(cudaStreamSynchronize(h->stream), "sync");
  });
}

int mlmc_learned_train(mlmc_hierarchy *h, const mlmc_train_params *p, float *weights_out, mlmc_train_report *rep) {
  return translate([&] {
    need(h);
    if (!p) fail(MLMC_ERR_INVALID_ARG, "null training parameters");
    if (h->prm.precision != MLMC_PREC_MIXED_FP32) fail(MLMC_ERR_UNSUPPORTED, "the learned correction runs in the mixed form");
    if (p->n_pairs < 2 || p->epochs < 1 || !(p->lr > 0.0) || !(p->tol > 0.0)) fail(MLMC_ERR_INVALID_ARG, "bad training parameters");
    H_t &H = *h;
    net_alloc(H);
    if (!H.conv_tuned) tune_conv(H);
    const Level &F = H.lv[0];
    const int k = H.kmax;
    cudaStream_t s = H.stream;
    mlmc_train_report R;
    std::memset(&R, 0, sizeof(R));
    R.n_weights = H.net_nw;
    // 1) residual/error pairs from plain solves (net off)
    auto t0 = std::chrono::steady_clock::now();
    size_t blocks = ((size_t)p->n_pairs + k - 1) / k;
    if (blocks < 2) blocks = 2;
    H.capture.alloc(blocks * F.n * (size_t)k * dtype_size(H.t32));
    H.capture_blocks = blocks;
    H.capture_n = 0;
    int was_on = H.net_on;
    H.net_on = 0;
    H.capturing = 1;
    for (uint64_t solve = 0; H.capture_n < H.capture_blocks && solve < 100000; ++solve) {
      launch_noise(H.complex_op ? 1 : 0, p->seed, key_hi(MLMC_PURPOSE_TRAIN, 1), solve * k, F.n, k, H.t64, H.xs[0].p, s);
      bool conv = true;
      solve_level(H, 0, H.xs[0].p, H.ys[0].p, k, p->tol, &conv);
    }
    H.capturing = 0;
    check_cuda(cudaStreamSynchronize(s), "sync");
    R.seconds_capture = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    R.blocks = (int)blocks;
    R.pairs = (int)(blocks * k);
    // 2) initial weights
    if (p->init_weights) {
      check_cuda(cudaMemcpyAsync(H.netW.p, p->init_weights, H.net_nw * sizeof(float), cudaMemcpyHostToDevice, s), "H2D W");
    } else {
      // Rademacher signs (Philox, purpose TRAIN, level 0) scaled by sqrt(2 / fan_in) / 2 per layer
      DevBuf tmp;
      tmp.alloc(H.net_nw * sizeof(double));
      launch_noise(0, p->seed, key_hi(MLMC_PURPOSE_TRAIN, 0), 0, (size_t)H.net_nw, 1, F64, tmp.p, s);
      std::vector<double> hw(H.net_nw);
      check_cuda(cudaMemcpyAsync(hw.data(), tmp.p, H.net_nw * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
      check_cuda(cudaStreamSynchronize(s), "sync");
      std::vector<float> w(H.net_nw);
      int c0 = H.net_c0;
      int n1 = 9 * NET_CH * c0, n2 = 9 * NET_CH * NET_CH;
      for (int i = 0; i < H.net_nw; ++i) {
        int fan_in = i < n1 ? 9 * c0 : 9 * NET_CH;
        (void)n2;
        w[i] = (float)(hw[i] * 0.5 * std::sqrt(2.0 / fan_in));
      }
      check_cuda(cudaMemcpyAsync(H.netW.p, w.data(), H.net_nw * sizeof(float), cudaMemcpyHostToDevice, s), "H2D W");
    }
    check_cuda(cudaMemsetAsync(H.netM.p, 0, H.net_nw * sizeof(float), s), "memset");
    check_cuda(cudaMemsetAsync(H.netV.p, 0, H.net_nw * sizeof(float), s), "memset");
    H.net_step = 0;
    // 3) Adam over the training blocks; the last block (at least 10%) is held out
    size_t nval = std::max<size_t>(1, blocks / 10);
    size_t ntrain = blocks - nval;
    auto blk = [&](size_t i) { return H.capture.as<char>() + i * F.n * (size_t)k * dtype_size(H.t32); };
    auto t1 = std::chrono::steady_clock::now();
    for (int ep = 0; ep < p->epochs; ++ep) {
      double sum = 0.0;
      for (size_t i = 0; i < ntrain; ++i) {
        bool rd = (ep == 0 || ep == p->epochs - 1);
        sum += net_loss_grad(H, blk(i), k, true, rd);
        launch_adam(H.netW.as<float>(), H.netG.as<float>(), H.netM.as<float>(), H.netV.as<float>(), H.net_nw,
                    (float)p->lr, ++H.net_step, s);
        H.launches++;
      }
      if (ep == 0) R.loss_first = sum / ntrain;
      if (ep == p->epochs - 1) R.loss_last = sum / ntrain;
    }
    double val = 0.0;
    for (size_t i = ntrain; i < blocks; ++i) val += net_loss_grad(H, blk(i), k, false, true);
    R.val_loss = val / nval;
    check_cuda(cudaStreamSynchronize(s), "sync");
    R.seconds_train = std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
    R.epochs = p->epochs;
    H.capture.release();
    H.capture_blocks = H.capture_n = 0;
    H.net_on = (p->enable && R.val_loss < 1.0) ? 1 : (p->enable ? 0 : was_on);
    R.enabled = H.net_on;
    if (weights_out)
      check_cuda(cudaMemcpyAsync(weights_out, H.netW.p, H.net_nw * sizeof(float), cudaMemcpyDeviceToHost, s), "D2H W");
    check_cuda(cudaStreamSynchronize(s), "sync");
    if (rep) *rep = R;
  });
}

int mlmc_set_block_width(mlmc_hierarchy *h, int k) {
  return translate([&] {
    need(h);
    if (k < 1 || k > h->kmax) fail(MLMC_ERR_INVALID_ARG, "block width must be in 1..block");
    h->kact = k;
  });
}

int mlmc_autotune_block(mlmc_hierarchy *h, int level, int noise, double tol, int *k_out, double *seconds_per_sample) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L - 1 : 0);
    if (noise == MLMC_NOISE_Z4 && !h->complex_op) fail(MLMC_ERR_INVALID_ARG, "Z4 noise needs a complex operator");
    H_t &H = *h;
    int best = H.kmax;
    double best_t = INFINITY;
    for (int k = 16; k <= H.kmax; k *= 2) {
      for (int rep = 0; rep < 2; ++rep) {      // first call captures graphs and warms caches
        bool conv = true;
        auto t0 = std::chrono::steady_clock::now();
        sample_block(H, level - 1, noise, 0x7e57ull, 0, k, tol, MLMC_PURPOSE_SETUP, &conv);
        check_cuda(cudaStreamSynchronize(H.stream), "sync");
        double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() / k;
        if (rep == 1 && t < best_t) {
          best_t = t;
          best = k;
        }
      }
      if (k * 2 > H.kmax && k != H.kmax) k = H.kmax / 2;   // also try kmax itself
    }
    H.kact = best;
    if (k_out) *k_out = best;
    if (seconds_per_sample) *seconds_per_sample = best_t;
  });
}

int mlmc_trace_estimate_batch(mlmc_hierarchy *const *hs, int count, const mlmc_estimate_params *params, int workers,
                              mlmc_estimate_result *results, int *status) {
  if (!hs || !params || !results || !status || count < 0 || workers < 1) {
    g_last_error = "bad batch arguments";
    return MLMC_ERR_INVALID_ARG;
  }
  std::atomic<int> next(0);
  auto work = [&] {
    for (;;) {
      int i = next.fetch_add(1);
      if (i >= count) return;
      status[i] = mlmc_trace_estimate(hs[i], &params[i], &results[i]);
    }
  };
  std::vector<std::thread> pool;
  int nw = std::min(workers, std::max(count, 1));
  for (int w = 0; w < nw; ++w) pool.emplace_back(work);
  for (auto &t : pool) t.join();
  for (int i = 0; i < count; ++i)
    if (status[i] != MLMC_OK) {
      g_last_error = "instance " + std::to_string(i) + " failed with status " + std::to_string(status[i]);
      return status[i];
    }
  return MLMC_OK;
}

int mlmc_launch_count(const mlmc_hierarchy *h, uint64_t *count) {
  return translate([&] {
    if (!h || !count) fail(MLMC_ERR_INVALID_ARG, "null argument");
    *count = h->launches;
  });
}

const char *mlmc_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
