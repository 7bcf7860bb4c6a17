// Host side of libmlmc: the C ABI of include/mlmc.h, hierarchy setup on the
// GPU (Sec. 4.1, Example 5.3), the batched flexible GMRES driver with its
// multigrid-cycle preconditioner (Remark 4.1), level-difference samples
// (Remark 4.3), the exact coarsest term (Remark 4.2) and the Sec. 5 estimate.
// Every numerical step runs in the kernels of the other translation units;
// this file only sequences launches and owns device memory.
#include <algorithm>
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

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf &operator=(DevBuf &&o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t nbytes) {
    release();
    if (nbytes == 0) nbytes = 16;
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      p = nullptr;
      fail(MLMC_ERR_OOM, "device allocation of " + std::to_string(nbytes) + " bytes failed");
    }
    check_cuda(e, "cudaMalloc");
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
  DevBuf Ainv64, Ainv32;                   // coarsest level only
};

// Workspace of one batched FGMRES (one level, one element type).
struct Krylov {
  DType t = F64;
  int hc = 0;               // complex Hessenberg data
  size_t n = 0;
  int k = 0, m = 0;
  DevBuf V, Z, partials, H, cs, sn, g, y, h2, bnorm, invnrm, resid, active, jdone, nactive;
  int *h_nactive = nullptr;
  ~Krylov() {
    if (h_nactive) cudaFreeHost(h_nactive);
  }
};

struct CycleBufs {
  DevBuf b, x, r;
  std::unique_ptr<Krylov> kcyc;   // K-cycle FGMRES on this level
};

}  // namespace

struct mlmc_hierarchy {
  cudaStream_t stream = nullptr;
  int complex_op = 0;
  DType t64 = F64, t32 = F32;
  mlmc_hierarchy_params prm{};
  int L = 0, kmax = 0;
  std::vector<Level> lv;
  std::vector<CycleBufs> cyc[2];                  // [0] FP64 cycle, [1] FP32 cycle
  std::vector<std::unique_ptr<Krylov>> outer;     // FP64 outer FGMRES per level
  std::vector<DevBuf> xs, ys;                     // sample blocks per level (FP64)
  DevBuf dots, samples, acc, err, trace;
  uint64_t launches = 0;
  double iters_accum[16] = {0}, solves_accum[16] = {0}, applies_accum[16] = {0};
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
  K.partials.alloc((size_t)multidot_parts(n, k) * (m + 1) * k * as);
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
  check_cuda(cudaMallocHost(&K.h_nactive, sizeof(int)), "cudaMallocHost");
}

int read_nactive(H_t &h, Krylov &K) {
  check_cuda(cudaMemcpyAsync(K.h_nactive, K.nactive.p, sizeof(int), cudaMemcpyDeviceToHost, h.stream), "D2H nactive");
  check_cuda(cudaStreamSynchronize(h.stream), "sync");
  return *K.h_nactive;
}

void apply_op(H_t &h, int l, int lo, const void *x, void *y, int k) {
  launch_stencil(view(h, l, lo), x, nullptr, y, k, 0, h.stream);
  h.launches++;
  if (!lo && l < 16) h.applies_accum[l] += k;
}

void residual_op(H_t &h, int l, int lo, const void *x, const void *b, void *r, int k) {
  launch_stencil(view(h, l, lo), x, b, r, k, 1, h.stream);
  h.launches++;
  if (!lo && l < 16) h.applies_accum[l] += k;
}

void dense_apply(H_t &h, int lo, const void *b, void *x, int k) {
  const Level &C = h.lv[h.L - 1];
  launch_dense_apply(lo ? h.t32 : h.t64, lo ? C.Ainv32.p : C.Ainv64.p, b, x, (int)C.n, k, h.stream);
  h.launches++;
}

void multidot(H_t &h, Krylov &K, const void *V, int nvec, const void *w, int k, void *out) {
  launch_multidot(K.t, V, K.n * (size_t)k, nvec, w, K.n, k, K.partials.p, multidot_parts(K.n, k), out,
                  K.hc ? C64 : F64, h.stream);
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
  cudaStream_t s = h.stream;

  check_cuda(cudaMemcpyAsync(Vj(0), b, blk * es, cudaMemcpyDeviceToDevice, s), "copy b");
  multidot(h, K, Vj(0), 1, Vj(0), k, K.g.p);
  check_cuda(cudaMemsetAsync(K.nactive.p, 0, sizeof(int), s), "memset");
  launch_arnoldi_init(K.hc, K.g.p, K.bnorm.as<double>(), K.invnrm.as<double>(), K.active.as<int>(),
                      K.jdone.as<int>(), k, fixed ? 0.0 : tol, 1, K.nactive.as<int>(), s);
  h.launches++;
  check_cuda(cudaMemsetAsync(x, 0, blk * es, s), "memset x");
  if (converged) *converged = true;
  if (!fixed && read_nactive(h, K) == 0) return 0;
  int its = 0;
  for (;;) {
    launch_scale_cols(K.t, Vj(0), Vj(0), K.invnrm.p, 0, K.n, k, s);
    h.launches++;
    int jlast = 0;
    for (int j = 0; j < m; ++j) {
      M(Vj(j), Zj(j));
      apply_op(h, l, lo, Zj(j), Vj(j + 1), k);
      multidot(h, K, K.V.p, j + 1, Vj(j + 1), k, Hcol(j));
      launch_multiaxpy(K.t, Vj(j + 1), K.V.p, blk, j + 1, Hcol(j), K.hc ? C64 : F64, k, -1.0, K.n, k, s);
      h.launches++;
      if (reorth) {
        multidot(h, K, K.V.p, j + 1, Vj(j + 1), k, K.h2.p);
        launch_multiaxpy(K.t, Vj(j + 1), K.V.p, blk, j + 1, K.h2.p, K.hc ? C64 : F64, k, -1.0, K.n, k, s);
        launch_add_acc(K.hc, Hcol(j), K.h2.p, (j + 1) * k, s);
        h.launches += 2;
      }
      multidot(h, K, Vj(j + 1), 1, Vj(j + 1), k, (char *)Hcol(j) + (size_t)(j + 1) * k * as);
      check_cuda(cudaMemsetAsync(K.nactive.p, 0, sizeof(int), s), "memset");
      launch_arnoldi_step(K.hc, K.H.p, K.cs.p, K.sn.p, K.g.p, j, m, k, K.active.as<int>(), K.jdone.as<int>(),
                          K.bnorm.as<double>(), tol, K.invnrm.as<double>(), K.resid.as<double>(),
                          K.nactive.as<int>(), fixed ? 1 : 0, s);
      launch_scale_cols(K.t, Vj(j + 1), Vj(j + 1), K.invnrm.p, 0, K.n, k, s);
      h.launches += 2;
      ++its;
      jlast = j + 1;
      if (fixed) {
        if (its >= fixed_its) break;
        continue;
      }
      if (read_nactive(h, K) == 0 || its >= maxit) break;
    }
    launch_trisolve(K.hc, K.H.p, K.g.p, K.y.p, K.jdone.as<int>(), m, k, s);
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
    if (read_nactive(h, K) == 0) return its;
    if (its >= maxit) {
      if (converged) *converged = false;
      return its;
    }
  }
}

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
  CycleBufs &cb = h.cyc[lo][l];
  CycleBufs &cn = h.cyc[lo][l + 1];
  launch_fill_zero(t, x, blk, s);
  StencilView A = view(h, l, lo);
  for (int it = 0; it < h.prm.smooth_pre; ++it) {
    launch_rbgs_half(A, x, b, k, 0, s);
    launch_rbgs_half(A, x, b, k, 1, s);
    h.launches += 2;
  }
  residual_op(h, l, lo, x, b, cb.r.p, k);
  launch_restrict(pview(h, l, lo), cb.r.p, cn.b.p, k, s);
  h.launches++;
  if (l + 1 == last) {
    dense_apply(h, lo, cn.b.p, cn.x.p, k);
  } else if (h.prm.cycle == MLMC_CYCLE_V) {
    cycle(h, lo, l + 1, cn.b.p, cn.x.p, k);
  } else {
    Precond M = [&h, lo, l, k](const void *v, void *z) { cycle(h, lo, l + 1, v, z, k); };
    fgmres(h, *cn.kcyc, l + 1, lo, cn.b.p, cn.x.p, k, 0.0, h.prm.kcycle_its, h.prm.kcycle_its, M, false, nullptr);
  }
  launch_prolong_add(pview(h, l, lo), cn.x.p, x, k, s);
  h.launches++;
  for (int it = 0; it < h.prm.smooth_post; ++it) {
    launch_rbgs_half(A, x, b, k, 1, s);
    launch_rbgs_half(A, x, b, k, 0, s);
    h.launches += 2;
  }
}

// FP64 preconditioner of the outer solve on level l: one cycle in FP64, or
// (mixed) the same cycle in FP32 between two precision conversions.
Precond outer_precond(H_t &h, int l, int k) {
  if (h.prm.precision == MLMC_PREC_FP64) {
    return [&h, l, k](const void *v, void *z) { cycle(h, 0, l, v, z, k); };
  }
  return [&h, l, k](const void *v, void *z) {
    CycleBufs &cb = h.cyc[1][l];
    size_t cnt = h.lv[l].n * (size_t)k;
    launch_convert(h.t32, cb.b.p, h.t64, v, cnt, h.stream);
    cycle(h, 1, l, cb.b.p, cb.x.p, k);
    launch_convert(h.t64, z, h.t32, cb.x.p, cnt, h.stream);
    h.launches += 2;
  };
}

// x = A_l^{-1} b in FP64 (dense inverse on the coarsest level).
int solve_level(H_t &h, int l, const void *b, void *x, int k, double tol, bool *conv) {
  if (conv) *conv = true;
  if (l == h.L - 1) {
    dense_apply(h, 0, b, x, k);
    return 0;
  }
  int its = fgmres(h, *h.outer[l], l, 0, b, x, k, tol, 0, h.prm.max_iter, outer_precond(h, l, k),
                   h.prm.reorth != 0, conv);
  if (l < 16) {
    h.iters_accum[l] += its;
    h.solves_accum[l] += 1;
  }
  return its;
}

uint64_t key_hi(int purpose, int level) { return ((uint64_t)purpose << 8) | (uint64_t)level; }

// ----------------------------------------------------------------- setup
void filter(H_t &h, int l, void *V, void *tmp, void *tmp2, int ntv, int kind, int sweeps, double omega) {
  StencilView A = view(h, l, 0);
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
  if (e) fail(MLMC_ERR_SINGULAR, std::string(what) + ": singular block or dependent test vectors (code " +
                                      std::to_string(e) + ")");
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
    col.alloc(C.n * es);
    launch_stencil_to_dense(view(h, h.L - 1, 0), dense.p, h.stream);
    launch_gauss_jordan(h.t64, dense.p, C.Ainv64.p, work.p, (int)C.n, h.err.as<int>(), col.p, h.stream);
    h.launches += 5 + 2 * C.n + 2;
    check_err(h, "coarsest inverse");
  }
  if (h.prm.precision == MLMC_PREC_MIXED_FP32) {
    for (int l = 0; l < h.L; ++l) {
      Level &Lv = h.lv[l];
      launch_convert(h.t32, Lv.coef32.p, h.t64, Lv.coef64.p, Lv.nsite * 5 * Lv.d * Lv.d, h.stream);
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

void validate(const mlmc_operator_desc *op, const mlmc_hierarchy_params *p) {
  if (!op || !p) fail(MLMC_ERR_INVALID_ARG, "null descriptor or parameters");
  if (op->kind != MLMC_OP_LAPLACE2D && op->kind != MLMC_OP_WILSON2D) fail(MLMC_ERR_INVALID_ARG, "unknown operator kind");
  if (op->nx < 2 || op->ny < 2) fail(MLMC_ERR_INVALID_ARG, "lattice too small");
  if (op->kind == MLMC_OP_WILSON2D && !op->links) fail(MLMC_ERR_INVALID_ARG, "Wilson operator needs links");
  if (p->levels < 2 || p->levels > 16) fail(MLMC_ERR_INVALID_ARG, "levels must be in 2..16");
  if (p->agg_x < 1 || p->agg_y < 1) fail(MLMC_ERR_INVALID_ARG, "bad aggregate shape");
  if (p->block < 1 || p->block > 256) fail(MLMC_ERR_INVALID_ARG, "block must be in 1..256");
  if (p->n_tv < 1 || p->n_tv > 16) fail(MLMC_ERR_INVALID_ARG, "n_tv must be in 1..16");
  if (p->setup_kind == MLMC_SETUP_CONSTANT && (p->n_tv != 1 || p->spin_split))
    fail(MLMC_ERR_INVALID_ARG, "constant setup needs n_tv = 1 and no spin split");
  if (p->fgmres_restart < 1 || p->fgmres_restart > 64) fail(MLMC_ERR_INVALID_ARG, "fgmres_restart must be in 1..64");
  if (p->max_iter < 1) fail(MLMC_ERR_INVALID_ARG, "max_iter must be positive");
  if (p->cycle == MLMC_CYCLE_K && (p->kcycle_its < 1 || p->kcycle_its > 8))
    fail(MLMC_ERR_INVALID_ARG, "kcycle_its must be in 1..8");
  if (p->precision != MLMC_PREC_FP64 && p->precision != MLMC_PREC_MIXED_FP32)
    fail(MLMC_ERR_INVALID_ARG, "unknown precision");
  long nx = op->nx, ny = op->ny;
  for (int l = 0; l + 1 < p->levels; ++l) {
    if (nx % p->agg_x || ny % p->agg_y) fail(MLMC_ERR_INVALID_ARG, "lattice not divisible by the aggregates");
    if (nx % 2 || ny % 2) fail(MLMC_ERR_INVALID_ARG, "smoothed levels need even lattice sizes");
    nx /= p->agg_x;
    ny /= p->agg_y;
  }
  int dc = p->n_tv * (p->spin_split ? 2 : 1);
  if (dc != 1 && dc != 2 && dc != 4 && dc != 8 && dc != 16)
    fail(MLMC_ERR_UNSUPPORTED, "coarse dofs per site must be 1, 2, 4, 8 or 16");
  if (nx * ny * dc > 8192) fail(MLMC_ERR_INVALID_ARG, "coarsest level larger than 8192 unknowns");
}

void setup(H_t &h, const mlmc_operator_desc *op, const mlmc_hierarchy_params *p, cudaStream_t stream) {
  validate(op, p);
  h.stream = stream;
  h.prm = *p;
  h.complex_op = op->kind == MLMC_OP_WILSON2D;
  h.t64 = h.complex_op ? C64 : F64;
  h.t32 = h.complex_op ? C32 : F32;
  h.L = p->levels;
  h.kmax = p->block;
  const bool mixed = p->precision == MLMC_PREC_MIXED_FP32;
  const int dc = p->n_tv * (p->spin_split ? 2 : 1);
  const size_t es = dtype_size(h.t64), es32 = dtype_size(h.t32);
  h.lv.resize(h.L);
  for (int l = 0; l < h.L; ++l) {
    Level &Lv = h.lv[l];
    Lv.nx = l == 0 ? op->nx : h.lv[l - 1].nx / p->agg_x;
    Lv.ny = l == 0 ? op->ny : h.lv[l - 1].ny / p->agg_y;
    Lv.d = l == 0 ? (h.complex_op ? 2 : 1) : dc;
    Lv.nsite = (size_t)Lv.nx * Lv.ny;
    Lv.n = Lv.nsite * Lv.d;
    Lv.coef64.alloc(Lv.nsite * 5 * Lv.d * Lv.d * es);
    if (mixed) Lv.coef32.alloc(Lv.nsite * 5 * Lv.d * Lv.d * es32);
    if (l + 1 < h.L) {
      Lv.ax = p->agg_x;
      Lv.ay = p->agg_y;
      Lv.dc = dc;
      Lv.dinv64.alloc(Lv.nsite * Lv.d * Lv.d * es);
      Lv.P64.alloc(Lv.n * dc * es);
      if (mixed) {
        Lv.dinv32.alloc(Lv.nsite * Lv.d * Lv.d * es32);
        Lv.P32.alloc(Lv.n * dc * es32);
      }
    } else {
      Lv.Ainv64.alloc(Lv.n * Lv.n * es);
      if (mixed) Lv.Ainv32.alloc(Lv.n * Lv.n * es32);
    }
  }
  // workspaces.  The FP64 cycle serves the solves in the FP64 form; in the
  // mixed form it only serves the setup bootstrap (n_tv columns) and the
  // FP32 cycle serves the solves.
  const int k = h.kmax;
  for (int lo = 0; lo < (mixed ? 2 : 1); ++lo) {
    DType t = lo ? h.t32 : h.t64;
    int kc = (lo == 0 && mixed) ? p->n_tv : std::max(k, p->n_tv);
    h.cyc[lo].resize(h.L);
    for (int l = 0; l < h.L; ++l) {
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
    h.xs[l].alloc(h.lv[l].n * (size_t)k * es);
    h.ys[l].alloc(h.lv[l].n * (size_t)k * es);
    if (l + 1 < h.L) {
      h.outer[l].reset(new Krylov());
      alloc_krylov(h, *h.outer[l], h.t64, h.lv[l].n, k, p->fgmres_restart);
    }
  }
  h.dots.alloc(2 * (size_t)k * 16);
  h.samples.alloc((size_t)k * 16);
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
int sample_block(H_t &h, int l, int noise, uint64_t seed, uint64_t first, int k, double tol, int purpose,
                 bool *conv) {
  const int kind = noise == MLMC_NOISE_Z4 ? 1 : 0;
  Level &Lv = h.lv[l];
  cudaStream_t s = h.stream;
  launch_noise(kind, seed, key_hi(purpose, l + 1), first, Lv.n, k, h.t64, h.xs[l].p, s);
  h.launches++;
  bool c1 = true, c2 = true;
  int its = solve_level(h, l, h.xs[l].p, h.ys[l].p, k, tol, &c1);
  char *dxy = h.dots.as<char>(), *dzw = dxy + (size_t)k * 16;
  auto coldot = [&](int lev, const void *a, const void *b, void *out) {
    launch_multidot(h.t64, a, h.lv[lev].n * (size_t)k, 1, b, h.lv[lev].n, k,
                    h.outer[0]->partials.p, multidot_parts(h.lv[lev].n, k), out, h.complex_op ? C64 : F64, s);
    h.launches += 2;
  };
  coldot(l, h.xs[l].p, h.ys[l].p, dxy);
  if (l + 1 < h.L) {
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
}

void need_level(const H_t *h, int level, int lo, int hi) {
  if (!h) fail(MLMC_ERR_INVALID_ARG, "null hierarchy");
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
  cudaStreamSynchronize(h->stream);
  delete h;
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

int mlmc_get_prolongation(const mlmc_hierarchy *h, int level, void *host_out) {
  return translate([&] {
    need_level(h, level, 1, h ? h->L - 1 : 0);
    if (!host_out) fail(MLMC_ERR_INVALID_ARG, "null output");
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
    check_cuda(cudaMemcpyAsync(host_out, Lv.coef64.p, Lv.nsite * 5 * Lv.d * Lv.d * dtype_size(h->t64),
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
    bool all_conv = true;
    for (int done = 0, b = 0; done < n_samples; ++b) {
      int k = std::min(h->kmax, n_samples - done);
      bool conv = true;
      int its = sample_block(*h, level - 1, noise, seed, first + done, k, tol, MLMC_PURPOSE_NOISE, &conv);
      copy_samples_out(*h, k, out_samples + done);
      if (out_iters) out_iters[b] = its;
      all_conv = all_conv && conv;
      done += k;
    }
    if (!all_conv) fail(MLMC_ERR_NOT_CONVERGED, "a level solve did not reach tol within max_iter");
  });
}

int mlmc_coarse_trace_exact(mlmc_hierarchy *h, mlmc_c64 *out) {
  return translate([&] {
    need(h);
    if (!out) fail(MLMC_ERR_INVALID_ARG, "null output");
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
    if (p->form != MLMC_FORM_SIMPLIFIED) fail(MLMC_ERR_UNSUPPORTED, "only the simplified form (Remark 4.3) is built");
    if (p->noise == MLMC_NOISE_Z4 && !h->complex_op) fail(MLMC_ERR_INVALID_ARG, "Z4 noise needs a complex operator");
    H_t &H = *h;
    const int L = H.L, nd = L - 1;
    std::memset(r, 0, sizeof(*r));
    r->levels = L;
    for (int l = 0; l < 16; ++l) H.iters_accum[l] = H.solves_accum[l] = H.applies_accum[l] = 0.0;
    auto t0 = std::chrono::steady_clock::now();
    mlmc_c64 TL;
    {
      const Level &C = H.lv[L - 1];
      launch_trace(H.t64, C.Ainv64.p, (int)C.n, H.trace.p, H.stream);
      H.launches++;
      check_cuda(cudaMemcpyAsync(&TL, H.trace.p, sizeof(TL), cudaMemcpyDeviceToHost, H.stream), "D2H trace");
      check_cuda(cudaStreamSynchronize(H.stream), "sync");
    }
    r->coarse_term = TL;
    // five warm-up estimates from the warm-up stream (Sec. 5)
    std::vector<mlmc_c64> tmp(std::max(5, H.kmax));
    double warm[5];
    for (int i = 0; i < 5; ++i) warm[i] = TL.re;
    const int kw = std::min(5, H.kmax);
    for (int l = 0; l < nd; ++l) {
      for (int done = 0; done < 5; done += kw) {
        int k = std::min(kw, 5 - done);
        bool conv = true;
        sample_block(H, l, p->noise, p->seed, done, k, p->tol, MLMC_PURPOSE_WARMUP, &conv);
        if (!conv) fail(MLMC_ERR_NOT_CONVERGED, "warm-up solve did not converge");
        copy_samples_out(H, k, tmp.data());
        for (int i = 0; i < k; ++i) warm[done + i] += tmp[i].re;
      }
    }
    double mean = 0.0;
    for (double v : warm) mean += v / 5.0;
    double ms = 0.0;
    for (double v : warm) ms += (v - mean) * (v - mean) / 5.0;
    double tau = mean - std::sqrt(ms);
    r->tau = tau;
    double wsum = 0.0;
    for (int l = 0; l < nd; ++l) wsum += p->weights[l];
    const int minN = p->min_samples > 0 ? p->min_samples : 5;
    const int maxN = p->max_samples > 0 ? p->max_samples : (1 << 24);
    double var_sum = 0.0;
    mlmc_c64 total = TL;
    for (int l = 0; l < nd; ++l) {
      double w = wsum > 0.0 ? p->weights[l] : 1.0 / nd;
      double rho = std::sqrt(w) * p->eps * std::fabs(tau);
      auto tl = std::chrono::steady_clock::now();
      check_cuda(cudaMemsetAsync(H.acc.p, 0, 4 * sizeof(double), H.stream), "memset acc");
      double acc[4] = {0, 0, 0, 0};
      for (;;) {
        int k = std::min(H.kmax, maxN - (int)acc[0]);
        if (k <= 0) break;
        bool conv = true;
        sample_block(H, l, p->noise, p->seed, (uint64_t)acc[0], k, p->tol, MLMC_PURPOSE_NOISE, &conv);
        if (!conv) fail(MLMC_ERR_NOT_CONVERGED, "level solve did not converge");
        launch_accumulate(H.samples.p, k, H.acc.as<double>(), H.stream);
        H.launches++;
        check_cuda(cudaMemcpyAsync(acc, H.acc.p, sizeof(acc), cudaMemcpyDeviceToHost, H.stream), "D2H acc");
        check_cuda(cudaStreamSynchronize(H.stream), "sync");
        double N = acc[0];
        double var = N > 1 ? acc[3] / (N - 1) : INFINITY;
        if (N >= minN && std::sqrt(var / N) <= rho) break;
      }
      double N = acc[0];
      double var = N > 1 ? acc[3] / (N - 1) : 0.0;
      r->n_samples[l] = (int)N;
      r->mean[l].re = acc[1];
      r->mean[l].im = acc[2];
      r->variance[l] = var;
      r->seconds[l] = std::chrono::duration<double>(std::chrono::steady_clock::now() - tl).count();
      total.re += acc[1];
      total.im += acc[2];
      if (N > 0) var_sum += var / N;
    }
    for (int l = 0; l < nd && l < 16; ++l) {
      double solves = H.solves_accum[l];
      r->iters[l] = solves > 0 ? H.iters_accum[l] / solves : 0.0;
    }
    // cost model (Sec. 5): nnz-weighted operator products per level
    for (int l = 0; l < L && l < 16; ++l) {
      const Level &Lv = H.lv[l];
      double nnz = (double)Lv.nsite * 5.0 * Lv.d * Lv.d;
      r->cost_nnz[l] = H.applies_accum[l] * nnz;
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
    if (k < 1 || k > h->kmax || reps < 1) fail(MLMC_ERR_INVALID_ARG, "bad k or reps");
    H_t &H = *h;
    int l = level - 1;
    int lo = which == 1 ? 1 : (which == 2 ? (H.prm.precision == MLMC_PREC_MIXED_FP32) : 0);
    if (lo && H.prm.precision != MLMC_PREC_MIXED_FP32) fail(MLMC_ERR_INVALID_ARG, "FP32 kernels need the mixed form");
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
    auto body = [&] {
      if (which == 2) {
        launch_rbgs_half(view(H, l, lo), y, x, k, 0, H.stream);
        launch_rbgs_half(view(H, l, lo), y, x, k, 1, H.stream);
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
    double coefb = const_coef ? 0.0 : (double)Lv.nsite * 5 * Lv.d * Lv.d * es;
    double bytes;
    if (which == 2) {
      // one sweep = two half-sweeps: each reads b and x on its colour, the
      // other colour's x as neighbours, writes x on its colour: 2 passes over
      // x plus b, plus the coefficient and inverse blocks
      double dinvb = (double)Lv.nsite * Lv.d * Lv.d * es;
      bytes = 3.0 * vec + (const_coef ? 0.0 : coefb + dinvb);
      if (ms_per_launch) *ms_per_launch = ms / reps;
    } else {
      bytes = 2.0 * vec + coefb;
      if (ms_per_launch) *ms_per_launch = ms / reps;
    }
    if (bytes_per_launch) *bytes_per_launch = bytes;
  });
}

int mlmc_launch_count(const mlmc_hierarchy *h, uint64_t *count) {
  return translate([&] {
    if (!h || !count) fail(MLMC_ERR_INVALID_ARG, "null argument");
    *count = h->launches;
  });
}

const char *mlmc_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
