"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances.  Noise is bit-exact (integer work).  Operator applies are FP64
with at most 9 products per entry: 1e-13 relative.  Solves run to relative
residual tol = 1e-12, so a sample x^* A^{-1} x differs from the exact value by
at most |x|^2 ||A^{-1}|| tol; the per-sample bar is 1e-9 relative (the FP64
form's target).  The mixed FP32-cycle form solves to 1e-10 under FP64 FGMRES:
1e-8 relative.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import estimator as E
from oracle.hierarchy import SetupParams, accumulated_prolongation, build_hierarchy
from oracle.operators import laplace2d, wilson2d
from oracle.philox import rademacher, z4, PURPOSE_NOISE, PURPOSE_SETUP
from paper_2108_11281_gb300.workloads import gauge_links


@pytest.fixture(scope="module")
def mlmc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_11281_gb300 import mlmc as m
    return m


def block_from_stencil(coef, nx, ny):
    """Sparse matrix of a [site][5][d][d] block stencil (periodic indexing)."""
    nsite, _, d, _ = coef.shape
    rows, cols, vals = [], [], []
    j, i = np.divmod(np.arange(nsite), nx)
    nbs = [np.arange(nsite), j * nx + (i + 1) % nx, j * nx + (i - 1) % nx,
           ((j + 1) % ny) * nx + i, ((j - 1) % ny) * nx + i]
    for dr, nb in enumerate(nbs):
        for a in range(d):
            for b in range(d):
                rows.append(np.arange(nsite) * d + a)
                cols.append(nb * d + b)
                vals.append(coef[:, dr, a, b])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nsite * d, nsite * d)).tocsr()
    A.sum_duplicates()
    return A


# ----------------------------------------------------------------- noise
@pytest.mark.parametrize("kind", ["rademacher", "z4"])
def test_noise_bit_exact(mlmc, kind):
    n, k, first, seed, level = 1000, 7, 123, 99, 3
    cplx = kind == "z4"
    out = torch.zeros((n, k), dtype=torch.complex128 if cplx else torch.float64, device="cuda")
    mlmc.noise(mlmc.NOISE_Z4 if cplx else mlmc.NOISE_RADEMACHER, seed, level, PURPOSE_NOISE, first, n, k,
               int(cplx), out.data_ptr())
    got = out.cpu().numpy()
    for c in range(k):
        ref = (z4 if cplx else rademacher)(n, seed, level, first + c)
        assert np.array_equal(got[:, c], ref)


# ----------------------------------------------------------------- operators and setup
def laplace_h(mlmc, N, levels, block=8, **kw):
    prm = mlmc.default_params(levels=levels, block=block, **kw)
    return mlmc.Hierarchy(mlmc.OP_LAPLACE2D, N, N, prm)


def test_laplace_apply_and_constant_galerkin(mlmc):
    N = 16
    h = laplace_h(mlmc, N, 2, n_tv=1, setup_kind=mlmc.SETUP_CONSTANT, bootstrap=0)
    A = laplace2d(N, N)
    x = torch.randn(N * N, 3, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    h.apply(1, x.data_ptr(), y.data_ptr(), 3)
    ref = A @ x.cpu().numpy()
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    lv = build_hierarchy(A, N, N, 1, SetupParams(levels=2, n_tv=1, kind="constant"))
    P = h.prolongation(1)
    assert np.array_equal(np.abs(P), np.full_like(P, 0.25))
    A2 = block_from_stencil(h.operator(2), N // 4, N // 4)
    assert np.abs((A2 - lv[1].A).toarray()).max() <= 1e-14
    tr = h.coarse_trace_exact()
    assert abs(tr - E.exact_coarse_trace(lv)) <= 1e-12 * abs(tr)
    h.close()


def test_wilson_apply(mlmc):
    N = 8
    U = gauge_links(N, N, 0.3, 5)
    prm = mlmc.default_params(levels=2, n_tv=2, spin_split=1, setup_kind=mlmc.SETUP_INVERSE, setup_sweeps=4,
                              coarse_sweeps=2, setup_omega=1.0, block=8, bootstrap=0)
    h = mlmc.Hierarchy(mlmc.OP_WILSON2D, N, N, prm, mass=0.1, links=U)
    S = wilson2d(N, N, 0.1, U)
    x = torch.randn(N * N * 2, 3, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    h.apply(1, x.data_ptr(), y.data_ptr(), 3)
    ref = S @ x.cpu().numpy()
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(block_from_stencil(h.operator(1), N, N) - S).max() <= 1e-15
    h.close()


@pytest.mark.parametrize("case", ["laplace-n64", "laplace-n1024", "laplace-n4096", "laplace-n4608", "wilson-n64",
                                  "wilson-n2048"])
def test_coarsest_inverse(mlmc, case):
    """The dense Gauss-Jordan inverse of the coarsest operator (Remark 4.2's exact term and
    the coarsest solves): its trace against numpy's inverse of the GPU's own coarsest
    stencil, and FP64 coarsest-level solves A_L x = b against the residual.  n_L = 64 and
    1024 run the in-place kernel with the rows in shared memory (1 and 7 rows per block);
    n_L = 4096 (27 rows per block, 884 KB) and the complex 2048 (14 rows, 458 KB) the same
    kernel with the rows in place in global memory; n_L = 4608 the kernel on [A | I]."""
    if case.startswith("laplace"):
        N, ntv = {"laplace-n64": (16, 4), "laplace-n1024": (64, 4), "laplace-n4096": (128, 4),
                  "laplace-n4608": (96, 8)}[case]
        h = laplace_h(mlmc, N, 2, n_tv=ntv, setup_sweeps=4, bootstrap=0)
    else:
        N, ntv = (16, 2) if case == "wilson-n64" else (64, 4)
        U = gauge_links(N, N, 0.3, 5)
        prm = mlmc.default_params(levels=2, n_tv=ntv, spin_split=1, setup_kind=mlmc.SETUP_INVERSE, setup_sweeps=4,
                                  setup_omega=1.0, block=8, bootstrap=0)
        h = mlmc.Hierarchy(mlmc.OP_WILSON2D, N, N, prm, mass=0.1, links=U)
    nx, ny, d = h.level_info(2)
    A2 = block_from_stencil(h.operator(2), nx, ny).toarray()
    n = A2.shape[0]
    assert n == int(case.split("-n")[1])
    inv = np.linalg.inv(A2)
    tr = h.coarse_trace_exact()
    assert abs(tr - np.trace(inv)) <= 1e-11 * abs(np.trace(inv))
    k = 5
    g = torch.Generator().manual_seed(11)
    dt = torch.complex128 if h.complex else torch.float64
    b = torch.randn(n, k, generator=g, dtype=torch.float64).to(dt).cuda()
    x = torch.zeros_like(b)
    h.solve(2, b.data_ptr(), x.data_ptr(), k, 1e-12)
    xn, bn = x.cpu().numpy(), b.cpu().numpy()
    assert np.abs(A2 @ xn - bn).max() <= 1e-10 * np.abs(bn).max() * np.abs(A2).max() * np.abs(inv).max()
    assert np.abs(xn - inv @ bn).max() <= 1e-10 * np.abs(inv @ bn).max()
    h.close()


def projector_distance(Pa, Pb):
    """max over aggregates of || Pa Pa^* - Pb Pb^* ||: independent of the basis inside each aggregate."""
    return max(np.abs(a @ a.conj().T - b @ b.conj().T).max() for a, b in zip(Pa, Pb))


@pytest.mark.parametrize("case", ["laplace", "wilson", "laplace-boot3"])
def test_setup_matches_oracle(mlmc, case):
    """GPU test vectors, bootstrap, MGS and Galerkin reproduce the oracle's hierarchy
    (same algorithm, FP64; agreement to rounding amplified by the setup's conditioning)."""
    if case.startswith("laplace"):
        N = 64
        nb, ni = (1, 2) if case == "laplace" else (2, 3)
        kw = dict(levels=3, n_tv=4, setup_sweeps=20, coarse_sweeps=10, bootstrap=nb, boot_iters=ni)
        h = laplace_h(mlmc, N, block=8, **kw)
        A = laplace2d(N, N)
        sp_ = SetupParams(levels=3, n_tv=4, sweeps=20, coarse_sweeps=10, bootstrap=nb, boot_iters=ni)
        lv = build_hierarchy(A, N, N, 1, sp_)
    else:
        N = 16
        U = gauge_links(N, N, 0.3, 7)
        kw = dict(levels=3, n_tv=2, spin_split=1, setup_kind=mlmc.SETUP_INVERSE, setup_sweeps=6, coarse_sweeps=4,
                  setup_omega=1.0, bootstrap=1, boot_iters=2, smooth_pre=2, smooth_post=2, block=8)
        prm = mlmc.default_params(**kw)
        h = mlmc.Hierarchy(mlmc.OP_WILSON2D, N, N, prm, mass=-0.05, links=U)
        A = wilson2d(N, N, -0.05, U)
        sp_ = SetupParams(levels=3, n_tv=2, spin_split=True, kind="inverse", sweeps=6, coarse_sweeps=4,
                          omega=1.0, noise_kind="z4", bootstrap=1, boot_iters=2, smooth_pre=2, smooth_post=2)
        lv = build_hierarchy(A, N, N, 2, sp_)
    for l in (1, 2):
        P = h.prolongation(l)
        assert projector_distance(P, lv[l - 1].P_blocks) <= 1e-9, l
        G = P.reshape(P.shape[0], -1, P.shape[2])
        assert max(np.abs(g.conj().T @ g - np.eye(g.shape[1])).max() for g in G) <= 1e-13
    tr = h.coarse_trace_exact()
    assert abs(tr - E.exact_coarse_trace(lv)) <= 1e-8 * abs(tr)
    # samples of the GPU-built hierarchy itself: in the hat form a sample depends on each
    # aggregate's range of P only (not on the basis inside it), so the GPU's and the oracle's
    # hierarchies give the same samples up to the setup's rounding (checked against the
    # size of the sample's first term, z^* A_l^{-1} z)
    kind = "rademacher" if case.startswith("laplace") else "z4"
    nz = mlmc.NOISE_RADEMACHER if kind == "rademacher" else mlmc.NOISE_Z4
    hats = [accumulated_prolongation(lv, l) for l in range(1, 4)]
    solv = E.LevelSolvers(lv)
    for level in (1, 2):
        got = h.sample_level_form(level, mlmc.FORM_HAT, nz, 5, 0, 6, 1e-12)
        ref = E.level_samples(lv, solv, level, kind, 5, 0, 6, form="hat", hats=hats)
        for j in range(6):
            x = (rademacher if kind == "rademacher" else z4)(lv[0].n, 5, level, j)
            z0 = hats[level - 1].conj().T @ x
            t0 = abs(np.vdot(z0, solv.solve(level - 1, z0)))
            assert abs(got[j] - ref[j]) <= 1e-7 * t0, (level, j, abs(got[j] - ref[j]) / t0)
    h.close()


# ----------------------------------------------------------------- solves and samples
def imported_laplace(mlmc, N=64, levels=3, **kw):
    A = laplace2d(N, N)
    lv = build_hierarchy(A, N, N, 1, SetupParams(levels=levels, n_tv=4, sweeps=20, coarse_sweeps=10))
    prm = mlmc.default_params(levels=levels, n_tv=4, **kw)
    h = mlmc.Hierarchy(mlmc.OP_LAPLACE2D, N, N, prm, user_P=[lv[i].P_blocks for i in range(levels - 1)])
    return h, lv


def test_galerkin_of_imported_P(mlmc):
    h, lv = imported_laplace(mlmc)
    for l in (2, 3):
        nx, ny, d = h.level_info(l)
        Al = block_from_stencil(h.operator(l), nx, ny)
        assert np.abs((Al - lv[l - 1].A).toarray()).max() <= 1e-13 * np.abs(lv[l - 1].A).max()
    h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_matches_exact(mlmc, precision):
    h, lv = imported_laplace(mlmc, block=5, precision=precision)
    k, n = 5, 64 * 64
    b = torch.randn(n, k, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    its = h.solve(1, b.data_ptr(), x.data_ptr(), k, 1e-12)
    assert 0 < its < 200
    A = lv[0].A
    bn, xn = b.cpu().numpy(), x.cpu().numpy()
    res = np.linalg.norm(bn - A @ xn, axis=0) / np.linalg.norm(bn, axis=0)
    assert res.max() <= 1e-12
    ref = E.exact_solver(A)(bn)
    assert np.linalg.norm(xn - ref) <= 1e-8 * np.linalg.norm(ref)
    h.close()


def compare_samples(got, ref, rtol):
    err = np.abs(got - ref) / np.abs(ref)
    assert err.max() <= rtol, (err.max(), np.argmax(err))


def test_config1_shape_samples(mlmc):
    """64x64 Dirichlet Laplacian, 2 levels, piecewise-constant P, Rademacher seed 0:
    70 level-1 samples (a full block of 64 and a ragged block of 6)."""
    N = 64
    h = laplace_h(mlmc, N, 2, block=64, n_tv=1, setup_kind=mlmc.SETUP_CONSTANT, bootstrap=0)
    got, its = h.sample_level(1, mlmc.NOISE_RADEMACHER, 0, 0, 70, 1e-12)
    lv = build_hierarchy(laplace2d(N, N), N, N, 1, SetupParams(levels=2, n_tv=1, kind="constant"))
    ref = E.level_samples(lv, E.LevelSolvers(lv), 1, "rademacher", 0, 0, 70)
    compare_samples(got, ref, 1e-9)
    h.close()


@pytest.mark.parametrize("precision,rtol", [(0, 1e-9), (1, 1e-8)])
def test_samples_three_levels(mlmc, precision, rtol):
    h, lv = imported_laplace(mlmc, block=8, precision=precision)
    solv = E.LevelSolvers(lv)
    tol = 1e-12 if precision == 0 else 1e-10
    for level, first, count in ((1, 3, 11), (2, 0, 8), (3, 5, 4)):
        got, _ = h.sample_level(level, mlmc.NOISE_RADEMACHER, 7, first, count, tol)
        ref = E.level_samples(lv, solv, level, "rademacher", 7, first, count) if level < 3 else \
            np.array([np.vdot(x, solv.solve(2, x)) for x in
                      [rademacher(lv[2].n, 7, 3, first + j) for j in range(count)]])
        compare_samples(got, ref, rtol)
    h.close()


@pytest.mark.parametrize("precision,rtol", [(0, 1e-9), (1, 1e-8)])
def test_samples_odd_aggregates(mlmc, precision, rtol):
    """3 x 3 aggregates (odd sides) on a 36^2 Laplacian, 3 levels, the oracle's P imported:
    the cycle's fused residual-restriction walks every site of an aggregate and skips the
    other colour; level-1 and level-2 samples against the oracle, in both forms."""
    N = 36
    A = laplace2d(N, N)
    sp_ = SetupParams(levels=3, agg_x=3, agg_y=3, n_tv=2, sweeps=10, coarse_sweeps=5, bootstrap=0)
    lv = build_hierarchy(A, N, N, 1, sp_)
    prm = mlmc.default_params(levels=3, agg_x=3, agg_y=3, n_tv=2, block=8, bootstrap=0, precision=precision)
    h = mlmc.Hierarchy(mlmc.OP_LAPLACE2D, N, N, prm, user_P=[lv[0].P_blocks, lv[1].P_blocks])
    solv = E.LevelSolvers(lv)
    tol = 1e-12 if precision == 0 else 1e-10
    for level in (1, 2):
        got, _ = h.sample_level(level, mlmc.NOISE_RADEMACHER, 5, 0, 6, tol)
        ref = E.level_samples(lv, solv, level, "rademacher", 5, 0, 6)
        compare_samples(got, ref, rtol)
    h.close()


def test_wilson_samples_imported_P(mlmc):
    N = 16
    U = gauge_links(N, N, 0.3, 11)
    S = wilson2d(N, N, 0.05, U)
    lv = build_hierarchy(S, N, N, 2, SetupParams(levels=3, n_tv=2, spin_split=True, kind="inverse", sweeps=6,
                                                 coarse_sweeps=4, omega=1.0, noise_kind="z4"))
    prm = mlmc.default_params(levels=3, n_tv=2, spin_split=1, block=4, smooth_pre=2, smooth_post=2)
    h = mlmc.Hierarchy(mlmc.OP_WILSON2D, N, N, prm, mass=0.05, links=U,
                       user_P=[lv[0].P_blocks, lv[1].P_blocks])
    solv = E.LevelSolvers(lv)
    for level in (1, 2):
        got, _ = h.sample_level(level, mlmc.NOISE_Z4, 3, 0, 6, 1e-12)
        ref = E.level_samples(lv, solv, level, "z4", 3, 0, 6)
        compare_samples(got, ref, 1e-9)
    tr = h.coarse_trace_exact()
    assert abs(tr - E.exact_coarse_trace(lv)) <= 1e-12 * abs(tr)
    h.close()


@pytest.mark.parametrize("precision,rtol", [(0, 1e-9), (1, 1e-8)])
def test_wilson_d8_level_apply_and_samples(mlmc, precision, rtol):
    """Coarse level with 8 dofs per site (4 test vectors x 2 spin halves), where the block
    apply and the block smoother take one thread per block row: the level-2 operator apply
    against its stencil matrix, and level-1 / level-2 samples against the oracle."""
    N = 32
    U = gauge_links(N, N, 0.3, 13)
    S = wilson2d(N, N, 0.05, U)
    lv = build_hierarchy(S, N, N, 2, SetupParams(levels=3, n_tv=4, spin_split=True, kind="inverse", sweeps=6,
                                                 coarse_sweeps=4, omega=1.0, noise_kind="z4"))
    prm = mlmc.default_params(levels=3, n_tv=4, spin_split=1, block=8, coarse_block=64, smooth_pre=2,
                              smooth_post=2, precision=precision)
    h = mlmc.Hierarchy(mlmc.OP_WILSON2D, N, N, prm, mass=0.05, links=U,
                       user_P=[lv[0].P_blocks, lv[1].P_blocks])
    nx, ny, d = h.level_info(2)
    assert (nx, ny, d) == (8, 8, 8)
    A2 = block_from_stencil(h.operator(2), nx, ny)
    assert abs(A2 - lv[1].A).max() <= 1e-12 * abs(lv[1].A).max()
    for k in (5, 64, 66):          # one column per thread; two (k even, >= 64), with a ragged chunk
        x = torch.randn(nx * ny * d, k, dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        h.apply(2, x.data_ptr(), y.data_ptr(), k)
        assert np.abs(y.cpu().numpy() - A2 @ x.cpu().numpy()).max() <= 1e-12 * abs(A2).max()
    solv = E.LevelSolvers(lv)
    # level 1 in blocks of 8; level 2 in one block of 64 columns (two columns per thread)
    for level, count in ((1, 6), (2, 64)):
        got, _ = h.sample_level(level, mlmc.NOISE_Z4, 5, 0, count, 1e-12 if precision == 0 else 1e-10)
        ref = E.level_samples(lv, solv, level, "z4", 5, 0, count)
        compare_samples(got, ref, rtol)
    h.close()


@pytest.mark.parametrize("tau_separate", [0, 1])
def test_trace_estimate_matches_oracle(mlmc, tau_separate):
    """Sec. 5 procedure on a 32x32 Laplacian, 2 levels: same tau, same N_l, same estimate;
    tau from samples 0..4 of the noise stream (counted in the means) or from five separate
    warm-up samples."""
    N = 32
    h = laplace_h(mlmc, N, 2, block=16, n_tv=1, setup_kind=mlmc.SETUP_CONSTANT, bootstrap=0)
    r = mlmc.result_dict(h.trace_estimate(eps=2e-2, noise=mlmc.NOISE_RADEMACHER, seed=4, tol=1e-12,
                                          tau_separate=tau_separate))
    lv = build_hierarchy(laplace2d(N, N), N, N, 1, SetupParams(levels=2, n_tv=1, kind="constant"))
    ref = E.trace_estimate(lv, "rademacher", seed=4, eps=2e-2, block=16, tau_separate=bool(tau_separate))
    assert r["n_samples"] == ref.n_samples
    assert abs(r["tau"] - ref.tau) <= 1e-9 * abs(ref.tau)
    assert abs(r["trace"] - ref.trace) <= 1e-9 * abs(ref.trace)
    assert abs(r["std_err"] - ref.std_err) <= 1e-6 * ref.std_err
    h.close()


def check_optimal_counts(r, eps, min_samples=5):
    """The estimate stops with every level at or above the oracle's Sec. 2 count for the
    variances and per-sample costs it ended with, and with the same weights."""
    nd = len(r["n_samples"])
    n = np.array(r["n_samples"], dtype=float)
    V = np.array(r["variance"], dtype=float)
    C = np.array(r["cost_nnz"][:nd], dtype=float) / n
    Nopt, _, w = E.optimal_allocation(V, C, eps * abs(r["tau"]), min_samples)
    for got, want in zip(n, Nopt):
        assert got >= max(min_samples, np.ceil(want * (1 - 1e-9)))
    assert np.allclose(r["weights_used"], w, rtol=1e-9, atol=0)


def test_optimal_allocation_estimate(mlmc):
    """Sec. 2 optimal allocation with the device-counted cost model (iteration counts
    included): the total variance meets (eps tau)^2 and every level ends at or above the
    Sec. 2 count for the variances and costs it reports."""
    N = 32
    h = laplace_h(mlmc, N, 3, block=16, n_tv=4, setup_sweeps=20, coarse_sweeps=10, smooth_pre=1, smooth_post=1)
    r = mlmc.result_dict(h.trace_estimate(eps=1e-2, noise=mlmc.NOISE_RADEMACHER, seed=2, tol=1e-12,
                                          allocation=mlmc.ALLOC_OPTIMAL))
    target = 1e-2 * abs(r["tau"])
    assert r["std_err"] <= target * (1 + 1e-12)
    assert all(n >= 5 for n in r["n_samples"])
    assert abs(sum(r["weights_used"]) - 1.0) < 1e-12
    check_optimal_counts(r, 1e-2)
    h.close()


def check_against_optimal_twin(mlmc, r, ref, lv, form="simplified"):
    """GPU estimate vs the oracle's adaptive Sec. 2 loop on the same samples: same N_l,
    tau and trace to 1e-9, the same nominal per-sample costs and weights."""
    assert r["n_samples"] == ref.n_samples
    assert abs(r["tau"] - ref.tau) <= 1e-9 * abs(ref.tau)
    assert abs(r["trace"] - ref.trace) <= 1e-9 * abs(ref.trace)
    assert abs(r["std_err"] - ref.std_err) <= 1e-6 * ref.std_err
    for l, n in enumerate(ref.n_samples, start=1):
        assert r["cost_nnz"][l - 1] == n * E.nominal_sample_cost(lv, l, form)
    assert np.allclose(r["weights_used"], ref.weights, rtol=1e-6, atol=0)


def test_optimal_allocation_matches_oracle_laplace(mlmc):
    """32^2 Laplacian, 3 levels, the oracle's P imported: the GPU's adaptive optimal
    allocation (nominal cost model) against the oracle's twin of the loop."""
    h, lv = imported_laplace(mlmc, N=32, levels=3, block=16, coarse_block=16)
    r = mlmc.result_dict(h.trace_estimate(eps=1e-2, noise=mlmc.NOISE_RADEMACHER, seed=2, tol=1e-12,
                                          allocation=mlmc.ALLOC_OPTIMAL, cost_model=mlmc.COST_NOMINAL))
    ref = E.optimal_trace_estimate(lv, "rademacher", seed=2, eps=1e-2, widths=[16, 16])
    assert sum(ref.n_samples) > 2 * 16            # the loop drew beyond the pilot blocks
    check_against_optimal_twin(mlmc, r, ref, lv)
    h.close()


def test_optimal_allocation_matches_oracle_wilson(mlmc):
    """16^2 Wilson operator, Z4 noise, imported P: the same comparison (complex samples,
    spin-split prolongations in the cost model)."""
    N = 16
    U = gauge_links(N, N, 0.3, 11)
    S = wilson2d(N, N, 0.05, U)
    lv = build_hierarchy(S, N, N, 2, SetupParams(levels=3, n_tv=2, spin_split=True, kind="inverse", sweeps=6,
                                                 coarse_sweeps=4, omega=1.0, noise_kind="z4"))
    prm = mlmc.default_params(levels=3, n_tv=2, spin_split=1, block=8, coarse_block=8, smooth_pre=2, smooth_post=2)
    h = mlmc.Hierarchy(mlmc.OP_WILSON2D, N, N, prm, mass=0.05, links=U, user_P=[lv[0].P_blocks, lv[1].P_blocks])
    r = mlmc.result_dict(h.trace_estimate(eps=1e-2, noise=mlmc.NOISE_Z4, seed=5, tol=1e-12,
                                          allocation=mlmc.ALLOC_OPTIMAL, cost_model=mlmc.COST_NOMINAL))
    ref = E.optimal_trace_estimate(lv, "z4", seed=5, eps=1e-2, widths=[8, 8])
    assert sum(ref.n_samples) > 2 * 8
    check_against_optimal_twin(mlmc, r, ref, lv)
    h.close()


def test_wilson_estimate_matches_oracle(mlmc):
    """Z4 estimate on a 16x16 Wilson operator (imported P): same N_l and estimate as the oracle."""
    N = 16
    U = gauge_links(N, N, 0.3, 11)
    S = wilson2d(N, N, 0.05, U)
    lv = build_hierarchy(S, N, N, 2, SetupParams(levels=3, n_tv=2, spin_split=True, kind="inverse", sweeps=6,
                                                 coarse_sweeps=4, omega=1.0, noise_kind="z4"))
    prm = mlmc.default_params(levels=3, n_tv=2, spin_split=1, block=8, smooth_pre=2, smooth_post=2)
    h = mlmc.Hierarchy(mlmc.OP_WILSON2D, N, N, prm, mass=0.05, links=U, user_P=[lv[0].P_blocks, lv[1].P_blocks])
    r = mlmc.result_dict(h.trace_estimate(eps=3e-2, noise=mlmc.NOISE_Z4, seed=5, tol=1e-12,
                                          weights=[0.4, 0.6]))
    ref = E.trace_estimate(lv, "z4", seed=5, eps=3e-2, block=8, weights=[0.4, 0.6])
    assert r["n_samples"] == ref.n_samples
    assert abs(r["trace"] - ref.trace) <= 1e-9 * abs(ref.trace)
    # tr(S^{-1}) is real (J-symmetry); a Z4 estimate carries only sampling noise in its imaginary part
    assert abs(r["trace"].imag) <= 4 * r["std_err"]
    h.close()


@pytest.mark.parametrize("cplx", [False, True])
def test_column_dots(mlmc, cplx):
    """Per-column conj(x) . y in FP64 against numpy (Remark 4.3 sample products)."""
    n, k = 5000, 37
    g = torch.Generator().manual_seed(1)
    dt = torch.complex128 if cplx else torch.float64
    if cplx:
        x = torch.complex(torch.randn(n, k, generator=g, dtype=torch.float64), torch.randn(n, k, generator=g, dtype=torch.float64))
        y = torch.complex(torch.randn(n, k, generator=g, dtype=torch.float64), torch.randn(n, k, generator=g, dtype=torch.float64))
    else:
        x = torch.randn(n, k, generator=g, dtype=dt)
        y = torch.randn(n, k, generator=g, dtype=dt)
    out = torch.zeros(k, dtype=dt, device="cuda")
    xd, yd = x.cuda(), y.cuda()          # keep the device copies alive during the call
    mlmc.column_dots(cplx, xd.data_ptr(), yd.data_ptr(), n, k, out.data_ptr())
    ref = np.einsum("ic,ic->c", x.numpy().conj(), y.numpy())
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max() * 10


def test_batch_matches_serial_and_autotune(mlmc):
    """Uneven batch (shifted Laplacians and Wilson operators of different sizes) run on
    worker threads with one stream per instance gives the same estimates as one-by-one
    runs; the autotuned block width does not change the samples."""
    def build(i):
        if i % 2 == 0:
            N = 32 * (1 + i // 2)
            prm = mlmc.default_params(levels=2, n_tv=4, setup_sweeps=20, coarse_sweeps=10, block=32,
                                      precision=mlmc.PREC_MIXED_FP32, inner_its=4, fgmres_restart=8)
            return mlmc.Hierarchy(mlmc.OP_LAPLACE2D, N, N, prm, shift=[1e-2, 1e-3][i // 2]), mlmc.NOISE_RADEMACHER
        N = 16 * (1 + i // 2)
        prm = mlmc.default_params(levels=2, n_tv=2, spin_split=1, setup_kind=mlmc.SETUP_INVERSE, setup_sweeps=6,
                                  setup_omega=1.0, block=32, precision=mlmc.PREC_MIXED_FP32, inner_its=4,
                                  fgmres_restart=8, smooth_pre=2, smooth_post=2)
        return mlmc.Hierarchy(mlmc.OP_WILSON2D, N, N, prm, mass=0.1, links=gauge_links(N, N, 0.3, 30 + i)), mlmc.NOISE_Z4
    built = [build(i) for i in range(4)]
    hs = [b[0] for b in built]
    params = [mlmc.estimate_params(eps=3e-2, noise=b[1], seed=i, tol=1e-10) for i, b in enumerate(built)]
    batch, status = mlmc.trace_estimate_batch(hs, params, workers=4)
    assert status == [0, 0, 0, 0]
    k, t = hs[0].autotune_block(1, mlmc.NOISE_RADEMACHER, 1e-10)
    assert k in (16, 32) and t > 0
    for i, h in enumerate(hs):
        r = mlmc.result_dict(h.trace_estimate(eps=3e-2, noise=built[i][1], seed=i, tol=1e-10,
                                              allocation=mlmc.ALLOC_OPTIMAL))
        if i == 0 and k != 32:
            # a different block width draws a different number of samples, but each sample is the same
            s, _ = h.sample_level(1, mlmc.NOISE_RADEMACHER, 0, 0, 8, 1e-10)
            h.set_block_width(32)
            s2, _ = h.sample_level(1, mlmc.NOISE_RADEMACHER, 0, 0, 8, 1e-10)
            assert np.allclose(s, s2, rtol=1e-8)
            continue
        assert r["n_samples"] == batch[i]["n_samples"]
        assert abs(r["trace"] - batch[i]["trace"]) <= 1e-12 * abs(r["trace"])
    for h in hs:
        h.close()


def test_hat_and_plain_forms(mlmc):
    """Hat form (noise on the fine space restricted by R^_l, Eq. tr_ml_dec) and plain
    Hutchinson (Eq. plain_tr_estimate) samples and estimates against the oracle."""
    h, lv = imported_laplace(mlmc, block=8)
    solv = E.LevelSolvers(lv)
    hats = [accumulated_prolongation(lv, l) for l in range(1, 4)]
    for level in (1, 2):
        got = h.sample_level_form(level, mlmc.FORM_HAT, mlmc.NOISE_RADEMACHER, 3, 2, 6, 1e-12)
        ref = E.level_samples(lv, solv, level, "rademacher", 3, 2, 6, form="hat", hats=hats)
        compare_samples(got, ref, 1e-9)
    got = h.sample_level_form(1, mlmc.FORM_PLAIN, mlmc.NOISE_RADEMACHER, 3, 0, 6, 1e-12)
    ref = E.level_samples(lv, solv, 1, "rademacher", 3, 0, 6, form="plain")
    compare_samples(got, ref, 1e-9)
    for form, name in ((mlmc.FORM_HAT, "hat"), (mlmc.FORM_PLAIN, "plain")):
        r = mlmc.result_dict(h.trace_estimate(eps=5e-2, noise=mlmc.NOISE_RADEMACHER, seed=1, tol=1e-12, form=form))
        ref = E.trace_estimate(lv, "rademacher", seed=1, eps=5e-2, block=8, form=name, solvers=solv)
        assert r["n_samples"] == ref.n_samples, name
        assert abs(r["trace"] - ref.trace) <= 1e-9 * abs(ref.trace), name
    h.close()


def test_block_width_growth_keeps_samples(mlmc):
    """Wider blocks on the coarse level differences (coarse_growth) change only the
    batching: samples are indexed (seed, level, j), so the same samples come back, the
    per-block iteration list has one entry per block, and an estimate with a fixed budget
    has the same mean."""
    N = 64
    kw = dict(n_tv=4, setup_sweeps=20, coarse_sweeps=10, block=4, coarse_block=8, bootstrap=0)
    h0 = laplace_h(mlmc, N, 4, **kw)
    h1 = laplace_h(mlmc, N, 4, coarse_growth=1, **kw)
    for level, width in ((2, 8), (3, 16)):
        s0, it0 = h0.sample_level(level, mlmc.NOISE_RADEMACHER, 1, 0, 40, 1e-12)
        s1, it1 = h1.sample_level(level, mlmc.NOISE_RADEMACHER, 1, 0, 40, 1e-12)
        assert np.abs(s0 - s1).max() <= 1e-9 * np.abs(s0).max()
        assert len(it0) == 5 and len(it1) == (40 + width - 1) // width
    r0 = mlmc.result_dict(h0.trace_estimate(noise=mlmc.NOISE_RADEMACHER, seed=2, tol=1e-12,
                                            allocation=mlmc.ALLOC_FIXED, n_fixed=[16, 16, 32]))
    r1 = mlmc.result_dict(h1.trace_estimate(noise=mlmc.NOISE_RADEMACHER, seed=2, tol=1e-12,
                                            allocation=mlmc.ALLOC_FIXED, n_fixed=[16, 16, 32]))
    assert r0["n_samples"] == r1["n_samples"] == [16, 16, 32]
    assert abs(r0["trace"] - r1["trace"]) <= 1e-9 * abs(r0["trace"])
    h0.close()
    h1.close()


@pytest.mark.parametrize("case, k", [("laplace", 8), ("laplace", 6), ("laplace", 40), ("laplace", 136),
                                     ("wilson", 8), ("wilson", 6), ("laplace-agg3", 8), ("laplace-agg3", 6)])
def test_fused_residual_restriction(mlmc, case, k):
    """The cycle's fused residual-and-restriction kernel against P^* m (b - A x) formed
    with the level's own operator and prolongation (m = the sites of one colour), on
    random blocks: the Example 5.1 fine level and a d = 4 aggregation level (Laplace),
    the complex d = 2 fine level of a Wilson operator with spin-split P, and 3 x 3
    aggregates (odd sides: the kernel walks every site and skips the other colour) on the
    fine level and a d = 2 level; FP64 data (1e-12 of scale) and, for the Laplacian, FP32
    data in the mixed form (1e-5).  k covers 16-byte and scalar column packs and blocks of
    8, 16 and 32 packs with a ragged last chunk."""
    if case == "laplace":
        N = 32
        h = laplace_h(mlmc, N, 3, block=8, n_tv=4, setup_sweeps=10, coarse_sweeps=5, bootstrap=0,
                      precision=mlmc.PREC_MIXED_FP32)
        A1 = laplace2d(N, N)
        levels = [(1, A1), (2, block_from_stencil(h.operator(2), *h.level_info(2)[:2]))]
        cplx = False
    elif case == "laplace-agg3":
        N = 36
        h = laplace_h(mlmc, N, 3, block=8, n_tv=2, setup_sweeps=10, coarse_sweeps=5, bootstrap=0, agg_x=3,
                      agg_y=3, precision=mlmc.PREC_MIXED_FP32)
        levels = [(1, laplace2d(N, N)), (2, block_from_stencil(h.operator(2), *h.level_info(2)[:2]))]
        cplx = False
    else:
        N = 16
        U = gauge_links(N, N, 0.3, 5)
        prm = mlmc.default_params(levels=3, n_tv=2, spin_split=1, setup_kind=mlmc.SETUP_INVERSE, setup_sweeps=4,
                                  setup_omega=1.0, block=8, bootstrap=0)
        h = mlmc.Hierarchy(mlmc.OP_WILSON2D, N, N, prm, mass=0.1, links=U)
        levels = [(1, wilson2d(N, N, 0.1, U))]
        cplx = True
    g = torch.Generator().manual_seed(3)
    for level, A in levels:
        nx, ny, d = h.level_info(level)
        Pb = h.prolongation(level)                       # [agg][ax*ay*d][dc]
        n, nc = A.shape[0], h.level_info(level + 1)[0] * h.level_info(level + 1)[1] * h.level_info(level + 1)[2]
        dt = torch.complex128 if cplx else torch.float64
        if cplx:
            x = torch.complex(torch.randn(n, k, generator=g, dtype=torch.float64),
                              torch.randn(n, k, generator=g, dtype=torch.float64))
            b = torch.complex(torch.randn(n, k, generator=g, dtype=torch.float64),
                              torch.randn(n, k, generator=g, dtype=torch.float64))
        else:
            x = torch.randn(n, k, generator=g, dtype=dt)
            b = torch.randn(n, k, generator=g, dtype=dt)
        r = b.numpy() - A @ x.numpy()
        j, i = np.divmod(np.arange(nx * ny), nx)
        ax, ay = h.params.agg_x, h.params.agg_y
        ncx = nx // ax
        for colour in (0, 1):
            mask = np.repeat(((i + j) % 2 == colour).astype(float), d)
            rm = r * mask[:, None]
            ref = np.zeros((nc, k), dtype=r.dtype)
            dc = Pb.shape[2]
            for I in range(Pb.shape[0]):
                bi, bj = I % ncx, I // ncx
                rows = []
                for loc in range(ax * ay):
                    jj, ii = divmod(loc, ax)
                    site = (bj * ay + jj) * nx + bi * ax + ii
                    rows.extend(site * d + a for a in range(d))
                ref[I * dc:(I + 1) * dc] = Pb[I].conj().T @ rm[rows]
            for prec in ((0, 1) if not cplx else (0,)):
                if prec == 0:
                    xs, bs, rc = x.cuda(), b.cuda(), torch.zeros(nc, k, dtype=dt, device="cuda")
                else:
                    xs, bs = x.to(torch.float32).cuda(), b.to(torch.float32).cuda()
                    rc = torch.zeros(nc, k, dtype=torch.float32, device="cuda")
                h.residual_restrict(level, mlmc.PREC_MIXED_FP32 if prec else mlmc.PREC_FP64, xs.data_ptr(),
                                    bs.data_ptr(), rc.data_ptr(), k, colour)
                tol = 1e-12 if prec == 0 else 1e-5
                got = rc.cpu().numpy()
                assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (level, colour, prec)
    h.close()


def test_prolongation_of_one_colour_is_exact(mlmc):
    """The cycle prolongates only colour 0: its post-smoothing starts with colour 1 and does
    not read x there.  With a zero-weight learned correction switched on, the fine level
    prolongates every site (the correction reads all of x) and adds exactly zero, so the
    samples must come out equal to the last bit."""
    h = laplace_h(mlmc, 32, 3, block=8, n_tv=4, setup_sweeps=10, coarse_sweeps=5, bootstrap=0,
                  precision=mlmc.PREC_MIXED_FP32)
    s0, _ = h.sample_level(1, mlmc.NOISE_RADEMACHER, 4, 0, 8, 1e-10)
    h.learned_set(np.zeros(h.net_weights(), dtype=np.float32), enable=1)
    s1, _ = h.sample_level(1, mlmc.NOISE_RADEMACHER, 4, 0, 8, 1e-10)
    assert np.array_equal(s0, s1)
    h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_512_column_blocks_on_a_coarse_difference(mlmc, precision):
    """coarse_growth = 2 widens the third level difference to 512 columns (real operators):
    its samples (two blocks, 512 + 88) agree with the oracle's exact solves (FP64 form 1e-9
    at tol 1e-12; mixed form 1e-8 at tol 1e-10), and the width is reported."""
    h, lv = imported_laplace(mlmc, N=64, levels=4, block=8, coarse_block=128, coarse_growth=2, precision=precision)
    assert [h.block_width(l) for l in (1, 2, 3)] == [8, 128, 512]
    tol, rtol = (1e-12, 1e-9) if precision == 0 else (1e-10, 1e-8)
    got, its = h.sample_level(3, mlmc.NOISE_RADEMACHER, 3, 0, 600, tol)
    ref = E.level_samples(lv, E.LevelSolvers(lv), 3, "rademacher", 3, 0, 600)
    assert len(its) == 2
    compare_samples(got, ref, rtol)
    h.close()


def test_sharded_driver_one_rank_matches_library_estimate(mlmc):
    """The multi-GPU driver (sharded.py) on one rank draws its blocks through
    mlmc_sample_block and merges their device statistics on the host: the same N_l, tau
    and trace (1e-12) as mlmc_trace_estimate's loop with nominal costs, and the sharded
    blocks reproduce mlmc_sample_level's samples."""
    from paper_2108_11281_gb300 import sharded
    h, lv = imported_laplace(mlmc, N=32, levels=3, block=16, coarse_block=16)
    r = mlmc.result_dict(h.trace_estimate(eps=1e-2, noise=mlmc.NOISE_RADEMACHER, seed=2, tol=1e-12,
                                          allocation=mlmc.ALLOC_OPTIMAL, cost_model=mlmc.COST_NOMINAL))
    smp = sharded.HierarchySampler(h, mlmc.NOISE_RADEMACHER, 2, 1e-12)
    s = sharded.sharded_trace_estimate(smp, lambda v: [v], 0, 1, eps=1e-2)
    assert s["n_samples"] == r["n_samples"]
    assert abs(s["tau"] - r["tau"]) <= 1e-12 * abs(r["tau"])
    assert abs(s["trace"] - r["trace"]) <= 1e-12 * abs(r["trace"])
    blk, stats, cost = h.sample_block(2, mlmc.FORM_SIMPLIFIED, mlmc.NOISE_RADEMACHER, 2, 16, 16, 1e-12)
    ref, _ = h.sample_level(2, mlmc.NOISE_RADEMACHER, 2, 16, 16, 1e-12)
    assert np.abs(blk - ref).max() <= 1e-12 * np.abs(ref).max()
    assert stats[0] == 16 and abs(stats[1] - blk.mean()) <= 1e-12 * abs(blk.mean())
    assert cost > 0 and h.block_width(1) == 16 and h.nominal_sample_cost(1) == E.nominal_sample_cost(lv, 1)
    h.close()
