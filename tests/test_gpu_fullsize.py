"""Full-size checks in the bench's launch configuration, plus edge cases.

At the workloads' full sizes the oracle cannot afford exact solves, so these
tests check sampled outputs the oracle computes one by one (noise columns,
operator rows) and properties that hold at any size: FP64 true residuals of
the solves, orthonormal prolongations, the Galerkin identity, J-symmetry of
every coarse Wilson operator, and the estimate against the closed-form trace
of Example 5.1.  Edge cases: one-column blocks, empty sample requests, a
periodic shifted Laplacian, and an iteration cap that must surface as
MLMC_ERR_NOT_CONVERGED rather than a wrong result.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import estimator as E
from oracle.hierarchy import SetupParams, build_hierarchy
from oracle.operators import laplace2d, spin_parity, wilson2d
from oracle.philox import rademacher, z4


@pytest.fixture(scope="module")
def mlmc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_11281_gb300 import mlmc as m
    return m


@pytest.fixture(scope="module")
def bench_mod():
    import bench
    return bench


def stencil_matrix(coef, nx, ny):
    nsite, _, d, _ = coef.shape
    j, i = np.divmod(np.arange(nsite), nx)
    nbs = [np.arange(nsite), j * nx + (i + 1) % nx, j * nx + (i - 1) % nx, ((j + 1) % ny) * nx + i,
           ((j - 1) % ny) * nx + i]
    rows, cols, vals = [], [], []
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


def test_laplace1024_full_size(mlmc, bench_mod):
    w = bench_mod.WORKLOADS["laplace1024"]
    h = bench_mod.make_hierarchy(mlmc, mlmc.PREC_MIXED_FP32, w, torch.cuda.current_stream().cuda_stream)
    n, k = w["nx"] * w["ny"], w["block"]
    # noise: three sampled columns of a full block, bit-exact against the oracle generator
    X = torch.zeros(n, k, dtype=torch.float64, device="cuda")
    mlmc.noise(mlmc.NOISE_RADEMACHER, 5, 1, mlmc.PURPOSE_NOISE, 1000, n, k, 0, X.data_ptr())
    Xc = X.cpu().numpy()
    for c in (0, 31, k - 1):
        assert np.array_equal(Xc[:, c], rademacher(n, 5, 1, 1000 + c))
    # operator apply against Example 5.1 on the full lattice (4 columns)
    A = laplace2d(w["nx"], w["ny"])
    Y = torch.empty(n, 4, dtype=torch.float64, device="cuda")
    X4 = X[:, :4].contiguous()
    h.apply(1, X4.data_ptr(), Y.data_ptr(), 4)
    ref = A @ Xc[:, :4]
    assert np.abs(Y.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
    # FP64 true residual of a full-width solve (the outer FGMRES acceptance gate)
    Z = torch.zeros_like(X)
    h.solve(1, X.data_ptr(), Z.data_ptr(), k, w["tol_mixed"])
    res = np.linalg.norm(Xc - A @ Z.cpu().numpy(), axis=0) / np.linalg.norm(Xc, axis=0)
    assert res.max() <= w["tol_mixed"]
    # orthonormal P on every level, Galerkin identity A_2 v = P^* A_1 P v on random vectors
    for l in range(1, w["levels"]):
        P = h.prolongation(l)
        G = np.einsum("iaq,iar->iqr", P.conj(), P)
        assert np.abs(G - np.eye(P.shape[2])[None]).max() <= 1e-12
    P1 = h.prolongation(1)
    nx2, ny2, d2 = h.level_info(2)
    A2 = stencil_matrix(h.operator(2), nx2, ny2)
    rng = np.random.default_rng(0)
    v = rng.normal(size=A2.shape[0])
    # P v assembled from the aggregate blocks (aggregate I = (bj, bi), local site jj*4 + ii)
    ncx = w["nx"] // 4
    Pv = np.zeros(n)
    blocks = np.einsum("iaq,iq->ia", P1, v.reshape(-1, d2))
    I = np.arange(blocks.shape[0])
    bi, bj = I % ncx, I // ncx
    for loc in range(16):
        ii, jj = loc % 4, loc // 4
        Pv[(bj * 4 + jj) * w["nx"] + bi * 4 + ii] = blocks[:, loc]
    APv = A @ Pv
    back = np.zeros_like(v).reshape(-1, d2)
    for loc in range(16):
        ii, jj = loc % 4, loc // 4
        back += P1[:, loc, :] * APv[(bj * 4 + jj) * w["nx"] + bi * 4 + ii][:, None]
    assert np.abs(A2 @ v - back.reshape(-1)).max() <= 1e-11 * np.abs(back).max()
    # the estimate in the bench's configuration against the closed form (Example 5.1)
    r = mlmc.result_dict(h.trace_estimate(eps=w["eps"], noise=mlmc.NOISE_RADEMACHER, seed=0, tol=w["tol_mixed"],
                                          allocation=mlmc.ALLOC_OPTIMAL))
    exact = bench_mod.closed_form(w)
    assert r["std_err"] <= w["eps"] * abs(r["tau"]) * (1 + 1e-12)
    assert abs(r["trace"].real - exact) <= 4 * r["std_err"]
    h.close()


def test_wilson128_full_size(mlmc, bench_mod):
    w = bench_mod.WORKLOADS["wilson128"]
    h = bench_mod.make_hierarchy(mlmc, mlmc.PREC_MIXED_FP32, w, torch.cuda.current_stream().cuda_stream)
    from paper_2108_11281_gb300.workloads import gauge_links
    S = wilson2d(w["nx"], w["ny"], w["mass"], gauge_links(w["nx"], w["ny"], w["link_sd"], w["link_seed"]))
    n, k = S.shape[0], w["block"]
    X = torch.zeros(n, k, dtype=torch.complex128, device="cuda")
    mlmc.noise(mlmc.NOISE_Z4, 3, 1, mlmc.PURPOSE_NOISE, 0, n, k, 1, X.data_ptr())
    Xc = X.cpu().numpy()
    assert np.array_equal(Xc[:, 7], z4(n, 3, 1, 7))
    Z = torch.zeros_like(X)
    h.solve(1, X.data_ptr(), Z.data_ptr(), k, w["tol_mixed"])
    res = np.linalg.norm(Xc - S @ Z.cpu().numpy(), axis=0) / np.linalg.norm(Xc, axis=0)
    assert res.max() <= w["tol_mixed"]
    # J A_l = A_l^* J on every level (spin-structure-preserving coarsening, Example 5.3)
    for l in range(1, w["levels"] + 1):
        nx, ny, d = h.level_info(l)
        Al = stencil_matrix(h.operator(l), nx, ny)
        J = sp.diags(spin_parity(nx * ny, d))
        assert abs(J @ Al - Al.conj().T @ J).max() <= 1e-12 * abs(Al).max()
    r = mlmc.result_dict(h.trace_estimate(eps=w["eps"], noise=mlmc.NOISE_Z4, seed=0, tol=w["tol_mixed"],
                                          allocation=mlmc.ALLOC_OPTIMAL))
    assert r["std_err"] <= w["eps"] * abs(r["tau"]) * (1 + 1e-12)
    assert abs(r["trace"].imag) <= 4 * r["std_err"]
    h.close()


def test_one_column_blocks_and_empty_requests(mlmc):
    N = 32
    prm = mlmc.default_params(levels=2, n_tv=1, setup_kind=mlmc.SETUP_CONSTANT, block=1, bootstrap=0)
    h = mlmc.Hierarchy(mlmc.OP_LAPLACE2D, N, N, prm)
    got, its = h.sample_level(1, mlmc.NOISE_RADEMACHER, 0, 3, 3, 1e-12)
    lv = build_hierarchy(laplace2d(N, N), N, N, 1, SetupParams(levels=2, n_tv=1, kind="constant"))
    ref = E.level_samples(lv, E.LevelSolvers(lv), 1, "rademacher", 0, 3, 3)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max() and len(its) == 3
    empty, its0 = h.sample_level(1, mlmc.NOISE_RADEMACHER, 0, 0, 0, 1e-12)
    assert len(empty) == 0 and its0 == []
    h.close()


def test_periodic_shifted_laplace(mlmc):
    N, shift = 32, 0.05
    prm = mlmc.default_params(levels=3, n_tv=4, setup_sweeps=20, coarse_sweeps=10, block=8)
    A = laplace2d(N, N, shift, periodic=True)
    lv = build_hierarchy(A, N, N, 1, SetupParams(levels=3, n_tv=4, sweeps=20, coarse_sweeps=10))
    h = mlmc.Hierarchy(mlmc.OP_LAPLACE2D, N, N, prm, shift=shift, periodic=1,
                       user_P=[lv[0].P_blocks, lv[1].P_blocks])
    x = torch.randn(N * N, 3, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    h.apply(1, x.data_ptr(), y.data_ptr(), 3)
    assert np.abs(y.cpu().numpy() - A @ x.cpu().numpy()).max() <= 1e-13 * 8
    got, _ = h.sample_level(1, mlmc.NOISE_RADEMACHER, 2, 0, 8, 1e-12)
    ref = E.level_samples(lv, E.LevelSolvers(lv), 1, "rademacher", 2, 0, 8)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    h.close()


def test_iteration_cap_reports_not_converged(mlmc):
    """A solve that cannot reach tol within max_iter returns MLMC_ERR_NOT_CONVERGED (host-side failure path)."""
    N = 64
    prm = mlmc.default_params(levels=2, n_tv=1, setup_kind=mlmc.SETUP_CONSTANT, block=4, bootstrap=0,
                              max_iter=1, fgmres_restart=1)
    h = mlmc.Hierarchy(mlmc.OP_LAPLACE2D, N, N, prm)
    with pytest.raises(mlmc.MLMCError) as ei:
        h.sample_level(1, mlmc.NOISE_RADEMACHER, 0, 0, 4, 1e-14)
    assert ei.value.status == mlmc.ERR_NOT_CONVERGED
    # the handle stays usable afterwards
    assert abs(h.coarse_trace_exact()) > 0
    h.close()
