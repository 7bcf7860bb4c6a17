"""The paper's hierarchy for Example 5.1 (Sec. 5) on the GPU against the oracle.

Bilinear interpolation between grids N_l = 2 N_{l+1} + 1, R = P^T, Galerkin
9-point coarse operators, 4-colour Gauss-Seidel on them, the hat form of the
estimator (R P != I) and its exact coarsest term tr(A_L^{-1} R^_L P^_L).

Tolerances as in the other parity tests: FP64 applies 1e-13 relative (at most
9 products per entry).  Samples from solves to relative residual tol differ
from the exact values by at most |z_l|^2 ||A_l^-1|| tol + |z_l+1|^2 ||A_l+1^-1|| tol
per sample (z = R^ x the restricted noise; the bound of the sample's two
solves); the tests check each sample against 1000 times that bound at
tol = 1e-12, and estimates within 1e-9 relative.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import estimator as E
from oracle.bilinear import build_bilinear_hierarchy
from oracle.hierarchy import accumulated_prolongation
from oracle.philox import rademacher

DX = [0, 1, -1, 0, 0, 1, -1, 1, -1]
DY = [0, 0, 0, 1, -1, 1, 1, -1, -1]


@pytest.fixture(scope="module")
def mlmc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_11281_gb300 import mlmc as m
    return m


def bil_h(mlmc, N, levels, shift=0.0, **kw):
    prm = mlmc.default_params(levels=levels, transfer=mlmc.TRANSFER_BILINEAR, **kw)
    return mlmc.Hierarchy(mlmc.OP_LAPLACE2D, N, N, prm, shift=shift)


def nine_point_matrix(coef, nx, ny):
    """Sparse matrix of a [site][9] stencil (Dirichlet: taps leaving the grid must be zero)."""
    rows, cols, vals = [], [], []
    for s in range(nx * ny):
        j, i = divmod(s, nx)
        for q in range(9):
            ii, jj = i + DX[q], j + DY[q]
            if 0 <= ii < nx and 0 <= jj < ny:
                rows.append(s)
                cols.append(jj * nx + ii)
                vals.append(coef[s, q])
            else:
                assert coef[s, q] == 0.0
    return sp.csr_matrix((vals, (rows, cols)), shape=(nx * ny, nx * ny))


def close_apply(got, ref, rtol):
    """Operator applies: every entry within rtol of the largest (at most 9 products each)."""
    got, ref = np.asarray(got), np.asarray(ref)
    assert np.abs(got - ref).max() <= rtol * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


def inv_norm(A):
    """||A^-1||_2 of a small symmetric positive definite level operator."""
    return 1.0 / np.linalg.eigvalsh(A.toarray()).min()


def close_per_sample(got, ref, lv, hats, level, seed, first, form, tol=1e-12, margin=1000.0):
    """Every sample within margin x its a-posteriori solve bound (see the module docstring)."""
    got, ref = np.asarray(got), np.asarray(ref)
    n1 = lv[0].n
    inv = {l: inv_norm(lv[l - 1].A) for l in ((1,) if form == "plain" else (level, level + 1))}
    for j in range(len(ref)):
        x = rademacher(n1, seed, level, first + j)
        if form == "plain":
            bound = x @ x * inv[1] * tol
        else:
            z0, z1 = hats[level - 1].T @ x, hats[level].T @ x
            bound = (z0 @ z0 * inv[level] + z1 @ z1 * inv[level + 1]) * tol
        assert abs(got[j] - ref[j]) <= margin * bound, (j, abs(got[j] - ref[j]), bound)


@pytest.mark.parametrize("shift", [0.0, 0.05])
def test_galerkin_levels_and_applies(mlmc, shift):
    N, L = 63, 4
    h = bil_h(mlmc, N, L, shift, block=8)
    lv = build_bilinear_hierarchy(N, L, shift)
    assert h.level_taps(1) == 5
    for l in range(2, L + 1):
        nx, ny, d = h.level_info(l)
        assert (nx, ny, d) == (lv[l - 1].nx, lv[l - 1].ny, 1) and h.level_taps(l) == 9
        Al = nine_point_matrix(h.operator(l)[:, :, 0, 0], nx, ny)
        assert abs(Al - lv[l - 1].A).max() <= 1e-13 * abs(lv[l - 1].A).max()
        # 9-point apply on the device
        x = torch.randn(nx * ny, 5, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        h.apply(l, x.data_ptr(), y.data_ptr(), 5)
        ref = lv[l - 1].A @ x.cpu().numpy()
        close_apply(y.cpu().numpy(), ref, 1e-13)
    assert abs(h.coarse_trace_exact().real - E.exact_coarse_trace(lv, "hat")) <= 1e-10 * abs(
        E.exact_coarse_trace(lv, "hat"))
    h.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solves_reach_exact_solution(mlmc, precision):
    """FGMRES with the V/K-cycle (red-black GS on the 5-point fine level, 4-colour GS
    on the 9-point levels, bilinear transfers, dense coarsest inverse) on levels 1-3."""
    N, L = 127, 4
    prec = mlmc.PREC_FP64 if precision == "fp64" else mlmc.PREC_MIXED_FP32
    tol = 1e-12 if precision == "fp64" else 1e-10
    h = bil_h(mlmc, N, L, block=8, precision=prec, inner_its=(0 if precision == "fp64" else 6))
    lv = build_bilinear_hierarchy(N, L)
    for l in (1, 2, 3):
        n = lv[l - 1].n
        b = np.stack([rademacher(n, 9, l, c) for c in range(8)], axis=1)
        bd = torch.from_numpy(b).cuda()
        xd = torch.zeros_like(bd)
        its = h.solve(l, bd.data_ptr(), xd.data_ptr(), 8, tol)
        x = xd.cpu().numpy()
        res = np.linalg.norm(b - lv[l - 1].A @ x, axis=0) / np.linalg.norm(b, axis=0)
        assert res.max() <= tol and its < 60, (l, res.max(), its)
    h.close()


def test_hat_samples_match_oracle(mlmc):
    N, L = 63, 3
    h = bil_h(mlmc, N, L, block=8)
    lv = build_bilinear_hierarchy(N, L)
    solv = E.LevelSolvers(lv)
    hats = [accumulated_prolongation(lv, l) for l in range(1, L + 1)]
    for level in (1, 2):
        got = h.sample_level_form(level, mlmc.FORM_HAT, mlmc.NOISE_RADEMACHER, 3, 2, 11, 1e-12)
        ref = E.level_samples(lv, solv, level, "rademacher", 3, 2, 11, form="hat", hats=hats)
        close_per_sample(got, ref, lv, hats, level, 3, 2, "hat")
    got = h.sample_level_form(1, mlmc.FORM_PLAIN, mlmc.NOISE_RADEMACHER, 3, 0, 6, 1e-12)
    close_per_sample(got, E.level_samples(lv, solv, 1, "rademacher", 3, 0, 6, form="plain"), lv, hats, 1, 3, 0,
                     "plain")
    # coarse-level blocks wider than the fine block: the hat form draws their noise on the
    # fine level (a block of 16 and a ragged block of 4)
    hw = bil_h(mlmc, N, L, block=4, coarse_block=16)
    got = hw.sample_level_form(2, mlmc.FORM_HAT, mlmc.NOISE_RADEMACHER, 3, 0, 20, 1e-12)
    ref = E.level_samples(lv, solv, 2, "rademacher", 3, 0, 20, form="hat", hats=hats)
    close_per_sample(got, ref, lv, hats, 2, 3, 0, "hat")
    hw.close()
    # the simplified form needs R P = I: rejected; P is applied, not stored
    with pytest.raises(mlmc.MLMCError) as ei:
        h.sample_level(1, mlmc.NOISE_RADEMACHER, 0, 0, 4, 1e-10)
    assert ei.value.status == mlmc.ERR_INVALID_ARG
    with pytest.raises(mlmc.MLMCError) as ei:
        h.prolongation(1)
    assert ei.value.status == mlmc.ERR_UNSUPPORTED
    h.close()


def test_hat_estimate_matches_oracle(mlmc):
    """Sec. 5 procedure in the hat form: same N_l, tau and estimate as the oracle."""
    N, L = 63, 3
    h = bil_h(mlmc, N, L, block=16)
    lv = build_bilinear_hierarchy(N, L)
    r = mlmc.result_dict(h.trace_estimate(eps=3e-2, noise=mlmc.NOISE_RADEMACHER, seed=5, tol=1e-12,
                                          form=mlmc.FORM_HAT))
    ref = E.trace_estimate(lv, "rademacher", seed=5, eps=3e-2, block=16, form="hat")
    assert r["n_samples"] == ref.n_samples
    assert abs(r["tau"] - ref.tau) <= 1e-9 * abs(ref.tau)
    assert abs(r["trace"] - ref.trace) <= 1e-9 * abs(ref.trace)
    assert abs(r["coarse_term"] - ref.coarse_term) <= 1e-10 * abs(ref.coarse_term)
    h.close()


def test_paper_size_estimate_against_closed_form(mlmc):
    """N = 511 with N_L = 15 (L = 6, as in Table 1), mixed form, optimal allocation:
    the estimate lies within 4 standard errors of the Example 5.1 closed form."""
    N, L = 511, 6
    h = bil_h(mlmc, N, L, block=32, coarse_block=64, precision=mlmc.PREC_MIXED_FP32, inner_its=8,
              fgmres_restart=8, smooth_pre=1, smooth_post=1)
    r = mlmc.result_dict(h.trace_estimate(eps=1e-2, noise=mlmc.NOISE_RADEMACHER, seed=0, tol=1e-8,
                                          form=mlmc.FORM_HAT, allocation=mlmc.ALLOC_OPTIMAL))
    c = 2 * np.cos(np.arange(1, N + 1) * np.pi / (N + 1))
    exact = float(np.sum(1.0 / (4.0 - c[:, None] - c[None, :])))
    assert r["std_err"] <= 1e-2 * abs(r["tau"]) * (1 + 1e-12)
    assert abs(r["trace"].real - exact) <= 4 * r["std_err"]
    assert len(r["n_samples"]) == L - 1
    h.close()
