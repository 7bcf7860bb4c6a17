"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names the passage it checks.  None of these compares the oracle
with itself: values come from closed forms, an independent generator
(numpy.random.Philox), exhaustive enumeration, dense linear algebra or the
table sizes printed in the paper.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import estimator as E
from oracle.hierarchy import SetupParams, build_hierarchy, accumulated_prolongation
from oracle.operators import laplace2d, wilson2d, spin_parity
from oracle.philox import philox4x64_10, rademacher, z4, noise_key, PURPOSE_NOISE
from oracle.solver import Cycle, fgmres, exact_solver, dense_inverse
from paper_2108_11281_gb300.workloads import gauge_links, pure_gauge_links


# ---------------------------------------------------------------- Philox / noise
def test_philox_matches_numpy_generator():
    """Philox4x64-10 (Salmon et al. 2011) vs numpy's independent implementation.
    numpy pre-increments its counter, so its first block is counter c+1."""
    rng = np.random.default_rng(5)
    for _ in range(5):
        key = rng.integers(0, 2**63, size=2, dtype=np.uint64)
        c0 = int(rng.integers(0, 2**40))
        ref = np.random.Philox(key=key, counter=np.array([c0, 7, 0, 0], dtype=np.uint64)).random_raw(4)
        ours = philox4x64_10(np.array([[c0 + 1], [7], [0], [0]], dtype=np.uint64), (key[0], key[1]))
        assert np.array_equal(ours[:, 0], ref)


def test_noise_bit_mapping_against_numpy_words():
    """Rademacher row 256b + 64q + bit uses bit `bit` of word q; Z4 uses 2 bits per row."""
    seed, level, sample = 11, 3, 42
    k0, k1 = noise_key(seed, level, PURPOSE_NOISE)
    x = rademacher(600, seed, level, sample)
    zc = z4(300, seed, level, sample)
    for blk in range(3):
        words = np.random.Philox(key=np.array([k0, k1], dtype=np.uint64),
                                 counter=np.array([blk - 1, sample, 0, 0] if blk else
                                                  [2**64 - 1, sample - 1, 0, 0],   # carry into word 1
                                                  dtype=np.uint64)).random_raw(4)
        for row in range(256 * blk, min(256 * (blk + 1), 600)):
            q, b = divmod(row - 256 * blk, 64)
            bit = (int(words[q]) >> b) & 1
            assert x[row] == (1.0 if bit == 0 else -1.0)
        for row in range(128 * blk, min(128 * (blk + 1), 300)):
            q, b = divmod(row - 128 * blk, 32)
            v = (int(words[q]) >> (2 * b)) & 3
            assert zc[row] == [1, 1j, -1, -1j][v]


def test_noise_moments():
    """Eq. P_assumptions: E[x_i] = 0, E[conj(x_i) x_j] = delta_ij (statistical, 4 sigma)."""
    X = np.stack([rademacher(64, 1, 1, j) for j in range(4000)])
    assert abs(X.mean()) < 4 / np.sqrt(X.size)
    C = X.T @ X / len(X)
    assert np.allclose(np.diag(C), 1.0)
    assert np.abs(C - np.eye(64)).max() < 5 / np.sqrt(len(X))
    Z = np.stack([z4(64, 1, 1, j) for j in range(4000)])
    assert np.allclose(np.abs(Z), 1.0)
    assert abs(Z.mean()) < 4 / np.sqrt(Z.size)
    assert abs((Z ** 2).mean()) < 4 / np.sqrt(Z.size)          # E[x^2] = 0 for Z4 (Cor. 3.2)


# ---------------------------------------------------------------- operators
def laplace_trace_inverse_closed_form(N, shift=0.0):
    """Example 5.1: eigenvalues 4 - 2cos(i pi/(N+1)) - 2cos(j pi/(N+1)) (+ shift)."""
    c = 2 * np.cos(np.arange(1, N + 1) * np.pi / (N + 1))
    return float(np.sum(1.0 / (4.0 + shift - c[:, None] - c[None, :])))


@pytest.mark.parametrize("N,shift", [(7, 0.0), (16, 0.0), (12, 0.05)])
def test_laplace_closed_form_trace(N, shift):
    A = laplace2d(N, N, shift)
    assert np.isclose(np.trace(np.linalg.inv(A.toarray())), laplace_trace_inverse_closed_form(N, shift),
                      rtol=1e-12)
    assert A.nnz == 5 * N * N - 4 * N                 # Table 1 nnz rule (1.96e4 for N = 63)


def test_laplace_table1_nnz():
    assert laplace2d(63, 63).nnz == 19593            # printed 1.96e4
    assert laplace2d(127, 127).nnz == 80137          # printed 8.01e4


def free_wilson_trace(N, m):
    """Eq. schwinger_coupling with U = 1 in momentum space: M(k) = a I + 2i(sin kx s1 + sin ky s2),
    a = 4 + m - 2cos kx - 2cos ky; s1, s2 anticommute and square to I, so
    tr M(k)^{-1} = 2a / (a^2 + 4 sin^2 kx + 4 sin^2 ky)."""
    k = 2 * np.pi * np.arange(N) / N
    kx, ky = k[None, :], k[:, None]
    a = 4 + m - 2 * np.cos(kx) - 2 * np.cos(ky)
    return float(np.sum(2 * a / (a ** 2 + 4 * np.sin(kx) ** 2 + 4 * np.sin(ky) ** 2)))


def test_wilson_free_field_closed_form():
    N, m = 8, 0.3
    S = wilson2d(N, N, m, np.ones((2, N, N), dtype=complex)).toarray()
    assert np.isclose(np.trace(np.linalg.inv(S)), free_wilson_trace(N, m), rtol=1e-12)


def test_wilson_gauge_covariance():
    """Pure-gauge links U_mu(x) = g(x) conj(g(x+mu)) give S' = G S_free G^*."""
    N, m = 6, 0.2
    U, g = pure_gauge_links(N, N, 3)
    S = wilson2d(N, N, m, U).toarray()
    S0 = wilson2d(N, N, m, np.ones((2, N, N), dtype=complex)).toarray()
    G = np.diag(np.repeat(g.reshape(-1), 2))
    assert np.allclose(S, G @ S0 @ G.conj().T, atol=1e-14)
    assert np.isclose(np.trace(np.linalg.inv(S)), free_wilson_trace(N, m), rtol=1e-11)


def test_wilson_table3_nnz_and_symmetry():
    """Table 3: nnz(S_1) = 2.94e5 at N = 128; Sec. 5: J S = S^* J."""
    N = 128
    S = wilson2d(N, N, -0.1, gauge_links(N, N, 0.3, 0))
    assert S.shape == (2 * N * N, 2 * N * N)
    assert S.nnz == 9 * 2 * N * N == 294912
    small = wilson2d(8, 8, -0.1, gauge_links(8, 8, 0.3, 0)).toarray()
    J = spin_parity(64, 2)
    assert np.allclose(J[:, None] * small, small.conj().T * J[None, :], atol=1e-15)


# ---------------------------------------------------------------- hierarchy
def wilson_hierarchy(N=16, levels=3, n_tv=(2, 4), agg=4):
    U = gauge_links(N, N, 0.3, 7)
    S = wilson2d(N, N, -0.05, U)
    prm = SetupParams(levels=levels, agg_x=agg, agg_y=agg, n_tv=list(n_tv), spin_split=True,
                      kind="inverse", sweeps=6,
                      coarse_sweeps=4, omega=1.0, noise_kind="z4", bootstrap=1)
    return S, build_hierarchy(S, N, N, 2, prm)


def test_hierarchy_orthonormal_galerkin_and_spin_structure():
    """Sec. 4.1 (A_{l+1} = R A P, R = P^*), Remark 4.3 (R P = I), Example 5.3 (J-symmetry kept)."""
    S, h = wilson_hierarchy()
    rng = np.random.default_rng(0)
    for lv, nxt in zip(h[:-1], h[1:]):
        P = lv.P
        assert np.abs((P.conj().T @ P).toarray() - np.eye(P.shape[1])).max() < 1e-13
        v = rng.normal(size=P.shape[1]) + 1j * rng.normal(size=P.shape[1])
        assert np.allclose(nxt.A @ v, P.conj().T @ (lv.A @ (P @ v)), atol=1e-12)
    for lv in h:
        J = spin_parity(lv.nx * lv.ny, lv.d)
        Ad = lv.A.toarray()
        assert np.abs(J[:, None] * Ad - Ad.conj().T * J[None, :]).max() < 1e-12
    # the exact coarse trace is real because of the J-symmetry
    assert abs(E.exact_coarse_trace(h).imag) < 1e-10 * abs(E.exact_coarse_trace(h))


def test_table3_level_sizes():
    """Table 3: n_l = 2*128^2, 4*32^2, 8*8^2, 8*2^2 with 4x4 aggregates, 2 then 4 test vectors,
    doubled by the spin split."""
    N = 128
    U = gauge_links(N, N, 0.3, 0)
    S = wilson2d(N, N, -0.1, U)
    prm = SetupParams(levels=4, n_tv=[2, 4, 4], spin_split=True, kind="inverse", sweeps=1,
                      coarse_sweeps=1, omega=1.0, noise_kind="z4", bootstrap=0)
    h = build_hierarchy(S, N, N, 2, prm)
    assert [lv.n for lv in h] == [2 * 128 ** 2, 4 * 32 ** 2, 8 * 8 ** 2, 8 * 2 ** 2]


def test_piecewise_constant_prolongation_entries():
    A = laplace2d(16, 16)
    h = build_hierarchy(A, 16, 16, 1, SetupParams(levels=2, n_tv=1, kind="constant"))
    assert np.allclose(np.abs(h[0].P.data), 0.25) and h[0].P.nnz == 256
    # Galerkin operator of the constant aggregation is exact in binary: (1/16) * integer sums
    assert np.array_equal(h[1].A.toarray() * 16, np.round(h[1].A.toarray() * 16))


# ---------------------------------------------------------------- telescoping and Hutchinson
def dense_level_traces(h):
    """tr(A_l^{-1}) and tr(P_l A_{l+1}^{-1} R_l) for every level from dense inverses."""
    inv = [np.linalg.inv(lv.A.toarray()) for lv in h]
    diffs = [np.trace(inv[i]) - np.trace(h[i].P.toarray() @ inv[i + 1] @ h[i].P.toarray().conj().T)
             for i in range(len(h) - 1)]
    return inv, diffs


def test_telescoping_identity_simplified_and_hat():
    """Eq. tr_ml_dec and Remark 4.3: the level differences plus the coarsest term give tr(A^{-1})."""
    S, h = wilson_hierarchy(N=8, levels=3, n_tv=(2, 2), agg=2)
    inv, diffs = dense_level_traces(h)
    total = np.trace(inv[0])
    assert np.isclose(sum(diffs) + np.trace(inv[-1]), total, rtol=1e-12)
    L = len(h)
    hats = [accumulated_prolongation(h, l).toarray() for l in range(1, L + 1)]
    hat_diffs = [np.trace(hats[i] @ inv[i] @ hats[i].conj().T) -
                 np.trace(hats[i + 1] @ inv[i + 1] @ hats[i + 1].conj().T) for i in range(L - 1)]
    assert np.isclose(sum(hat_diffs) + E.exact_coarse_trace(h, "hat"), total, rtol=1e-12)
    assert np.isclose(E.exact_coarse_trace(h, "hat"), E.exact_coarse_trace(h), rtol=1e-12)


def _enumerate_level_samples(h, kind, n):
    solv = E.LevelSolvers(h)
    if kind == "rademacher":
        vecs = itertools.product([1.0, -1.0], repeat=n)
    else:
        vecs = itertools.product([1, 1j, -1, -1j], repeat=n)
    return np.array([E.sample(h, solv, 1, np.array(v, dtype=complex)) for v in vecs])


def test_hutchinson_unbiased_and_variance_real_noise():
    """Thm. 3.1 and Cor. 3.2 by enumerating all 2^n sign vectors: the mean of the
    level-1 samples is tr(B), B = A_1^{-1} - P A_2^{-1} R, and their variance is
    (1/2) ||offdiag(B + B^T)||_F^2."""
    A = laplace2d(4, 2, 0.3)
    h = build_hierarchy(A, 4, 2, 1, SetupParams(levels=2, agg_x=2, agg_y=2, n_tv=1, kind="constant"))
    s = _enumerate_level_samples(h, "rademacher", 8)
    B = np.linalg.inv(A.toarray()) - h[0].P.toarray() @ np.linalg.inv(h[1].A.toarray()) @ h[0].P.toarray().T
    assert np.isclose(s.mean(), np.trace(B), rtol=1e-12)
    off = B + B.T
    np.fill_diagonal(off, 0)
    assert np.isclose(np.mean(np.abs(s - s.mean()) ** 2), 0.5 * np.sum(off ** 2), rtol=1e-10)


def test_hutchinson_unbiased_and_variance_z4_noise():
    """Same for Z4 noise on a complex Wilson level: variance ||offdiag(B)||_F^2 (Cor. 3.2)."""
    U = gauge_links(2, 2, 0.5, 4)
    S = wilson2d(2, 2, 0.4, U)
    h = build_hierarchy(S, 2, 2, 2, SetupParams(levels=2, agg_x=2, agg_y=2, n_tv=1, spin_split=True,
                                                kind="inverse", sweeps=2, omega=1.0,
                                                noise_kind="z4", bootstrap=0))
    s = _enumerate_level_samples(h, "z4", 8)
    P = h[0].P.toarray()
    B = np.linalg.inv(S.toarray()) - P @ np.linalg.inv(h[1].A.toarray()) @ P.conj().T
    assert np.isclose(s.mean(), np.trace(B), rtol=1e-12)
    off = B.copy()
    np.fill_diagonal(off, 0)
    assert np.isclose(np.mean(np.abs(s - s.mean()) ** 2), np.sum(np.abs(off) ** 2), rtol=1e-10)


# ---------------------------------------------------------------- solver and estimator
@pytest.mark.parametrize("cycle", ["V", "K"])
def test_fgmres_multigrid_reaches_exact_solve(cycle):
    A = laplace2d(64, 64)
    h = build_hierarchy(A, 64, 64, 1, SetupParams(levels=3, n_tv=4, sweeps=20, coarse_sweeps=10))
    M = Cycle(h, 0, 1, 1, cycle, 2)
    b = rademacher(A.shape[0], 0, 1, 0)
    x, its, res = fgmres(A, b, M, tol=1e-11, m=30)
    assert res <= 1e-11
    ref = exact_solver(A)(b)
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)


def test_wilson_fgmres_multigrid():
    S, h = wilson_hierarchy(N=16, levels=3, n_tv=(4, 4))
    M = Cycle(h, 0, 2, 2, "K", 2)
    b = z4(S.shape[0], 0, 1, 0)
    x, its, res = fgmres(S, b, M, tol=1e-10, m=30)
    assert res <= 1e-10
    assert np.allclose(x, exact_solver(S)(b), rtol=0, atol=1e-7 * np.abs(x).max())


def test_small_laplace_estimate_against_closed_form():
    """64x64 Laplacian, 2 levels, piecewise-constant P: the MLMC estimate is within
    4 standard errors of the closed-form trace, and the exact coarse term equals the
    dense tr(A_2^{-1})."""
    N = 64
    A = laplace2d(N, N)
    h = build_hierarchy(A, N, N, 1, SetupParams(levels=2, n_tv=1, kind="constant"))
    res = E.trace_estimate(h, "rademacher", seed=0, eps=1e-2, block=64)
    exact = laplace_trace_inverse_closed_form(N)
    assert abs(res.trace.real - exact) <= 4 * res.std_err
    assert np.isclose(res.coarse_term, np.trace(np.linalg.inv(h[1].A.toarray())), rtol=1e-12)
    assert all(n >= 5 for n in res.n_samples)


def test_optimal_allocation_minimises_cost():
    """Sec. 2: the counts minimise sum N_l C_l subject to sum V_l / N_l = eps^2, checked
    against a numerical constrained minimisation (scipy SLSQP, from several starts), the
    constraint itself, and the minimal cost eps^-2 (sum sqrt(V_l C_l))^2 printed there."""
    from scipy.optimize import minimize
    rng = np.random.default_rng(3)
    for _ in range(5):
        L = int(rng.integers(2, 5))
        V = rng.uniform(0.1, 50.0, L)
        C = rng.uniform(1.0, 100.0, L)
        eps = rng.uniform(0.05, 0.5)
        N, counts, w = E.optimal_allocation(V, C, eps, min_samples=1)
        assert abs(np.sum(V / N) - eps ** 2) <= 1e-12 * eps ** 2
        assert abs(np.dot(N, C) - np.sum(np.sqrt(V * C)) ** 2 / eps ** 2) <= 1e-10 * np.dot(N, C)
        assert abs(w.sum() - 1.0) <= 1e-14 and np.allclose(V / N, w * eps ** 2, rtol=1e-12)
        assert counts == [max(1, int(np.ceil(n))) for n in N]
        best = None
        for start in (np.full(L, 10.0), rng.uniform(1.0, 1e3, L)):
            res = minimize(lambda n: np.dot(n, C) / np.dot(N, C), start * N.mean() / start.mean(),
                           constraints=[{"type": "eq", "fun": lambda n: np.sum(V / n) / eps ** 2 - 1.0}],
                           bounds=[(1e-6, None)] * L, method="SLSQP", options={"ftol": 1e-14, "maxiter": 500})
            if res.success and (best is None or res.fun < best.fun):
                best = res
        assert best is not None
        assert np.allclose(best.x, N, rtol=1e-4)
        assert best.fun >= 1.0 - 1e-9          # nothing feasible is cheaper than the closed form


def test_stopping_rule_closed_form(monkeypatch):
    """Sec. 5 stopping rule on synthetic samples with a closed form.  Level l draws
    s_i = mu_l + sigma_l (-1)^i (sample index i), the coarse term is T_L.  Then the five
    full estimates are m + S (-1)^i with m = T_L + sum mu_l, S = sum sigma_l, so
    tau = m + S/5 - sqrt(0.96) S (population deviation of +,-,+,-,+).  For an even count n
    the unbiased variance is n sigma^2 / (n - 1), so level l stops at the first multiple of
    the block (and >= 5) with sigma_l^2 / (n - 1) <= rho_l^2, rho_l = sqrt(w_l) eps tau, and
    the estimate is exactly m."""
    mu, sigma, TL = [10.0, 5.0], [3.0, 1.0], 100.0

    def fake_samples(levels, solvers, l, kind, seed, first, count, form="simplified", purpose=0, hats=None):
        i = np.arange(first, first + count)
        return mu[l - 1] + sigma[l - 1] * (-1.0) ** i + 0j

    monkeypatch.setattr(E, "level_samples", fake_samples)
    monkeypatch.setattr(E, "exact_coarse_trace", lambda levels, form="simplified": TL)
    eps, block = 0.01, 8
    for weights in (None, [0.8, 0.2]):
        r = E.trace_estimate([None, None, None], "rademacher", eps=eps, weights=weights, block=block,
                             solvers=object())
        m, S = TL + sum(mu), sum(sigma)
        tau = m + S / 5 - np.sqrt(0.96) * S
        assert abs(r.tau - tau) <= 1e-12 * tau
        w = [0.5, 0.5] if weights is None else weights
        for l in range(2):
            rho2 = w[l] * (eps * tau) ** 2
            n = block
            while not (n >= 5 and sigma[l] ** 2 / (n - 1) <= rho2):
                n += block
            assert r.n_samples[l] == n
            assert abs(r.variances[l] - n * sigma[l] ** 2 / (n - 1)) <= 1e-12 * sigma[l] ** 2
        assert abs(r.trace - m) <= 1e-12 * m
        se = np.sqrt(sum(sigma[l] ** 2 / (r.n_samples[l] - 1) for l in range(2)))
        assert abs(r.std_err - se) <= 1e-12 * se


def test_tau_from_separate_warmup_samples(monkeypatch):
    """Sec. 5 with tau from separate samples: the five full estimates use the warm-up
    stream (level l: s_i = 2 mu_l + 3 sigma_l (-1)^i there), the level means only the noise
    stream (s_i = mu_l + sigma_l (-1)^i), so tau = m' + S'/5 - sqrt(0.96) S' with
    m' = T_L + 2 sum mu_l, S' = 3 sum sigma_l, and the estimate is still exactly m."""
    from oracle.philox import PURPOSE_WARMUP
    mu, sigma, TL = [10.0, 5.0], [3.0, 1.0], 100.0

    def fake_samples(levels, solvers, l, kind, seed, first, count, form="simplified", purpose=0, hats=None):
        i = np.arange(first, first + count)
        if purpose == PURPOSE_WARMUP:
            return 2 * mu[l - 1] + 3 * sigma[l - 1] * (-1.0) ** i + 0j
        return mu[l - 1] + sigma[l - 1] * (-1.0) ** i + 0j

    monkeypatch.setattr(E, "level_samples", fake_samples)
    monkeypatch.setattr(E, "exact_coarse_trace", lambda levels, form="simplified": TL)
    m2, S2 = TL + 2 * sum(mu), 3 * sum(sigma)
    tau = m2 + S2 / 5 - np.sqrt(0.96) * S2
    for run in (lambda: E.trace_estimate([None] * 3, "rademacher", eps=0.01, block=8, solvers=object(),
                                         tau_separate=True),
                lambda: E.optimal_trace_estimate([None] * 3, "rademacher", eps=0.01, widths=8, costs=[10.0, 1.0],
                                                 solvers=object(), tau_separate=True)):
        r = run()
        assert abs(r.tau - tau) <= 1e-12 * tau
        assert abs(r.trace - (TL + sum(mu))) <= 1e-12 * (TL + sum(mu))


def test_nominal_sample_cost_hand_counts():
    """Sec. 5 cost model (a product B x costs nnz(B)) of one sample, counted by hand.
    64^2 Dirichlet Laplacian, 2 levels, piecewise-constant P: nnz(A_1) = 5*4096 - 4*64
    (Example 5.1), n_2 = 256 so the coarsest dense inverse has 256^2 entries, and P_1
    has one entry per fine row.  32^2 with 4 test vectors and 3 levels: level 2 is 8^2
    sites of 4 dofs with full 4 x 4 blocks for each of the 5*64 - 4*8 coupled site
    pairs, P_1 has 4 entries per fine row, P_2 4 per level-2 row, n_3 = 2*2*4 = 16."""
    lv = build_hierarchy(laplace2d(64, 64), 64, 64, 1, SetupParams(levels=2, n_tv=1, kind="constant"))
    assert E.nominal_sample_cost(lv, 1) == 20224 + 65536 + 4096
    assert E.nominal_sample_cost(lv, 1, "plain") == 20224
    lv = build_hierarchy(laplace2d(32, 32), 32, 32, 1, SetupParams(levels=3, n_tv=4, sweeps=5, coarse_sweeps=3,
                                                                     bootstrap=0))
    a1, a2, p1, p2 = 5 * 1024 - 4 * 32, 16 * (5 * 64 - 4 * 8), 1024 * 4, 256 * 4
    assert E.nominal_sample_cost(lv, 1) == a1 + a2 + p1
    assert E.nominal_sample_cost(lv, 2) == a2 + 16 ** 2 + p2
    assert E.nominal_sample_cost(lv, 2, "hat") == a2 + 16 ** 2 + p1 + p2


def _constant_variance_stream(mu, V, width):
    """Samples of one level difference whose unbiased variance is exactly V after every
    whole block of `width` (even) samples and whose mean is exactly mu: within block m
    the values are mu + a_m (-1)^j, a_0 = sqrt(V (width - 1) / width), a_m = sqrt(V) after
    (each block has mean mu, so the sums of squared deviations add: V (width - 1) for
    the first block, V width for every further one)."""
    a0 = np.sqrt(V * (width - 1) / width)

    def values(first, count):
        i = np.arange(first, first + count)
        a = np.where(i < width, a0, np.sqrt(V))
        return mu + a * (-1.0) ** (i % width) + 0j
    return values, a0


def test_optimal_allocation_loop_closed_form(monkeypatch):
    """Sec. 2 optimal allocation, run adaptively, on sample streams with constant variances
    V_l and fixed per-sample costs C_l.  The five full estimates are m + A (-1)^i with
    m = T_L + sum mu_l and A = sum a_0,l, so tau = m + A/5 - sqrt(0.96) A (Sec. 5).  The
    optimum of Sec. 2 for the target T = eps tau is N_l* = sqrt(V_l / C_l) S / T^2 with
    S = sum_j sqrt(V_j C_j); whole blocks are drawn until N_l >= max(5, ceil(N_l*)), at
    which point sum V_l / N_l <= T^2 holds, so each level ends at the first block multiple
    at or above that count; the estimate is exactly m and the weights are
    sqrt(V_l C_l) / S.  A multiplier read as printed (sqrt(V_j / C_j) in S), V and C
    swapped, or a wrong tau changes the counts."""
    TL = 50.0
    for mu, V, C, widths, eps in [([10.0, 5.0], [400.0, 90.0], [1000.0, 30.0], [8, 16], 0.02),
                                  ([3.0, 2.0, 1.0], [90.0, 60.0, 40.0], [5000.0, 400.0, 20.0], [6, 8, 16], 0.03)]:
        streams = [_constant_variance_stream(m_, v, w) for m_, v, w in zip(mu, V, widths)]

        def fake_samples(levels, solvers, l, kind, seed, first, count, form="simplified", purpose=0, hats=None):
            return streams[l - 1][0](first, count)

        monkeypatch.setattr(E, "level_samples", fake_samples)
        monkeypatch.setattr(E, "exact_coarse_trace", lambda levels, form="simplified": TL)
        r = E.optimal_trace_estimate([None] * (len(mu) + 1), "rademacher", eps=eps, widths=widths, costs=C,
                                     solvers=object())
        m, A = TL + sum(mu), sum(a0 for _, a0 in streams)
        tau = m + A / 5 - np.sqrt(0.96) * A
        assert abs(r.tau - tau) <= 1e-12 * tau
        T2 = (eps * tau) ** 2
        S = sum(np.sqrt(v * c) for v, c in zip(V, C))
        for l in range(len(mu)):
            need = max(5, int(np.ceil(np.sqrt(V[l] / C[l]) * S / T2)))
            want = widths[l] * max(1, -(-need // widths[l]))
            assert r.n_samples[l] == want
            assert abs(r.variances[l] - V[l]) <= 1e-9 * V[l]
            assert abs(r.weights[l] - np.sqrt(V[l] * C[l]) / S) <= 1e-12
        assert abs(r.trace - m) <= 1e-12 * m
        assert r.std_err ** 2 <= T2 * (1 + 1e-12)
        assert any(n > w for n, w in zip(r.n_samples, widths))      # the loop did draw beyond the pilot


def test_optimal_allocation_loop_one_level_reestimates(monkeypatch):
    """One level difference with s_i = mu + sigma (-1)^i: after an even count N the unbiased
    variance is N sigma^2 / (N - 1), so V changes as samples arrive.  With one level Sec. 2
    gives N* = V / T^2 (S = sqrt(V C)), independent of C; the loop stops at the first
    block multiple N with N >= ceil(N sigma^2 / ((N - 1) T^2))."""
    mu, sigma, TL, block, eps = 4.0, 2.0, 30.0, 8, 0.01

    def fake_samples(levels, solvers, l, kind, seed, first, count, form="simplified", purpose=0, hats=None):
        i = np.arange(first, first + count)
        return mu + sigma * (-1.0) ** i + 0j

    monkeypatch.setattr(E, "level_samples", fake_samples)
    monkeypatch.setattr(E, "exact_coarse_trace", lambda levels, form="simplified": TL)
    for C in (1.0, 1e6):
        r = E.optimal_trace_estimate([None, None], "rademacher", eps=eps, widths=block, costs=[C], solvers=object())
        tau = (TL + mu) + sigma / 5 - np.sqrt(0.96) * sigma
        T2 = (eps * tau) ** 2
        n = block
        while n < np.ceil(n * sigma ** 2 / ((n - 1) * T2)):
            n += block
        assert r.n_samples == [n]
        assert abs(r.trace - (TL + mu)) <= 1e-12 * (TL + mu)


# ---------------------------------------------------------------- learned correction (no paper basis)
@pytest.mark.parametrize("case", ["wilson", "laplace"])
def test_learned_gradient_matches_finite_differences(case):
    """The network's loss gradient (oracle/learned.py) against central differences in FP64."""
    from oracle import learned as NN
    rng = np.random.default_rng(3)
    if case == "wilson":
        A = wilson2d(4, 4, 0.2, gauge_links(4, 4, 0.3, 1))
        d, cplx, per, n = 2, True, True, 32
        R = rng.normal(size=(n, 2)) + 1j * rng.normal(size=(n, 2))
    else:
        A = laplace2d(4, 4)
        d, cplx, per, n = 1, False, False, 16
        R = rng.normal(size=(n, 2))
    Ws = NN.init_weights(NN.channels_of(d, cplx), 5)
    _, G = NN.loss_and_grad(A, R, Ws, 4, 4, d, cplx, per)
    h = 1e-6
    for li, idx in [(0, (1, 0, 2, 1)), (1, (5, 7, 1, 1)), (2, (0, 3, 0, 2))]:
        Wp = [W.copy() for W in Ws]
        Wm = [W.copy() for W in Ws]
        Wp[li][idx] += h
        Wm[li][idx] -= h
        fd = (NN.loss_and_grad(A, R, Wp, 4, 4, d, cplx, per)[0] - NN.loss_and_grad(A, R, Wm, 4, 4, d, cplx, per)[0]) / (2 * h)
        assert abs(fd - G[li][idx]) <= 1e-6 * max(abs(fd), 1e-3)


def test_learned_linear_special_case():
    """With every pre-activation positive the network is the linear map W3*W2*W1: a
    single-tap identity chain must reproduce its input exactly (net(r) = r)."""
    from oracle import learned as NN
    c0 = 4
    W1 = np.zeros((16, c0, 3, 3)); W2 = np.zeros((16, 16, 3, 3)); W3 = np.zeros((c0, 16, 3, 3))
    for c in range(c0):
        W1[c, c, 1, 1] = 1.0
        W1[c + c0, c, 1, 1] = -1.0          # ReLU(x) - ReLU(-x) = x
        W2[c, c, 1, 1] = 1.0
        W2[c + c0, c + c0, 1, 1] = 1.0
        W3[c, c, 1, 1] = 1.0
        W3[c, c + c0, 1, 1] = -1.0
    rng = np.random.default_rng(1)
    r = rng.normal(size=32) + 1j * rng.normal(size=32)
    e, _ = NN.forward(r, [W1, W2, W3], 4, 4, 2, True, True)
    assert np.allclose(e, r, atol=1e-15)


def test_plain_hutchinson_sample_is_unbiased():
    """Eq. plain_tr_estimate: the mean of x^T A^{-1} x over all 2^n sign vectors is tr(A^{-1})."""
    A = laplace2d(4, 2, 0.2)
    h = build_hierarchy(A, 4, 2, 1, SetupParams(levels=2, agg_x=2, agg_y=2, n_tv=1, kind="constant"))
    solv = E.LevelSolvers(h)
    vals = [E.sample(h, solv, 1, np.array(v), form="plain") for v in itertools.product([1.0, -1.0], repeat=8)]
    assert np.isclose(np.mean(vals), np.trace(np.linalg.inv(A.toarray())), rtol=1e-12)


# ---------------------------------------------------------------- the paper's bilinear Laplace hierarchy

def _table1_rows():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_laplace_hierarchy.txt")
    rows = []
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            rows.append((int(line[0]), int(line[1]), int(line[2]), float(line[3])))
    return rows


def test_bilinear_hierarchy_table1_sizes_and_nnz():
    """Table 1: n_l and nnz(L^N_l) of the Example 5.1 hierarchy (bilinear P, Galerkin,
    N_{l+1} = floor(N_l/2), N_L = 15) for N = 63, 127, 255, 511."""
    from oracle.bilinear import build_bilinear_hierarchy
    rows = _table1_rows()
    for N in sorted({r[0] for r in rows}):
        mine = [r for r in rows if r[0] == N]
        lv = build_bilinear_hierarchy(N, len(mine))
        for (_, l, n_l, nnz_printed), L in zip(mine, lv):
            assert L.n == n_l
            assert float("%.2e" % L.A.nnz) == nnz_printed, (N, l, L.A.nnz)


def _tri(n, off, diag):
    return sp.diags([off * np.ones(n - 1), diag * np.ones(n), off * np.ones(n - 1)], [-1, 0, 1])


@pytest.mark.parametrize("shift", [0.0, 0.05])
def test_bilinear_galerkin_operators_closed_form(shift):
    """Galerkin coarse operators of Example 5.1 under bilinear P, derived by hand:
    A_1 = T (x) I + I (x) T (+ s I (x) I) with T = tridiag(-1, 2, -1); P = p (x) p, so
    A_l = T_l (x) M_l + M_l (x) T_l + s M_l (x) M_l with T_{l+1} = p^T T_l p = T_l / 2
    (at every size, also next to the Dirichlet edge) and M_{l+1} = p^T M_l p, where
    p^T tridiag(a, b) p = tridiag(b/4 + a, 3b/2 + 2a); M_1 = I."""
    from oracle.bilinear import build_bilinear_hierarchy
    lv = build_bilinear_hierarchy(63, 4, shift)
    t_scale, (a, b) = 1.0, (0.0, 1.0)
    for L in lv:
        n = L.nx
        T = t_scale * _tri(n, -1.0, 2.0)
        M = _tri(n, a, b)
        ref = sp.kron(T, M) + sp.kron(M, T) + shift * sp.kron(M, M)
        assert abs(L.A - ref).max() <= 1e-13
        t_scale, (a, b) = t_scale / 2.0, (b / 4.0 + a, 1.5 * b + 2.0 * a)
    # interior 9-point stencil of level 2 (shift 0): [-1/4 -1/2 -1/4; -1/2 3 -1/2; -1/4 -1/2 -1/4]
    A2 = build_bilinear_hierarchy(15, 2)[1].A.toarray()
    c = 3 * 7 + 3
    assert np.allclose([A2[c, c], A2[c, c + 1], A2[c, c + 7], A2[c, c + 8], A2[c, c - 6]],
                       [3.0, -0.5, -0.5, -0.25, -0.25], atol=1e-15)


def test_bilinear_four_colour_gauss_seidel_is_well_defined():
    """9-point stencils couple diagonal neighbours: the 4-colour order (i mod 2, j mod 2)
    leaves no coupling inside a colour (so each partial sweep solves its rows exactly),
    while red-black would not; and R P != I, so the simplified form does not apply."""
    from oracle.bilinear import build_bilinear_hierarchy
    from oracle.solver import site_colour
    lv = build_bilinear_hierarchy(31, 3)
    for L in lv[1:]:
        r, c = L.A.nonzero()
        off = r != c
        col4 = site_colour(L.nx, L.ny, 1, 4)
        col2 = site_colour(L.nx, L.ny, 1, 2)
        assert np.all(col4[r[off]] != col4[c[off]])
        assert np.any(col2[r[off]] == col2[c[off]])
    RP = (lv[0].P.T @ lv[0].P).toarray()
    assert np.abs(RP - np.eye(RP.shape[0])).max() > 0.1


def test_bilinear_hat_telescoping_against_closed_form():
    """Eq. tr_ml_dec with the exact term of Remark 4.2, tr(A_L^{-1} R^_L P^_L): the hat-form
    level differences plus that term equal the closed-form tr(A^{-1}) of Example 5.1."""
    from oracle.bilinear import build_bilinear_hierarchy
    N = 31
    lv = build_bilinear_hierarchy(N, 3)
    hats = [accumulated_prolongation(lv, l).toarray() for l in range(1, 4)]
    inv = [np.linalg.inv(L.A.toarray()) for L in lv]
    diffs = [np.trace(hats[i] @ inv[i] @ hats[i].T) - np.trace(hats[i + 1] @ inv[i + 1] @ hats[i + 1].T)
             for i in range(2)]
    exact = E.exact_coarse_trace(lv, "hat")
    assert np.isclose(sum(diffs) + exact, laplace_trace_inverse_closed_form(N, 0.0), rtol=1e-12)
    assert not np.isclose(exact, np.trace(inv[-1]), rtol=1e-3)     # R^ P^ != I matters


def test_bilinear_multigrid_reaches_exact_solve():
    """FGMRES with the multigrid cycle on the bilinear hierarchy (red-black GS on the
    5-point fine level, 4-colour GS on the 9-point coarse levels) reaches the exact solve."""
    from oracle.bilinear import build_bilinear_hierarchy
    lv = build_bilinear_hierarchy(63, 3)
    for cycle in ("V", "K"):
        M = Cycle(lv, 0, 1, 1, cycle, 2)
        b = rademacher(lv[0].n, 0, 1, 0)
        x, its, res = fgmres(lv[0].A, b, M, tol=1e-11, m=30)
        assert res <= 1e-11 and its < 30
        ref = exact_solver(lv[0].A)(b)
        assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
