"""Multilevel Monte-Carlo estimator of tr(A^{-1}) (Secs. 2 and 4).

Oracle (test infrastructure only): imported by tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py``; never by the product path.

Per-level difference samples:
  simplified form (Remark 4.3, needs R_l P_l = I): x in F^{n_l},
      s = x^* A_l^{-1} x - (R_l x)^* A_{l+1}^{-1} (R_l x)
  hat form (Eq. tr_ml_dec and the estimator after it): x in F^{n_1},
      s = (R^_l x)^* A_l^{-1} (R^_l x) - (R^_{l+1} x)^* A_{l+1}^{-1} (R^_{l+1} x)
      using x^* P^_l = (R^_l x)^* since R = P^*.
The coarsest term is exact (Remark 4.2): tr(A_L^{-1} R^_L P^_L), which is
tr(A_L^{-1}) in the simplified form.

Estimate (Sec. 2): sum over levels of the sample means plus the exact term;
variance sum_l V_l / N_l with V_l the unbiased sample variance of |s - mean|^2
(complex variance convention of Sec. 3).

Optimal allocation (Sec. 2), run adaptively (``optimal_trace_estimate``):
after the first block of every level, repeatedly set
N_l = max(5, ceil(sqrt(V_l / C_l) sum_j sqrt(V_j C_j) / (eps tau)^2)) from the
current variance estimates V_l and per-sample costs C_l (the Sec. 5 cost
model), draw a block on every level below its count, and stop when no level
is below its count and sum_l V_l / N_l <= (eps tau)^2.

Stopping rule (Sec. 5): five full estimates t_1..t_5 (one sample per level
difference plus the exact term) give tau = mean(t) - rms(t - mean(t)) (real
parts).  They are samples 0..4 of each level's noise stream, taken from the
first block every level draws, and they also count in the level means (or,
with tau_separate, samples 0..4 of the warm-up stream, which do not).
rho_l = sqrt(w_l) eps |tau| with sum w_l = 1 (default w_l = 1/(L-1)); level l
then draws further blocks of `block` samples until N_l >= 5 and the standard
error sqrt(V_l / N_l) <= rho_l.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .hierarchy import accumulated_prolongation
from .philox import noise, PURPOSE_NOISE, PURPOSE_WARMUP
from .solver import exact_solver, dense_inverse


class LevelSolvers:
    """Exact solves y = A_l^{-1} x for every level (sparse LU; dense inverse on the coarsest)."""

    def __init__(self, levels):
        self.levels = levels
        self.coarse_inv = dense_inverse(levels[-1].A)
        self.solvers = [exact_solver(L.A) for L in levels[:-1]]

    def solve(self, l, b):           # l is 0-based
        if l == len(self.levels) - 1:
            return self.coarse_inv @ b
        return self.solvers[l](b)


def exact_coarse_trace(levels, form="simplified"):
    """Remark 4.2: tr(P^_L A_L^{-1} R^_L) = tr(A_L^{-1} R^_L P^_L)."""
    Ainv = dense_inverse(levels[-1].A)
    if form == "simplified":
        return np.trace(Ainv)
    L = len(levels)
    Ph = accumulated_prolongation(levels, L)
    RP = (Ph.conj().T @ Ph).toarray()
    return np.trace(Ainv @ RP)


def sample(levels, solvers, l, x, form="simplified", hats=None):
    """One difference sample at level l (1-based, l < L) for the noise vector x.

    form "plain" (Eq. plain_tr_estimate): x^* A_1^{-1} x, level 1 only."""
    i = l - 1
    if form == "plain":
        return np.vdot(x, solvers.solve(0, x))
    if form == "simplified":
        y = solvers.solve(i, x)
        z = levels[i].P.conj().T @ x
        w = solvers.solve(i + 1, z)
        return np.vdot(x, y) - np.vdot(z, w)
    zl = hats[i].conj().T @ x
    zl1 = hats[i + 1].conj().T @ x
    return np.vdot(zl, solvers.solve(i, zl)) - np.vdot(zl1, solvers.solve(i + 1, zl1))


def noise_length(levels, l, form):
    return levels[l - 1].n if form == "simplified" else levels[0].n   # hat and plain: fine space


def level_samples(levels, solvers, l, kind, seed, first, count, form="simplified",
                  purpose=PURPOSE_NOISE, hats=None):
    """Samples first..first+count-1 of level l (1-based)."""
    n = noise_length(levels, l, form)
    out = np.zeros(count, dtype=np.complex128)
    for j in range(count):
        x = noise(n, kind, seed, l, first + j, purpose)
        out[j] = sample(levels, solvers, l, x, form, hats)
    return out


@dataclass
class Accumulator:
    n: int = 0
    values: List[complex] = field(default_factory=list)

    def add(self, s):
        self.values.extend(list(s))
        self.n = len(self.values)

    def mean(self):
        return np.mean(self.values) if self.n else 0.0

    def var(self):
        if self.n < 2:
            return np.inf
        v = np.asarray(self.values)
        return float(np.sum(np.abs(v - v.mean()) ** 2) / (self.n - 1))


@dataclass
class EstimateResult:
    trace: complex
    std_err: float
    tau: float
    coarse_term: complex
    n_samples: List[int]
    means: List[complex]
    variances: List[float]
    warmup: List[complex]
    weights: Optional[List[float]] = None     # optimal allocation: w_l = sqrt(V_l C_l) / sum_j sqrt(V_j C_j)


def optimal_allocation(variances, costs, target, min_samples=5):
    """Sec. 2: the sample counts minimising sum_l N_l C_l subject to
    sum_l V_l / N_l = target^2.  Stationarity of the Lagrangian gives
    N_l = mu sqrt(V_l / C_l); the constraint then fixes
    mu = target^-2 sum_j sqrt(V_j C_j).  (The multiplier printed in Sec. 2 has
    sqrt(V_j / C_j) in the sum, which does not satisfy the constraint; the
    minimal cost printed there, target^-2 (sum_j sqrt(V_j C_j))^2, agrees with
    this reading.)
    Returns the real optimum N_l, the whole counts max(min_samples, ceil(N_l))
    and the weights w_l = sqrt(V_l C_l) / sum_j sqrt(V_j C_j), with which the
    optimum is the split rho_l^2 = w_l target^2 of the Sec. 5 stopping rule."""
    V = np.asarray(variances, dtype=float)
    C = np.asarray(costs, dtype=float)
    S = 0.0
    for v, c in zip(V, C):
        S += np.sqrt(v * c)
    N = np.sqrt(V / C) * S / (target * target)
    counts = [max(min_samples, int(np.ceil(n))) for n in N]
    return N, counts, np.sqrt(V * C) / S


def five_estimates(levels, solvers, kind, seed, TL, form, hats, acc, separate):
    """The five full estimates of Sec. 5 (one sample per level difference plus the exact
    term): samples 0..4 of every level's noise stream (held in acc), or, separate, samples
    0..4 of the warm-up stream (Philox purpose 1), which do not enter the level means."""
    warm = np.zeros(5, dtype=np.complex128) + TL
    for l, a in enumerate(acc, start=1):
        if separate:
            warm += level_samples(levels, solvers, l, kind, seed, 0, 5, form, PURPOSE_WARMUP, hats)
        else:
            warm += np.asarray(a.values[:5])
    return warm


def trace_estimate(levels, kind, seed=0, eps=1e-3, weights=None, block=64, min_samples=5,
                   max_samples=1 << 20, form="simplified", solvers=None, tau_separate=False):
    """Sec. 5 procedure; returns an EstimateResult."""
    L = len(levels)
    solvers = solvers or LevelSolvers(levels)
    hats = None
    if form == "hat":
        hats = [accumulated_prolongation(levels, l) for l in range(1, L + 1)]
    if form == "plain":                 # Hutchinson on A_1 alone: one level, no exact term
        L = 2
        TL = 0.0
    else:
        TL = exact_coarse_trace(levels, form)
    # first block of every level; its first five samples give the five full estimates of tau
    acc = [Accumulator() for _ in range(L - 1)]
    for l in range(1, L):
        while acc[l - 1].n < 5:
            a = acc[l - 1]
            a.add(level_samples(levels, solvers, l, kind, seed, a.n, block, form, PURPOSE_NOISE, hats))
    warm = five_estimates(levels, solvers, kind, seed, TL, form, hats, acc, tau_separate)
    tr = warm.real
    tau = tr.mean() - np.sqrt(np.mean((tr - tr.mean()) ** 2))
    w = np.full(L - 1, 1.0 / (L - 1)) if weights is None else np.asarray(weights, dtype=float)
    rho = np.sqrt(w) * eps * abs(tau)
    for l in range(1, L):
        a = acc[l - 1]
        while a.n < max_samples:
            if a.n >= min_samples and np.sqrt(a.var() / a.n) <= rho[l - 1]:
                break
            a.add(level_samples(levels, solvers, l, kind, seed, a.n, block, form, PURPOSE_NOISE, hats))
    est = TL + sum(a.mean() for a in acc)
    se = np.sqrt(sum(a.var() / a.n for a in acc))
    return EstimateResult(est, se, tau, TL, [a.n for a in acc], [a.mean() for a in acc],
                          [a.var() for a in acc], list(warm))


def nominal_sample_cost(levels, l, form="simplified"):
    """Cost of one sample of level difference l (1-based) in the Sec. 5 cost
    model, where a product B x costs nnz(B), counted without the solver's
    iteration counts: the restrictions the sample's noise goes through (each
    R_j = P_j^* costs nnz(P_j)), plus one product with each operator the sample
    solves with; the coarsest level is solved with its dense inverse, n_L^2
    entries.  An optimal multigrid solve costs a level-independent multiple of
    one product with its operator, and a common factor cancels in the optimal
    N_l of Sec. 2.

    simplified form: R_l x, then solves on levels l and l+1;
    hat form:        R^_l x and R^_{l+1} x = R_l ... R_1 x, i.e. P_1 .. P_l;
    plain form:      one solve on level 1."""
    L = len(levels)

    def solve(i):                         # 0-based level
        if i == L - 1:
            return float(levels[i].n) ** 2
        return float(levels[i].A.count_nonzero())

    if form == "plain":
        return solve(0)
    i = l - 1
    c = solve(i) + solve(i + 1)
    for j in (range(i + 1) if form == "hat" else [i]):
        c += float(levels[j].P.count_nonzero())
    return c


def optimal_trace_estimate(levels, kind, seed=0, eps=1e-3, widths=64, min_samples=5, max_samples=1 << 24,
                           form="simplified", solvers=None, costs=None, tau_separate=False):
    """Sec. 2's optimal sample allocation, with V_l and C_l estimated as the samples arrive.

    widths: samples per block, one value for every level difference or a list (the
    last value repeats).  costs: per-sample cost C_l of every level difference;
    default ``nominal_sample_cost``.  Steps:
      1. the exact coarsest term T_L (Remark 4.2);
      2. every level difference draws blocks until it holds 5 samples; samples 0..4 of
         each level plus T_L are the five full estimates that give tau (Sec. 5);
      3. target T = eps |tau|;
      4. repeat: with S = sum_j sqrt(V_j C_j) from the current unbiased variances,
         go through the levels in order; level l wants
         N_l* = max(min_samples, ceil(sqrt(V_l / C_l) S / T^2)) (Sec. 2, reading the
         multiplier from the constraint, see ``optimal_allocation``) and draws one block
         if it holds fewer (and fewer than max_samples).  When no level drew and
         sum_l V_l / N_l <= T^2 (variances as they stood before the pass) the estimate
         stops.  When no level drew but the sum is above T^2 (only possible when a level
         is held at max_samples), one block goes to the level whose next block lowers
         sum V/N most per unit of cost, and when no level can draw any more, it stops."""
    L = len(levels)
    solvers = solvers or LevelSolvers(levels)
    hats = None
    if form == "hat":
        hats = [accumulated_prolongation(levels, l) for l in range(1, L + 1)]
    if form == "plain":
        nd, TL = 1, 0.0
    else:
        nd, TL = L - 1, exact_coarse_trace(levels, form)
    if isinstance(widths, int):
        widths = [widths]
    width = [int(widths[min(i, len(widths) - 1)]) for i in range(nd)]
    if costs is None:
        costs = [nominal_sample_cost(levels, l, form) for l in range(1, nd + 1)]
    C = [float(c) for c in costs]
    acc = [Accumulator() for _ in range(nd)]

    def draw(i):
        k = min(width[i], max_samples - acc[i].n)
        if k <= 0:
            return False
        acc[i].add(level_samples(levels, solvers, i + 1, kind, seed, acc[i].n, k, form, PURPOSE_NOISE, hats))
        return True

    for i in range(nd):
        while acc[i].n < 5:
            if not draw(i):
                raise ValueError("max_samples allows fewer than five samples per level")
    warm = five_estimates(levels, solvers, kind, seed, TL, form, hats, acc, tau_separate)
    tr = warm.real
    tau = tr.mean() - np.sqrt(np.mean((tr - tr.mean()) ** 2))
    T2 = (eps * abs(tau)) ** 2
    w = [0.0] * nd
    while True:
        V = [a.var() for a in acc]
        S = 0.0
        for i in range(nd):
            S += np.sqrt(V[i] * C[i])
        drew, total = False, 0.0
        for i in range(nd):
            want = max(float(min_samples), np.ceil(np.sqrt(V[i] / C[i]) * S / T2))
            w[i] = np.sqrt(V[i] * C[i]) / S
            total += V[i] / acc[i].n
            if acc[i].n < want and acc[i].n < max_samples:
                drew = True
                draw(i)
        if drew:
            continue
        if total <= T2:
            break
        best, gain = -1, -1.0
        for i in range(nd):
            n, v = acc[i].n, acc[i].var()
            k = min(width[i], max_samples - n)
            if k <= 0:
                continue
            g = (v / n - v / (n + k)) / (C[i] * k)
            if g > gain:
                best, gain = i, g
        if best < 0:
            break
        draw(best)
    est = TL + sum(a.mean() for a in acc)
    se = np.sqrt(sum(a.var() / a.n for a in acc))
    return EstimateResult(est, se, tau, TL, [a.n for a in acc], [a.mean() for a in acc],
                          [a.var() for a in acc], list(warm), list(w))
