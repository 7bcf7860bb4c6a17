"""One MLMC estimate of tr(A^-1) with its samples spread over ranks (Secs. 2 and 5).

The samples of a level difference are independent and indexed by (seed, level,
sample index), so ranks draw disjoint blocks of the same sample stream: in a
round on level difference l, rank r draws block b0 + r, i.e. samples
(b0 + r) k_l ... (b0 + r + 1) k_l - 1, on its own GPU (``mlmc_sample_block``:
the solves and the block's (N, mean, M2) run in the library's kernels).  One
exchange per round (an all-gather of ten doubles per rank) gives every rank the
statistics of all blocks of the round, which it merges into the level's
running (N, mean, M2) in block order with the pairwise update of Chan, Golub
and LeVeque.  The merged statistics therefore depend on which blocks were
drawn, not on how many ranks drew them, and every rank takes the same stopping
decisions from them.  The exact coarsest term (Remark 4.2) is rank 0's, shared
by the first exchange; tau comes from samples 0..4 of every level (Sec. 5).

Allocation: Sec. 2's optimal N_l (nominal per-sample costs, the loop of
``mlmc_trace_estimate`` with MLMC_COST_NOMINAL), the Sec. 5 rho split, or fixed
counts.  Rounds draw `world` blocks at a time, so N_l can overshoot by up to
world - 1 blocks more than one rank would draw.

``allgather(values) -> list of per-rank value lists`` (rank order), e.g.
``torch.distributed.all_gather`` of a float64 tensor over NCCL or gloo.
"""
import math

from . import mlmc as _m


class HierarchySampler:
    """Blocks of level-difference samples from one GPU hierarchy (the library)."""

    def __init__(self, h, noise, seed, tol, form=_m.FORM_SIMPLIFIED):
        self.h, self.noise, self.seed, self.tol, self.form = h, noise, seed, tol, form
        self.n_differences = 1 if form == _m.FORM_PLAIN else h.params.levels - 1

    def width(self, l):
        return self.h.block_width(l)

    def cost(self, l):
        return self.h.nominal_sample_cost(l, self.form)

    def coarse_term(self):
        return 0.0 if self.form == _m.FORM_PLAIN else self.h.coarse_trace_exact().real

    def block(self, l, first, k):
        """(samples, (N, mean, M2)) of samples first .. first + k - 1 of level difference l."""
        samples, stats, _ = self.h.sample_block(l, self.form, self.noise, self.seed, first, k, self.tol)
        return samples, stats


def merge(a, b):
    """Pairwise update (Chan, Golub, LeVeque) of running (N, mean, M2) with a block's."""
    na, ma, qa = a
    nb, mb, qb = b
    if nb == 0:
        return a
    if na == 0:
        return (nb, mb, qb)
    n = na + nb
    d = mb - ma
    return (n, ma + d * (nb / n), qa + qb + abs(d) ** 2 * (na * nb / n))


def sharded_trace_estimate(sampler, allgather, rank=0, world=1, eps=1e-3, allocation="optimal", weights=None,
                           n_fixed=None, min_samples=5, max_samples=1 << 24):
    """The estimate (Sec. 2 estimator, Sec. 5 tau and stopping) over `world` ranks; every
    rank returns the same dict: trace, std_err, tau, coarse_term, n_samples, mean,
    variance, weights_used, rounds."""
    nd = sampler.n_differences
    acc = [(0, 0j, 0.0) for _ in range(nd)]
    nblk = [0] * nd
    warm = [0.0] * 5
    term = [None]
    rounds = [0]

    def cap(l):
        return n_fixed[l] if allocation == "fixed" else max_samples

    def draw(l):
        """One round on level difference l (0-based): every rank one block."""
        kl = sampler.width(l + 1)
        first = (nblk[l] + rank) * kl
        k = min(kl, cap(l) - first)
        vec = [0.0] * 10
        if k > 0:
            samples, (n, mean, q) = sampler.block(l + 1, first, k)
            vec[0:4] = [float(n), mean.real, mean.imag, float(q)]
            for i in range(first, min(first + k, 5)):
                vec[4 + i] = samples[i - first].real
        if term[0] is None and rank == 0:
            vec[9] = sampler.coarse_term()
        got = allgather(vec)
        if term[0] is None:
            term[0] = got[0][9]
        for r in range(world):
            g = got[r]
            acc[l] = merge(acc[l], (int(g[0]), complex(g[1], g[2]), g[3]))
            for i in range(5):
                warm[i] += g[4 + i]
        nblk[l] += world
        rounds[0] += 1
        return any(g[0] > 0 for g in got)

    def var(l):
        n, _, q = acc[l]
        return q / (n - 1) if n > 1 else math.inf

    for l in range(nd):
        while acc[l][0] < 5:
            if not draw(l):
                raise ValueError("max_samples allows fewer than five samples per level")
    tr = [term[0] + v for v in warm]
    mu = sum(tr) / 5.0
    tau = mu - math.sqrt(sum((t - mu) ** 2 for t in tr) / 5.0)
    target = eps * abs(tau)
    T2 = target * target
    w = [0.0] * nd
    if allocation == "fixed":
        for l in range(nd):
            while acc[l][0] < n_fixed[l]:
                draw(l)
    elif allocation == "rho":
        ws = [1.0 / nd] * nd if weights is None else [x / sum(weights) for x in weights]
        for l in range(nd):
            w[l] = ws[l]
            rho = math.sqrt(ws[l]) * target
            while not (acc[l][0] >= min_samples and math.sqrt(var(l) / acc[l][0]) <= rho):
                if acc[l][0] >= max_samples or not draw(l):
                    break
    else:
        C = [sampler.cost(l + 1) for l in range(nd)]
        while True:
            V = [var(l) for l in range(nd)]
            S = sum(math.sqrt(V[l] * C[l]) for l in range(nd))
            drew, total = False, 0.0
            for l in range(nd):
                want = max(float(min_samples), math.ceil(math.sqrt(V[l] / C[l]) * S / T2))
                w[l] = math.sqrt(V[l] * C[l]) / S
                total += V[l] / acc[l][0]
                if acc[l][0] < want and acc[l][0] < max_samples:
                    drew = True
                    draw(l)
            if drew:
                continue
            if total <= T2:
                break
            best, gain = -1, -1.0
            for l in range(nd):
                n, v = acc[l][0], var(l)
                k = min(sampler.width(l + 1) * world, max_samples - n)
                if k <= 0:
                    continue
                g = (v / n - v / (n + k)) / (C[l] * k)
                if g > gain:
                    best, gain = l, g
            if best < 0:
                break
            draw(best)
    trace = complex(term[0]) + sum(a[1] for a in acc)
    return {"trace": trace, "std_err": math.sqrt(sum(var(l) / acc[l][0] for l in range(nd))), "tau": tau,
            "coarse_term": term[0], "n_samples": [a[0] for a in acc], "mean": [a[1] for a in acc],
            "variance": [var(l) for l in range(nd)], "weights_used": w, "rounds": rounds[0]}


def torch_allgather(device="cpu"):
    """allgather over the default torch.distributed process group (NCCL: device="cuda")."""
    import torch
    import torch.distributed as dist

    def gather(vec):
        t = torch.tensor(vec, dtype=torch.float64, device=device)
        out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
        dist.all_gather(out, t)
        return [o.cpu().tolist() for o in out]
    return gather
