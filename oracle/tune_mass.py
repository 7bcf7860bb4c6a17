"""Tune the Wilson mass m so that sigma_min(S) / sigma_max(S) is about 1e-3.

Oracle tool (test infrastructure): calls only oracle/ and the seeded link
generator.  sigma_max by power iteration on S^* S, sigma_min by inverse
iteration on S^* S with sparse-LU solves; bisection on m.  The workloads
record the printed masses.

usage: python -m oracle.tune_mass NX NY LINK_SD LINK_SEED [TARGET [LO HI SCAN]]
       python -m oracle.tune_mass NX NY LINK_SD LINK_SEED TARGET --bisect M_CRIT M_HI STEPS
         (bisection on [M_CRIT, M_HI], the physical side above a known critical mass)
"""
import sys

import numpy as np
import scipy.sparse.linalg as spla

from .operators import wilson2d
from paper_2108_11281_gb300.workloads import gauge_links


def sigma_extremes(S, iters=30, seed=0):
    rng = np.random.default_rng(seed)
    n = S.shape[0]
    v = rng.normal(size=n) + 1j * rng.normal(size=n)
    for _ in range(iters):
        v = S.conj().T @ (S @ v)
        v /= np.linalg.norm(v)
    smax = np.sqrt(np.linalg.norm(S.conj().T @ (S @ v)))
    lu = spla.splu(S.tocsc())
    luh = spla.splu(S.conj().T.tocsc())
    u = rng.normal(size=n) + 1j * rng.normal(size=n)
    lam = 0.0
    for _ in range(iters):
        u = lu.solve(luh.solve(u))          # (S^* S)^{-1} u = S^{-1} S^{-*} u
        lam = np.linalg.norm(u)
        u /= lam
    return 1.0 / np.sqrt(lam), smax


def tune(nx, ny, sd, seed, target=1e-3, lo=-0.4, hi=0.1, scan=21, steps=30):
    """sigma_min(m) dips to ~0 at the critical mass m_c; the physical side is m > m_c
    (spectrum in the right half plane, Example 5.3).  Scan for the dip, then bisect
    on [m_c, m_c + spacing] where the ratio increases with m."""
    U = gauge_links(nx, ny, sd, seed)

    def ratio_of(m):
        smin, smax = sigma_extremes(wilson2d(nx, ny, m, U))
        return smin / smax

    grid = np.linspace(lo, hi, scan)
    vals = []
    for m in grid:
        vals.append(ratio_of(m))
        print("scan m %.4f ratio %.3e" % (m, vals[-1]), flush=True)
    i = int(np.argmin(vals))
    a, b = grid[max(i - 1, 0)], grid[min(i + 1, scan - 1)]
    for _ in range(40):                      # golden-section refinement of the dip
        m1, m2 = a + 0.382 * (b - a), a + 0.618 * (b - a)
        if ratio_of(m1) < ratio_of(m2):
            b = m2
        else:
            a = m1
    mc = 0.5 * (a + b)
    if ratio_of(mc) > target:
        raise ValueError("the ratio never reaches the target on this configuration")
    a, b = mc, mc + (grid[1] - grid[0]) * 2
    r = None
    for _ in range(steps):
        m = 0.5 * (a + b)
        r = ratio_of(m)
        if abs(np.log(r / target)) < np.log(1.02):
            return m, r
        if r > target:
            b = m
        else:
            a = m
    return m, r


if __name__ == "__main__":
    a = sys.argv[1:]
    nx, ny, sd, seed = int(a[0]), int(a[1]), float(a[2]), int(a[3])
    target = float(a[4]) if len(a) > 4 else 1e-3
    if len(a) > 5 and a[5] == "--bisect":
        U = gauge_links(nx, ny, sd, seed)
        lo, hi = float(a[6]), float(a[7])
        for _ in range(int(a[8])):
            m = 0.5 * (lo + hi)
            smin, smax = sigma_extremes(wilson2d(nx, ny, m, U))
            ratio = smin / smax
            print("bisect m %.6f ratio %.4e" % (m, ratio), flush=True)
            if ratio > target:
                hi = m
            else:
                lo = m
        print("mass %.10f ratio %.4e" % (m, ratio))
        sys.exit(0)
    rng = dict(lo=float(a[5]), hi=float(a[6]), scan=int(a[7])) if len(a) > 7 else {}
    m, ratio = tune(nx, ny, sd, seed, target, **rng)
    print("mass %.10f ratio %.4e" % (m, ratio))
