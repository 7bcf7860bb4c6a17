"""Aggregation multigrid hierarchy (Sec. 4.1 and the Schwinger sketch of Example 5.3).

Oracle (test infrastructure only): imported by tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py``; never by the product path.

Levels l = 1..L carry A_l (n_l x n_l, Petrov-Galerkin A_{l+1} = R_l A_l P_l with
R_l = P_l^*), and P_l (n_l x n_{l+1}) for l < L.  The lattice of level l is
divided into non-overlapping agg_x x agg_y aggregates; each aggregate becomes
one site of level l+1.  P_l is block diagonal over aggregates: its columns
are test vectors restricted to the aggregate (optionally split into the two
spin halves of each site's dofs, which doubles the coarse dofs and keeps
J A = A^* J), orthonormalised by modified Gram-Schmidt applied twice to each
column (smooth test vectors are nearly dependent on an aggregate; one pass
leaves |P^* P - I| ~ 1e-10).  So R_l P_l = I and Remark 4.3 applies.

Test vectors (the paper says only "quite inexact approximations to the d
smallest eigenvectors"; this is the project's reading): n_tv Philox noise
vectors (purpose SETUP, sample index = vector index, level = l), then
  kind "smooth":  nu times  v <- v - omega D^{-1} A v          (damped Jacobi on A v = 0)
  kind "inverse": nu times  v <- two damped-Jacobi steps on A x = v from x = 0
with D = diag(A_l).  No normalisation: Gram-Schmidt removes the scale.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np
import scipy.sparse as sp

from .philox import noise, PURPOSE_SETUP


@dataclass
class Level:
    A: sp.csr_matrix
    nx: int
    ny: int
    d: int
    P: Optional[sp.csr_matrix] = None       # n_l x n_{l+1}; None on the coarsest level
    P_blocks: Optional[np.ndarray] = None   # [aggregate][loc*d + a][q], same entries as P
    colours: int = 2                        # site colours of the Gauss-Seidel smoother: 2 for
                                            # nearest-neighbour stencils, 4 for 9-point stencils

    @property
    def n(self):
        return self.nx * self.ny * self.d


@dataclass
class SetupParams:
    levels: int
    agg_x: int = 4
    agg_y: int = 4
    n_tv: object = 4              # int, or one count per coarsening (fresh noise fills any increase)
    spin_split: bool = False
    kind: str = "smooth"          # "smooth" | "inverse" | "constant" (n_tv = 1, P = 1/sqrt(|agg|))
    sweeps: int = 40              # filter sweeps on level 1
    coarse_sweeps: int = 20       # filter sweeps on levels >= 2 (after restriction)
    omega: float = 2.0 / 3.0
    seed: int = 0
    noise_kind: str = "rademacher"  # test-vector noise: "rademacher" | "z4"
    bootstrap: int = 1            # rounds of test-vector improvement by the solver's cycle
    boot_iters: int = 2           # v <- v - M A v applications per round
    smooth_pre: int = 1           # red-black GS sweeps of the cycle used by the bootstrap
    smooth_post: int = 1
    kcycle_its: int = 2
    coarse_smooth: int = 0        # > 0: sweeps on levels >= 2 in that cycle


def tv_count(params, lvl):
    """Number of test vectors used to build P_lvl (lvl is 1-based)."""
    if isinstance(params.n_tv, (list, tuple)):
        return int(params.n_tv[lvl - 1])
    return int(params.n_tv)


def jacobi_filter(A, V, kind, sweeps, omega):
    """Apply the test-vector filter column by column."""
    if kind == "constant":
        return V
    Dinv = 1.0 / A.diagonal()
    V = V.copy()
    for _ in range(sweeps):
        if kind == "smooth":
            V = V - omega * (Dinv[:, None] * (A @ V))
        elif kind == "inverse":
            x1 = omega * (Dinv[:, None] * V)
            x2 = x1 + omega * (Dinv[:, None] * (V - A @ x1))
            V = x2
        else:
            raise ValueError(kind)
    return V


def aggregate_of_sites(nx, ny, ax, ay):
    """For each site s = j*nx+i: (aggregate index, local site index inside it)."""
    j, i = np.divmod(np.arange(nx * ny), nx)
    agg = (j // ay) * (nx // ax) + (i // ax)
    loc = (j % ay) * ax + (i % ax)
    return agg, loc


def build_prolongation(V, nx, ny, d, ax, ay, spin_split):
    """P from test vectors V (n x n_tv): per aggregate, MGS in column order.

    Column q of aggregate I: q = h*n_tv + t (spin half h, test vector t) when
    spin_split, else q = t.  Global coarse dof = I*dc + q; global fine dof = s*d + a.
    Returns (P as a sparse matrix, dense blocks [I][loc*d + a][q]).
    All aggregates are processed together; each one is an independent MGS.
    """
    n_tv = V.shape[1]
    dc = n_tv * (2 if spin_split else 1)
    nagg = (nx // ax) * (ny // ay)
    agg, loc = aggregate_of_sites(nx, ny, ax, ay)
    m = ax * ay * d                                   # fine dofs per aggregate
    fine_index = np.zeros((nagg, m), dtype=np.int64)
    s = np.arange(nx * ny)
    for a in range(d):
        fine_index[agg, loc * d + a] = s * d + a
    dtype = np.result_type(V.dtype, np.float64)
    local = V[fine_index].astype(dtype)               # nagg x m x n_tv
    if spin_split:
        upper = (np.arange(m) % d) < d // 2           # first half of each site's dofs
        cols = [local[:, :, t] * upper for t in range(n_tv)] + \
               [local[:, :, t] * ~upper for t in range(n_tv)]
    else:
        cols = [local[:, :, t] for t in range(n_tv)]
    Q = np.zeros((nagg, m, dc), dtype=dtype)
    for q, v in enumerate(cols):
        v = v.copy()
        for _ in range(2):                            # modified Gram-Schmidt, each column twice
            for p in range(q):
                coef = np.einsum("im,im->i", Q[:, :, p].conj(), v)
                v = v - coef[:, None] * Q[:, :, p]
        nrm = np.sqrt(np.einsum("im,im->i", v.conj(), v).real)
        if np.any(nrm == 0.0):
            raise ValueError("test vectors are linearly dependent on an aggregate")
        Q[:, :, q] = v / nrm[:, None]
    rows = np.repeat(fine_index[:, :, None], dc, axis=2)
    colsidx = np.broadcast_to(np.arange(nagg)[:, None, None] * dc + np.arange(dc)[None, None, :],
                              Q.shape)
    P = sp.csr_matrix((Q.ravel(), (rows.ravel(), colsidx.ravel())),
                      shape=(nx * ny * d, nagg * dc))
    return P, Q


def _coarsen(levels_in, V1, params: SetupParams):
    """Levels 2..L from level-1 test vectors V1 (Sec. 4.1 / Example 5.3).

    Level l >= 2 starts from the previous level's test vectors restricted,
    V_l = R_{l-1} V_{l-1}, which represent them exactly because each is a
    column of P_{l-1} before orthonormalisation; then `coarse_sweeps` filter
    sweeps with A_l.
    """
    A1, nx, ny, d = levels_in.A, levels_in.nx, levels_in.ny, levels_in.d
    levels = [Level(sp.csr_matrix(A1), nx, ny, d)]
    V = V1
    for lvl in range(1, params.levels):
        cur = levels[-1]
        if cur.nx % params.agg_x or cur.ny % params.agg_y:
            raise ValueError("lattice not divisible by the aggregate size")
        nt = tv_count(params, lvl)
        if lvl > 1:
            if V.shape[1] > nt:
                V = V[:, :nt]
            elif V.shape[1] < nt:                       # extra fresh vectors on this level
                extra = np.stack([noise(cur.n, params.noise_kind, params.seed, lvl, t, PURPOSE_SETUP)
                                  for t in range(V.shape[1], nt)], axis=1)
                V = np.concatenate([V, extra.astype(np.result_type(V, extra))], axis=1)
            V = jacobi_filter(cur.A, V, params.kind, params.coarse_sweeps, params.omega)
        P, blocks = build_prolongation(V, cur.nx, cur.ny, cur.d, params.agg_x, params.agg_y,
                                       params.spin_split)
        cur.P, cur.P_blocks = P, blocks
        Ac = sp.csr_matrix(P.conj().T @ cur.A @ P)     # A_{l+1} = R_l A_l P_l, R_l = P_l^*
        dc = nt * (2 if params.spin_split else 1)
        levels.append(Level(Ac, cur.nx // params.agg_x, cur.ny // params.agg_y, dc))
        V = P.conj().T @ V                              # R_l V_l
    return levels


def level1_test_vectors(A1, n, params: SetupParams):
    if params.kind == "constant":
        return np.ones((n, 1))
    V = np.stack([noise(n, params.noise_kind, params.seed, 1, t, PURPOSE_SETUP)
                  for t in range(tv_count(params, 1))], axis=1)
    return jacobi_filter(A1, V, params.kind, params.sweeps, params.omega)


def build_hierarchy(A1, nx, ny, d, params: SetupParams):
    """Levels 1..L: test vectors, aggregation, Galerkin coarsening, bootstrap.

    Bootstrap round (the paper's test vectors are "quite inexact
    approximations to the smallest eigenvectors"; improving them with the
    solver itself is the project's reading): each level-1 test vector v is
    replaced `boot_iters` times by v - M(A v), with M one cycle (class
    ``Cycle``) of the current hierarchy, and the hierarchy is rebuilt.
    """
    from .solver import Cycle      # local import: the cycle needs built levels
    base = Level(sp.csr_matrix(A1), nx, ny, d)
    V = level1_test_vectors(base.A, base.n, params)
    levels = _coarsen(base, V, params)
    for _ in range(params.bootstrap if params.kind != "constant" else 0):
        M = Cycle(levels, 0, params.smooth_pre, params.smooth_post, "K", params.kcycle_its,
                  coarse_smooth=params.coarse_smooth)
        for _ in range(params.boot_iters):
            V = np.stack([V[:, t] - M(base.A @ V[:, t]) for t in range(V.shape[1])], axis=1)
        levels = _coarsen(base, V, params)
    return levels


def accumulated_prolongation(levels, l):
    """P-hat_l = P_1 ... P_{l-1} (Sec. 4.1); identity for l = 1.  l is 1-based."""
    n1 = levels[0].n
    Ph = sp.identity(n1, format="csr", dtype=levels[0].A.dtype)
    for k in range(l - 1):
        Ph = Ph @ levels[k].P
    return sp.csr_matrix(Ph)
