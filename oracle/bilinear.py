"""The paper's own hierarchy for Example 5.1 (Sec. 5, the 2d Laplace study).

Oracle (test infrastructure only): imported by tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py``; never by the product path.

Level l has an N_l x N_l grid (Dirichlet, site s = j*N + i, x fastest) with
N_{l+1} = floor(N_l / 2); the grids used are N_l odd, N_l = 2 N_{l+1} + 1, so
coarse point I sits on fine point 2I + 1.  P_l is standard bilinear
interpolation from level l+1 to level l, the tensor product of the 1-D
interpolation p with p[2I+1, I] = 1 and p[2I, I] = p[2I+2, I] = 1/2; the
restriction is its adjoint R_l = P_l^T, and A_{l+1} = R_l A_l P_l (Galerkin).
Coarse operators are 9-point stencils, smoothed by 4-colour Gauss-Seidel.
P_l is not orthonormal (R_l P_l != I), so the estimator must use the hat form
(Eq. tr_ml_dec) and the exact term tr(A_L^{-1} R^_L P^_L) (Remark 4.2).
"""
import numpy as np
import scipy.sparse as sp

from .hierarchy import Level
from .operators import laplace2d


def interpolation_1d(nf):
    """p (nf x nc), nc = (nf - 1) / 2: linear interpolation from the coarse 1-D grid."""
    if nf % 2 != 1 or nf < 3:
        raise ValueError("bilinear coarsening needs an odd grid side >= 3")
    nc = (nf - 1) // 2
    I = np.arange(nc)
    rows = np.concatenate([2 * I + 1, 2 * I, 2 * I + 2])
    cols = np.concatenate([I, I, I])
    vals = np.concatenate([np.ones(nc), 0.5 * np.ones(nc), 0.5 * np.ones(nc)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


def bilinear_prolongation(nx, ny):
    """P = p_y (x) p_x for site order s = j*nx + i."""
    return sp.csr_matrix(sp.kron(interpolation_1d(ny), interpolation_1d(nx)))


def build_bilinear_hierarchy(N, levels, shift=0.0):
    """Levels 1..L of the Example 5.1 hierarchy with bilinear P (Sec. 5)."""
    A = laplace2d(N, N, shift)
    out = [Level(A, N, N, 1, colours=2)]
    for _ in range(1, levels):
        cur = out[-1]
        P = bilinear_prolongation(cur.nx, cur.ny)
        cur.P = P
        Ac = sp.csr_matrix(P.T @ cur.A @ P)
        Ac.eliminate_zeros()
        out.append(Level(Ac, (cur.nx - 1) // 2, (cur.ny - 1) // 2, 1, colours=4))
    return out
