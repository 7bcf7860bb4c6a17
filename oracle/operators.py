"""Fine-level operators written out from their definitions.

Oracle (test infrastructure only): imported by tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py``; never by the product path.

Site order everywhere: s = j*nx + i (x fastest); dofs of a site are
contiguous, global dof index = s*d + a.
"""
import numpy as np
import scipy.sparse as sp


def laplace2d(nx, ny, shift=0.0, periodic=False):
    """Example 5.1: L = B (x) I + I (x) B with B = tridiag(-1, 2, -1), plus shift*I.

    Dirichlet (periodic=False) drops couplings that leave the grid; the
    periodic variant closes B into a circulant.  Real, symmetric.
    """
    def one_d(n):
        B = sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="lil")
        if periodic and n > 2:
            B[0, n - 1] = -1.0
            B[n - 1, 0] = -1.0
        return B.tocsr()
    Bx, By = one_d(nx), one_d(ny)
    # site s = j*nx + i: the x index is the fast one, so Bx acts on the right factor
    A = sp.kron(sp.identity(ny), Bx) + sp.kron(By, sp.identity(nx))
    if shift != 0.0:
        A = A + shift * sp.identity(nx * ny)
    return sp.csr_matrix(A, dtype=np.float64)


SIGMA1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SIGMA2 = np.array([[0, 1j], [-1j, 0]], dtype=np.complex128)   # as printed in Example 5.3
ID2 = np.eye(2, dtype=np.complex128)


def wilson2d(nx, ny, mass, links):
    """Example 5.3, Eq. schwinger_coupling: the 2-spin periodic Schwinger/Wilson operator.

    Row of site (i,j):  (4+m) u_ij - U^x_ij (I - s1) u_{i+1,j} - U^y_ij (I - s2) u_{i,j+1}
                        - conj(U^x_{i-1,j}) (I + s1) u_{i-1,j} - conj(U^y_{i,j-1}) (I + s2) u_{i,j-1}
    links: complex array (2, ny, nx); links[0] = exp(i Theta) on the x-link
    (i,j)->(i+1,j), links[1] = exp(i Phi) on the y-link (i,j)->(i,j+1).
    Indices are taken mod N (periodic).
    """
    links = np.asarray(links, dtype=np.complex128)
    n = nx * ny
    rows, cols, vals = [], [], []

    def add(site_rows, site_cols, coef, block):
        for a in range(2):
            for b in range(2):
                if block[a, b] != 0:
                    rows.append(2 * site_rows + a)
                    cols.append(2 * site_cols + b)
                    vals.append(coef * block[a, b])

    j, i = np.divmod(np.arange(n), nx)
    s = j * nx + i
    xp = j * nx + (i + 1) % nx
    xm = j * nx + (i - 1) % nx
    yp = ((j + 1) % ny) * nx + i
    ym = ((j - 1) % ny) * nx + i
    Ux = links[0].reshape(n)
    Uy = links[1].reshape(n)
    add(s, s, np.full(n, 4.0 + mass, dtype=np.complex128), ID2)
    add(s, xp, -Ux[s], ID2 - SIGMA1)
    add(s, yp, -Uy[s], ID2 - SIGMA2)
    add(s, xm, -np.conj(Ux[xm]), ID2 + SIGMA1)
    add(s, ym, -np.conj(Uy[ym]), ID2 + SIGMA2)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(2 * n, 2 * n)).tocsr()
    A.sum_duplicates()
    return A


def spin_parity(n_sites, d):
    """Diagonal of J: +1 on the first half of each site's dofs, -1 on the second (Sec. 5, Ex. 5.3)."""
    half = np.concatenate([np.ones(d // 2), -np.ones(d // 2)])
    return np.tile(half, n_sites)
