"""Linear solves for the level systems A_l y = x.

Oracle (test infrastructure only): imported by tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py``; never by the product path.

Two routes:
  * ``exact_solver``: sparse LU (SuperLU) of A_l, i.e. the definition
    y = A_l^{-1} x up to rounding.  Used for the per-sample reference values.
  * ``fgmres`` preconditioned by ``Cycle``: the multigrid solver of Example
    5.3 and Remark 4.1 (flexible GMRES whose preconditioner is one multigrid
    cycle over levels l..L with Gauss-Seidel pre- and post-smoothing and a
    direct solve on the coarsest level).  Two choices here are the project's
    own and shared with the GPU path: the Gauss-Seidel sweep uses red-black
    site order with d x d site blocks (sites of one colour do not couple in a
    nearest-neighbour operator, so the sweep is a well-defined block
    Gauss-Seidel), and the coarse-grid correction may be Krylov-accelerated
    (K-cycle: a fixed number of FGMRES steps on level l+1 preconditioned by
    the cycle on l+1).  Used for the setup bootstrap, the CPU baseline and to
    pin that the solver reaches the exact solve.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class exact_solver:
    """y = A^{-1} x by a sparse (or, for small A, dense) LU factorisation."""

    def __init__(self, A):
        self.n = A.shape[0]
        if self.n <= 2048:
            self.lu = sla.lu_factor(A.toarray())
            self._solve = lambda b: sla.lu_solve(self.lu, b)
        else:
            self.lu = spla.splu(sp.csc_matrix(A))
            self._solve = self.lu.solve

    def __call__(self, b):
        return self._solve(b)


def dense_inverse(A):
    """A^{-1} of the (small) coarsest operator, by LU with partial pivoting."""
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A)
    lu = sla.lu_factor(Ad)
    return sla.lu_solve(lu, np.eye(Ad.shape[0], dtype=Ad.dtype))


def site_colour(nx, ny, d, colours=2):
    """Colour of every dof.  2 colours: red (0) / black (1) = parity of i + j of
    its site.  4 colours (9-point stencils, whose diagonal neighbours share the
    red-black colour): (i mod 2) + 2 (j mod 2)."""
    j, i = np.divmod(np.arange(nx * ny), nx)
    c = (i + j) % 2 if colours == 2 else (i % 2) + 2 * (j % 2)
    return np.repeat(c, d)


class RedBlackGS:
    """Block Gauss-Seidel in multi-colour site order on one level (red-black for
    nearest-neighbour stencils, four colours for 9-point stencils).

    A partial sweep over colour c sets, for every site s of colour c,
        x_s <- x_s + D_s^{-1} (b - A x)_s,     D_s = the d x d diagonal block,
    which equals solving the site's row block exactly given its neighbours.
    Pre-smoothing visits the colours in increasing order, post-smoothing in
    decreasing order.
    """

    def __init__(self, level):
        A = sp.csr_matrix(level.A)
        d, nsite = level.d, level.nx * level.ny
        dense_blocks = np.zeros((nsite, d, d), dtype=A.dtype)
        rows, cols = A.nonzero()
        same = rows // d == cols // d
        r, c = rows[same], cols[same]
        dense_blocks[r // d, r % d, c % d] = np.asarray(A[r, c]).ravel()
        inv = np.linalg.inv(dense_blocks)
        bi = np.repeat(np.arange(nsite) * d, d * d) + np.tile(np.repeat(np.arange(d), d), nsite)
        bj = np.repeat(np.arange(nsite) * d, d * d) + np.tile(np.tile(np.arange(d), d), nsite)
        self.Dinv = sp.csr_matrix((inv.ravel(), (bi, bj)), shape=A.shape)
        self.A = A
        self.ncol = getattr(level, "colours", 2)
        colour = site_colour(level.nx, level.ny, d, self.ncol)
        self.mask = [(colour == c).astype(float) for c in range(self.ncol)]

    def half(self, x, b, c):
        upd = self.Dinv @ (b - self.A @ x)
        m = self.mask[c] if x.ndim == 1 else self.mask[c][:, None]
        return x + m * upd

    def pre(self, x, b, sweeps):
        for _ in range(sweeps):
            for c in range(self.ncol):
                x = self.half(x, b, c)
        return x

    def post(self, x, b, sweeps):
        for _ in range(sweeps):
            for c in reversed(range(self.ncol)):
                x = self.half(x, b, c)
        return x


class Cycle:
    """One multigrid cycle started on level index `first` (0-based) of `levels`.

    cycle(l, b): x = pre-smooth(0, b); r = b - A_l x; rc = P_l^* r;
                 ec = A_L^{-1} rc                          if l+1 is the coarsest level,
                      cycle(l+1, rc)                       for a V-cycle,
                      `kcycle_its` FGMRES steps on A_{l+1} ec = rc
                      preconditioned by cycle(l+1)         for a K-cycle;
                 x += P_l ec; x = post-smooth(x, b).
    """

    def __init__(self, levels, first=0, pre=1, post=1, kind="K", kcycle_its=2, coarse_inv=None, coarse_smooth=0):
        self.levels, self.first = levels, first
        self.pre, self.post = pre, post
        self.coarse_smooth = coarse_smooth      # > 0: sweeps on every level below the finest
        self.kind, self.kits = kind, kcycle_its
        self.smoothers = [RedBlackGS(L) if i < len(levels) - 1 else None
                          for i, L in enumerate(levels)]
        self.coarse_inv = dense_inverse(levels[-1].A) if coarse_inv is None else coarse_inv

    def cycle(self, l, b):
        last = len(self.levels) - 1
        if l == last:
            return self.coarse_inv @ b
        L = self.levels[l]
        pre = self.coarse_smooth if (l > 0 and self.coarse_smooth > 0) else self.pre
        post = self.coarse_smooth if (l > 0 and self.coarse_smooth > 0) else self.post
        x = self.smoothers[l].pre(np.zeros_like(b), b, pre)
        r = b - L.A @ x
        rc = L.P.conj().T @ r
        if l + 1 == last or self.kind == "V":
            ec = self.cycle(l + 1, rc)
        else:
            ec, _, _ = fgmres(self.levels[l + 1].A, rc, lambda v: self.cycle(l + 1, v),
                              tol=0.0, m=self.kits, maxit=self.kits)
        x = x + L.P @ ec
        return self.smoothers[l].post(x, b, post)

    def __call__(self, b):
        return self.cycle(self.first, b)


def fgmres(A, b, M, tol=1e-10, m=20, maxit=1000):
    """Flexible GMRES(m) (Saad, Iterative Methods for Sparse Linear Systems, Alg. 9.6), x0 = 0.

    Stops when the residual estimate |g_{j+1}| <= tol ||b|| or after maxit
    iterations; restarts every m iterations from the true residual.
    Returns (x, iterations, true relative residual).
    """
    n = b.shape[0]
    dtype = np.result_type(A.dtype, b.dtype)
    x = np.zeros(n, dtype=dtype)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    its = 0
    while its < maxit:
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            break
        V = np.zeros((n, m + 1), dtype=dtype)
        Z = np.zeros((n, m), dtype=dtype)
        H = np.zeros((m + 1, m), dtype=dtype)
        V[:, 0] = r / beta
        g = np.zeros(m + 1, dtype=dtype)
        g[0] = beta
        cs = np.zeros(m, dtype=dtype)
        sn = np.zeros(m, dtype=dtype)
        j_done = 0
        for j in range(m):
            Z[:, j] = M(V[:, j])
            w = A @ Z[:, j]
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.vdot(V[:, i], w)
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[:, j + 1] = w / H[j + 1, j]
            for i in range(j):                           # earlier Givens rotations
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = np.conj(cs[i]) * hi + np.conj(sn[i]) * hi1
                H[i + 1, j] = -sn[i] * hi + cs[i] * hi1
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            cs[j], sn[j] = (a / den, c / den) if den != 0 else (1.0, 0.0)
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            its += 1
            j_done = j + 1
            if abs(g[j + 1]) <= tol * bnorm or its >= maxit or den == 0:
                break
        y = sla.solve_triangular(H[:j_done, :j_done], g[:j_done])
        x = x + Z[:, :j_done] @ y
    res = np.linalg.norm(b - A @ x) / bnorm
    return x, its, res
