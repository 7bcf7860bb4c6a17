"""Learned smoother: a bias-free 3-layer 3x3 convolutional network (FP64 reference).

Oracle (test infrastructure only): imported by tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py``; never by the product path.

The paper has no learned component; this is the project's definition of the
learned correction used inside the multigrid cycle.  With nothing in the paper
to pin it to, it is pinned by mathematics alone: its gradients against central
differences of its loss, and the exact linear special case.

Network: channels c0 -> 16 -> 16 -> c0 with ReLU after the first two layers,
3x3 taps on the lattice (periodic wrap, or zero padding for Dirichlet
lattices), no biases.  The input of a lattice vector u (dofs d per site) is
its real channels per site: [Re u_0, Im u_0, Re u_1, Im u_1, ...] for complex
u, [u_0, ...] for real u; the output maps back the same way.
Weights W[layer] have shape (c_out, c_in, 3, 3); tap (ty, tx) reads the
neighbour at (i + tx - 1, j + ty - 1).

Training objective for a residual r (error e with A e = r):
    loss(r) = || A net(r) - r ||^2 / ||r||^2   (= ||A (net(r) - e)||^2 / ||r||^2),
averaged over the batch.  Optimiser: Adam (Kingma & Ba 2015) with the usual
bias corrections.
"""
import numpy as np

CHANNELS = 16


def channels_of(d, is_complex):
    return d * (2 if is_complex else 1)


def to_channels(u, nx, ny, d, is_complex):
    """Lattice vector (n,) -> array (ny, nx, c)."""
    u = u.reshape(ny, nx, d)
    if not is_complex:
        return u.real.astype(np.float64)
    out = np.empty((ny, nx, 2 * d))
    out[..., 0::2] = u.real
    out[..., 1::2] = u.imag
    return out


def from_channels(a, d, is_complex):
    ny, nx, _ = a.shape
    if not is_complex:
        return a.reshape(-1).copy()
    return (a[..., 0::2] + 1j * a[..., 1::2]).reshape(-1)


def shift(a, tx, ty, periodic):
    """b[j, i] = a[j + ty, i + tx] (wrap or zero outside)."""
    if periodic:
        return np.roll(np.roll(a, -ty, axis=0), -tx, axis=1)
    ny, nx = a.shape[:2]
    b = np.zeros_like(a)
    js = slice(max(0, -ty), min(ny, ny - ty))
    is_ = slice(max(0, -tx), min(nx, nx - tx))
    jd = slice(max(0, ty), min(ny, ny + ty))
    id_ = slice(max(0, tx), min(nx, nx + tx))
    b[js, is_] = a[jd, id_]
    return b


def conv(a, W, periodic):
    """out[j, i, co] = sum_{ty,tx,ci} W[co, ci, ty, tx] a[j + ty - 1, i + tx - 1, ci]."""
    out = np.zeros(a.shape[:2] + (W.shape[0],))
    for ty in range(3):
        for tx in range(3):
            out += shift(a, tx - 1, ty - 1, periodic) @ W[:, :, ty, tx].T
    return out


def conv_backward(a, W, gout, periodic):
    """Gradients of sum(gout * conv(a, W)) with respect to a and W."""
    gW = np.zeros_like(W)
    ga = np.zeros_like(a)
    for ty in range(3):
        for tx in range(3):
            sa = shift(a, tx - 1, ty - 1, periodic)
            gW[:, :, ty, tx] = np.tensordot(gout, sa, axes=([0, 1], [0, 1]))
            # a contributes to out at (j - ty + 1, i - tx + 1): shift gout back
            ga += shift(gout @ W[:, :, ty, tx], -(tx - 1), -(ty - 1), periodic)
    return ga, gW


def forward(u, Ws, nx, ny, d, is_complex, periodic):
    """net(u) and the intermediate activations (input, pre-ReLU values)."""
    a0 = to_channels(u, nx, ny, d, is_complex)
    z1 = conv(a0, Ws[0], periodic)
    a1 = np.maximum(z1, 0.0)
    z2 = conv(a1, Ws[1], periodic)
    a2 = np.maximum(z2, 0.0)
    z3 = conv(a2, Ws[2], periodic)
    return from_channels(z3, d, is_complex), (a0, z1, a1, z2, a2)


def backward(gout_vec, cache, Ws, nx, ny, d, is_complex, periodic):
    """Weight gradients of <gout, net(u)> (real inner product of the channel arrays)."""
    a0, z1, a1, z2, a2 = cache
    g3 = to_channels(gout_vec, nx, ny, d, is_complex)
    ga2, gW3 = conv_backward(a2, Ws[2], g3, periodic)
    gz2 = ga2 * (z2 > 0)
    ga1, gW2 = conv_backward(a1, Ws[1], gz2, periodic)
    gz1 = ga1 * (z1 > 0)
    _, gW1 = conv_backward(a0, Ws[0], gz1, periodic)
    return [gW1, gW2, gW3]


def loss_and_grad(A, R, Ws, nx, ny, d, is_complex, periodic):
    """Mean over the columns r of R of ||A net(r) - r||^2 / ||r||^2, and its weight gradients."""
    total = 0.0
    grads = [np.zeros_like(W) for W in Ws]
    nb = R.shape[1]
    AH = A.conj().T
    for c in range(nb):
        r = R[:, c]
        e, cache = forward(r, Ws, nx, ny, d, is_complex, periodic)
        res = A @ e - r
        nr2 = np.vdot(r, r).real
        total += np.vdot(res, res).real / nr2
        # d/d(e) of |A e - r|^2 in the real sense: 2 A^H (A e - r)
        g = 2.0 * (AH @ res) / nr2
        gs = backward(g, cache, Ws, nx, ny, d, is_complex, periodic)
        for i in range(3):
            grads[i] += gs[i]
    return total / nb, [g / nb for g in grads]


def init_weights(c0, seed, scale=None):
    """He-style normal initial weights from numpy's PCG64 (passed to both sides as data)."""
    rng = np.random.default_rng(seed)
    shapes = [(CHANNELS, c0, 3, 3), (CHANNELS, CHANNELS, 3, 3), (c0, CHANNELS, 3, 3)]
    Ws = []
    for sh in shapes:
        fan_in = sh[1] * 9
        Ws.append(rng.normal(0.0, np.sqrt(2.0 / fan_in) if scale is None else scale, size=sh))
    return Ws


class Adam:
    def __init__(self, Ws, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros_like(W) for W in Ws]
        self.v = [np.zeros_like(W) for W in Ws]
        self.t = 0

    def step(self, Ws, grads):
        self.t += 1
        out = []
        for i, (W, g) in enumerate(zip(Ws, grads)):
            self.m[i] = self.b1 * self.m[i] + (1 - self.b1) * g
            self.v[i] = self.b2 * self.v[i] + (1 - self.b2) * g * g
            mh = self.m[i] / (1 - self.b1 ** self.t)
            vh = self.v[i] / (1 - self.b2 ** self.t)
            out.append(W - self.lr * mh / (np.sqrt(vh) + self.eps))
        return out
