"""GPU learned correction against the FP64 oracle (oracle/learned.py).

The network runs in FP32; forward values are compared to 1e-5 of the output
scale and gradients to 1e-3 of the gradient scale (FP32 sums over 9*16 taps
and all lattice sites)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import learned as NN
from oracle.operators import laplace2d, wilson2d
from paper_2108_11281_gb300.workloads import gauge_links


@pytest.fixture(scope="module")
def mlmc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_11281_gb300 import mlmc as m
    return m


def make(mlmc, case, N=8, k=3):
    if case == "wilson":
        U = gauge_links(N, N, 0.3, 2)
        prm = mlmc.default_params(levels=2, n_tv=2, spin_split=1, setup_kind=mlmc.SETUP_INVERSE, setup_sweeps=4,
                                  setup_omega=1.0, precision=mlmc.PREC_MIXED_FP32, block=k, bootstrap=0)
        h = mlmc.Hierarchy(mlmc.OP_WILSON2D, N, N, prm, mass=0.2, links=U)
        A = wilson2d(N, N, 0.2, U)
        return h, A, 2, True, True
    prm = mlmc.default_params(levels=2, n_tv=1, setup_kind=mlmc.SETUP_CONSTANT, precision=mlmc.PREC_MIXED_FP32,
                              block=k, bootstrap=0)
    h = mlmc.Hierarchy(mlmc.OP_LAPLACE2D, N, N, prm)
    return h, laplace2d(N, N), 1, False, False


def flat(Ws):
    return np.concatenate([W.astype(np.float32).ravel() for W in Ws])


@pytest.mark.parametrize("k", [3, 16])
@pytest.mark.parametrize("case", ["wilson", "laplace"])
def test_forward_and_gradient_match_oracle(mlmc, case, k):
    """k = 3: the CUDA-core convolutions; k = 16: the tensor-core ones (tiles of 8 sites)."""
    N = 8
    h, A, d, cplx, per = make(mlmc, case, N, k)
    h.set_conv_kernel(mlmc.CONV_TC if k == 16 else mlmc.CONV_SIMT)
    c0 = NN.channels_of(d, cplx)
    Ws = [W.astype(np.float32).astype(np.float64) for W in NN.init_weights(c0, 9)]
    h.learned_set(flat(Ws), enable=0)
    n = N * N * d
    g = torch.Generator().manual_seed(0)
    if cplx:
        R = torch.complex(torch.randn(n, k, generator=g), torch.randn(n, k, generator=g)).to(torch.complex64).cuda()
    else:
        R = torch.randn(n, k, generator=g, dtype=torch.float32).cuda()
    E = torch.zeros_like(R)
    h.learned_apply(R.data_ptr(), E.data_ptr(), k)
    Rn = R.cpu().numpy().astype(np.complex128 if cplx else np.float64)
    En = E.cpu().numpy()
    for c in range(k):
        ref, _ = NN.forward(Rn[:, c], Ws, N, N, d, cplx, per)
        assert np.abs(En[:, c] - ref).max() <= 1e-5 * np.abs(ref).max()
    loss, grad = h.learned_grad(R.data_ptr(), k)
    ref_loss, ref_g = NN.loss_and_grad(A, Rn, Ws, N, N, d, cplx, per)
    ref_flat = np.concatenate([x.ravel() for x in ref_g])
    assert abs(loss - ref_loss) <= 1e-4 * abs(ref_loss)
    assert np.abs(grad - ref_flat).max() <= 1e-3 * np.abs(ref_flat).max()
    h.close()


def test_tensor_core_convolutions_match_cuda_cores(mlmc):
    """The tcgen05 implicit-GEMM convolutions (three TF32 products per term) against the
    FP32 CUDA-core kernels on a 32x32 Wilson lattice (periodic) and a 32x32 Dirichlet
    Laplacian, k = 32: the network output to 1e-5 and the loss gradient to 1e-4 of their
    scales (both FP32, summed in different orders)."""
    for case in ("wilson", "laplace"):
        N, k = 32, 32
        h, A, d, cplx, per = make(mlmc, case, N, k)
        c0 = NN.channels_of(d, cplx)
        Ws = [W.astype(np.float32).astype(np.float64) for W in NN.init_weights(c0, 4)]
        h.learned_set(flat(Ws), enable=0)
        n = N * N * d
        g = torch.Generator().manual_seed(1)
        if cplx:
            R = torch.complex(torch.randn(n, k, generator=g), torch.randn(n, k, generator=g)).to(torch.complex64).cuda()
        else:
            R = torch.randn(n, k, generator=g, dtype=torch.float32).cuda()
        out = {}
        for which in (mlmc.CONV_TC, mlmc.CONV_SIMT):
            h.set_conv_kernel(which)
            E = torch.zeros_like(R)
            h.learned_apply(R.data_ptr(), E.data_ptr(), k)
            loss, grad = h.learned_grad(R.data_ptr(), k)
            out[which] = (E.cpu().numpy(), loss, grad)
        (Et, lt, gt), (Es, ls, gs) = out[mlmc.CONV_TC], out[mlmc.CONV_SIMT]
        assert np.abs(Et - Es).max() <= 1e-5 * np.abs(Es).max()
        assert abs(lt - ls) <= 1e-5 * abs(ls)
        assert np.abs(gt - gs).max() <= 1e-4 * np.abs(gs).max()
        h.close()


def wilson32(mlmc, max_iter=2000):
    N, k = 32, 16
    U = gauge_links(N, N, 0.3, 4)
    prm = mlmc.default_params(levels=3, n_tv=2, spin_split=1, setup_kind=mlmc.SETUP_INVERSE, setup_sweeps=8,
                              coarse_sweeps=4, setup_omega=1.0, precision=mlmc.PREC_MIXED_FP32, block=k,
                              smooth_pre=1, smooth_post=1, inner_its=6, fgmres_restart=10, max_iter=max_iter)
    return mlmc.Hierarchy(mlmc.OP_WILSON2D, N, N, prm, mass=0.02, links=U), wilson2d(N, N, 0.02, U), N, k


def solve_checked(h, A, N, k, tol=1e-10, seed=0):
    """Solve a seeded complex block on level 1 and check the FP64 true residual."""
    n = N * N * 2
    g = torch.Generator().manual_seed(seed)
    b = torch.complex(torch.randn(n, k, generator=g, dtype=torch.float64),
                      torch.randn(n, k, generator=g, dtype=torch.float64)).cuda()
    x = torch.zeros_like(b)
    its = h.solve(1, b.data_ptr(), x.data_ptr(), k, tol)
    bn, xn = b.cpu().numpy(), x.cpu().numpy()
    assert (np.linalg.norm(bn - A @ xn, axis=0) / np.linalg.norm(bn, axis=0)).max() <= tol
    return its


def test_training_on_gpu_and_gain(mlmc):
    """Train on residuals captured from plain solves of a 32x32 Wilson operator
    (m = 0.02, one pre- and one post-sweep, inner FGMRES(6)); the network must lower
    its training loss, solves with it must still meet the FP64 tolerance, and on this
    operator it must save outer iterations: fewer with it than without it."""
    h, A, N, k = wilson32(mlmc)
    W, rep = h.learned_train(n_pairs=32 * k, epochs=4, lr=2e-3, tol=1e-6, seed=1, enable=1)
    assert rep["loss_last"] < rep["loss_first"]
    assert np.isfinite(W).all() and rep["n_weights"] == W.size
    assert rep["enabled"] == 1 and h.learned_stats()[0] == 1
    its_net = solve_checked(h, A, N, k)
    h.learned_set(None, enable=0)
    its_plain = solve_checked(h, A, N, k)
    print("learned: val_loss %.3f, outer iterations with net %d, without %d" % (rep["val_loss"], its_net, its_plain))
    assert its_net < its_plain
    assert h.learned_stats() == (0, 0)
    h.close()


def test_learned_fallback_to_plain_smoother(mlmc):
    """The plain smoother is the fallback and the FP64 true residual the judge.  Weights
    scaled up 100-fold make the correction useless: the solve with it does not converge
    within max_iter, is repeated without it (the fallback count rises) and still meets
    the tolerance.  All-zero weights add nothing: the same iterations as the plain cycle."""
    h, A, N, k = wilson32(mlmc, max_iter=40)
    its_plain = solve_checked(h, A, N, k)
    assert its_plain < 40
    nw = h.net_weights()
    rng = np.random.default_rng(3)
    h.learned_set(np.zeros(nw, dtype=np.float32), enable=1)
    assert solve_checked(h, A, N, k) == its_plain
    assert h.learned_stats() == (1, 0)
    h.learned_set((100.0 * rng.standard_normal(nw)).astype(np.float32), enable=1)
    solve_checked(h, A, N, k)
    enabled, fallbacks = h.learned_stats()
    assert enabled == 1 and fallbacks >= 1
    h.close()
