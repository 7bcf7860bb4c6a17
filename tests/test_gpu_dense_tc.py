"""Coarsest-level dense apply on the tensor cores (tcgen05, three TF32 products
per term) against the plain FP64 product, element by element.

The FP32 cycle applies the dense inverse of the coarsest operator (Sec. 4: the
coarsest system is solved directly).  The definition is Y = A B; the check is
the FP32 error bound of a length-n dot product, |Y - AB| <= c n u (|A||B|),
with u = 2^-24, far below the ~2^-11 relative error a single TF32 product
would leave, so a dropped correction term fails it.  Shapes cover several row
tiles, column tiles and K slices, ragged edges (n, k not multiples of the tile,
rows not 16-byte multiples), one-by-one, and the complex (Wilson) embedding.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mlmc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_11281_gb300 import mlmc as m
    return m


def run(mlmc, cplx, n, k, which, seed=0):
    rng = np.random.default_rng(seed)
    if cplx:
        A = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))).astype(np.complex64)
        B = (rng.choice([1, 1j, -1, -1j], size=(n, k))).astype(np.complex64)
    else:
        A = rng.normal(size=(n, n)).astype(np.float32)
        B = rng.normal(size=(n, k)).astype(np.float32)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Yd = torch.full_like(Bd, float("nan"))
    mlmc.dense_apply(cplx, Ad.data_ptr(), Bd.data_ptr(), Yd.data_ptr(), n, k, which,
                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy().astype(np.complex128 if cplx else np.float64)
    A64 = A.astype(np.complex128 if cplx else np.float64)
    B64 = B.astype(np.complex128 if cplx else np.float64)
    ref = A64 @ B64
    scale = np.abs(A64) @ np.abs(B64)
    return Y, ref, scale


SHAPES = [(0, 1024, 64), (0, 1024, 128), (0, 130, 5), (0, 1, 1), (0, 300, 130), (0, 256, 4096 // 16),
          (1, 512, 32), (1, 512, 128), (1, 40, 3), (1, 129, 70)]


@pytest.mark.parametrize("cplx,n,k", SHAPES)
def test_tensor_core_apply_matches_fp64_product(mlmc, cplx, n, k):
    Y, ref, scale = run(mlmc, cplx, n, k, mlmc.DENSE_TC)
    assert np.isfinite(Y).all()
    u = 2.0 ** -24
    bound = 4 * max(np.sqrt(2 * n), 8) * u * scale + 1e-30
    assert (np.abs(Y - ref) <= bound).all(), np.max(np.abs(Y - ref) / (scale + 1e-30))
    # and the product is far more accurate than a single TF32 product could be
    rel = np.max(np.abs(Y - ref) / (scale + 1e-30))
    assert rel < 2.0 ** -16


@pytest.mark.parametrize("cplx,n,k", [(0, 1024, 64), (1, 512, 32), (0, 130, 5)])
def test_cuda_core_apply_matches_fp64_product(mlmc, cplx, n, k):
    Y, ref, scale = run(mlmc, cplx, n, k, mlmc.DENSE_SIMT)
    bound = 4 * max(np.sqrt(2 * n), 8) * 2.0 ** -24 * scale
    assert (np.abs(Y - ref) <= bound).all()


def test_withheld_commit_times_out_and_context_survives(mlmc):
    """The bounded mbarrier wait: with its MMAs withheld the kernel gives up,
    reports MLMC_ERR_TIMEOUT, frees its tensor memory, and the next call works."""
    with pytest.raises(mlmc.MLMCError) as ei:
        run(mlmc, 0, 64, 16, mlmc.DENSE_TC_WITHHOLD)
    assert ei.value.status == mlmc.ERR_TIMEOUT
    Y, ref, scale = run(mlmc, 0, 256, 32, mlmc.DENSE_TC, seed=1)
    assert (np.abs(Y - ref) <= 4 * 32 * 2.0 ** -24 * scale).all()


def test_hierarchy_dense_kernels_agree(mlmc):
    """The same level samples with the coarsest apply on the tensor cores and on
    the CUDA cores: both are preconditioners under the FP64 outer FGMRES, so
    the samples agree to the solve tolerance."""
    from paper_2108_11281_gb300.workloads import gauge_links
    N = 64
    prm = mlmc.default_params(levels=3, n_tv=4, spin_split=1, setup_kind=mlmc.SETUP_INVERSE, setup_sweeps=10,
                              coarse_sweeps=5, setup_omega=1.0, precision=mlmc.PREC_MIXED_FP32, block=16,
                              bootstrap=0)
    h = mlmc.Hierarchy(mlmc.OP_WILSON2D, N, N, prm, mass=0.1, links=gauge_links(N, N, 0.3, 7))
    got, launches, iters = {}, {}, {}
    for which in (mlmc.DENSE_TC, mlmc.DENSE_SIMT):
        h.set_dense_kernel(which)
        n0 = h.launch_count()
        s, its = h.sample_level(2, mlmc.NOISE_Z4, 3, 0, 16, 1e-12)
        launches[which], iters[which], got[which] = h.launch_count() - n0, list(its), s
    a, b = got[mlmc.DENSE_TC], got[mlmc.DENSE_SIMT]
    assert np.abs(a - b).max() <= 1e-8 * np.abs(b).max()
    # the switch reaches the captured inner solves: the tensor-core apply is two
    # launches (products, slice sum), the CUDA-core one a single launch
    if iters[mlmc.DENSE_TC] == iters[mlmc.DENSE_SIMT]:
        assert launches[mlmc.DENSE_TC] > launches[mlmc.DENSE_SIMT]
    ms = {}
    for which in (mlmc.DENSE_TC, mlmc.DENSE_SIMT):
        h.set_dense_kernel(which)
        ms[which], _ = h.profile_kernel(5, 3, 16, 5)
    assert ms[mlmc.DENSE_TC] > 0 and ms[mlmc.DENSE_SIMT] > 0
    h.close()
