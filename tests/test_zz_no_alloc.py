"""The allocation-free column dots against the allocating entry point.

mlmc_column_dots_noalloc exists for callers that cannot let a library
allocate device memory (an application memory manager that owns the whole
device budget, loops that must not pay an allocator's synchronisation in the
middle of a run).  It must give the same numbers as mlmc_column_dots: both run
the same two kernels in the same summation order, so the bar is bit-equality.
Two calls in a row (different sizes, so the second reuses a shared scratch
array that still holds the first call's partial sums) check that the reuse
is safe.  This file is collected last so that a run stopping at its first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_11281_gb300 import mlmc
    f = mlmc.lib.mlmc_column_dots_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    mlmc.lib.mlmc_noalloc_last_error.restype = ctypes.c_char_p
    return mlmc


@pytest.mark.parametrize("cplx", [False, True])
def test_noalloc_matches_allocating_entry_point(lib, cplx):
    dt = torch.complex128 if cplx else torch.float64
    for call, (n, k) in enumerate([(100003, 64), (777, 5)]):
        g = torch.Generator(device="cuda").manual_seed(10 + call)
        x = torch.randn(n, k, generator=g, device="cuda", dtype=dt)
        y = torch.randn(n, k, generator=g, device="cuda", dtype=dt)
        ref = torch.zeros(k, dtype=dt, device="cuda")
        got = torch.full((k,), float("nan"), dtype=dt, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        lib.column_dots(cplx, x.data_ptr(), y.data_ptr(), n, k, ref.data_ptr(), stream)
        st = lib.lib.mlmc_column_dots_noalloc(int(cplx), x.data_ptr(), y.data_ptr(), n, k, got.data_ptr(), stream)
        assert st == 0, lib.lib.mlmc_noalloc_last_error()
        assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_rejects_too_many_columns(lib):
    x = torch.zeros(10, 257, dtype=torch.float64, device="cuda")
    out = torch.zeros(257, dtype=torch.float64, device="cuda")
    st = lib.lib.mlmc_column_dots_noalloc(0, x.data_ptr(), x.data_ptr(), 10, 257, out.data_ptr(), None)
    assert st == 1 and b"256" in lib.lib.mlmc_noalloc_last_error()
