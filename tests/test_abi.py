"""CPU checks of the C-ABI library: it builds, loads, and exports every entry
point include/mlmc.h declares.  No compute call is made (no GPU here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mlmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|const char \*)\s*(mlmc_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_11281_gb300 import mlmc
    lib = ctypes.CDLL(mlmc.LIB_PATH)
    names = declared_functions()
    assert "mlmc_setup_hierarchy" in names and "mlmc_trace_estimate" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(mlmc.EXPORTED)


def test_invalid_arguments_are_rejected_without_a_gpu():
    from paper_2108_11281_gb300 import mlmc
    h = ctypes.c_void_p()
    st = mlmc.lib.mlmc_setup_hierarchy(None, None, None, ctypes.byref(h))
    assert st == mlmc.ERR_INVALID_ARG
    assert b"null" in mlmc.lib.mlmc_last_error()
    desc = mlmc.OperatorDesc(kind=mlmc.OP_LAPLACE2D, nx=30, ny=30)
    prm = mlmc.default_params(levels=3)
    st = mlmc.lib.mlmc_setup_hierarchy(ctypes.byref(desc), ctypes.byref(prm), None, ctypes.byref(h))
    assert st == mlmc.ERR_INVALID_ARG                     # 30 is not divisible by 4 twice
    st = mlmc.lib.mlmc_sample_level(None, 1, 0, 0, 0, 1, 1e-8, None, None)
    assert st == mlmc.ERR_INVALID_ARG
