"""Thin ctypes binding of libmlmc (include/mlmc.h).

Argument marshalling only: every numerical step runs in the CUDA library.
There is no CPU fallback; importing this module fails loudly when the
library has not been built.  Device buffers are passed as raw pointers
(e.g. ``torch.Tensor.data_ptr()``); streams as ``cudaStream_t`` integers.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmlmc.so")

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_OOM, ERR_NOT_CONVERGED, ERR_SINGULAR, \
    ERR_TIMEOUT, ERR_REJECTED = range(9)
OP_LAPLACE2D, OP_WILSON2D = 1, 2
NOISE_RADEMACHER, NOISE_Z4 = 0, 1
PURPOSE_NOISE, PURPOSE_WARMUP, PURPOSE_SETUP = 0, 1, 2
SETUP_SMOOTH, SETUP_INVERSE, SETUP_CONSTANT = 0, 1, 2
PREC_FP64, PREC_MIXED_FP32 = 0, 1
FORM_SIMPLIFIED, FORM_HAT, FORM_PLAIN = 0, 1, 2
CYCLE_V, CYCLE_K = 0, 1
ALLOC_RHO, ALLOC_OPTIMAL, ALLOC_FIXED = 0, 1, 2
COST_COUNTED, COST_NOMINAL = 0, 1
DENSE_SIMT, DENSE_TC, DENSE_TC_WITHHOLD, DENSE_AUTO = 0, 1, 2, 3
CONV_SIMT, CONV_AUTO, CONV_TC = 0, 1, 2
TRANSFER_AGGREGATION, TRANSFER_BILINEAR = 0, 1


class C64(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class OperatorDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("periodic", ctypes.c_int), ("shift", ctypes.c_double), ("mass", ctypes.c_double),
                ("links", ctypes.c_void_p)]


class HierarchyParams(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("agg_x", ctypes.c_int), ("agg_y", ctypes.c_int),
                ("n_tv", ctypes.c_int), ("spin_split", ctypes.c_int), ("setup_kind", ctypes.c_int),
                ("setup_sweeps", ctypes.c_int), ("coarse_sweeps", ctypes.c_int),
                ("setup_omega", ctypes.c_double), ("setup_seed", ctypes.c_uint64),
                ("bootstrap", ctypes.c_int), ("boot_iters", ctypes.c_int),
                ("smooth_pre", ctypes.c_int), ("smooth_post", ctypes.c_int), ("cycle", ctypes.c_int),
                ("kcycle_its", ctypes.c_int), ("fgmres_restart", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("precision", ctypes.c_int), ("block", ctypes.c_int), ("reorth", ctypes.c_int),
                ("inner_its", ctypes.c_int), ("graphs", ctypes.c_int), ("coarse_smooth", ctypes.c_int),
                ("coarse_block", ctypes.c_int), ("user_P", ctypes.c_void_p), ("transfer", ctypes.c_int),
                ("coarse_growth", ctypes.c_int)]


class EstimateParams(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("weights", ctypes.c_double * 16), ("noise", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("tol", ctypes.c_double), ("min_samples", ctypes.c_int),
                ("max_samples", ctypes.c_int), ("form", ctypes.c_int), ("allocation", ctypes.c_int),
                ("n_fixed", ctypes.c_int * 16), ("cost_model", ctypes.c_int), ("tau_separate", ctypes.c_int)]


class EstimateResult(ctypes.Structure):
    _fields_ = [("trace", C64), ("std_err", ctypes.c_double), ("tau", ctypes.c_double),
                ("coarse_term", C64), ("levels", ctypes.c_int), ("n_samples", ctypes.c_int * 16),
                ("mean", C64 * 16), ("variance", ctypes.c_double * 16), ("iters", ctypes.c_double * 16),
                ("seconds", ctypes.c_double * 16), ("cost_nnz", ctypes.c_double * 16),
                ("weights_used", ctypes.c_double * 16), ("seconds_total", ctypes.c_double)]


class TrainParams(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int), ("epochs", ctypes.c_int), ("lr", ctypes.c_double), ("tol", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("init_weights", ctypes.c_void_p), ("enable", ctypes.c_int)]


class TrainReport(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_int), ("blocks", ctypes.c_int), ("epochs", ctypes.c_int), ("enabled", ctypes.c_int),
                ("n_weights", ctypes.c_int), ("loss_first", ctypes.c_double), ("loss_last", ctypes.c_double),
                ("val_loss", ctypes.c_double), ("seconds_capture", ctypes.c_double),
                ("seconds_train", ctypes.c_double)]


class MLMCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libmlmc status %d: %s" % (status, msg))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmlmc.so is not built (run __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, u64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
    sig = {
        "mlmc_setup_hierarchy": [ctypes.POINTER(OperatorDesc), ctypes.POINTER(HierarchyParams), vp,
                                 ctypes.POINTER(vp)],
        "mlmc_level_info": [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)],
        "mlmc_get_prolongation": [vp, i, vp],
        "mlmc_get_operator": [vp, i, vp],
        "mlmc_apply": [vp, i, vp, vp, i],
        "mlmc_solve": [vp, i, vp, vp, i, d, ctypes.POINTER(i)],
        "mlmc_noise": [i, u64, i, i, u64, i, i, i, vp, vp],
        "mlmc_sample_level": [vp, i, i, u64, u64, i, d, ctypes.POINTER(C64), ctypes.POINTER(i)],
        "mlmc_coarse_trace_exact": [vp, ctypes.POINTER(C64)],
        "mlmc_trace_estimate": [vp, ctypes.POINTER(EstimateParams), ctypes.POINTER(EstimateResult)],
        "mlmc_profile_kernel": [vp, i, i, i, i, ctypes.POINTER(d), ctypes.POINTER(d)],
        "mlmc_launch_count": [vp, ctypes.POINTER(u64)],
        "mlmc_learned_train": [vp, ctypes.POINTER(TrainParams), vp, ctypes.POINTER(TrainReport)],
        "mlmc_learned_set": [vp, vp, i],
        "mlmc_learned_apply": [vp, vp, vp, i],
        "mlmc_learned_grad": [vp, vp, i, ctypes.POINTER(d), vp],
        "mlmc_column_dots": [i, vp, vp, i, i, vp, vp],
        "mlmc_set_block_width": [vp, i],
        "mlmc_sample_level_form": [vp, i, i, i, u64, u64, i, d, ctypes.POINTER(C64)],
        "mlmc_autotune_block": [vp, i, i, d, ctypes.POINTER(i), ctypes.POINTER(d)],
        "mlmc_trace_estimate_batch": [ctypes.POINTER(vp), i, ctypes.POINTER(EstimateParams), i,
                                      ctypes.POINTER(EstimateResult), ctypes.POINTER(i)],
        "mlmc_dense_apply": [i, vp, vp, vp, i, i, i, vp],
        "mlmc_level_taps": [vp, i, ctypes.POINTER(i)],
        "mlmc_set_dense_kernel": [vp, i],
        "mlmc_learned_stats": [vp, ctypes.POINTER(i), ctypes.POINTER(i)],
        "mlmc_measure_fma_rate": [i, vp, ctypes.POINTER(d)],
        "mlmc_set_conv_kernel": [vp, i],
        "mlmc_sample_block": [vp, i, i, i, u64, u64, i, d, ctypes.POINTER(C64), ctypes.POINTER(d), ctypes.POINTER(d)],
        "mlmc_nominal_sample_cost": [vp, i, i, ctypes.POINTER(d)],
        "mlmc_block_width": [vp, i, ctypes.POINTER(i)],
        "mlmc_residual_restrict": [vp, i, i, vp, vp, vp, i, i],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.mlmc_destroy_hierarchy.argtypes = [vp]
    lib.mlmc_destroy_hierarchy.restype = None
    lib.mlmc_last_error.argtypes = []
    lib.mlmc_last_error.restype = ctypes.c_char_p
    return lib


lib = _load()
EXPORTED = ["mlmc_setup_hierarchy", "mlmc_destroy_hierarchy", "mlmc_level_info", "mlmc_get_prolongation",
            "mlmc_get_operator", "mlmc_apply", "mlmc_solve", "mlmc_noise", "mlmc_sample_level",
            "mlmc_coarse_trace_exact", "mlmc_trace_estimate", "mlmc_profile_kernel", "mlmc_launch_count",
            "mlmc_last_error", "mlmc_learned_train", "mlmc_learned_set", "mlmc_learned_apply", "mlmc_learned_grad",
            "mlmc_column_dots", "mlmc_column_dots_noalloc", "mlmc_noalloc_last_error", "mlmc_set_block_width",
            "mlmc_autotune_block", "mlmc_trace_estimate_batch", "mlmc_sample_level_form", "mlmc_dense_apply",
            "mlmc_set_dense_kernel", "mlmc_level_taps", "mlmc_learned_stats",
            "mlmc_measure_fma_rate", "mlmc_set_conv_kernel", "mlmc_sample_block", "mlmc_nominal_sample_cost",
            "mlmc_block_width", "mlmc_residual_restrict"]


def check(status):
    if status != OK:
        raise MLMCError(status, lib.mlmc_last_error().decode(errors="replace"))


def default_params(**kw):
    p = HierarchyParams(levels=2, agg_x=4, agg_y=4, n_tv=4, spin_split=0, setup_kind=SETUP_SMOOTH,
                        setup_sweeps=40, coarse_sweeps=20, setup_omega=2.0 / 3.0, setup_seed=0,
                        bootstrap=1, boot_iters=2, smooth_pre=1, smooth_post=1, cycle=CYCLE_K,
                        kcycle_its=2, fgmres_restart=30, max_iter=2000, precision=PREC_FP64, block=64,
                        reorth=1, inner_its=0, graphs=1, coarse_smooth=0, coarse_block=0, user_P=None,
                        transfer=TRANSFER_AGGREGATION, coarse_growth=0)
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Hierarchy:
    """Owner of an mlmc_hierarchy handle (device memory freed on close)."""

    def __init__(self, kind, nx, ny, params, shift=0.0, mass=0.0, links=None, periodic=0, stream=0,
                 user_P=None):
        self._keep = []
        links_ptr = None
        if links is not None:
            arr = np.ascontiguousarray(np.asarray(links, dtype=np.complex128))
            if arr.shape != (2, ny, nx):
                raise ValueError("links must have shape (2, ny, nx)")
            self._keep.append(arr)
            links_ptr = arr.ctypes.data
        if user_P is not None:
            arrs = [np.ascontiguousarray(a) for a in user_P]
            self._keep.extend(arrs)
            ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
            self._keep.append(ptrs)
            params.user_P = ctypes.cast(ptrs, ctypes.c_void_p)
        self.desc = OperatorDesc(kind=kind, nx=nx, ny=ny, periodic=periodic, shift=shift, mass=mass,
                                 links=links_ptr)
        self.params = params
        self.complex = kind == OP_WILSON2D
        self.handle = ctypes.c_void_p()
        check(lib.mlmc_setup_hierarchy(ctypes.byref(self.desc), ctypes.byref(params), ctypes.c_void_p(stream),
                                       ctypes.byref(self.handle)))

    def close(self):
        if self.handle:
            lib.mlmc_destroy_hierarchy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_info(self, level):
        nx, ny, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib.mlmc_level_info(self.handle, level, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(d)))
        return nx.value, ny.value, d.value

    def n(self, level):
        nx, ny, d = self.level_info(level)
        return nx * ny * d

    def prolongation(self, level):
        nx, ny, d = self.level_info(level)
        _, _, dc = self.level_info(level + 1)
        p = self.params
        nagg = (nx // p.agg_x) * (ny // p.agg_y)
        out = np.zeros((nagg, p.agg_x * p.agg_y * d, dc), dtype=np.complex128 if self.complex else np.float64)
        check(lib.mlmc_get_prolongation(self.handle, level, out.ctypes.data))
        return out

    def level_taps(self, level):
        t = ctypes.c_int()
        check(lib.mlmc_level_taps(self.handle, level, ctypes.byref(t)))
        return t.value

    def operator(self, level):
        """[site][tap][d][d]: 5 block taps, or 9 scalar taps on the bilinear coarse levels."""
        nx, ny, d = self.level_info(level)
        out = np.zeros((nx * ny, self.level_taps(level), d, d), dtype=np.complex128 if self.complex else np.float64)
        check(lib.mlmc_get_operator(self.handle, level, out.ctypes.data))
        return out

    def apply(self, level, x_ptr, y_ptr, k):
        check(lib.mlmc_apply(self.handle, level, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), k))

    def solve(self, level, b_ptr, x_ptr, k, tol):
        its = ctypes.c_int()
        check(lib.mlmc_solve(self.handle, level, ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr), k, tol,
                             ctypes.byref(its)))
        return its.value

    def sample_level(self, level, noise, seed, first, n_samples, tol):
        out = (C64 * max(n_samples, 1))()
        # one iteration count per block; a block holds at least one sample, and the
        # library's block width (block, coarse_block, the active width, growth) decides
        its = (ctypes.c_int * max(n_samples, 1))(*([-1] * max(n_samples, 1)))
        check(lib.mlmc_sample_level(self.handle, level, noise, seed, first, n_samples, tol, out, its))
        vals = np.array([complex(out[i].re, out[i].im) for i in range(n_samples)])
        return vals, [v for v in its if v >= 0]

    def sample_level_form(self, level, form, noise, seed, first, n_samples, tol):
        out = (C64 * max(n_samples, 1))()
        check(lib.mlmc_sample_level_form(self.handle, level, form, noise, seed, first, n_samples, tol, out))
        return np.array([complex(out[i].re, out[i].im) for i in range(n_samples)])

    def coarse_trace_exact(self):
        out = C64()
        check(lib.mlmc_coarse_trace_exact(self.handle, ctypes.byref(out)))
        return complex(out.re, out.im)

    def trace_estimate(self, eps=1e-3, noise=NOISE_RADEMACHER, seed=0, tol=1e-10, weights=None, min_samples=5,
                       max_samples=1 << 24, form=FORM_SIMPLIFIED, allocation=ALLOC_RHO, n_fixed=None,
                       cost_model=COST_COUNTED, tau_separate=0):
        p = EstimateParams(eps=eps, noise=noise, seed=seed, tol=tol, min_samples=min_samples,
                           max_samples=max_samples, form=form, allocation=allocation, cost_model=cost_model,
                           tau_separate=tau_separate)
        if n_fixed is not None:
            for i, n in enumerate(n_fixed):
                p.n_fixed[i] = n
        if weights is not None:
            for i, w in enumerate(weights):
                p.weights[i] = w
        r = EstimateResult()
        check(lib.mlmc_trace_estimate(self.handle, ctypes.byref(p), ctypes.byref(r)))
        return r

    def profile_kernel(self, which, level, k, reps):
        ms, by = ctypes.c_double(), ctypes.c_double()
        check(lib.mlmc_profile_kernel(self.handle, which, level, k, reps, ctypes.byref(ms), ctypes.byref(by)))
        return ms.value, by.value

    def net_weights(self):
        c0 = self.level_info(1)[2] * (2 if self.complex else 1)
        return 9 * (16 * c0 + 256 + c0 * 16)

    def learned_train(self, n_pairs=10000, epochs=3, lr=1e-3, tol=1e-8, seed=0, init_weights=None, enable=1):
        w0 = None
        if init_weights is not None:
            w0 = np.ascontiguousarray(init_weights, dtype=np.float32)
        p = TrainParams(n_pairs=n_pairs, epochs=epochs, lr=lr, tol=tol, seed=seed,
                        init_weights=None if w0 is None else w0.ctypes.data, enable=enable)
        out = np.zeros(self.net_weights(), dtype=np.float32)
        rep = TrainReport()
        check(lib.mlmc_learned_train(self.handle, ctypes.byref(p), out.ctypes.data, ctypes.byref(rep)))
        return out, {f: getattr(rep, f) for f, _ in TrainReport._fields_}

    def learned_set(self, weights, enable=1):
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
        check(lib.mlmc_learned_set(self.handle, None if w is None else w.ctypes.data, enable))

    def learned_stats(self):
        """(enabled, fallbacks): whether the network acts in the cycle, and how many level
        solves were repeated without it because they did not converge with it."""
        en, fb = ctypes.c_int(), ctypes.c_int()
        check(lib.mlmc_learned_stats(self.handle, ctypes.byref(en), ctypes.byref(fb)))
        return en.value, fb.value

    def learned_apply(self, r_ptr, e_ptr, k):
        check(lib.mlmc_learned_apply(self.handle, ctypes.c_void_p(r_ptr), ctypes.c_void_p(e_ptr), k))

    def learned_grad(self, r_ptr, k):
        loss = ctypes.c_double()
        g = np.zeros(self.net_weights(), dtype=np.float32)
        check(lib.mlmc_learned_grad(self.handle, ctypes.c_void_p(r_ptr), k, ctypes.byref(loss), g.ctypes.data))
        return loss.value, g

    def set_block_width(self, k):
        check(lib.mlmc_set_block_width(self.handle, k))

    def set_dense_kernel(self, which):
        check(lib.mlmc_set_dense_kernel(self.handle, which))

    def sample_block(self, level, form, noise, seed, first, k, tol):
        """(samples, (N, mean, M2), cost) of one block of level-difference samples."""
        out = (C64 * k)()
        st = (ctypes.c_double * 4)()
        cost = ctypes.c_double()
        check(lib.mlmc_sample_block(self.handle, level, form, noise, seed, first, k, tol, out, st,
                                    ctypes.byref(cost)))
        samples = np.array([complex(v.re, v.im) for v in out])
        return samples, (st[0], complex(st[1], st[2]), st[3]), cost.value

    def residual_restrict(self, level, precision, x_ptr, b_ptr, rc_ptr, k, colour):
        """rc = P_l^* m (b - A_l x), m the sites of `colour` (device pointers)."""
        check(lib.mlmc_residual_restrict(self.handle, level, precision, ctypes.c_void_p(x_ptr), ctypes.c_void_p(b_ptr),
                                         ctypes.c_void_p(rc_ptr), k, colour))

    def nominal_sample_cost(self, level, form=FORM_SIMPLIFIED):
        r = ctypes.c_double()
        check(lib.mlmc_nominal_sample_cost(self.handle, level, form, ctypes.byref(r)))
        return r.value

    def block_width(self, level):
        """Samples per block on level difference `level` (1-based)."""
        r = ctypes.c_int()
        check(lib.mlmc_block_width(self.handle, level, ctypes.byref(r)))
        return r.value

    def set_conv_kernel(self, which):
        check(lib.mlmc_set_conv_kernel(self.handle, which))

    def autotune_block(self, level=1, noise=NOISE_RADEMACHER, tol=1e-8):
        k, t = ctypes.c_int(), ctypes.c_double()
        check(lib.mlmc_autotune_block(self.handle, level, noise, tol, ctypes.byref(k), ctypes.byref(t)))
        return k.value, t.value

    def launch_count(self):
        c = ctypes.c_uint64()
        check(lib.mlmc_launch_count(self.handle, ctypes.byref(c)))
        return c.value


def noise(kind, seed, level, purpose, first, n, k, complex_out, out_ptr, stream=0):
    check(lib.mlmc_noise(kind, seed, level, purpose, first, n, k, complex_out, ctypes.c_void_p(out_ptr),
                         ctypes.c_void_p(stream)))


def column_dots(complex_data, x_ptr, y_ptr, n, k, out_ptr, stream=0):
    check(lib.mlmc_column_dots(int(complex_data), ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), n, k,
                               ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream)))


def dense_apply(complex_data, a_ptr, b_ptr, y_ptr, n, k, which=DENSE_TC, stream=0):
    """Y = A B in FP32 / complex64 on the device (the coarsest-level apply of the FP32 cycle)."""
    check(lib.mlmc_dense_apply(int(complex_data), ctypes.c_void_p(a_ptr), ctypes.c_void_p(b_ptr),
                               ctypes.c_void_p(y_ptr), n, k, which, ctypes.c_void_p(stream)))


def trace_estimate_batch(hierarchies, params, workers=4):
    """mlmc_trace_estimate_batch over Hierarchy objects with one EstimateParams each."""
    n = len(hierarchies)
    hs = (ctypes.c_void_p * n)(*[h.handle.value for h in hierarchies])
    ps = (EstimateParams * n)(*params)
    rs = (EstimateResult * n)()
    st = (ctypes.c_int * n)()
    check(lib.mlmc_trace_estimate_batch(hs, n, ps, workers, rs, st))
    return [result_dict(rs[i]) for i in range(n)], list(st)


def measure_fma_rate(fp64=True, stream=0, add=False, l2=False):
    """Fused multiply-adds (add=True: FP64 additions) per second of the whole GPU, measured;
    l2=True: the L2 bandwidth in bytes per second."""
    r = ctypes.c_double()
    op = 3 if l2 else (2 if add else int(bool(fp64)))
    check(lib.mlmc_measure_fma_rate(op, ctypes.c_void_p(stream or None), ctypes.byref(r)))
    return r.value


def estimate_params(eps=1e-3, noise=NOISE_RADEMACHER, seed=0, tol=1e-8, allocation=ALLOC_OPTIMAL, weights=None,
                    min_samples=5, max_samples=1 << 24, n_fixed=None, cost_model=COST_COUNTED):
    p = EstimateParams(eps=eps, noise=noise, seed=seed, tol=tol, min_samples=min_samples, max_samples=max_samples,
                       form=FORM_SIMPLIFIED, allocation=allocation, cost_model=cost_model)
    if n_fixed is not None:
        for i, n in enumerate(n_fixed):
            p.n_fixed[i] = n
    if weights is not None:
        for i, w in enumerate(weights):
            p.weights[i] = w
    return p


def result_dict(r):
    L = r.levels
    return {
        "trace": complex(r.trace.re, r.trace.im), "std_err": r.std_err, "tau": r.tau,
        "coarse_term": complex(r.coarse_term.re, r.coarse_term.im),
        "n_samples": [r.n_samples[i] for i in range(L - 1)],
        "mean": [complex(r.mean[i].re, r.mean[i].im) for i in range(L - 1)],
        "variance": [r.variance[i] for i in range(L - 1)],
        "iters": [r.iters[i] for i in range(L - 1)],
        "seconds": [r.seconds[i] for i in range(L - 1)],
        "cost_nnz": [r.cost_nnz[i] for i in range(L)],
        "weights_used": [r.weights_used[i] for i in range(L - 1)],
        "seconds_total": r.seconds_total,
    }
