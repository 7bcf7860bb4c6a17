"""Time-to-trace benchmark of the MLMC trace estimator on one GB300.

A step is one complete Sec. 5 estimate of tr(A^{-1}) to relative accuracy
eps = 1e-3 (exact coarsest term, five warm-up estimates, per-level sampling
until every level meets its standard-error target) on the 1024 x 1024
Dirichlet Laplacian with a 4-level 4x4-aggregation hierarchy (4 smoothed test
vectors per aggregate) and blocks of 64 Rademacher vectors, in the mixed form
(FP32 multigrid cycle under FP64 flexible GMRES).  The hierarchy is built once
before the timed region; `e2e` repeats the step through the C ABI including
the setup from the host-side operator descriptor.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(test infrastructure) on a bounded sample of the same workload instead.
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import ctypes
import json
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# `python -m oracle.tune_mass 256 256 0.4 2 1e-3 --bisect -0.25 -0.20 7`: sigma_min / sigma_max = 1.019e-3
WILSON256_MASS = -0.2417968750

WORKLOADS = {
    # the 1024^2 Dirichlet Laplacian, 4 levels of 4x4 aggregation, 4 smoothed test vectors
    "laplace1024": dict(name="laplace2d-1024x1024-L4-4tv-k64", kind="laplace", nx=1024, ny=1024, levels=4, n_tv=4,
                        spin_split=0, setup="smooth", setup_sweeps=160, coarse_sweeps=20, omega=2.0 / 3.0,
                        bootstrap=2, boot_iters=5, smooth_pre=2, smooth_post=2, kcycle_its=2, restart=8,
                        # blocks of 64 / 128 / 512 on the three level differences (growth 4x beyond the
                        # second: 0.158 s per trace against 0.163 s with 256 on the third)
                        inner_its=8, block=64, coarse_block=128, coarse_growth=2, noise="rademacher", eps=1e-3,
                        tol_fp64=1e-10,
                        tol_mixed=1e-8,
                        # one classical Gram-Schmidt pass in the outer Arnoldi (both forms): the
                        # same iterations and trace as two passes, 1.5-3.5 % less time per trace
                        reorth=0,
                        seed=0, learned=False),
    # the paper's own hierarchy for Example 5.1 (Sec. 5, Table 1): bilinear P, N_{l+1} = (N_l - 1)/2,
    # Galerkin 9-point coarse levels down to N_L = 15; the hat form of the estimator (R P != I)
    "laplace1023bil": dict(name="laplace2d-1023x1023-bilinear-L7-k64", kind="laplace", transfer="bilinear",
                           form="hat", nx=1023, ny=1023, levels=7, n_tv=1, spin_split=0, setup="smooth",
                           setup_sweeps=0, coarse_sweeps=0, omega=2.0 / 3.0, bootstrap=0, boot_iters=0,
                           smooth_pre=1, smooth_post=1, kcycle_its=2, restart=8, inner_its=8, block=64,
                           coarse_block=128, noise="rademacher", eps=1e-3, tol_fp64=1e-10, tol_mixed=1e-8,
                           seed=0, learned=False),
    # the paper's Fig. 5 setting: N = 127, bilinear hierarchy to N_L = 15 (L = 4), blocks of 8
    # samples so that large eps are not held at a 64-sample minimum (the paper's minimum is 5)
    "laplace127bil": dict(name="laplace2d-127x127-bilinear-L4-k8", kind="laplace", transfer="bilinear",
                          form="hat", nx=127, ny=127, levels=4, n_tv=1, spin_split=0, setup="smooth",
                          setup_sweeps=0, coarse_sweeps=0, omega=2.0 / 3.0, bootstrap=0, boot_iters=0,
                          smooth_pre=1, smooth_post=1, kcycle_its=2, restart=8, inner_its=8, block=8,
                          coarse_block=8, noise="rademacher", eps=1e-3, tol_fp64=1e-10, tol_mixed=1e-8,
                          seed=0, learned=False),
    # 2-spin Wilson operator 128^2, theta ~ N(0, 0.3^2), m0 tuned to sigma_min / sigma_max = 1e-3
    "wilson128": dict(name="wilson2d-128x128-L3-8dof-k32", kind="wilson", nx=128, ny=128, levels=3, n_tv=4,
                      spin_split=1, setup="inverse", setup_sweeps=20, coarse_sweeps=10, omega=1.0, bootstrap=4,
                      boot_iters=4, smooth_pre=2, smooth_post=2, kcycle_its=2, restart=10, inner_its=8, block=32,
                      coarse_block=128,
                      noise="z4", eps=1e-3, tol_fp64=1e-10, tol_mixed=1e-8, seed=0, link_sd=0.3, link_seed=1,
                      mass=-0.1317442871, learned=False,
                      # the counted cost model: 0.131 s against 0.144 s per trace with the nominal one
                      cost_model="counted"),
    # 2-spin Wilson operator 256^2, theta ~ N(0, 0.4^2), complex64 cycle with the learned correction
    # trained on 10^4 residual/error pairs from plain multigrid solves (training is setup, not timed)
    "wilson256": dict(name="wilson2d-256x256-L3-8dof-k32-learned", kind="wilson", nx=256, ny=256, levels=3,
                      n_tv=4, spin_split=1, setup="inverse", setup_sweeps=20, coarse_sweeps=10, omega=1.0,
                      bootstrap=4, boot_iters=4, smooth_pre=2, smooth_post=2, kcycle_its=2, restart=10,
                      inner_its=8, block=32, coarse_block=128, noise="z4", eps=1e-3, tol_fp64=1e-10,
                      tol_mixed=1e-8, seed=0, link_sd=0.4, link_seed=2, mass=WILSON256_MASS, learned=True, train_pairs=10000,
                      train_epochs=3, train_lr=1e-3, cost_model="counted"),
}
WORKLOAD = WORKLOADS["laplace1024"]
# ncu DRAM traffic (read + write bytes) per launch unit of the roofline kernel, keyed by
# (workload, kernel row); only for the kernel version the capture was taken on
TRAFFIC = {
    # k_rbgs_half_p<float,4,4> (resident grid, colour 1 from the last row), level 2
    # (256^2 x 4, k = 128), both halves of one sweep after six warm launches, caches kept
    # between launches (ncu --cache-control none, 1 pass each): dram__bytes_read
    # 127.47 + 127.13 MB, dram__bytes_write 69.69 + 67.33 MB
    ("laplace2d-1024x1024-L4-4tv-k64", "rbgs_sweep_fp32_level2"): 391.62e6,
}
METRIC = "Seconds to tr(A^-1) at 1e-3 rel. error, mixed+learned vs plain FP64; HBM %"
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-form", action="store_true")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the config-4 leg (Wilson 256^2 with and without the learned correction)")
    ap.add_argument("--profile-sample", action="store_true",
                    help="for ncu only: after setup, one warm block and one profiled 64-sample block per level "
                         "difference inside cudaProfilerStart/Stop; prints no bench line")
    ap.add_argument("--profile-kernel", default="",
                    choices=["", "multidot", "multiaxpy", "rbgs", "rbgs2", "stencil", "stencil64", "dense", "restrict",
                             "prolong", "restrict2", "prolong2", "rr", "rr2", "rr3", "net", "net_simt"],
                    help="with --profile-sample: instead of sample blocks, the one kernel launch the bench's "
                         "roofline measures (3 warm launches, then 1), inside cudaProfilerStart/Stop")
    ap.add_argument("--profile-step", action="store_true",
                    help="for ncu launch lists only: setup, --warmup estimates, then one estimate inside "
                         "cudaProfilerStart/Stop; prints no bench line")
    ap.add_argument("--profile-nx", type=int, default=0,
                    help="with --profile-sample: lattice side for a smaller capture (default: the workload's)")
    ap.add_argument("--workload", default="laplace1024", choices=sorted(WORKLOADS) + ["batch48"],
                    help="laplace1024 (default, the headline), wilson128, wilson256 (learned correction)")
    ap.add_argument("--eps-sweep", action="store_true",
                    help="MLMC vs plain Hutchinson (Eq. plain_tr_estimate) over eps = 10^-1 .. 10^-3 on the "
                         "workload: seconds, device-counted cost (Sec. 5 model) and N per method; one JSON line")
    ap.add_argument("--alloc", default="optimal", choices=["optimal", "rho"],
                    help="Sec. 2 optimal allocation (default) or the Sec. 5 equal rho split")
    ap.add_argument("--coarse-growth", type=int, default=-1,
                    help="override the workload's block-width growth exponent on coarse level differences")
    ap.add_argument("--set", action="append", default=[], metavar="KEY=INT",
                    help="override an integer workload parameter (smooth_pre, smooth_post, coarse_smooth, "
                         "inner_its, kcycle_its, restart, coarse_block, block)")
    ap.add_argument("--replicas", action="store_true",
                    help="with several GPUs: independent estimates (disjoint seeds) instead of one estimate whose "
                         "samples are spread over the GPUs")
    ap.add_argument("--cost-model", default="", choices=["", "counted", "nominal"],
                    help="per-sample cost C_l of the optimal allocation: products the solves performed "
                         "(counted) or one product per operator solved with (nominal, solver-independent); "
                         "default: the workload's (nominal for the Laplacians, counted for Wilson)")
    return ap.parse_args()


def workload_of(args):
    """The workload named by --workload with the --coarse-growth and --set overrides."""
    w = dict(WORKLOADS[args.workload])
    if args.coarse_growth >= 0:
        w["coarse_growth"] = args.coarse_growth
    for kv in args.set:
        key, val = kv.split("=")
        if key not in ("smooth_pre", "smooth_post", "coarse_smooth", "inner_its", "kcycle_its", "restart",
                       "coarse_block", "block"):
            raise SystemExit("--set: unknown parameter " + key)
        w[key] = int(val)
    return w


def hierarchy_params(mlmc, precision, w=None):
    w = w or WORKLOAD
    kind = {"smooth": mlmc.SETUP_SMOOTH, "inverse": mlmc.SETUP_INVERSE}[w["setup"]]
    return mlmc.default_params(levels=w["levels"], n_tv=w["n_tv"], spin_split=w["spin_split"], setup_kind=kind,
                               setup_sweeps=w["setup_sweeps"], coarse_sweeps=w["coarse_sweeps"],
                               setup_omega=w["omega"], bootstrap=w["bootstrap"], boot_iters=w["boot_iters"],
                               smooth_pre=w["smooth_pre"], smooth_post=w["smooth_post"], cycle=mlmc.CYCLE_K,
                               kcycle_its=w["kcycle_its"], fgmres_restart=w["restart"], max_iter=5000,
                               precision=precision, block=w["block"], reorth=w.get("reorth", 1),
                               inner_its=w["inner_its"],
                               coarse_block=w.get("coarse_block", 0), coarse_growth=w.get("coarse_growth", 0),
                               coarse_smooth=w.get("coarse_smooth", 0),
                               transfer=(mlmc.TRANSFER_BILINEAR if w.get("transfer") == "bilinear"
                                         else mlmc.TRANSFER_AGGREGATION))


def make_hierarchy(mlmc, precision, w, stream=0):
    """Hierarchy of workload w (the Wilson links come from the seeded generator)."""
    prm = hierarchy_params(mlmc, precision, w)
    if w["kind"] == "laplace":
        return mlmc.Hierarchy(mlmc.OP_LAPLACE2D, w["nx"], w["ny"], prm, stream=stream)
    from paper_2108_11281_gb300.workloads import gauge_links
    U = gauge_links(w["nx"], w["ny"], w["link_sd"], w["link_seed"])
    return mlmc.Hierarchy(mlmc.OP_WILSON2D, w["nx"], w["ny"], prm, mass=w["mass"], links=U, stream=stream)


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + CLOCK_FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self, gpu_index=0):
        if not self.proc:
            return None
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != gpu_index:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names[1:], parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d.get("hbm_gbs")), "measured"
        except (ValueError, TypeError):
            pass
    return 6800.0, "fallback"


def host_info():
    """Host cores and CPU model of the machine the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model}


def oracle_levels(w):
    """The oracle's FP64 hierarchy of workload w, built on the host."""
    from oracle.hierarchy import SetupParams, build_hierarchy
    from oracle.operators import laplace2d, wilson2d
    if w.get("transfer") == "bilinear":
        from oracle.bilinear import build_bilinear_hierarchy
        return build_bilinear_hierarchy(w["nx"], w["levels"])
    if w["kind"] == "laplace":
        A, d = laplace2d(w["nx"], w["ny"], w.get("shift", 0.0)), 1
    else:
        from paper_2108_11281_gb300.workloads import gauge_links
        A, d = wilson2d(w["nx"], w["ny"], w["mass"], gauge_links(w["nx"], w["ny"], w["link_sd"], w["link_seed"])), 2
    if w["setup"] == "constant":
        return build_hierarchy(A, w["nx"], w["ny"], d, SetupParams(levels=w["levels"], n_tv=1, kind="constant"))
    return build_hierarchy(A, w["nx"], w["ny"], d, SetupParams(
        levels=w["levels"], n_tv=w["n_tv"], spin_split=bool(w["spin_split"]), kind=w["setup"],
        sweeps=w["setup_sweeps"], coarse_sweeps=w["coarse_sweeps"], omega=w["omega"],
        noise_kind="z4" if w["kind"] == "wilson" else "rademacher", bootstrap=w["bootstrap"],
        boot_iters=w["boot_iters"], smooth_pre=w["smooth_pre"], smooth_post=w["smooth_post"],
        kcycle_its=w["kcycle_its"]))


# per worker process of the oracle pool (spawned: the parent may already hold a CUDA context)
_POOL = {}


def _pool_init(levels, w, tol):
    _POOL.clear()
    _POOL.update(levels=levels, w=w, tol=tol, cycles={})


def _oracle_sample(task):
    """One level-difference sample (simplified form, Remark 4.3) with the oracle's own solver:
    FGMRES(30) preconditioned by one K-cycle (oracle/solver.py) to the workload's tolerance on
    level l, the same on level l+1 or the dense inverse on the coarsest level.  Returns
    (level, sample index, value, seconds); the cycle's set-up is not timed."""
    from oracle.philox import noise
    from oracle.solver import Cycle, dense_inverse, fgmres
    import numpy as np
    l, j, seed = task
    lv, w, tol, cyc = _POOL["levels"], _POOL["w"], _POOL["tol"], _POOL["cycles"]
    L = len(lv)
    for i in (l - 1, l):
        if i not in cyc:
            cyc[i] = dense_inverse(lv[i].A) if i == L - 1 else \
                Cycle(lv, i, w["smooth_pre"], w["smooth_post"], "K", w["kcycle_its"])
    t = time.time()
    x = noise(lv[l - 1].n, w["noise"], seed, l, j)
    y = fgmres(lv[l - 1].A, x, cyc[l - 1], tol=tol, m=30, maxit=5000)[0]
    z = lv[l - 1].P.conj().T @ x
    if l == L - 1:
        v = cyc[l] @ z
    else:
        v = fgmres(lv[l].A, z, cyc[l], tol=tol, m=30, maxit=5000)[0]
    s = np.vdot(x, y) - np.vdot(z, v)
    return l, j, complex(s), time.time() - t


def oracle_pool(levels, w, tol, procs):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(procs, initializer=_pool_init, initargs=(levels, w, tol))


def oracle_plan(w, levels, pool, procs, seed):
    """The oracle's own pilot (Sec. 5 and Sec. 2): samples 0..4 of every level difference,
    computed concurrently on `procs` single-threaded processes, give tau, V_l and the seconds
    per sample; N_l follows from the Sec. 2 optimal allocation with the nominal cost model.
    Nothing here comes from the GPU."""
    import numpy as np
    from oracle import estimator as E
    nd = len(levels) - 1
    t0 = time.time()
    res = pool.map(_oracle_sample, [(l, j, seed) for j in range(5) for l in range(1, nd + 1)], chunksize=1)
    wall = time.time() - t0
    TL = E.exact_coarse_trace(levels).real
    vals = {l: [r[2] for r in res if r[0] == l] for l in range(1, nd + 1)}
    secs = {l: [r[3] for r in res if r[0] == l] for l in range(1, nd + 1)}
    t_est = np.array([TL + sum(vals[l][i] for l in vals).real for i in range(5)])
    tau = t_est.mean() - np.sqrt(np.mean((t_est - t_est.mean()) ** 2))
    V = [float(np.var(np.array(vals[l]), ddof=1)) for l in range(1, nd + 1)]
    C = [E.nominal_sample_cost(levels, l) for l in range(1, nd + 1)]
    _, counts, _ = E.optimal_allocation(V, C, w["eps"] * abs(tau))
    return {"tau": float(tau), "variance": V, "n_samples": counts,
            "sec_per_sample": [float(np.mean(secs[l])) for l in range(1, nd + 1)],
            "pilot_wall_s": wall, "pilot_samples": 5 * nd, "procs": procs}


def trace_seconds(plan):
    """Seconds to trace: sum_l N_l x seconds per sample; the samples are independent, so
    `procs` processes share them (per-sample times were measured with all of them busy)."""
    one = sum(n * t for n, t in zip(plan["n_samples"], plan["sec_per_sample"]))
    return one, one / plan["procs"]


def config1_oracle(procs):
    """Config 1 end to end with the oracle (measured, not extrapolated): 64^2 Dirichlet
    Laplacian, 2 levels, piecewise-constant P, 1000 Rademacher samples (seed 0) at level 1,
    tol 1e-10, plus the exact coarse term; once on one process, once on `procs`."""
    import numpy as np
    from oracle import estimator as E
    w1 = dict(WORKLOADS["laplace1024"], nx=64, ny=64, levels=2, setup="constant", smooth_pre=1, smooth_post=1)
    t0 = time.time()
    lv = oracle_levels(w1)
    tasks = [(1, j, 0) for j in range(1000)]
    _pool_init(lv, w1, 1e-10)
    vals = [_oracle_sample(tk)[2] for tk in tasks]
    one = time.time() - t0
    pool = oracle_pool(lv, w1, 1e-10, procs)
    try:
        pool.map(_oracle_sample, tasks[:procs], chunksize=1)          # workers up and warm
        t0 = time.time()
        par = pool.map(_oracle_sample, tasks, chunksize=8)
        allc = time.time() - t0
    finally:
        pool.close()
        pool.join()
    trace = E.exact_coarse_trace(lv).real + float(np.mean(np.array(vals).real))
    assert all(a[2] == b for a, b in zip(par, vals))      # the same samples on one and on many processes
    return {"workload": "laplace2d-64x64-L2-constP-1000samples", "seconds_1core": one, "seconds_all_cores": allc,
            "procs": procs, "trace": trace, "closed_form": closed_form(w1), "measured": True}


def cpu_baseline(w):
    """The FP64 oracle (as it stands) on the host cores, with nothing taken from the GPU run:
    its own hierarchy, its own pilot (five samples per level difference, concurrently on all
    cores), N_l from its own variances (Sec. 2 allocation, nominal costs), seconds to trace
    extrapolated as sum N_l x seconds per sample; and config 1 measured end to end."""
    procs = max(1, min(os.cpu_count() or 1, 16))
    t0 = time.time()
    lv = oracle_levels(w)
    setup_s = time.time() - t0
    pool = oracle_pool(lv, w, w["tol_mixed"], procs)
    try:
        plan = oracle_plan(w, lv, pool, procs, w["seed"])
    finally:
        pool.close()
        pool.join()
    one, allc = trace_seconds(plan)
    cfg1 = config1_oracle(procs)
    return {"value": allc, "unit": "s (extrapolated)", "cores": procs, "kind": "oracle",
            "single_core_s": one, "setup_s": setup_s, "plan": plan, "host": host_info(),
            "config1_end_to_end": cfg1,
            "sample": "oracle FP64 FGMRES(30)+K-cycle at tol %g: its own hierarchy (setup %.1f s, excluded), "
                      "samples 0..4 of each level difference on %d processes (%.1f s wall); N_l %s from its "
                      "own pilot (Sec. 2, nominal costs); value = sum N_l x s/sample / %d processes" %
                      (w["tol_mixed"], setup_s, procs, plan["pilot_wall_s"], plan["n_samples"], procs)}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, on the machine's host cores.  Setup:
    the oracle's hierarchy and its own pilot (N_l, seconds per sample).  Each step is a bounded
    sample of the workload: one level difference in rotation, one sample per process
    concurrently; the step's value is the seconds to trace with that level's per-sample time
    re-measured (the other levels' from their latest measurement)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    procs = max(1, min(os.cpu_count() or 1, 16))
    lv = oracle_levels(w)
    pool = oracle_pool(lv, w, w["tol_mixed"], procs)
    steps = []
    try:
        plan = oracle_plan(w, lv, pool, procs, w["seed"])
        nd = len(lv) - 1
        nxt = 5
        for i in range(args.warmup + args.steps):
            l = 1 + i % nd
            res = pool.map(_oracle_sample, [(l, nxt + q, w["seed"]) for q in range(procs)], chunksize=1)
            nxt += procs
            plan["sec_per_sample"][l - 1] = sum(r[3] for r in res) / len(res)
            if i >= args.warmup:
                steps.append(trace_seconds(plan)[1])
    finally:
        pool.close()
        pool.join()
    v = statistics.mean(steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w, args.alloc), "form": "FP64 CPU oracle (FGMRES + K-cycle)",
            "cpu_baseline": {"value": v, "unit": "s (extrapolated)", "kind": "oracle", "cores": procs,
                             "host": host_info(), "n_samples": plan["n_samples"],
                             "sample": "oracle FP64 FGMRES(30)+K-cycle at tol %g; N_l %s from its own 5-sample "
                                       "pilot (Sec. 2, nominal costs); each step re-times one level "
                                       "difference (one sample on each of %d processes); value = sum N_l x "
                                       "s/sample / %d" % (w["tol_mixed"], plan["n_samples"], procs, procs)},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(w, alloc="optimal"):
    """The workload, identical for both arms (the implementation is named in `form`)."""
    blk = w["nx"] * w["ny"] * (2 if w["kind"] == "wilson" else 1) * w["block"] * (16 if w["kind"] == "wilson" else 8)
    return {"workload": w["name"], "nx": w["nx"], "ny": w["ny"], "levels": w["levels"],
            "n_tv": w["n_tv"], "block": w["block"], "eps": w["eps"], "noise": w["noise"],
            "outer_gram_schmidt_passes": 2 if w.get("reorth", 1) else 1,
            "allocation": alloc,
            "l2": ("inputs larger than L2 (a level-1 block is %d MiB in FP64)" % (blk >> 20)) if blk > 130e6 else
                  ("level-1 block %d MiB: L2-resident working set, no flush" % (blk >> 20))}


def profile_sample(args):
    """One block per level difference inside cudaProfilerStart/Stop (ncu launch lists / captures)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_11281_gb300 import mlmc
    w = workload_of(args)
    if args.profile_nx:
        w["nx"] = w["ny"] = args.profile_nx
    nz = mlmc.NOISE_Z4 if w["noise"] == "z4" else mlmc.NOISE_RADEMACHER
    h = make_hierarchy(mlmc, mlmc.PREC_MIXED_FP32, w, torch.cuda.current_stream().cuda_stream)
    if args.profile_kernel:
        which = {"stencil": 1, "stencil64": 0, "rbgs": 2, "rbgs2": 2, "multidot": 3, "multiaxpy": 4, "dense": 5,
                 "restrict": 6, "restrict2": 6, "prolong": 7, "prolong2": 7, "net": 8,
                 "net_simt": 8, "rr": 9, "rr2": 9, "rr3": 9}[args.profile_kernel]
        level, kk = 1, w["block"]
        if which == 5:
            level, kk = w["levels"], w.get("coarse_block") or w["block"]
        elif args.profile_kernel in ("rbgs2", "restrict2", "prolong2", "rr2"):
            level, kk = 2, w.get("coarse_block") or w["block"]
        elif args.profile_kernel == "rr3":
            level, kk = 3, w.get("coarse_block") or w["block"]
        if which == 8:
            h.set_conv_kernel(mlmc.CONV_SIMT if args.profile_kernel == "net_simt" else mlmc.CONV_TC)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        h.profile_kernel(which, level, kk, 1)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        h.close()
        return
    form = mlmc.FORM_HAT if w.get("form") == "hat" else mlmc.FORM_SIMPLIFIED
    for lvl in range(1, w["levels"]):
        h.sample_level_form(lvl, form, nz, 0, 0, w["block"], w["tol_mixed"])
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for lvl in range(1, w["levels"]):
        h.sample_level_form(lvl, form, nz, 0, w["block"], w["block"], w["tol_mixed"])
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    h.close()


def replica_seed(base_seed, rank):
    """Replicas draw disjoint noise: replica r uses seed base + 1000 r (Philox key)."""
    return base_seed + 1000 * rank


def max_over_ranks(t, device="cuda"):
    """The job's time per step is the slowest replica's: all-reduce MAX over the process
    group (the identity for one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(t_step_max, world):
    """Whole-job metric: seconds per trace when `world` replicas estimate concurrently."""
    return t_step_max / world


def profile_step(args):
    """One estimate of the workload inside cudaProfilerStart/Stop, after setup and --warmup
    estimates (the launch list of exactly what one timed bench step runs)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_11281_gb300 import mlmc
    w = WORKLOADS[args.workload]
    nz = mlmc.NOISE_Z4 if w["noise"] == "z4" else mlmc.NOISE_RADEMACHER
    form = mlmc.FORM_HAT if w.get("form") == "hat" else mlmc.FORM_SIMPLIFIED
    h = make_hierarchy(mlmc, mlmc.PREC_MIXED_FP32, w, torch.cuda.current_stream().cuda_stream)
    for _ in range(args.warmup):
        h.trace_estimate(eps=w["eps"], noise=nz, seed=w["seed"], tol=w["tol_mixed"], form=form,
                         allocation=mlmc.ALLOC_OPTIMAL)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    h.trace_estimate(eps=w["eps"], noise=nz, seed=w["seed"], tol=w["tol_mixed"], form=form,
                     allocation=mlmc.ALLOC_OPTIMAL)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    h.close()


def eps_sweep(args):
    """Time-to-trace and arithmetic cost of MLMC (simplified form, Sec. 2 optimal allocation) and
    of plain Hutchinson on the fine operator, for eps = 10^-1, 10^-1.5, ..., 10^-3 (the study of
    the paper's Fig. 5 and Sec. 5 cost model), on one GPU with the same solver, noise and seed."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_11281_gb300 import mlmc
    w = WORKLOADS[args.workload]
    nz = mlmc.NOISE_Z4 if w["noise"] == "z4" else mlmc.NOISE_RADEMACHER
    h = make_hierarchy(mlmc, mlmc.PREC_MIXED_FP32, w, torch.cuda.current_stream().cuda_stream)
    rows = []
    for e in (1.0, 1.5, 2.0, 2.5, 3.0):
        eps = 10.0 ** -e
        row = {"eps": eps}
        mlmc_form = mlmc.FORM_HAT if w.get("form") == "hat" else mlmc.FORM_SIMPLIFIED
        for name, form in (("mlmc", mlmc_form), ("plain", mlmc.FORM_PLAIN)):
            torch.cuda.synchronize()
            t = time.time()
            r = mlmc.result_dict(h.trace_estimate(eps=eps, noise=nz, seed=w["seed"], tol=w["tol_mixed"],
                                                  form=form, allocation=mlmc.ALLOC_OPTIMAL))
            torch.cuda.synchronize()
            row[name] = {"seconds": time.time() - t, "trace": r["trace"].real, "std_err": r["std_err"],
                         "n_samples": r["n_samples"], "cost_nnz": float(sum(r["cost_nnz"]))}
        row["cost_ratio_plain_over_mlmc"] = row["plain"]["cost_nnz"] / row["mlmc"]["cost_nnz"]
        row["time_ratio_plain_over_mlmc"] = row["plain"]["seconds"] / row["mlmc"]["seconds"]
        rows.append(row)
    h.close()
    print(json.dumps({"eps_sweep": rows, "workload": w["name"], "closed_form": closed_form(w),
                      "form": "mixed: FP32 K-cycle under FP64 FGMRES", "allocation": "optimal"}), flush=True)


def batch_instances(seed=2026):
    """48 uneven instances (seeded): 24 shifted Dirichlet Laplacians, sides 256..2048,
    shift ~ U[1e-4, 1e-1]; 24 Wilson operators, sides 64..256, theta ~ N(0, 0.3^2),
    mass -0.10 (above the critical mass, about -0.14 at this link spread); per level
    difference a sample budget ~ U{16..128}."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for i in range(48):
        lap = i < 24
        side = int(rng.choice([256, 512, 1024, 2048] if lap else [64, 128, 256]))
        levels = 1
        s_ = side
        while s_ > 16 and s_ % 4 == 0 and (s_ // 4) >= 2:
            s_ //= 4
            levels += 1
        if levels < 2:
            levels = 2
        inst = dict(kind="laplace" if lap else "wilson", side=side, levels=levels, index=i,
                    n_fixed=[int(rng.integers(16, 129)) for _ in range(levels - 1)])
        if lap:
            inst["shift"] = float(rng.uniform(1e-4, 1e-1))
        else:
            inst["link_seed"] = 100 + i
        out.append(inst)
    return out


def run_batch(args):
    """Config 5: the 48 instances through a pool of worker threads; each worker builds the
    hierarchy (mixed form), autotunes the block width, runs the fixed-budget estimate and
    frees the hierarchy.  Value: seconds for the whole batch."""
    import threading
    from concurrent.futures import ThreadPoolExecutor
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_11281_gb300 import mlmc
    from paper_2108_11281_gb300.workloads import gauge_links
    insts = batch_instances()
    base = WORKLOADS["laplace1024"]
    wb = WORKLOADS["wilson128"]
    tuned = {}                 # (kind, side) -> block width chosen by the autotuner
    tuned_lock = threading.Lock()

    def one(inst):
        t0 = time.time()
        if inst["kind"] == "laplace":
            # no width growth on the coarse differences: the setup's 32-bit indexing bound
            # counts the widest block on the fine level (hat-form noise), and the 2048^2
            # instances reach it with 512 columns
            w = dict(base, nx=inst["side"], ny=inst["side"], levels=inst["levels"], coarse_growth=0)
            w["block"] = 128 if inst["side"] <= 512 else (64 if inst["side"] <= 1024 else 32)
            prm = hierarchy_params(mlmc, mlmc.PREC_MIXED_FP32, w)
            h = mlmc.Hierarchy(mlmc.OP_LAPLACE2D, inst["side"], inst["side"], prm, shift=inst["shift"])
            nz = mlmc.NOISE_RADEMACHER
        else:
            w = dict(wb, nx=inst["side"], ny=inst["side"], levels=inst["levels"], block=128)
            prm = hierarchy_params(mlmc, mlmc.PREC_MIXED_FP32, w)
            U = gauge_links(inst["side"], inst["side"], 0.3, inst["link_seed"])
            h = mlmc.Hierarchy(mlmc.OP_WILSON2D, inst["side"], inst["side"], prm, mass=-0.10, links=U)
            nz = mlmc.NOISE_Z4
        t_setup = time.time() - t0
        # the autotuner runs once per (operator kind, lattice side); the other instances of
        # that class reuse its choice
        key = (inst["kind"], inst["side"])
        with tuned_lock:
            k = tuned.get(key)
        if k is None:
            k, _ = h.autotune_block(1, nz, 1e-8)
            with tuned_lock:
                tuned[key] = k
        else:
            h.set_block_width(k)
        t1 = time.time()
        r = mlmc.result_dict(h.trace_estimate(noise=nz, seed=inst["index"], tol=1e-8, allocation=mlmc.ALLOC_FIXED,
                                              n_fixed=inst["n_fixed"]))
        t_est = time.time() - t1
        launches = h.launch_count()
        h.close()
        return dict(index=inst["index"], kind=inst["kind"], side=inst["side"], block=k, setup_s=t_setup,
                    estimate_s=t_est, total_s=time.time() - t0, trace=r["trace"].real, std_err=r["std_err"],
                    n_samples=r["n_samples"], launches=launches)

    workers = 4
    for _ in range(args.warmup if args.warmup < 1 else 1):
        one(insts[0])
    torch.cuda.synchronize()
    t0 = time.time()
    with ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(one, insts))
    torch.cuda.synchronize()
    wall = time.time() - t0
    # roofline: the level-2 block Gauss-Seidel sweep (the headline's dominant kernel family) on a
    # 1024^2 Laplace instance of the batch, timed alone with CUDA events
    peak, peak_kind = measured_peaks()
    w = dict(base, nx=1024, ny=1024, levels=4, block=128)
    hp = mlmc.Hierarchy(mlmc.OP_LAPLACE2D, 1024, 1024, hierarchy_params(mlmc, mlmc.PREC_MIXED_FP32, w), shift=1e-2)
    kern = {}
    for name, which, lvl in (("rbgs_sweep_fp32_level1", 2, 1), ("rbgs_sweep_fp32_level2", 2, 2),
                             ("stencil_fp32_level2", 1, 2), ("restrict_fp32_level1", 6, 1)):
        kms, kbytes = hp.profile_kernel(which, lvl, 128, 20)
        kern[name] = {"ms": kms, "bytes": kbytes, "gbs": kbytes / kms / 1e6, "k": 128}
    hp.close()
    dom = kern["rbgs_sweep_fp32_level2"]
    roofline = {"bound": "hbm", "kernel": "k_rbgs_half_p (level-2 block GS of a 1024^2 instance, k=128, one sweep)",
                "achieved": dom["gbs"], "peak": peak, "unit": "GB/s", "frac": dom["gbs"] / peak,
                "peak_source": peak_kind, "traffic": None, "algorithmic_bytes": dom["bytes"], "kernels": kern}
    cpu = None if args.no_cpu_baseline else batch_cpu_baseline(insts)
    h2d = sum(2 * r["side"] * r["side"] * 16 for r in res if r["kind"] == "wilson")
    line = {"metric": METRIC, "value": wall, "unit": "s (48-instance batch)", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": wall * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64/f32", "data": "synthetic",
            "config": {"workload": "batch48-uneven", "workers": workers, "instances": len(insts),
                       "allocation": "fixed budget per level ~ U{16..128}", "form": "mixed"},
            "e2e": {"value": wall, "unit": "s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": len(insts) * ctypes.sizeof(mlmc.EstimateResult),
                    "includes": "every instance's setup from its host descriptor (links copied in), block-width "
                                "autotuning, the estimate and the result read-back"},
            "roofline": roofline, "cpu_baseline": cpu,
            "instances_per_s": len(insts) / wall, "gpu_launches": int(sum(r["launches"] for r in res)),
            "sum_instance_seconds": sum(r["total_s"] for r in res), "instances": res}
    print(json.dumps(line), flush=True)


def batch_cpu_baseline(insts):
    """The oracle on a bounded sample of the batch: per (kind, side) class up to 512^2 sites it
    builds the class's oracle hierarchy and times samples 0..4 of every level difference on all
    host cores (single-threaded processes); larger classes are scaled from the largest timed
    class of their kind by the number of unknowns.  Seconds for the batch = sum over instances
    and levels of n_fixed x seconds per sample, shared by the processes (extrapolated)."""
    procs = max(1, min(os.cpu_count() or 1, 16))
    per_class = {}
    t0 = time.time()
    for kind in ("wilson", "laplace"):
        sides = sorted({i["side"] for i in insts if i["kind"] == kind})
        timed = [sd for sd in sides if sd <= 512][:2]
        for sd in timed:
            inst = next(i for i in insts if i["kind"] == kind and i["side"] == sd)
            if kind == "laplace":
                w = dict(WORKLOADS["laplace1024"], nx=sd, ny=sd, levels=inst["levels"], shift=inst["shift"])
            else:
                w = dict(WORKLOADS["wilson128"], nx=sd, ny=sd, levels=inst["levels"], mass=-0.10,
                         link_seed=inst["link_seed"])
            lv = oracle_levels(w)
            pool = oracle_pool(lv, w, 1e-8, procs)
            try:
                plan = oracle_plan(w, lv, pool, procs, 0)
            finally:
                pool.close()
                pool.join()
            per_class[(kind, sd)] = plan["sec_per_sample"]
    total = 0.0
    for inst in insts:
        key = (inst["kind"], inst["side"])
        if key in per_class:
            sec = per_class[key]
        else:
            ref = max(sd for (kd, sd) in per_class if kd == inst["kind"])
            scale = (inst["side"] / ref) ** 2
            sec = [v * scale for v in per_class[(inst["kind"], ref)]]
            sec += [sec[-1]] * (len(inst["n_fixed"]) - len(sec))
        total += sum(n * t for n, t in zip(inst["n_fixed"], sec))
    return {"value": total / procs, "unit": "s (extrapolated)", "cores": procs, "kind": "oracle",
            "single_core_s": total, "host": host_info(), "timed_classes": sorted("%s%d" % k for k in per_class),
            "seconds_measuring": time.time() - t0,
            "sample": "oracle FP64 FGMRES(30)+K-cycle at tol 1e-8, samples 0..4 per level difference of one "
                      "instance per class up to 512^2 sites on %d processes; larger classes scaled by unknowns; "
                      "value = sum n_fixed x s/sample / %d" % (procs, procs)}


def learned_leg(mlmc, stream, warmup, steps, seed=0):
    """Config 4: Wilson 256^2 (theta ~ N(0, 0.4^2)), mixed form, with the learned correction
    trained on the GPU (10^4 residual/error pairs from plain solves; training is setup) and
    without it (plain multigrid smoother), the same warm-up and number of estimates timed
    between CUDA events for both."""
    import torch
    w = WORKLOADS["wilson256"]
    nz = mlmc.NOISE_Z4
    cm = mlmc.COST_COUNTED if w.get("cost_model") == "counted" else mlmc.COST_NOMINAL
    t0 = time.time()
    h = make_hierarchy(mlmc, mlmc.PREC_MIXED_FP32, w, stream)
    setup_s = time.time() - t0
    t0 = time.time()
    _, rep = h.learned_train(n_pairs=w["train_pairs"], epochs=w["train_epochs"], lr=w["train_lr"],
                             tol=w["tol_mixed"], seed=7, enable=1)
    train_s = time.time() - t0

    def timed():
        for _ in range(warmup):
            h.trace_estimate(eps=w["eps"], noise=nz, seed=seed, tol=w["tol_mixed"], allocation=mlmc.ALLOC_OPTIMAL,
                             cost_model=cm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            r = mlmc.result_dict(h.trace_estimate(eps=w["eps"], noise=nz, seed=seed, tol=w["tol_mixed"],
                                                  allocation=mlmc.ALLOC_OPTIMAL, cost_model=cm))
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps, r

    # the network alone on a fine-level block: tensor-core vs CUDA-core convolutions
    kern = {}
    c0 = 4
    flops = 2.0 * 9 * (16 * c0 + 256 + 16 * c0) * w["nx"] * w["ny"] * w["block"]
    for name, which in (("net_forward_tc", mlmc.CONV_TC), ("net_forward_simt", mlmc.CONV_SIMT)):
        h.set_conv_kernel(which)
        kms, kbytes = h.profile_kernel(8, 1, w["block"], 20)
        kern[name] = {"ms": kms, "bytes": kbytes, "gbs": kbytes / kms / 1e6, "tflops": flops / kms / 1e9}
    h.set_conv_kernel(mlmc.CONV_AUTO)
    net_on = h.learned_stats()[0]
    t_net, r_net = timed()
    fallbacks = h.learned_stats()[1]
    h.learned_set(None, enable=0)
    t_plain, r_plain = timed()
    h.close()
    return {"workload": w["name"], "train": dict(rep, seconds_total=train_s), "setup_s": setup_s,
            "net_enabled": net_on, "fallbacks": fallbacks,
            "with_net_s": t_net, "plain_s": t_plain, "speedup_plain_over_net": t_plain / t_net,
            "with_net_iters": r_net["iters"], "plain_iters": r_plain["iters"],
            "with_net_n_samples": r_net["n_samples"], "plain_n_samples": r_plain["n_samples"],
            "trace_with_net": r_net["trace"].real, "trace_plain": r_plain["trace"].real,
            "std_err": r_plain["std_err"], "steps": steps, "warmup": warmup, "kernels": kern}


def gpu_config1(mlmc, stream, warmup, steps=3):
    """Config 1 on the GPU, FP64 form: 64^2 Dirichlet Laplacian, 2 levels, piecewise-constant
    P, exactly 1000 Rademacher samples (seed 0) at level 1 in blocks of 200, tol 1e-10, plus
    the exact coarse term; setup outside, estimates between CUDA events after warm-up."""
    import torch
    prm = mlmc.default_params(levels=2, n_tv=1, setup_kind=mlmc.SETUP_CONSTANT, bootstrap=0,
                              precision=mlmc.PREC_FP64, block=200, smooth_pre=1, smooth_post=1)
    t0 = time.time()
    h = mlmc.Hierarchy(mlmc.OP_LAPLACE2D, 64, 64, prm, stream=stream)
    setup_s = time.time() - t0

    def one():
        return mlmc.result_dict(h.trace_estimate(noise=mlmc.NOISE_RADEMACHER, seed=0, tol=1e-10,
                                                 allocation=mlmc.ALLOC_FIXED, n_fixed=[1000]))
    for _ in range(max(1, warmup)):
        one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        r = one()
    e1.record()
    torch.cuda.synchronize()
    h.close()
    cf = closed_form(dict(kind="laplace", nx=64, ny=64))
    return {"workload": "laplace2d-64x64-L2-constP-1000samples", "form": "fp64", "seconds": e0.elapsed_time(e1) / 1e3 / steps,
            "setup_s": setup_s, "trace": r["trace"].real, "std_err": r["std_err"], "closed_form": cf,
            "n_samples": r["n_samples"], "within_4se": abs(r["trace"].real - cf) <= 4 * r["std_err"]}


def closed_form(w):
    """Example 5.1: tr(A^{-1}) = sum over the eigenvalues 4 + shift - 2cos(i pi/(N+1)) - 2cos(j pi/(N+1))
    (Dirichlet Laplacian; None for other operators)."""
    if w["kind"] != "laplace":
        return None
    import numpy as np
    cx = 2 * np.cos(np.arange(1, w["nx"] + 1) * np.pi / (w["nx"] + 1))
    cy = 2 * np.cos(np.arange(1, w["ny"] + 1) * np.pi / (w["ny"] + 1))
    return float(np.sum(1.0 / (4.0 + w.get("shift", 0.0) - cy[:, None] - cx[None, :])))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch48":
        run_batch(args)
        return
    if args.profile_sample:
        profile_sample(args)
        return
    if args.eps_sweep:
        eps_sweep(args)
        return
    if args.profile_step:
        profile_step(args)
        return
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_11281_gb300 import mlmc
    w = workload_of(args)
    nz = mlmc.NOISE_Z4 if w["noise"] == "z4" else mlmc.NOISE_RADEMACHER
    stream = torch.cuda.current_stream().cuda_stream
    h = make_hierarchy(mlmc, mlmc.PREC_MIXED_FP32, w, stream)

    alloc = mlmc.ALLOC_OPTIMAL if args.alloc == "optimal" else mlmc.ALLOC_RHO

    form = mlmc.FORM_HAT if w.get("form") == "hat" else mlmc.FORM_SIMPLIFIED

    if not args.cost_model:
        args.cost_model = w.get("cost_model", "nominal")
    cost_model = mlmc.COST_NOMINAL if args.cost_model == "nominal" else mlmc.COST_COUNTED

    def step(hh, tol, seed):
        return mlmc.result_dict(hh.trace_estimate(eps=w["eps"], noise=nz, seed=seed, tol=tol,
                                                  allocation=alloc, form=form, cost_model=cost_model))

    if world > 1 and not args.replicas:
        # one estimate over all ranks: disjoint blocks of one sample stream per rank, block
        # statistics all-gathered over NCCL after every round (sharded.py); nominal costs
        from paper_2108_11281_gb300 import sharded
        gather = sharded.torch_allgather("cuda")
        serial_step = step

        def step(hh, tol, seed):
            if hh is not h:
                return serial_step(hh, tol, seed)
            smp = sharded.HierarchySampler(hh, nz, w["seed"], tol, form)
            r = sharded.sharded_trace_estimate(smp, gather, rank, world, eps=w["eps"],
                                               allocation="optimal" if args.alloc == "optimal" else "rho")
            r.update(trace=complex(r["trace"]), coarse_term=complex(r["coarse_term"]),
                     iters=None, seconds=None, cost_nnz=None)
            return r

    if w.get("learned"):
        h.learned_train(n_pairs=w["train_pairs"], epochs=w["train_epochs"], lr=w["train_lr"],
                        tol=w["tol_mixed"], seed=7, enable=1)
    # replicas (--replicas) draw disjoint noise; the sharded estimate shares one stream
    seed = replica_seed(w["seed"], rank) if args.replicas else w["seed"]
    for _ in range(args.warmup):
        res = step(h, w["tol_mixed"], seed)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    l0 = h.launch_count()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(os.environ.get("MLMC_CLOCKS_CSV", os.path.join(tempfile.gettempdir(), "clocks_bench.csv")))
    results = []
    with sampler:
        torch.cuda.profiler.start()      # no-op unless a profiler is attached (launch lists)
        ev0.record()
        t0 = time.time()
        for _ in range(args.steps):
            results.append(step(h, w["tol_mixed"], seed))
        ev1.record()
        barrier()
        wall = time.time() - t0
        torch.cuda.profiler.stop()
    ms = ev0.elapsed_time(ev1)
    launches = (h.launch_count() - l0) // max(args.steps, 1)
    t_step = max_over_ranks(ms / 1e3 / args.steps, "cuda")
    # replicas: seconds per trace over all of them; sharded: the one estimate's seconds
    value = job_value(t_step, world) if args.replicas else t_step
    res = results[-1]

    # dominant kernels, timed alone with CUDA events on the hierarchy's stream
    peak, peak_kind = measured_peaks()
    kern = {}
    for name, which in (("multidot_fp32", 3), ("multiaxpy_fp32", 4), ("rbgs_sweep_fp32", 2), ("stencil_fp32", 1),
                        ("stencil_fp64", 0)):
        kms, kbytes = h.profile_kernel(which, 1, w["block"], 20)
        kern[name] = {"ms": kms, "bytes": kbytes, "gbs": kbytes / kms / 1e6}
    # the coarse-level smoother sweeps (block stencils, k = the coarse block)
    kcb = w.get("coarse_block") or w["block"]
    for lvl in range(2, w["levels"]):
        kms, kbytes = h.profile_kernel(2, lvl, kcb, 20)
        kern["rbgs_sweep_fp32_level%d" % lvl] = {"ms": kms, "bytes": kbytes, "gbs": kbytes / kms / 1e6, "k": kcb}
        kms, kbytes = h.profile_kernel(1, lvl, kcb, 20)
        kern["stencil_fp32_level%d" % lvl] = {"ms": kms, "bytes": kbytes, "gbs": kbytes / kms / 1e6, "k": kcb}
    # the coarsest dense apply of the FP32 cycle (tensor cores vs CUDA cores), k = the coarse block
    nxL, nyL, dL = h.level_info(w["levels"])
    nL, kc = nxL * nyL * dL, (w.get("coarse_block") or w["block"])
    for name, wk in (("dense_apply_tc", mlmc.DENSE_TC), ("dense_apply_simt", mlmc.DENSE_SIMT)):
        h.set_dense_kernel(wk)
        kms, kbytes = h.profile_kernel(5, w["levels"], kc, 20)
        flops = (8.0 if w["kind"] == "wilson" else 2.0) * nL * nL * kc
        kern[name] = {"ms": kms, "bytes": kbytes, "flops": flops, "tflops": flops / kms / 1e9, "n": nL, "k": kc}
    h.set_dense_kernel(mlmc.DENSE_AUTO)
    # the transfers (Sec. 4.1 aggregation P_l and R_l = P_l^*) on every level pair, k = that
    # level difference's block (the fine pair at the fine block width)
    for lvl in range(1, w["levels"]):
        kt = w["block"] if lvl == 1 else kcb
        for name, which in (("restrict", 6), ("prolong", 7)):
            kms, kbytes = h.profile_kernel(which, lvl, kt, 20)
            kern["%s_fp32_level%d" % (name, lvl)] = {"ms": kms, "bytes": kbytes, "gbs": kbytes / kms / 1e6, "k": kt}
        # the cycle's fused residual and restriction (levels whose stencil and P it supports)
        try:
            kms, kbytes = h.profile_kernel(9, lvl, kt, 20)
        except mlmc.MLMCError:
            continue
        kern["residual_restrict_fp32_level%d" % lvl] = {"ms": kms, "bytes": kbytes, "gbs": kbytes / kms / 1e6, "k": kt}
    # the arithmetic ceilings the FP64 kernels meet: measured FMA rates
    fma64 = mlmc.measure_fma_rate(True, stream)
    fma32 = mlmc.measure_fma_rate(False, stream)
    add64 = mlmc.measure_fma_rate(True, stream, add=True)
    l2bw = mlmc.measure_fma_rate(stream=stream, l2=True)
    kern["fma_rate"] = {"fp64_tfma_s": fma64 / 1e12, "fp32_tfma_s": fma32 / 1e12, "fp64_tadd_s": add64 / 1e12,
                        "l2_copy_gbs": l2bw / 1e9}
    # kernels whose working set fits in L2 (< 100 MB per launch): their fraction of the measured
    # L2 copy bandwidth, not of HBM
    for name, v in kern.items():
        if "bytes" in v and "gbs" in v and "flops" not in v and v["bytes"] < 100e6:
            v["bound"] = "l2"
            v["l2_frac"] = v["gbs"] * 1e9 / l2bw
    # the FP64 fine-level apply: 4 FP64 operations per element (3 additions, 1 FMA)
    if w["kind"] == "laplace" and w.get("transfer") != "bilinear":
        st = kern["stencil_fp64"]
        ops = 4.0 * w["nx"] * w["ny"] * w["block"]
        st["fp64_ops_per_s"] = ops / (st["ms"] * 1e-3)
        st["alu_frac_of_measured_fma_rate"] = st["fp64_ops_per_s"] / fma64
        # 3 additions and 1 FMA per element at the measured rates: the FP64 ALU time floor
        floor_s = w["nx"] * w["ny"] * w["block"] * (3.0 / add64 + 1.0 / fma64)
        st["alu_floor_ms"] = floor_s * 1e3
        st["alu_frac"] = floor_s * 1e3 / st["ms"]
    # dominant kernel of the timed step (largest share of the step's ncu launch list): the
    # coarse-level block Gauss-Seidel k_rbgs_half on level 2; one sweep = two launches
    dom_name = "rbgs_sweep_fp32_level2" if w["levels"] > 2 else "multidot_fp32"
    dom = kern[dom_name]
    # DRAM bytes per sweep of this kernel version from an ncu capture (None until taken)
    traffic = TRAFFIC.get((w["name"], dom_name))
    if dom_name == "multidot_fp32":
        label = "k_multidot_partial<float> (inner Arnoldi: 4 basis blocks + w, level 1, k=%d)" % w["block"]
    elif w["kind"] == "wilson":
        label = ("k_rbgs_half_rows<cfloat,8> (coarse-level red-black block GS, level 2, d = 8, one sweep = "
                 "2 launches, k=%d; L2-resident working set)" % kcb)
    else:
        label = "k_rbgs_half_p (coarse-level red-black block GS, level 2, one sweep = 2 launches, k=%d)" % kcb
    roofline = {"bound": "hbm", "kernel": label,
                "achieved": dom["gbs"], "peak": peak, "unit": "GB/s", "frac": dom["gbs"] / peak,
                "peak_source": peak_kind, "traffic": traffic, "algorithmic_bytes": dom["bytes"], "kernels": kern}

    fp64 = None
    if not args.no_fp64_form and rank == 0:
        # the plain FP64 form (FP64 cycle, FP64 tolerance), timed like the mixed form: the same
        # warm-up estimates, then the same number of steps between CUDA events
        h.close()
        h64 = make_hierarchy(mlmc, mlmc.PREC_FP64, w, stream)
        for _ in range(args.warmup):
            step(h64, w["tol_fp64"], seed)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            r64 = step(h64, w["tol_fp64"], seed)
        e1.record()
        barrier()
        fp64 = {"seconds": e0.elapsed_time(e1) / 1e3 / args.steps,
                "unit": "s per estimate (%d warm-up, %d timed; same allocation and noise)" % (args.warmup, args.steps),
                "trace": r64["trace"].real, "std_err": r64["std_err"],
                "n_samples": r64["n_samples"], "iters": r64["iters"]}
        h64.close()
    else:
        h.close()

    # end to end through the C ABI: setup from the host descriptor + estimate + result read-back
    torch.cuda.synchronize()
    t = time.time()
    he = make_hierarchy(mlmc, mlmc.PREC_MIXED_FP32, w, stream)
    if w.get("learned"):
        he.learned_train(n_pairs=w["train_pairs"], epochs=w["train_epochs"], lr=w["train_lr"],
                         tol=w["tol_mixed"], seed=7, enable=1)
    step(he, w["tol_mixed"], seed)
    he.close()
    torch.cuda.synchronize()
    e2e = time.time() - t

    cfg1 = gpu_config1(mlmc, stream, args.warmup) if rank == 0 else None
    # config 4 (Wilson 256^2): the learned correction against the plain smoother
    learned = None
    if rank == 0 and not args.no_learned:
        learned = learned_leg(mlmc, stream, args.warmup, args.steps, seed)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)
    if rank == 0:
        import ctypes
        line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
                "scaling": "weak" if (args.replicas or world == 1) else "strong", "vs_baseline": None,
                "dtype": "f64/f32", "data": "synthetic",
                "config": config_dict(w, args.alloc), "form": "mixed: FP32 K-cycle under FP64 FGMRES",
                "cost_model": args.cost_model,
                "clocks": sampler.summary(local), "gpu_launches": int(launches), "wall_s_timed": wall,
                "e2e": {"value": e2e, "unit": "s",
                        "h2d_bytes_per_step": 0 if w["kind"] == "laplace" else 2 * w["nx"] * w["ny"] * 16,
                        "d2h_bytes_per_step": ctypes.sizeof(mlmc.EstimateResult),
                        "includes": "hierarchy setup from the host descriptor" +
                                    (" + network training" if w.get("learned") else "") +
                                    " + estimate + result read-back"},
                "roofline": roofline, "cpu_baseline": cpu,
                "result": {"trace": res["trace"].real, "std_err": res["std_err"], "tau": res["tau"],
                           "closed_form": closed_form(w),
                           "coarse_term": res["coarse_term"].real, "n_samples": res["n_samples"],
                           "iters": res["iters"], "seconds_per_level": res["seconds"]},
                "fp64_form": fp64, "learned": learned, "config1": cfg1}
        if fp64 is not None:
            # the mixed form's trace against the plain FP64 form's on the same samples
            line["result"]["rel_diff_vs_fp64_form"] = abs(res["trace"].real - fp64["trace"]) / abs(fp64["trace"])
        if closed_form(w) is not None:
            line["result"]["rel_err_vs_closed_form"] = abs(res["trace"].real - closed_form(w)) / closed_form(w)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
