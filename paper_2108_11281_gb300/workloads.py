"""Seeded synthetic inputs shaped like the paper's matrix classes.

This module holds input generation only (no arithmetic of the method): gauge
links for the Wilson/Schwinger operator and the parameter sets of the
workloads.  Both the CUDA path and the CPU oracle's tests take their inputs
from here.

Links (Example 5.3 uses a thermalized configuration that is not available;
the stand-in is i.i.d. phases): theta ~ N(0, sd^2) per link from numpy's
PCG64 generator seeded with `seed`, U = cos(theta) + i sin(theta) from the
host libm.  Layout (2, ny, nx): [0] = x-links Theta_ij on (i,j)->(i+1,j),
[1] = y-links Phi_ij on (i,j)->(i,j+1).
"""
import numpy as np


def gauge_links(nx, ny, sd, seed):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0.0, sd, size=(2, ny, nx))
    return np.cos(theta) + 1j * np.sin(theta)


def pure_gauge_links(nx, ny, seed):
    """U_mu(x) = g(x) conj(g(x + mu)) for random phases g: gauge-equivalent to U = 1."""
    rng = np.random.default_rng(seed)
    g = np.exp(1j * rng.uniform(0.0, 2 * np.pi, size=(ny, nx)))
    ux = g * np.conj(np.roll(g, -1, axis=1))
    uy = g * np.conj(np.roll(g, -1, axis=0))
    return np.stack([ux, uy]), g


# Workloads: synthetic operators with the sizes and classes of the paper's examples (Sec. 5).
LAPLACE_SMALL = dict(name="laplace2d-64x64-L2-const", kind="laplace", nx=64, ny=64, shift=0.0,
                     levels=2, n_tv=1, setup="constant", noise="rademacher", block=64,
                     tol=1e-10, samples=1000)
LAPLACE_1024 = dict(name="laplace2d-1024x1024-L4", kind="laplace", nx=1024, ny=1024, shift=0.0,
                    levels=4, n_tv=4, setup="smooth", sweeps=160, coarse_sweeps=20,
                    noise="rademacher", block=64, tol=1e-10, eps=1e-3)
# mass from `python -m oracle.tune_mass 128 128 0.3 1`: sigma_min / sigma_max = 1.0015e-3
WILSON_128 = dict(name="wilson2d-128x128-L3", kind="wilson", nx=128, ny=128, link_sd=0.3,
                  link_seed=1, mass=-0.1317442871, levels=3, n_tv=4, spin_split=True, setup="inverse",
                  sweeps=20, noise="z4", block=32, tol=1e-10, eps=1e-3)
# mass from `python -m oracle.tune_mass 256 256 0.4 2 1e-3 --bisect -0.25 -0.20 7`: ratio 1.019e-3
WILSON_256 = dict(name="wilson2d-256x256-L3", kind="wilson", nx=256, ny=256, link_sd=0.4, link_seed=2,
                  mass=-0.2417968750, levels=3, n_tv=4, spin_split=True, setup="inverse", sweeps=20,
                  noise="z4", block=32, tol=1e-8, eps=1e-3)
