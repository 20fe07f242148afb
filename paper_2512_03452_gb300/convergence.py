"""The convergence study of Sec. 5.1 on the GPU: runs of the uniform-ball set-up
(unit ball of density 60/pi, M0 = 80, L = 8, mu = chi = 1, eps = 1e-4,
k = 0.1, tau = 1e-5, N_T = 2000 steps, automatic filter scale) for given
particle numbers P, grid sizes H and seeds, each seed drawing both the initial
positions and the Brownian increments; the result of a run is the radius
|X_p| of every particle at T, from which the study's radial quantiles are taken.
Runs of one (P, H) with H >= 32 go through the batched engine together.
"""
from __future__ import annotations

import math

import numpy as np

from . import Batch, Simulation, params_from_workload, workloads


def final_radii(P, H, seeds, steps=2000, precision=32):
    """|X^(N)_p| of the Sec. 5.1 run for each seed (list of float64 arrays)."""
    ws = [workloads.uniform_ball(P=P, H=H, seed=int(s)) for s in seeds]
    params = [params_from_workload(w, precision=precision) for w in ws]
    X0s = [workloads.sample_positions(w) for w in ws]
    if H >= 32 and len(ws) > 1:
        with Batch(params, X0s) as b:
            b.step(steps)
            b.sync()
            return [np.linalg.norm(b.positions(r), axis=1) for r in range(len(ws))]
    out = []
    for p, X0 in zip(params, X0s):
        with Simulation(p, X0) as sim:
            sim.step(steps)
            sim.sync()
            out.append(np.linalg.norm(sim.positions(), axis=1))
    return out


def quantile_levels(n=1000):
    """j/n for j = 0..m, m = ceil(3n/4) - 1: the levels the study compares."""
    m = int(math.ceil(3 * n / 4)) - 1
    return np.arange(m + 1) / n


def radial_quantiles(radii, levels):
    """q_a = inf{r : #{|X_p| <= r} / P >= a} (the ceil(a P)-th smallest radius)."""
    r = np.sort(np.asarray(radii, dtype=np.float64))
    k = np.ceil(np.asarray(levels) * r.shape[0] - 1e-12).astype(np.int64)
    return np.where(k <= 0, 0.0, r[np.clip(k, 1, r.shape[0]) - 1])


def fitted_slope(xs, errs):
    """Least-squares slope of log2(err) against log2(x)."""
    return float(np.polyfit(np.log2(np.asarray(xs, dtype=np.float64)), np.log2(np.asarray(errs)), 1)[0])
