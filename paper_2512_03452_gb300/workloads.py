"""Seeded synthetic inputs for the SIPF-PIC step.

This module holds only input generation: the physical parameters of each
workload and i.i.d. samples of the initial particle positions X^(0) (the
sampling line of Algorithm 4). It contains none of the method's arithmetic,
so both the CUDA path and the FP64 oracle can be fed from it.

The paper's own experiments use analytic initial shapes (uniform ball, Sec.
5.1; uniform torus, Sec. 5.4); the workloads below use shapes of the same kind
(Gaussian blob, Gaussian torus plus a uniform background) at the sizes of the
benchmark configurations.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Workload:
    """Physical and numerical parameters of one run (names follow Sec. 2.2)."""
    name: str
    P: int                 # particles
    H: int                 # grid points / Fourier modes per dimension
    L: float = 1.0         # periodic box [-L/2, L/2)^3
    mass: float = 10.0     # M0
    chi: float = 1.0
    mu: float = 1.0
    eps: float = 1.0
    k: float = 1.0
    dt: float = 1e-3       # tau
    steps: int = 20
    seed: int = 0
    shape: str = "gaussian"        # gaussian | torus
    sigma: float = 0.1             # blob std or torus minor-radius std, in units of L
    major: float = 0.25            # torus major radius, in units of L
    background: float = 0.0        # fraction of particles uniform on the box
    radius: float = 0.125          # ball radius, in units of L (shape "ball")
    H0: float = -1.0               # Gaussian filter resolution; <0 auto, 0 off


def wrap_into_box(X: np.ndarray, L: float) -> np.ndarray:
    """Map sampled points into [-L/2, L/2) by periodicity (input preparation)."""
    Y = np.mod(X + 0.5 * L, L) - 0.5 * L
    Y[Y >= 0.5 * L] -= L
    return Y


def sample_positions(w: Workload, seed: int | None = None) -> np.ndarray:
    """i.i.d. samples of X^(0) as a (P, 3) float64 array inside the box."""
    rng = np.random.default_rng(w.seed if seed is None else seed)
    L = w.L
    if w.shape == "gaussian":
        X = rng.normal(0.0, w.sigma * L, size=(w.P, 3))
    elif w.shape == "torus":
        n_bg = int(round(w.background * w.P))
        n_t = w.P - n_bg
        phi = rng.uniform(0.0, 2.0 * math.pi, size=n_t)
        s1 = rng.normal(0.0, w.sigma * L, size=n_t)
        s2 = rng.normal(0.0, w.sigma * L, size=n_t)
        r = w.major * L + s1
        T = np.stack([r * np.cos(phi), r * np.sin(phi), s2], axis=1)
        B = rng.uniform(-0.5 * L, 0.5 * L, size=(n_bg, 3))
        X = np.concatenate([T, B], axis=0)
        X = X[rng.permutation(w.P)]
    elif w.shape == "ball":
        # uniform in the ball |x| <= radius L: radius r U^(1/3), uniform direction
        v = rng.normal(size=(w.P, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        X = (w.radius * L) * np.cbrt(rng.uniform(size=(w.P, 1))) * v
    elif w.shape == "uniform":
        X = rng.uniform(-0.5 * L, 0.5 * L, size=(w.P, 3))
    else:
        raise ValueError(f"unknown shape {w.shape!r}")
    return wrap_into_box(X, L)


# Benchmark workloads: plain FP64 small case, blow-up blob, torus at scale.
def small_blob() -> Workload:
    """P=1e4 Gaussian blob, H=16, 20 steps (the case the oracle runs in seconds)."""
    return Workload("gaussian_blob_P1e4_H16", P=10_000, H=16, L=1.0, mass=10.0,
                    chi=1.0, mu=1.0, eps=1.0, k=1.0, dt=1e-3, steps=20, seed=0,
                    shape="gaussian", sigma=0.1)


def blowup_blob() -> Workload:
    """P=1e6 supercritical Gaussian blob (M0=200, sigma=0.05L), H=64, L=2."""
    return Workload("blowup_blob_P1e6_H64", P=1_000_000, H=64, L=2.0, mass=200.0,
                    chi=1.0, mu=1.0, eps=1.0, k=0.5, dt=1e-4, steps=1000, seed=0,
                    shape="gaussian", sigma=0.05)


def torus_ring(H: int = 128, P: int = 10_000_000) -> Workload:
    """Ring-shaped data: torus (R=0.25L, sigma=0.03L) + 5% uniform, M0=300."""
    return Workload(f"torus_ring_P{P:.0e}_H{H}".replace("+0", "").replace("+", ""),
                    P=P, H=H, L=1.0, mass=300.0, chi=1.0, mu=0.5, eps=1.0, k=1.0,
                    dt=5e-5, steps=500, seed=0, shape="torus", sigma=0.03,
                    major=0.25, background=0.05)


def uniform_ball(P: int = 2 ** 14, H: int = 32, seed: int = 0) -> Workload:
    """The initial data of the Sec. 5.1 convergence study: uniform density
    60/pi on the unit ball (M0 = 80), L = 8, mu = chi = 1, eps = 1e-4,
    k = 0.1, tau = 1e-5, T = 0.02 (2000 steps)."""
    return Workload(f"uniform_ball_P{P}_H{H}", P=P, H=H, L=8.0, mass=80.0, chi=1.0, mu=1.0,
                    eps=1e-4, k=0.1, dt=1e-5, steps=2000, seed=seed, shape="ball", radius=1.0 / 8.0)


def ensemble(n_runs: int = 256, seed: int = 0) -> list[Workload]:
    """Batched ensemble: P log-uniform in [1e4, 1e6], H in {32, 64}, chi in
    [0.5, 2], mass in [10, 200], Gaussian blobs with per-run seeds."""
    rng = np.random.default_rng(seed)
    runs = []
    for i in range(n_runs):
        P = int(10 ** rng.uniform(4.0, 6.0))
        H = int(rng.choice([32, 64]))
        chi = float(rng.uniform(0.5, 2.0))
        mass = float(rng.uniform(10.0, 200.0))
        runs.append(Workload(f"ensemble_{i}", P=P, H=H, L=1.0, mass=mass, chi=chi,
                             mu=1.0, eps=1.0, k=1.0, dt=1e-4, steps=200, seed=i,
                             shape="gaussian", sigma=0.1))
    return runs


def adjoint_case(small: bool = False) -> Workload:
    """Adjoint workload: P=1e6, H=64, 200 steps (small: P=1e4, H=16)."""
    if small:
        return Workload("adjoint_P1e4_H16", P=10_000, H=16, L=1.0, mass=10.0,
                        chi=1.0, mu=1.0, eps=1.0, k=1.0, dt=1e-4, steps=20,
                        seed=0, shape="gaussian", sigma=0.1)
    return Workload("adjoint_P1e6_H64", P=1_000_000, H=64, L=1.0, mass=10.0,
                    chi=1.0, mu=1.0, eps=1.0, k=1.0, dt=1e-4, steps=200, seed=0,
                    shape="gaussian", sigma=0.1)
