"""Plain FP64 CPU oracle of the 2D SIPF-PIC step (the parabolic-elliptic
variant of Sec. 5.2: the Keller-Segel system with eps = 0 in two dimensions).

TEST INFRASTRUCTURE, like sipf_oracle: only the tests and the benchmark's CPU
legs may import it; the library never does, and it shares no code with the
CUDA path.

The method is Algorithm 4 restricted to two dimensions:
  * domain [-L/2, L/2)^2, H x H nodes x_j = j h (j in [-H/2, H/2), stored at
    j mod H), particle weight M0/P;
  * deposit with the 2D fourth-order stencil (12 nodes; the 2D analogue of
    Eq. (4ord)): inner 2 x 2 nodes carry the bilinear weight times
    1 + sum_k lambda_k (1 - lambda_k)/2 over the two axes, an outer node with
    index -1 or 2 on one axis the cubic factor of Eq. (4ord) on that axis times
    the linear weight of the other; or the bilinear stencil (order 2);
  * beta_q = L^-2 sum_j phi_j e^{-i y_q . x_j} (F_H in 2D);
  * eps = 0: c-hat solves (|y|^2 + k^2) alpha = beta (the zero mode is left at
    0 when k = 0: the periodic problem determines c up to a constant, and
    only its gradient enters); eps > 0: the implicit update of Eq.
    (alpha_hat_update);
  * gradient G_d = i y_d Phi_q alpha, Phi_q = exp(-2 pi^2 |q|^2 / H0^2), with
    component d zeroed on the line q_d = -H/2;
  * move with the bilinear gather: Z = X + W^- + chi tau I*(grad c)(X + W^-),
    X^n = Z + W^+, W^+- ~ N(0, mu tau I), periodic wrap.
Readings (also listed with the library's design notes): with eps = 0 the
field of level n-1 is the elliptic solution for rho^(n-1) and drives the move
of step n (the time level Algorithm 4 uses for the drift); the noise of
particle p at step n is the first Philox block of the 3D generator's counter
(p lo, p hi, n, 0): W^- = s (z0, z1), W^+ = s (z2, z3) (plain Euler-Maruyama:
W = s (z0, z1) with s = sqrt(2 mu tau)).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .sipf_oracle import auto_H0, philox4x32_10, MASK32, TWO_PI


def normals2(seed: int, step: int, P: int, first: int = 0):
    """Four standard normals per particle from Philox block 0 of the counter
    (p lo, p hi, step, 0): Box-Muller on the pairs (u0, u1), (u2, u3) with
    u = (x + 1/2) 2^-32."""
    p = np.arange(first, first + P, dtype=np.uint64)
    k0, k1 = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    w = philox4x32_10(p & MASK32, p >> np.uint64(32), np.full(P, step & 0xFFFFFFFF, dtype=np.uint64),
                      np.zeros(P, dtype=np.uint64), k0, k1)
    u = (np.stack(w, axis=1).astype(np.float64) + 0.5) * 2.0 ** -32
    z = np.empty((P, 4))
    for j in range(2):
        r = np.sqrt(-2.0 * np.log(u[:, 2 * j]))
        th = TWO_PI * u[:, 2 * j + 1]
        z[:, 2 * j] = r * np.cos(th)
        z[:, 2 * j + 1] = r * np.sin(th)
    return z


def _lin(j, lam):
    return 1.0 - j + (2.0 * j - 1.0) * lam


GAMMA2_2D = np.array([(a, b) for a in (0, 1) for b in (0, 1)], dtype=np.int64)


def _gamma4_2d_offsets():
    outer = []
    for axis in range(2):
        for e in (-1, 2):
            for a in (0, 1):
                o = [0, 0]
                o[axis] = e
                o[1 - axis] = a
                outer.append(tuple(o))
    return np.array([tuple(o) for o in GAMMA2_2D] + outer, dtype=np.int64)


GAMMA4_2D = _gamma4_2d_offsets()


def stencil2(lam, order):
    """(offsets (n, 2), weights (P, n)) of the 2D stencil of the given order."""
    if order == 2:
        W = np.ones((lam.shape[0], 4))
        for g, off in enumerate(GAMMA2_2D):
            for s in range(2):
                W[:, g] *= _lin(off[s], lam[:, s])
        return GAMMA2_2D, W
    if order != 4:
        raise ValueError("order must be 2 or 4")
    W = np.empty((lam.shape[0], 12))
    boost = 1.0 + np.sum(lam * (1.0 - lam), axis=1) / 2.0
    for g, off in enumerate(GAMMA4_2D):
        outer = [s for s in range(2) if off[s] in (-1, 2)]
        if not outer:
            w = boost * _lin(off[0], lam[:, 0]) * _lin(off[1], lam[:, 1])
        else:
            s = outer[0]
            l = lam[:, s]
            w = -(1.0 + l) * (1.0 - l) * l / 6.0 if off[s] == 2 else -(2.0 - l) * l * (1.0 - l) / 6.0
            w = w * _lin(off[1 - s], lam[:, 1 - s])
        W[:, g] = w
    return GAMMA4_2D, W


def cell_and_lambda(X, H, L):
    u = X * (H / L)
    cell = np.floor(u)
    return cell.astype(np.int64), u - cell


def stencil_indices(cell, offsets, H):
    idx = (cell[:, None, :] + offsets[None, :, :]) % H
    return idx[..., 0] * H + idx[..., 1]


def deposit(X, w, H, L, order=4):
    """phi[q_{p,gamma}] += w F_{p,gamma} (Algorithm 2 in 2D); H x H masses."""
    cell, lam = cell_and_lambda(X, H, L)
    offs, F = stencil2(lam, order)
    idx = stencil_indices(cell, offs, H)
    return np.bincount(idx.ravel(), weights=(w * F).ravel(), minlength=H * H).reshape(H, H)


def gather(f, X, H, L, order=2):
    """f_p = sum_gamma F_{p,gamma} f[q_{p,gamma}] (Algorithm 3 in 2D); f (..., H, H)."""
    cell, lam = cell_and_lambda(X, H, L)
    offs, F = stencil2(lam, order)
    idx = stencil_indices(cell, offs, H)
    flat = f.reshape(f.shape[:-2] + (H * H,))
    return np.sum(flat[..., idx] * F, axis=-1)


def mode_numbers(H):
    q = np.arange(H)
    q = np.where(q < H // 2, q, q - H)
    qy = np.arange(H // 2 + 1)
    qy = np.where(qy < H // 2, qy, qy - H)
    return q[:, None], qy[None, :]


def forward_ft(phi, L):
    """beta_q = L^-2 sum_j phi_j e^{-i 2 pi q.j / H} (half layout H x (H/2+1))."""
    return np.fft.rfftn(phi) / L ** 2


def inverse_ft(G, H):
    """f(x_j) = sum_q G_q e^{i 2 pi q.j / H} over the full Hermitian spectrum."""
    return np.fft.irfftn(G, s=(H, H), axes=(0, 1)) * (H * H)


def wrap(X, L):
    Y = X - L * np.floor(X / L + 0.5)
    Y[Y >= 0.5 * L] -= L
    Y[Y < -0.5 * L] += L
    return Y


def min_image(D, L):
    return D - L * np.round(D / L)


@dataclasses.dataclass
class Params2D:
    P: int
    H: int
    L: float = 8.0
    mass: float = 20.0
    chi: float = 1.0
    mu: float = 1.0
    eps: float = 0.0
    k: float = 0.0
    dt: float = 5e-4
    H0: float = -1.0
    seed: int = 0
    p2g_order: int = 4
    g2p_order: int = 2
    splitting: str = "half"

    @property
    def H0_eff(self):
        return auto_H0(self.H, self.L) if self.H0 < 0 else float(self.H0)


def solve_field(beta, alpha_prev, p):
    """alpha at level n-1 from beta of level n-1: (|y|^2 + k^2) alpha = beta for
    eps = 0; for eps > 0 the implicit update of Eq. (alpha_hat_update) from
    alpha_prev."""
    qx, qy = mode_numbers(p.H)
    y2 = (2.0 * math.pi / p.L) ** 2 * (qx ** 2 + qy ** 2).astype(np.float64)
    lam = y2 + p.k ** 2
    if p.eps == 0.0:
        out = np.zeros_like(beta)
        nz = lam > 0
        out[nz] = beta[nz] / lam[nz]
        return out
    return alpha_prev / (1.0 + p.dt / p.eps * lam) + beta / (lam + p.eps / p.dt)


def gradient_grids(alpha, p):
    """grad c on the nodes: F_H^-1 of i y_d Phi_q alpha, d = 1, 2, with
    component d zeroed on the line q_d = -H/2.  Returns (2, H, H)."""
    H = p.H
    qx, qy = mode_numbers(H)
    q2 = (qx ** 2 + qy ** 2).astype(np.float64)
    H0 = p.H0_eff
    Phi = np.ones_like(q2) if H0 == 0 else np.exp(-2.0 * math.pi ** 2 * q2 / (H0 * H0))
    out = []
    for d, q in enumerate((qx, qy)):
        y = 2.0 * math.pi * q / p.L
        G = 1j * np.broadcast_to(y, alpha.shape) * Phi * alpha
        G = np.where(np.broadcast_to(q, alpha.shape) == -H // 2, 0.0, G)
        out.append(inverse_ft(G, H))
    return np.stack(out)


def move(X, grads, p, n, first=0):
    z = normals2(p.seed, n, X.shape[0], first)
    if p.splitting == "half":
        s = math.sqrt(p.mu * p.dt)
        Y = X + s * z[:, 0:2]
        drift = gather(grads, Y, p.H, p.L, p.g2p_order).T
        return wrap(Y + p.chi * p.dt * drift + s * z[:, 2:4], p.L)
    s = math.sqrt(2.0 * p.mu * p.dt)
    drift = gather(grads, X, p.H, p.L, p.g2p_order).T
    return wrap(X + p.chi * p.dt * drift + s * z[:, 0:2], p.L)


@dataclasses.dataclass
class State2D:
    X: np.ndarray
    alpha: np.ndarray      # field of the last level (eps > 0: alpha^(n))
    n: int = 0


def init_state(X0, p):
    return State2D(wrap(np.array(X0, dtype=np.float64), p.L),
                   np.zeros((p.H, p.H // 2 + 1), dtype=np.complex128), 0)


def step(state, p):
    """One step: the field of level n-1 from rho^(n-1) (eps = 0: the elliptic
    solution; eps > 0: the implicit update of alpha, whose drift then uses
    alpha^(n-1) as in Algorithm 4), then the move of all particles."""
    n = state.n + 1
    phi = deposit(state.X, p.mass / p.P, p.H, p.L, p.p2g_order)
    beta = forward_ft(phi, p.L)
    if p.eps == 0.0:
        field = solve_field(beta, None, p)
        alpha_next = field
    else:
        field = state.alpha
        alpha_next = solve_field(beta, state.alpha, p)
    X = move(state.X, gradient_grids(field, p), p, n)
    return State2D(X, alpha_next, n)


def second_moment(X):
    """m2-hat = (1/P) sum_p |X_p|^2 (Sec. 5.2)."""
    return float(np.mean(np.sum(X ** 2, axis=1)))
