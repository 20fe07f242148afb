"""Plain FP64 CPU oracle of the SIPF-PIC time step (Algorithm 4).

TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU
baseline may import this module; the library never does, and it shares no
code with the CUDA path (its own Philox, its own stencils, numpy's FFT).

Everything is float64 and written to be checked against the paper by eye:
each function follows one numbered piece of the method, in the paper's order
and notation, with no blocking or fusion beyond vectorising the per-particle
loops of Algorithms 2 and 3 over the particle axis.

Readings taken where the paper is silent or garbled (each one is also listed
with the design notes of the library):
  * Mode set: q_d in {-H/2, ..., H/2-1} (the usual DFT set of H points per
    axis); the gradient component d is zeroed on the plane q_d = -H/2 so the
    gradient field stays real (Eq. (U) prints H+1 points per axis).
  * Source term of the implicit-Euler update: beta / (|y|^2 + k^2 + eps/tau),
    as in Eq. (alpha_hat_update) and Algorithm 4.
  * Gradient time level: grad c^(n-1) is built from alpha^(n-1), before the
    update (Algorithm 4); the Gaussian filter Phi multiplies the gradient.
  * Grid: node j in [-H/2, H/2) sits at x_j = j*h and is stored at j mod H,
    so F_H of the deposited masses is a plain index DFT over storage order.
  * Noise: Philox4x32-10 keyed by the 64-bit seed, counter
    (particle lo, particle hi, step, block), then Box-Muller; see normals().
  * Wrap: x -> x - L*floor(x/L + 1/2) after the full move; the pre-diffused
    point X + W^- is not wrapped (stencil indices are wrapped instead).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TWO_PI = 2.0 * math.pi
MASK32 = np.uint64(0xFFFFFFFF)


# ---------------------------------------------------------------------------
# Counter-based noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
# random numbers: as easy as 1, 2, 3", SC'11) + Box-Muller.  The paper only
# asks for W^-, W^+ ~ N(0, mu*tau*I) independent per particle and step
# (Algorithm 4); a counter-based generator lets the GPU draw the same numbers.
# ---------------------------------------------------------------------------
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on 32-bit words held in uint64 arrays.

    One round: (hi0, lo0) = M0*c0, (hi1, lo1) = M1*c2 (full 64-bit products),
    then c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by the
    Weyl constants (W0, W1) between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK32 for v in (c0, c1, c2, c3))
    k0 = np.uint64(k0) & MASK32
    k1 = np.uint64(k1) & MASK32
    for r in range(10):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniforms(seed: int, step: int, P: int, first: int = 0):
    """Eight uniforms in (0,1) per particle: blocks 0 and 1 of Philox with
    counter (p mod 2^32, p >> 32, step, block) and key (seed lo, seed hi);
    u = (x + 1/2) * 2^-32."""
    p = np.arange(first, first + P, dtype=np.uint64)
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    lo, hi = p & MASK32, p >> np.uint64(32)
    st = np.full(P, step & 0xFFFFFFFF, dtype=np.uint64)
    out = []
    for block in (0, 1):
        out.extend(philox4x32_10(lo, hi, st, np.full(P, block, dtype=np.uint64), k0, k1))
    x = np.stack(out, axis=1).astype(np.float64)
    return (x + 0.5) * 2.0 ** -32


def normals(seed: int, step: int, P: int, first: int = 0):
    """Six standard normals z0..z5 per particle via Box-Muller on the uniform
    pairs (u0,u1), (u2,u3), (u4,u5): z = sqrt(-2 ln u_a) (cos, sin)(2 pi u_b)."""
    u = uniforms(seed, step, P, first)
    z = np.empty((P, 6))
    for j in range(3):
        r = np.sqrt(-2.0 * np.log(u[:, 2 * j]))
        th = TWO_PI * u[:, 2 * j + 1]
        z[:, 2 * j] = r * np.cos(th)
        z[:, 2 * j + 1] = r * np.sin(th)
    return z


# ---------------------------------------------------------------------------
# Particle-grid weights (Sec. 3.1).  lambda = (H/L) X - floor((H/L) X).
# ---------------------------------------------------------------------------
def cell_and_lambda(X, H, L):
    u = X * (H / L)
    cell = np.floor(u)
    return cell.astype(np.int64), u - cell


def _lin(j, lam):
    """1D factor of the second-order weights: 1 - j + (2j - 1) lambda."""
    return 1.0 - j + (2.0 * j - 1.0) * lam


GAMMA2 = np.array([(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1)], dtype=np.int64)


def weights_gamma2(lam):
    """F^(2)_{j1 j2 j3}(lambda) = prod_s (1 - j_s + (2 j_s - 1) lambda_s), Eq. (2ord).
    Returns (offsets (8,3), weights (P,8))."""
    W = np.ones((lam.shape[0], 8))
    for g, off in enumerate(GAMMA2):
        for s in range(3):
            W[:, g] *= _lin(off[s], lam[:, s])
    return GAMMA2, W


def _gamma4_offsets():
    inner = [tuple(o) for o in GAMMA2]
    outer = []
    for axis in range(3):
        for e in (-1, 2):
            for a in (0, 1):
                for b in (0, 1):
                    o = [0, 0, 0]
                    o[axis] = e
                    others = [s for s in range(3) if s != axis]
                    o[others[0]] = a
                    o[others[1]] = b
                    outer.append(tuple(o))
    return np.array(inner + outer, dtype=np.int64)


GAMMA4 = _gamma4_offsets()


def weights_gamma4(lam):
    """Fourth-order 32-point weights of Eq. (4ord).

    Inner nodes (j in {0,1}^3): trilinear weight times (1 + sum_k lambda_k (1 - lambda_k)/2).
    Outer node with index 2 on axis s: -(1 + l)(1 - l) l / 6 times the bilinear
    weight of the other two axes; index -1 on axis s: -(2 - l) l (1 - l) / 6 times
    the same bilinear weight (l = lambda_s).  The paper prints axis 1 and states
    cubic symmetry for axes 2 and 3.
    Returns (offsets (32,3), weights (P,32))."""
    P = lam.shape[0]
    W = np.empty((P, 32))
    boost = 1.0 + np.sum(lam * (1.0 - lam), axis=1) / 2.0
    for g, off in enumerate(GAMMA4):
        outer_axes = [s for s in range(3) if off[s] in (-1, 2)]
        if not outer_axes:
            w = boost.copy()
            for s in range(3):
                w *= _lin(off[s], lam[:, s])
        else:
            s = outer_axes[0]
            l = lam[:, s]
            if off[s] == 2:
                w = -(1.0 + l) * (1.0 - l) * l / 6.0
            else:
                w = -(2.0 - l) * l * (1.0 - l) / 6.0
            for t in range(3):
                if t != s:
                    w = w * _lin(off[t], lam[:, t])
        W[:, g] = w
    return GAMMA4, W


def stencil(lam, order):
    if order == 2:
        return weights_gamma2(lam)
    if order == 4:
        return weights_gamma4(lam)
    raise ValueError("order must be 2 or 4")


def stencil_indices(cell, offsets, H):
    """Storage index of X_{p,gamma}: (floor(H X / L) + gamma) mod H per axis."""
    idx = (cell[:, None, :] + offsets[None, :, :]) % H
    return (idx[..., 0] * H + idx[..., 1]) * H + idx[..., 2]


# ---------------------------------------------------------------------------
# Algorithm 2 (particle-to-grid) and Algorithm 3 (grid-to-particle).
# ---------------------------------------------------------------------------
def deposit(X, weights, H, L, order=4, chunk=1 << 20):
    """phi[q_{p,gamma}] += w_p F_{p,gamma} over all particles and stencil
    points (Algorithm 2 without its final FFT).  `weights` is w_p (scalar M0/P
    or a per-particle array).  Particles are taken in chunks only to bound
    memory.  Returns the H^3 mass grid (float64)."""
    w = np.broadcast_to(np.asarray(weights, dtype=np.float64), (X.shape[0],))
    phi = np.zeros(H ** 3)
    for s in range(0, X.shape[0], chunk):
        cell, lam = cell_and_lambda(X[s:s + chunk], H, L)
        offs, F = stencil(lam, order)
        idx = stencil_indices(cell, offs, H)
        phi += np.bincount(idx.ravel(), weights=(w[s:s + chunk, None] * F).ravel(), minlength=H ** 3)
    return phi.reshape(H, H, H)


def gather(f, X, H, L, order=2):
    """f_p = sum_gamma F_{p,gamma} f[q_{p,gamma}] (Algorithm 3).  `f` has shape
    (..., H, H, H); returns (..., P)."""
    cell, lam = cell_and_lambda(X, H, L)
    offs, F = stencil(lam, order)
    idx = stencil_indices(cell, offs, H)
    flat = f.reshape(f.shape[:-3] + (H ** 3,))
    return np.sum(flat[..., idx] * F, axis=-1)


# ---------------------------------------------------------------------------
# Fourier side (Sec. 3.1 convention F_H, Eq. (alpha_hat_update), filter Phi).
# Half spectrum layout (H, H, H/2+1), index m <-> q = m for m < H/2, m - H else.
# ---------------------------------------------------------------------------
def mode_numbers(H):
    """Integer q per axis for the half-spectrum layout: (qx, qy, qz) broadcastable."""
    q = np.arange(H)
    q = np.where(q < H // 2, q, q - H)
    qz = np.arange(H // 2 + 1)
    qz = np.where(qz < H // 2, qz, qz - H)   # index H/2 is q = -H/2
    return q[:, None, None], q[None, :, None], qz[None, None, :]


def auto_H0(H, L):
    """H0 = ceil(8 H^(8/13) L^(5/13)), the filter scale used in Sec. 5.1.

    Evaluated exactly: the smallest integer m >= 0 with m^13 >= 8^13 H^8 L^5,
    L taken as the exact rational value of the float.  (A floating-point power
    can land just above an exact integer -- 8 * 8^(8/13) * 8^(5/13) = 64
    evaluates to 64.00000000000001 -- and its ceiling is then one too large.)"""
    from fractions import Fraction
    target = Fraction(8) ** 13 * Fraction(H) ** 8 * Fraction(L) ** 5
    m = max(0, math.ceil(8.0 * H ** (8.0 / 13.0) * L ** (5.0 / 13.0)) - 2)
    while Fraction(m) ** 13 < target:
        m += 1
    return float(m)


def filter_phi(H, H0):
    """Phi_q = exp(-2 pi^2 |q|^2 / H0^2); H0 == 0 means no filter."""
    qx, qy, qz = mode_numbers(H)
    q2 = (qx ** 2 + qy ** 2 + qz ** 2).astype(np.float64)
    if H0 == 0:
        return np.ones_like(q2)
    return np.exp(-2.0 * math.pi ** 2 * q2 / (H0 * H0))


def forward_ft(phi, L):
    """beta_q = F_H(I rho-hat)(2 pi q / L) = L^-3 sum_j phi_j e^{-i 2 pi q.j / H}."""
    return np.fft.rfftn(phi) / L ** 3


def inverse_ft(G, H):
    """F_H^{-1} G at the grid nodes: sum_q G_q e^{+i 2 pi q.j / H} (unnormalised)."""
    return np.fft.irfftn(G, s=(H, H, H), axes=(-3, -2, -1)) * float(H) ** 3


def update_alpha(alpha, beta, p):
    """Implicit-Euler update, Eq. (alpha_hat_update):
    alpha^n = alpha^{n-1} / (1 + tau/eps (|y|^2 + k^2)) + beta^{n-1} / (|y|^2 + k^2 + eps/tau)."""
    H = alpha.shape[0]
    qx, qy, qz = mode_numbers(H)
    y2 = (TWO_PI / p.L) ** 2 * (qx ** 2 + qy ** 2 + qz ** 2)
    return alpha / (1.0 + p.dt / p.eps * (y2 + p.k ** 2)) + beta / (y2 + p.k ** 2 + p.eps / p.dt)


def update_alpha_exp(alpha, beta, p):
    """Exponential propagator of Sec. 3.4: alpha^{n+1} = kappa (alpha^n + tau beta^n),
    kappa = exp(-tau/eps (|y|^2 + k^2))."""
    H = alpha.shape[0]
    qx, qy, qz = mode_numbers(H)
    y2 = (TWO_PI / p.L) ** 2 * (qx ** 2 + qy ** 2 + qz ** 2)
    return np.exp(-p.dt / p.eps * (y2 + p.k ** 2)) * (alpha + p.dt * beta)


def gradient_spectrum(alpha, p):
    """G_d = (2 pi i q_d / L) alpha_q Phi_q for d = 1..3 (Algorithm 4), with
    component d set to zero on its Nyquist plane q_d = -H/2."""
    H = alpha.shape[0]
    qs = mode_numbers(H)
    Phi = filter_phi(H, p.H0_eff)
    G = np.empty((3,) + alpha.shape, dtype=np.complex128)
    for d in range(3):
        qd = np.broadcast_to(qs[d], alpha.shape)
        Gd = 1j * (TWO_PI * qd / p.L) * alpha * Phi
        Gd = np.where(qd == -(H // 2), 0.0, Gd)
        G[d] = Gd
    return G


def gradient_grids(alpha, p):
    """grad c-hat at the grid nodes: F_H^{-1}(2 pi i q / L alpha Phi), shape (3,H,H,H)."""
    G = gradient_spectrum(alpha, p)
    H = alpha.shape[0]
    return np.stack([inverse_ft(G[d], H) for d in range(3)])


def wrap(X, L):
    """Periodic wrap into [-L/2, L/2): x - L floor(x/L + 1/2)."""
    Y = X - L * np.floor(X / L + 0.5)
    Y = np.where(Y >= 0.5 * L, Y - L, Y)
    Y = np.where(Y < -0.5 * L, Y + L, Y)
    return Y


def min_image(D, L):
    """Minimum-image difference for comparing periodic positions."""
    return D - L * np.round(D / L)


# ---------------------------------------------------------------------------
# Algorithm 4: one SIPF-PIC step.
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    P: int
    H: int
    L: float = 1.0
    mass: float = 10.0
    chi: float = 1.0
    mu: float = 1.0
    eps: float = 1.0
    k: float = 1.0
    dt: float = 1e-3
    H0: float = -1.0         # <0: auto (Sec. 5 rule); 0: filter off
    seed: int = 0
    p2g_order: int = 4
    g2p_order: int = 2
    splitting: str = "half"  # "half" (Algorithm 4) or "plain" (Eq. (rho_hat_update))
    propagator: str = "implicit"   # "implicit" (Eq. alpha_hat_update) or "exp" (Sec. 3.4)

    @property
    def H0_eff(self):
        return auto_H0(self.H, self.L) if self.H0 < 0 else float(self.H0)

    @classmethod
    def from_workload(cls, w, **kw):
        d = dict(P=w.P, H=w.H, L=w.L, mass=w.mass, chi=w.chi, mu=w.mu, eps=w.eps,
                 k=w.k, dt=w.dt, H0=w.H0, seed=w.seed)
        d.update(kw)
        return cls(**d)


@dataclasses.dataclass
class State:
    X: np.ndarray          # (P, 3) positions X^(n)
    alpha: np.ndarray      # (H, H, H/2+1) complex alpha^(n)
    n: int = 0


def init_state(X0, p):
    """alpha^(0) = 0 and the sampled X^(0) (Algorithm 4, initialisation)."""
    return State(np.array(X0, dtype=np.float64, copy=True),
                 np.zeros((p.H, p.H, p.H // 2 + 1), dtype=np.complex128), 0)


def move(X, grads, p, n, first=0):
    """Particle update of step n with the gradient grids of grad c^(n-1).

    half:  Z = X + W^- + chi tau I*(grad c)(X + W^-),  X^n = Z + W^+,
           W^-, W^+ ~ N(0, mu tau I)  (Algorithm 4)
    plain: X^n = X + chi tau I*(grad c)(X) + W, W ~ N(0, 2 mu tau I)  (Eq. (rho_hat_update))
    The rows of X are particles first, first+1, ... (their noise indices).
    """
    z = normals(p.seed, n, X.shape[0], first=first)
    if p.splitting == "half":
        s = math.sqrt(p.mu * p.dt)
        Y = X + s * z[:, 0:3]
        drift = gather(grads, Y, p.H, p.L, p.g2p_order).T
        return wrap(Y + p.chi * p.dt * drift + s * z[:, 3:6], p.L)
    s = math.sqrt(2.0 * p.mu * p.dt)
    drift = gather(grads, X, p.H, p.L, p.g2p_order).T
    return wrap(X + p.chi * p.dt * drift + s * z[:, 0:3], p.L)


def step(state, p):
    """State at t_{n-1} -> state at t_n (one pass of the loop of Algorithm 4)."""
    n = state.n + 1
    phi = deposit(state.X, p.mass / p.P, p.H, p.L, p.p2g_order)
    beta = forward_ft(phi, p.L)
    grads = gradient_grids(state.alpha, p)           # grad c^(n-1) from alpha^(n-1)
    if p.propagator == "exp":
        alpha = update_alpha_exp(state.alpha, beta, p)
    else:
        alpha = update_alpha(state.alpha, beta, p)
    X = move(state.X, grads, p, n)
    return State(X, alpha, n)


def run(X0, p, nsteps):
    s = init_state(X0, p)
    for _ in range(nsteps):
        s = step(s, p)
    return s


# ---------------------------------------------------------------------------
# Algorithm 1 operators (direct O(P H^3) sums), used as a brute-force pin.
# Full-cube layout (H, H, H), q from the DFT order.
# ---------------------------------------------------------------------------
def _q_full(H):
    q = np.arange(H)
    return np.where(q < H // 2, q, q - H)


def direct_beta(X, weights, H, L, chunk=2048):
    """beta_q = (1/L^3) sum_p w_p e^{-2 pi i q.X_p / L} for all q (Eq. (beta_hat_comp))."""
    q = _q_full(H)
    w = np.broadcast_to(np.asarray(weights, dtype=np.float64), (X.shape[0],))
    out = np.zeros((H, H, H), dtype=np.complex128)
    for s in range(0, X.shape[0], chunk):
        Xc = X[s:s + chunk]
        e = [np.exp(-1j * TWO_PI / L * np.outer(Xc[:, d], q)) for d in range(3)]
        out += np.einsum("p,pa,pb,pc->abc", w[s:s + chunk], e[0], e[1], e[2], optimize=True)
    return out / L ** 3


def direct_gradient(alpha_full, X, p, chunk=2048):
    """grad c(X) = sum_q (2 pi i q / L) Phi_q alpha_q e^{2 pi i q.X / L} (Eq. (gradc),
    with Algorithm 4's filter and the Nyquist-plane rule).  Returns (P, 3)."""
    H = alpha_full.shape[0]
    q = _q_full(H)
    qx, qy, qz = np.meshgrid(q, q, q, indexing="ij")
    Phi = np.ones(qx.shape) if p.H0_eff == 0 else np.exp(
        -2.0 * math.pi ** 2 * (qx ** 2 + qy ** 2 + qz ** 2) / p.H0_eff ** 2)
    out = np.zeros((X.shape[0], 3))
    for d, qd in enumerate((qx, qy, qz)):
        G = 1j * (TWO_PI * qd / p.L) * Phi * alpha_full
        G = np.where(qd == -(H // 2), 0.0, G)
        for s in range(0, X.shape[0], chunk):
            Xc = X[s:s + chunk]
            e = [np.exp(1j * TWO_PI / p.L * np.outer(Xc[:, dd], q)) for dd in range(3)]
            out[s:s + chunk, d] = np.einsum("abc,pa,pb,pc->p", G, e[0], e[1], e[2],
                                            optimize=True).real
    return out


def direct_update_alpha(alpha_full, beta_full, p):
    q = _q_full(p.H)
    qx, qy, qz = np.meshgrid(q, q, q, indexing="ij")
    y2 = (TWO_PI / p.L) ** 2 * (qx ** 2 + qy ** 2 + qz ** 2)
    return alpha_full / (1.0 + p.dt / p.eps * (y2 + p.k ** 2)) + beta_full / (y2 + p.k ** 2 + p.eps / p.dt)


def direct_step(X, alpha_full, p, n):
    """One step of the direct-sum method with Algorithm 4's move and filter:
    exact beta (Eq. (beta_hat_comp)) and exact gradient (Eq. (gradc)) in place
    of the interpolations I and I*.  Returns (X^n, alpha^n)."""
    beta = direct_beta(X, p.mass / p.P, p.H, p.L)
    z = normals(p.seed, n, X.shape[0])
    if p.splitting == "half":
        s = math.sqrt(p.mu * p.dt)
        Y = X + s * z[:, 0:3]
        drift = direct_gradient(alpha_full, Y, p)
        Xn = wrap(Y + p.chi * p.dt * drift + s * z[:, 3:6], p.L)
    else:
        s = math.sqrt(2.0 * p.mu * p.dt)
        drift = direct_gradient(alpha_full, X, p)
        Xn = wrap(X + p.chi * p.dt * drift + s * z[:, 0:3], p.L)
    return Xn, direct_update_alpha(alpha_full, beta, p)


# ---------------------------------------------------------------------------
# Diagnostics (Sec. 5): mass, zero mode, rho_num peak, high-frequency energy
# share, second moment, ring radius.
# ---------------------------------------------------------------------------
def density_num(phi, p):
    """rho_num = F_H^{-1}(Phi F_H I rho-hat) on the grid (rho-hat convolved with
    the Gaussian N(0, (L/H0)^2 I)); H0 = 0 gives the plain deposited density."""
    beta = forward_ft(phi, p.L)
    return inverse_ft(filter_phi(p.H, p.H0_eff) * beta, p.H)


def hf_energy_fraction(alpha, qmin=4.0):
    """Share of sum |alpha_q|^2 held by modes with ||q|| >= qmin (full spectrum
    recovered from the half layout by Hermitian symmetry)."""
    H = alpha.shape[0]
    qx, qy, qz = mode_numbers(H)
    mult = np.full(alpha.shape[2], 2.0)
    mult[0] = 1.0
    if H % 2 == 0:
        mult[H // 2] = 1.0
    e = np.abs(alpha) ** 2 * mult[None, None, :]
    hi = np.sqrt(qx ** 2 + qy ** 2 + qz ** 2) >= qmin
    tot = e.sum()
    return float(e[np.broadcast_to(hi, e.shape)].sum() / tot) if tot > 0 else 0.0


def diagnostics(state, p):
    phi = deposit(state.X, p.mass / p.P, p.H, p.L, p.p2g_order)
    rho = density_num(phi, p)
    r = np.sqrt(state.X[:, 0] ** 2 + state.X[:, 1] ** 2)
    return dict(mass=float(phi.sum()),
                alpha0=float(state.alpha[0, 0, 0].real),
                peak=float(rho.max()),
                hf_frac=hf_energy_fraction(state.alpha),
                m2=float(np.mean(np.sum(state.X ** 2, axis=1))),
                ring_radius=float(np.mean(r)))
