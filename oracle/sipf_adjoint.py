"""Plain FP64 CPU adjoint (reverse mode) of N steps of SIPF-PIC (Algorithm 4)
with the noise held fixed.

TEST INFRASTRUCTURE, like sipf_oracle: only the tests, the smoke check and the
benchmark may import it; the library never does and shares no code with it.

The forward map (sipf_oracle.step, repeated N times from X^0 with alpha^0 = 0)
is differentiated by hand, operator by operator, in reverse order:

  phi^{n-1} = I rho-hat(X^{n-1})               deposit, Gamma_4 weights (Alg. 2)
  beta^{n-1} = F_H phi^{n-1}                   L^-3 DFT
  alpha^n = A alpha^{n-1} + B beta^{n-1}       Eq. (alpha_hat_update) (or Sec. 3.4)
  g^{n-1} = F_H^-1 (i y Phi alpha^{n-1})       gradient grids (Nyquist planes zero)
  Y = X^{n-1} + s W^-,  V = I* g^{n-1}(Y)      gather, Gamma_2 weights (Alg. 3)
  X^n = Y + chi tau V + s W^+                  (wrap: a translation, derivative 1)

The output is the deposited density rho(T) = phi^N / h^3 on the grid; the
caller supplies rho-bar = dJ/drho(T) and gets dJ/dchi, dJ/dmu and dJ/dX^0.
Adjoints of the linear Fourier maps use the real inner product of full
(Hermitian) spectra, Re sum_q conj(u_q) v_q: the transpose of F_H is
L^-3 F_H^-1, the transpose of F_H^-1 (complex-to-real) is the unnormalised
forward DFT, a pointwise factor m_q turns into conj(m_q).  Every spectrum in
the chain is Hermitian, so the half layout carries it without weights.  The
deposit I and the gather I* are transposes of each other (the relation
<I rho, f> = <rho, I* f> stated after Def. grid2particle, Sec. 3.1); the particle-position derivatives come
from the derivatives of the weight polynomials of Eqs. (2ord) and (4ord).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import sipf_oracle as O


# ---------------------------------------------------------------------------
# Weight polynomials and their derivatives in lambda (Eqs. (2ord), (4ord)).
# ---------------------------------------------------------------------------
def _dlin(j):
    """d/dlambda of the 1D factor 1 - j + (2j - 1) lambda."""
    return 2.0 * j - 1.0


def stencil_grad(lam, order):
    """Offsets, weights F (P, n) and dF/dlambda (P, n, 3) of the order-2 or
    order-4 stencil at fractional positions lam (P, 3)."""
    offs, F = O.stencil(lam, order)
    P, n = F.shape
    dF = np.empty((P, n, 3))
    if order == 2:
        for g, off in enumerate(offs):
            for e in range(3):
                d = np.full(P, _dlin(off[e]))
                for s in range(3):
                    if s != e:
                        d = d * O._lin(off[s], lam[:, s])
                dF[:, g, e] = d
        return offs, F, dF
    boost = 1.0 + np.sum(lam * (1.0 - lam), axis=1) / 2.0
    for g, off in enumerate(offs):
        outer = [s for s in range(3) if off[s] in (-1, 2)]
        if not outer:
            tri = np.ones(P)
            for s in range(3):
                tri = tri * O._lin(off[s], lam[:, s])
            for e in range(3):
                others = np.ones(P)
                for s in range(3):
                    if s != e:
                        others = others * O._lin(off[s], lam[:, s])
                # d/dl_e [boost * prod lin] = (1 - 2 l_e)/2 * prod lin + boost * lin'_e * prod_{s != e} lin
                dF[:, g, e] = 0.5 * (1.0 - 2.0 * lam[:, e]) * tri + boost * _dlin(off[e]) * others
        else:
            s = outer[0]
            l = lam[:, s]
            if off[s] == 2:
                f = -(1.0 + l) * (1.0 - l) * l / 6.0          # -(l - l^3)/6
                df = -(1.0 - 3.0 * l * l) / 6.0
            else:
                f = -(2.0 - l) * l * (1.0 - l) / 6.0          # -(2l - 3l^2 + l^3)/6
                df = -(2.0 - 6.0 * l + 3.0 * l * l) / 6.0
            ts = [t for t in range(3) if t != s]
            lin = {t: O._lin(off[t], lam[:, t]) for t in ts}
            dF[:, g, s] = df * lin[ts[0]] * lin[ts[1]]
            dF[:, g, ts[0]] = f * _dlin(off[ts[0]]) * lin[ts[1]]
            dF[:, g, ts[1]] = f * lin[ts[0]] * _dlin(off[ts[1]])
    return offs, F, dF


def gather_jacobian(f, X, H, L, order):
    """J[p, d, e] = d/dX_e of (I* f_d)(X_p) for component grids f (ncomp, H, H, H):
    (H/L) sum_gamma dF_gamma/dlambda_e f_d[q_{p,gamma}]."""
    cell, lam = O.cell_and_lambda(X, H, L)
    offs, _, dF = stencil_grad(lam, order)
    idx = O.stencil_indices(cell, offs, H)
    flat = f.reshape(f.shape[0], H ** 3)
    return (H / L) * np.einsum("dpg,pge->pde", flat[:, idx], dF)


def deposit_adjoint(X, w, phibar, H, L, order):
    """Transpose of X -> I rho-hat(X) applied to a grid cotangent phibar:
    dX_p = w (H/L) sum_gamma grad_lambda F_gamma(lambda(X_p)) phibar[q_{p,gamma}], shape (P, 3)."""
    cell, lam = O.cell_and_lambda(X, H, L)
    offs, _, dF = stencil_grad(lam, order)
    idx = O.stencil_indices(cell, offs, H)
    return w * (H / L) * np.einsum("pg,pge->pe", phibar.reshape(-1)[idx], dF)


# ---------------------------------------------------------------------------
# The Fourier-side factors and transposes.
# ---------------------------------------------------------------------------
def propagator_factors(p, H):
    """(A_q, B_q) with alpha^n = A alpha^{n-1} + B beta^{n-1}."""
    qx, qy, qz = O.mode_numbers(H)
    y2 = (O.TWO_PI / p.L) ** 2 * (qx ** 2 + qy ** 2 + qz ** 2)
    if p.propagator == "exp":
        kap = np.exp(-p.dt / p.eps * (y2 + p.k ** 2))
        return kap, kap * p.dt
    return 1.0 / (1.0 + p.dt / p.eps * (y2 + p.k ** 2)), 1.0 / (y2 + p.k ** 2 + p.eps / p.dt)


def gradient_multipliers(p, H):
    """m_d(q) = 2 pi i q_d / L * Phi_q, zero on the plane q_d = -H/2 (shape (3, H, H, H/2+1))."""
    qs = O.mode_numbers(H)
    Phi = O.filter_phi(H, p.H0_eff)
    shape = (H, H, H // 2 + 1)
    m = np.empty((3,) + shape, dtype=np.complex128)
    for d in range(3):
        qd = np.broadcast_to(qs[d], shape)
        m[d] = np.where(qd == -(H // 2), 0.0, 1j * (O.TWO_PI * qd / p.L) * Phi)
    return m


def forward_ft_T(betabar, p):
    """Transpose of phi -> F_H phi: L^-3 F_H^{-1} betabar (a real grid)."""
    return O.inverse_ft(betabar, p.H) / p.L ** 3


def gradient_grids_T(gbar, p):
    """Transpose of alpha -> gradient grids: sum_d conj(m_d) DFT(gbar_d) (half spectrum)."""
    m = gradient_multipliers(p, p.H)
    return sum(np.conj(m[d]) * np.fft.rfftn(gbar[d]) for d in range(3))


def spectral_inner(u, v):
    """Re sum over the full spectrum of conj(u) v, from half spectra of real fields."""
    H = u.shape[0]
    mult = np.full(u.shape[2], 2.0)
    mult[0] = 1.0
    mult[H // 2] = 1.0
    return float(np.sum(mult[None, None, :] * np.real(np.conj(u) * v)))


# ---------------------------------------------------------------------------
# Forward with stored states, and the reverse sweep.
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Trajectory:
    X: list        # X^0 .. X^N (P, 3)
    alpha: list    # alpha^0 .. alpha^N


def forward(X0, p, nsteps):
    s = O.init_state(X0, p)
    traj = Trajectory([s.X.copy()], [s.alpha.copy()])
    for _ in range(nsteps):
        s = O.step(s, p)
        traj.X.append(s.X.copy())
        traj.alpha.append(s.alpha.copy())
    return traj


def density(X, p):
    """rho(T) on the grid: the deposited masses over the cell volume, phi / h^3."""
    h3 = (p.L / p.H) ** 3
    return O.deposit(X, p.mass / p.P, p.H, p.L, p.p2g_order) / h3


def loss(rho, rho_star):
    """J = sum_j (rho_j - rho*_j)^2 and its cotangent dJ/drho."""
    d = rho - rho_star
    return float(np.sum(d * d)), 2.0 * d


@dataclasses.dataclass
class Gradients:
    chi: float
    mu: float
    X0: np.ndarray


def adjoint(traj, p, rhobar):
    """dJ/dchi, dJ/dmu, dJ/dX^0 for J with dJ/drho(T) = rhobar, by the reverse
    sweep over the stored trajectory (noise regenerated from its counter)."""
    H, L, P = p.H, p.L, p.P
    N = len(traj.X) - 1
    w = p.mass / P
    h3 = (L / H) ** 3
    A, B = propagator_factors(p, H)
    half = p.splitting == "half"
    s = math.sqrt(p.mu * p.dt) if half else math.sqrt(2.0 * p.mu * p.dt)
    ds_dmu = 0.5 * s / p.mu if p.mu > 0 else 0.0
    # terminal cotangents: rho(T) = phi^N / h^3 and nothing reads alpha^N
    Xbar = deposit_adjoint(traj.X[N], w, rhobar / h3, H, L, p.p2g_order)
    abar = np.zeros_like(traj.alpha[0])
    chibar = 0.0
    sbar = 0.0
    for n in range(N, 0, -1):
        Xp, ap = traj.X[n - 1], traj.alpha[n - 1]
        grads = O.gradient_grids(ap, p)
        z = O.normals(p.seed, n, P)
        Xq = Xp + s * z[:, 0:3] if half else Xp          # point where the gradient is gathered
        V = O.gather(grads, Xq, H, L, p.g2p_order).T
        Jac = gather_jacobian(grads, Xq, H, L, p.g2p_order)
        chibar += p.dt * float(np.sum(V * Xbar))
        Ybar = Xbar + p.chi * p.dt * np.einsum("pde,pd->pe", Jac, Xbar)
        if half:
            sbar += float(np.sum(z[:, 0:3] * Ybar) + np.sum(z[:, 3:6] * Xbar))
        else:
            sbar += float(np.sum(z[:, 0:3] * Xbar))
        gbar = np.stack([O.deposit(Xq, p.chi * p.dt * Xbar[:, d], H, L, p.g2p_order) for d in range(3)])
        # alpha^n = A alpha^{n-1} + B beta^{n-1};  g^{n-1} = Gop alpha^{n-1}
        betabar = B * abar
        abar = A * abar + gradient_grids_T(gbar, p)
        phibar = forward_ft_T(betabar, p)
        Xbar = Ybar + deposit_adjoint(Xp, w, phibar, H, L, p.p2g_order)
    return Gradients(chibar, sbar * ds_dmu, Xbar)


def loss_and_gradients(X0, p, nsteps, rho_star):
    traj = forward(X0, p, nsteps)
    J, rhobar = loss(density(traj.X[-1], p), rho_star)
    return J, adjoint(traj, p, rhobar)
