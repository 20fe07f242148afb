"""Pins of the FP64 CPU adjoint (oracle/sipf_adjoint.py) against things other
than itself: derivatives of the weight polynomials by central differences,
the transposition identities of the linear operators (<A x, y> = <x, A^T y>,
spectra under the real inner product of full Hermitian spectra), and the
whole reverse sweep against central differences of the forward oracle.
"""
import math

import numpy as np
import pytest

from oracle import sipf_adjoint as A
from oracle import sipf_oracle as O


@pytest.mark.parametrize("order", [2, 4])
def test_stencil_derivatives_match_central_differences(order):
    rng = np.random.default_rng(order)
    lam = rng.uniform(0.02, 0.98, size=(200, 3))
    _, F, dF = A.stencil_grad(lam, order)
    _, F0 = O.stencil(lam, order)
    assert np.array_equal(F, F0)
    h = 1e-6
    for e in range(3):
        lp, lm = lam.copy(), lam.copy()
        lp[:, e] += h
        lm[:, e] -= h
        fd = (O.stencil(lp, order)[1] - O.stencil(lm, order)[1]) / (2 * h)
        assert np.max(np.abs(fd - dF[:, :, e])) < 1e-8


@pytest.mark.parametrize("order", [2, 4])
def test_weight_derivatives_sum_to_zero(order):
    """Partition of unity (sum_gamma F_gamma = 1) makes the derivatives sum to 0,
    and first-moment reproduction makes sum_gamma gamma_e dF/dl_f = delta_ef."""
    lam = np.random.default_rng(7).uniform(0, 1, size=(100, 3))
    offs, _, dF = A.stencil_grad(lam, order)
    assert np.max(np.abs(dF.sum(axis=1))) < 1e-13
    mom = np.einsum("ge,pgf->pef", offs.astype(float), dF)
    assert np.max(np.abs(mom - np.eye(3)[None])) < 1e-13


def test_deposit_and_gather_are_transposes():
    """<I w, f> = <w, I* f> (the relation after Def. grid2particle, Sec. 3.1) and the position derivative of <I w, f>."""
    rng = np.random.default_rng(1)
    H, L, P = 8, 1.3, 50
    X = rng.uniform(-L / 2, L / 2, size=(P, 3))
    w = rng.normal(size=P)
    f = rng.normal(size=(H, H, H))
    for order in (2, 4):
        lhs = np.sum(O.deposit(X, w, H, L, order) * f)
        rhs = np.sum(w * O.gather(f[None], X, H, L, order)[0])
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))
    # d/dX <I(w0 X), f> = deposit_adjoint, checked by central differences
    w0, h = 0.7, 1e-6
    G = A.deposit_adjoint(X, w0, f, H, L, 4)
    for p, e in [(0, 0), (3, 1), (17, 2), (49, 0)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[p, e] += h
        Xm[p, e] -= h
        fd = (np.sum(O.deposit(Xp, w0, H, L, 4) * f) - np.sum(O.deposit(Xm, w0, H, L, 4) * f)) / (2 * h)
        assert abs(fd - G[p, e]) < 1e-6 * max(1.0, abs(fd))


def test_fourier_transposes():
    rng = np.random.default_rng(2)
    p = O.Params(P=1, H=8, L=1.7, H0=5.0)
    phi = rng.normal(size=(8, 8, 8))
    bbar = np.fft.rfftn(rng.normal(size=(8, 8, 8)))
    assert abs(A.spectral_inner(O.forward_ft(phi, p.L), bbar) - np.sum(phi * A.forward_ft_T(bbar, p))) < 1e-10
    alpha = np.fft.rfftn(rng.normal(size=(8, 8, 8)))
    gbar = rng.normal(size=(3, 8, 8, 8))
    lhs = np.sum(O.gradient_grids(alpha, p) * gbar)
    rhs = A.spectral_inner(alpha, A.gradient_grids_T(gbar, p))
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def _case(**kw):
    d = dict(P=120, H=8, L=1.0, mass=12.0, chi=1.3, mu=0.8, eps=1.0, k=1.0, dt=2e-3, seed=11)
    d.update(kw)
    p = O.Params(**d)
    rng = np.random.default_rng(5)
    X0 = O.wrap(rng.normal(scale=0.15, size=(p.P, 3)), p.L)
    rho_star = rng.uniform(0, 2 * p.mass / p.L ** 3, size=(p.H,) * 3)
    return p, X0, rho_star


def _J(p, X0, nsteps, rho_star):
    return A.loss(A.density(O.run(X0, p, nsteps).X, p), rho_star)[0]


@pytest.mark.parametrize("variant", [{}, dict(splitting="plain"), dict(propagator="exp"),
                                     dict(p2g_order=2, g2p_order=4), dict(H0=0.0)])
def test_adjoint_matches_central_differences(variant):
    p, X0, rho_star = _case(**variant)
    nsteps = 5
    J, g = A.loss_and_gradients(X0, p, nsteps, rho_star)
    assert abs(J - _J(p, X0, nsteps, rho_star)) < 1e-12 * J
    h = 1e-6
    for name in ("chi", "mu"):
        v = getattr(p, name)
        pp = O.Params(**{**p.__dict__, name: v * (1 + h)})
        pm = O.Params(**{**p.__dict__, name: v * (1 - h)})
        fd = (_J(pp, X0, nsteps, rho_star) - _J(pm, X0, nsteps, rho_star)) / (2 * h * v)
        assert abs(fd - getattr(g, name)) < 1e-5 * max(abs(fd), 1e-3 * J), name
    hx = 1e-6 * p.L
    for (i, e) in [(0, 0), (7, 1), (33, 2), (119, 1)]:
        Xp, Xm = X0.copy(), X0.copy()
        Xp[i, e] += hx
        Xm[i, e] -= hx
        fd = (_J(p, Xp, nsteps, rho_star) - _J(p, Xm, nsteps, rho_star)) / (2 * hx)
        assert abs(fd - g.X0[i, e]) < 1e-5 * max(abs(fd), 1e-3 * np.max(np.abs(g.X0))), (i, e)


def test_adjoint_of_free_diffusion_is_closed_form():
    """chi = 0: X^N = X^0 + s sum_n (W^-_n + W^+_n) exactly, so dJ/dX^0 is the
    deposit adjoint at X^N and dJ/dmu = sum_p dJ/dX^N_p . (ds/dmu) sum_n (W^- + W^+)."""
    p, X0, rho_star = _case(chi=0.0)
    nsteps = 4
    J, g = A.loss_and_gradients(X0, p, nsteps, rho_star)
    traj = A.forward(X0, p, nsteps)
    _, rhobar = A.loss(A.density(traj.X[-1], p), rho_star)
    XbarN = A.deposit_adjoint(traj.X[-1], p.mass / p.P, rhobar / (p.L / p.H) ** 3, p.H, p.L, 4)
    assert np.max(np.abs(g.X0 - XbarN)) < 1e-12 * np.max(np.abs(XbarN))
    S = sum(O.normals(p.seed, n, p.P)[:, 0:3] + O.normals(p.seed, n, p.P)[:, 3:6] for n in range(1, nsteps + 1))
    s = math.sqrt(p.mu * p.dt)
    assert abs(g.mu - np.sum(XbarN * S) * s / (2 * p.mu)) < 1e-12 * abs(g.mu)
    assert g.chi != 0.0
