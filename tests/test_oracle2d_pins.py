"""Pins of the 2D oracle (oracle/sipf2d_oracle.py, the parabolic-elliptic
variant of Sec. 5.2) to facts fixed by the paper and by mathematics: the
fourth-order 2D stencil's exactness on cubic polynomials, the transforms on
planted modes, the elliptic solve and gradient of a planted density mode in
closed form, the deposit + F_H against the direct sum over stencil points,
the noise against the 3D generator, pure diffusion for chi = 0, and the
second-moment law dm2/dt = 4 M0 (1 - M0 / (8 pi)) of Eq. (second_moment)."""
import itertools
import math

import numpy as np
import pytest

from oracle import sipf2d_oracle as O2
from oracle import sipf_oracle as O


def _lam(n, seed=1):
    return np.random.default_rng(seed).uniform(size=(n, 2))


@pytest.mark.parametrize("order,maxdeg", [(2, 1), (4, 3)])
def test_stencil_reproduces_polynomials(order, maxdeg):
    lam = _lam(500)
    offs, W = O2.stencil2(lam, order)
    assert np.max(np.abs(W.sum(axis=1) - 1.0)) < 1e-14
    d = offs[None, :, :] - lam[:, None, :]
    for a, b in itertools.product(range(maxdeg + 2), repeat=2):
        if a + b > maxdeg + 1:
            continue
        err = np.max(np.abs((W * d[..., 0] ** a * d[..., 1] ** b).sum(axis=1) - (1.0 if a + b == 0 else 0.0)))
        if a + b <= maxdeg:
            assert err < 1e-13, (a, b)
        elif order == 4 and (a, b) in ((4, 0), (0, 4)):
            assert err > 1e-3          # not exact at degree 4


def test_inverse_transform_of_a_planted_mode():
    """One stored entry at q = (1, 2) stands for the pair q, -q: f_j = 2 cos(2 pi (j1 + 2 j2)/H)."""
    H = 16
    G = np.zeros((H, H // 2 + 1), dtype=complex)
    G[1, 2] = 1.0
    j1, j2 = np.meshgrid(np.arange(H), np.arange(H), indexing="ij")
    assert np.max(np.abs(O2.inverse_ft(G, H) - 2.0 * np.cos(2 * math.pi * (j1 + 2 * j2) / H))) < 1e-13


def test_deposit_fft_equals_direct_sum_over_stencil_points():
    """beta_q = L^-2 sum_p sum_gamma w F_{p,gamma} e^{-i y_q . x_{p,gamma}}, with
    x_{p,gamma} = (floor(H X/L) + gamma) h (F_H of the deposit, Sec. 3.1)."""
    H, L, P = 8, 1.7, 40
    X = O2.wrap(np.random.default_rng(2).uniform(-L, L, size=(P, 2)), L)
    w = 0.3
    beta = O2.forward_ft(O2.deposit(X, w, H, L, 4), L)
    cell, lam = O2.cell_and_lambda(X, H, L)
    offs, F = O2.stencil2(lam, 4)
    pts = (cell[:, None, :] + offs[None, :, :]) * (L / H)
    qx, qy = O2.mode_numbers(H)
    for a in range(H):
        for b in range(H // 2 + 1):
            y = 2 * math.pi * np.array([qx[a, 0], qy[0, b]]) / L
            ref = np.sum(w * F * np.exp(-1j * (pts @ y))) / L ** 2
            assert abs(beta[a, b] - ref) < 1e-12


def test_elliptic_gradient_of_a_planted_density_mode():
    """eps = k = 0: masses phi_j = A cos(y . x_j) give beta = A H^2/(2 L^2) at +-q and
    c = (A H^2 / (L^2 |y|^2)) cos(y . x), so grad c = -(A H^2/(L^2 |y|^2)) y sin(y . x)."""
    H, L, A = 32, 3.0, 0.7
    p = O2.Params2D(P=1, H=H, L=L, H0=0.0)
    j1, j2 = np.meshgrid(np.arange(H), np.arange(H), indexing="ij")
    q = np.array([3, -2])
    y = 2 * math.pi * q / L
    ang = (j1 * q[0] + j2 * q[1]) * (2 * math.pi / H)
    phi = A * np.cos(ang)
    alpha = O2.solve_field(O2.forward_ft(phi, L), None, p)
    g = O2.gradient_grids(alpha, p)
    amp = A * H ** 2 / (L ** 2 * (y @ y))
    assert np.max(np.abs(g[0] + amp * y[0] * np.sin(ang))) < 1e-10 * amp
    assert np.max(np.abs(g[1] + amp * y[1] * np.sin(ang))) < 1e-10 * amp


def test_noise_is_the_first_block_of_the_3d_generator():
    z2 = O2.normals2(12345, 7, 300, first=99)
    z3 = O.normals(12345, 7, 300, first=99)
    assert np.array_equal(z2, z3[:, :4])


def test_chi0_moves_are_the_summed_noise():
    p = O2.Params2D(P=500, H=16, L=4.0, chi=0.0, mu=0.7, dt=1e-3, seed=3)
    X0 = O2.wrap(np.random.default_rng(4).normal(0, 0.5, size=(p.P, 2)), p.L)
    s = O2.init_state(X0, p)
    disp = np.zeros_like(X0)
    for n in range(1, 6):
        s = O2.step(s, p)
        z = O2.normals2(p.seed, n, p.P)
        disp += math.sqrt(p.mu * p.dt) * (z[:, :2] + z[:, 2:])
    assert np.max(np.abs(O2.min_image(s.X - X0 - disp, p.L))) < 1e-13


def _disk(P, M0, seed):
    rng = np.random.default_rng(seed)
    r = np.sqrt(rng.uniform(size=P))
    th = rng.uniform(0, 2 * math.pi, size=P)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


@pytest.mark.parametrize("M0", [10.0, 20.0])
def test_second_moment_law(M0):
    """Sec. 5.2, Eq. (second_moment): on the whole plane, with (k, eps, mu, chi)
    = (0, 0, 1, 1), m2(t)/M0 = m2(0)/M0 + 4 t (1 - M0/(8 pi)) (for the unit disk
    m2(0)/M0 = 1/2, so m2(2)/M0 = 17/2 - M0/pi).  The oracle's particle second
    moment on a box of side 12 (the disk spreads to radius ~2) follows the law
    over 400 steps of 5e-4: the fitted rate within 6% of 4 (1 - M0/(8 pi)).  A
    wrong sign or factor of the drift moves the rate by far more (M0 = 20: 0.82
    against 7.2 repulsive or -2.4 doubled)."""
    P = 2 ** 13
    p = O2.Params2D(P=P, H=128, L=12.0, mass=M0, dt=5e-4, seed=11)
    s = O2.init_state(_disk(P, M0, 5), p)
    ts, m2 = [0.0], [O2.second_moment(s.X)]
    for n in range(1, 401):
        s = O2.step(s, p)
        if n % 50 == 0:
            ts.append(n * p.dt)
            m2.append(O2.second_moment(s.X))
    rate = np.polyfit(ts, m2, 1)[0]
    law = 4.0 * (1.0 - M0 / (8.0 * math.pi))
    assert abs(rate - law) < 0.06 * 4.0, (rate, law)
