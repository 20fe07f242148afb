"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these re-types an oracle formula: each checks a property the paper
states (constants, identities, error bounds, conservation laws) or a closed
form / brute-force result that a wrong sign, index, factor or dropped term in
the oracle would violate.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import sipf_oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _rand_lam(n, seed=1):
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(n, 3))


# ----------------------------------------------------------------- stencils
@pytest.mark.parametrize("order", [2, 4])
def test_partition_of_unity(order):
    lam = _rand_lam(1000)
    _, W = O.stencil(lam, order)
    assert np.max(np.abs(W.sum(axis=1) - 1.0)) < 1e-14


@pytest.mark.parametrize("order,maxdeg", [(2, 1), (4, 3)])
def test_polynomial_reproduction(order, maxdeg):
    """I_eta is exact on polynomials of degree <= eta-1 (Sec. 3.3, proof of
    Thm:P2G); the local coordinate of node gamma relative to X is gamma - lambda."""
    lam = _rand_lam(500)
    offs, W = O.stencil(lam, order)
    for a, b, c in itertools.product(range(maxdeg + 1), repeat=3):
        if a + b + c > maxdeg:
            continue
        d = offs[None, :, :] - lam[:, None, :]
        vals = d[..., 0] ** a * d[..., 1] ** b * d[..., 2] ** c
        target = 1.0 if a + b + c == 0 else 0.0
        assert np.max(np.abs((W * vals).sum(axis=1) - target)) < 1e-13, (a, b, c)


def test_gamma4_not_exact_at_degree_four():
    lam = _rand_lam(200)
    offs, W = O.stencil(lam, 4)
    d = offs[None, :, :] - lam[:, None, :]
    err = np.abs((W * d[..., 0] ** 4).sum(axis=1))
    assert err.max() > 1e-3


def test_gamma2_multilinear_and_nonnegative():
    lam = _rand_lam(500)
    offs, W = O.stencil(lam, 2)
    assert W.min() >= 0.0
    d = offs[None, :, :] - lam[:, None, :]
    vals = d[..., 0] * d[..., 1] * d[..., 2]
    assert np.max(np.abs((W * vals).sum(axis=1))) < 1e-14      # trilinear is exact on x1 x2 x3


def test_gamma4_cluster_identity_and_signs():
    """-(F_211 + F_121 + F_112) = l1 l2 l3 (3 - |l|^2)/6; outer weights <= 0,
    inner >= 0; sum of outer weights >= -1/2 (Sec. 3.3, proof of Thm:P2G)."""
    lam = _rand_lam(1000)
    offs, W = O.stencil(lam, 4)
    col = {tuple(o): i for i, o in enumerate(offs)}
    lhs = -(W[:, col[(2, 1, 1)]] + W[:, col[(1, 2, 1)]] + W[:, col[(1, 1, 2)]])
    l1, l2, l3 = lam.T
    rhs = l1 * l2 * l3 * (3.0 - l1 ** 2 - l2 ** 2 - l3 ** 2) / 6.0
    assert np.max(np.abs(lhs - rhs)) < 1e-15
    inner = np.all((offs >= 0) & (offs <= 1), axis=1)
    assert W[:, inner].min() >= 0.0
    assert W[:, ~inner].max() <= 0.0
    assert W[:, ~inner].sum(axis=1).min() >= GOLD["outer_sum_bound"]["value"] - 1e-15
    # the eight clusters add up to -sum_k lambda_k (1 - lambda_k)/2
    assert np.max(np.abs(W[:, ~inner].sum(axis=1) + np.sum(lam * (1 - lam), axis=1) / 2)) < 1e-15


@pytest.mark.parametrize("order", [2, 4])
def test_deposit_continuous_across_cell_faces(order):
    """Moving a particle across a cell face changes the deposited grid
    continuously (the floor() in lambda does not leak into the result)."""
    H, L = 8, 1.0
    h = L / H
    base = np.array([[0.13, -0.21, 0.07]])
    for axis in range(3):
        face = np.floor(base[0, axis] / h) * h + h
        Xa, Xb = base.copy(), base.copy()
        Xa[0, axis] = face - 1e-12
        Xb[0, axis] = face + 1e-12
        da = O.deposit(Xa, 1.0, H, L, order)
        db = O.deposit(Xb, 1.0, H, L, order)
        assert np.max(np.abs(da - db)) < 1e-9


# ----------------------------------------------------------------- deposit / FFT
def test_fft_matches_brute_force_dft():
    """forward_ft / inverse_ft equal the defining sums of F_H and F_H^{-1}
    (Sec. 3.1) evaluated by brute force at H = 8."""
    H, L = 8, 1.7
    rng = np.random.default_rng(3)
    phi = rng.normal(size=(H, H, H))
    j = np.arange(H)
    q = np.where(j < H // 2, j, j - H)
    beta = O.forward_ft(phi, L)
    # physical node x_j = j h with j in [-H/2, H/2) stored at j mod H
    jphys = np.where(j < H // 2, j, j - H)
    for (a, b, c) in [(0, 0, 0), (1, 2, 3), (7, 5, 4), (4, 4, 4), (3, 6, 2)]:
        y = 2 * np.pi / L * np.array([q[a], q[b], q[c] if c < H // 2 else -(H // 2)])
        tot = 0j
        for i1, i2, i3 in itertools.product(range(H), repeat=3):
            x = L / H * np.array([jphys[i1], jphys[i2], jphys[i3]])
            tot += np.exp(-1j * y @ x) * phi[i1, i2, i3]
        assert abs(beta[a, b, c] - tot / L ** 3) < 1e-12 * (1 + abs(tot))
    # inverse: sum_q G_q e^{i y x_j} with a Hermitian G built from a real field
    G = beta
    g = O.inverse_ft(G, H)
    full = np.fft.fftn(phi) / L ** 3
    for (i1, i2, i3) in [(0, 0, 0), (1, 2, 3), (7, 7, 1)]:
        x = L / H * np.array([jphys[i1], jphys[i2], jphys[i3]])
        tot = 0j
        for a, b, c in itertools.product(range(H), repeat=3):
            y = 2 * np.pi / L * np.array([q[a], q[b], q[c]])
            tot += full[a, b, c] * np.exp(1j * y @ x)
        assert abs(g[i1, i2, i3] - tot.real) < 1e-11
        assert abs(g[i1, i2, i3] - phi[i1, i2, i3] * H ** 3 / L ** 3) < 1e-10


def test_deposit_fft_equals_direct_sum_over_stencil_points():
    """F_H I(rho-hat)(y) = M0/(P L^3) sum_p sum_gamma F_{p,gamma} e^{-i y.X_{p,gamma}}
    (Eq. (FH)), with X_{p,gamma} the physical (unwrapped) stencil points."""
    H, L, M0, P = 8, 1.3, 5.0, 37
    rng = np.random.default_rng(4)
    X = rng.uniform(-L / 2, L / 2, size=(P, 3))
    beta = O.forward_ft(O.deposit(X, M0 / P, H, L, 4), L)
    cell, lam = O.cell_and_lambda(X, H, L)
    offs, F = O.stencil(lam, 4)
    pts = (cell[:, None, :] + offs[None]) * (L / H)            # (P, 32, 3)
    qx, qy, qz = O.mode_numbers(H)
    for (a, b, c) in [(0, 0, 0), (1, 0, 0), (2, 7, 3), (5, 5, 4), (4, 1, 2)]:
        y = 2 * np.pi / L * np.array([qx[a, 0, 0], qy[0, b, 0], qz[0, 0, c]])
        direct = (M0 / (P * L ** 3)) * np.sum(F * np.exp(-1j * pts @ y))
        assert abs(beta[a, b, c] - direct) < 1e-13


def test_mass_conservation_and_zero_mode():
    """int I rho-hat = M0 (Sec. 3.4) and beta_0 = M0 / L^3."""
    H, L, M0, P = 16, 2.0, 7.5, 5000
    X = np.random.default_rng(5).uniform(-L / 2, L / 2, size=(P, 3))
    for order in (2, 4):
        phi = O.deposit(X, M0 / P, H, L, order)
        assert abs(phi.sum() - M0) < 1e-12 * M0
        assert abs(O.forward_ft(phi, L)[0, 0, 0] - M0 / L ** 3) < 1e-12


@pytest.mark.parametrize("order,Ckey,eta", [(2, "C2", 2), (4, "C4", 4)])
def test_p2g_spectral_error_bound(order, Ckey, eta):
    """|F_H I_eta rho-hat - F_H rho-hat|(y) <= C_eta M0 L^-3 |y|^eta (L/H)^eta
    per mode (Thm:P2G), against the direct sum of Eq. (beta_hat_comp)."""
    H, L, M0, P = 16, 1.0, 10.0, 400
    X = np.random.default_rng(6).normal(0, 0.15, size=(P, 3))
    X = O.wrap(X, L)
    beta_pic = O.forward_ft(O.deposit(X, M0 / P, H, L, order), L)
    beta_dir = O.direct_beta(X, M0 / P, H, L)[:, :, : H // 2 + 1]
    qx, qy, qz = O.mode_numbers(H)
    # direct_beta's kz axis uses q in [0, H/2) then -H/2: same as mode_numbers
    y = 2 * np.pi / L * np.sqrt(qx ** 2 + qy ** 2 + qz ** 2)
    bound = GOLD[Ckey]["value"] * M0 / L ** 3 * y ** eta * (L / H) ** eta
    err = np.abs(beta_pic - beta_dir)
    assert np.all(err <= bound + 1e-12)
    # and the error is genuinely of that order for the larger modes
    assert err.max() > 1e-6


# ----------------------------------------------------------------- gather / gradient
def _planted(H, L, qv, amp):
    """alpha with a single real cosine mode: c(x) = 2 Re(amp e^{i y.x})."""
    alpha = np.zeros((H, H, H // 2 + 1), dtype=np.complex128)
    a, b, c = (qv[0] % H, qv[1] % H, qv[2])
    alpha[a, b, c] = amp
    return alpha


def test_gradient_grid_of_planted_mode_is_analytic():
    """grad c at the nodes equals the analytic gradient of the planted
    trigonometric polynomial (sign of e^{+iyx}, factor 2 pi / L, filter Phi)."""
    H, L = 16, 1.5
    p = O.Params(P=1, H=H, L=L, H0=9.0)
    qv = np.array([2, -3, 1])
    amp = 0.3 - 0.4j
    alpha = _planted(H, L, qv, amp)
    g = O.gradient_grids(alpha, p)
    j = np.arange(H)
    jp = np.where(j < H // 2, j, j - H) * (L / H)
    x = np.stack(np.meshgrid(jp, jp, jp, indexing="ij"), axis=-1)
    y = 2 * np.pi / L * qv
    phase = x @ y
    Phi = math.exp(-2 * math.pi ** 2 * np.sum(qv ** 2) / 81.0)
    # c = amp e^{i y x} + conj; grad = 2 Re(i y amp e^{iyx}) Phi
    ana = np.stack([2 * np.real(1j * y[d] * amp * np.exp(1j * phase)) * Phi for d in range(3)])
    assert np.max(np.abs(g - ana)) < 1e-12


def test_gradient_nyquist_plane_zeroed_and_field_real():
    H, L = 8, 1.0
    p = O.Params(P=1, H=H, L=L, H0=0)
    rng = np.random.default_rng(7)
    field = rng.normal(size=(H, H, H))
    alpha = O.forward_ft(field, L)
    G = O.gradient_spectrum(alpha, p)
    assert np.all(G[0][H // 2] == 0) and np.all(G[1][:, H // 2] == 0) and np.all(G[2][:, :, H // 2] == 0)
    # spectral derivative of a band-limited field: check d/dx of a pure mode
    g = O.gradient_grids(alpha, p)
    assert np.all(np.isfinite(g))


def test_g2p_error_bound_planted_mode():
    """|I*_2 f - f| <= (9/2) max|D^2 f| h^2 (Thm:G2P) for f = d c/dx_d of a
    planted mode, with f known exactly at any point."""
    H, L = 32, 1.0
    p = O.Params(P=1, H=H, L=L, H0=0)
    qv = np.array([1, -2, 1])          # half layout stores q_z >= 0
    amp = 0.5 + 0.1j
    alpha = _planted(H, L, qv, amp)
    g = O.gradient_grids(alpha, p)
    X = np.random.default_rng(8).uniform(-L / 2, L / 2, size=(300, 3))
    got = O.gather(g, X, H, L, 2)
    y = 2 * np.pi / L * qv
    e = np.exp(1j * X @ y)
    exact = np.stack([2 * np.real(1j * y[d] * amp * e) for d in range(3)])
    # |D^2 f| <= 2 |amp| |y_d| |y|^2 for each second derivative
    for d in range(3):
        K2 = GOLD["K2_factor"]["value"] * 2 * abs(amp) * abs(y[d]) * np.max(np.abs(y)) ** 2
        assert np.max(np.abs(got[d] - exact[d])) <= K2 * (L / H) ** 2
    assert np.max(np.abs(got - exact)) > 1e-6      # not trivially exact


@pytest.mark.parametrize("order", [2, 4])
def test_adjoint_relation(order):
    """<I rho, f> = <rho, I* f> for the same stencil (Sec. 3.1)."""
    H, L, P = 8, 1.0, 50
    rng = np.random.default_rng(9)
    X = rng.uniform(-L / 2, L / 2, size=(P, 3))
    w = rng.uniform(0.5, 2.0, size=P)
    f = rng.normal(size=(H, H, H))
    lhs = np.sum(O.deposit(X, w, H, L, order) * f)
    rhs = np.sum(w * O.gather(f, X, H, L, order))
    assert abs(lhs - rhs) < 1e-12 * (1 + abs(lhs))


# ----------------------------------------------------------------- spectral update
def test_zero_mode_recurrence_and_ode():
    """With beta_0 = M0/L^3 fixed, the zero mode obeys alpha0^n = a*(1 - r^n),
    a* = M0/(L^3 k^2), r = 1/(1 + tau k^2/eps), and approaches the solution of
    eps c0' = -k^2 c0 + M0/L^3 to O(tau)."""
    H, L, M0, k, eps, tau = 8, 1.0, 10.0, 1.0, 1.0, 1e-3
    p = O.Params(P=1, H=H, L=L, mass=M0, k=k, eps=eps, dt=tau)
    alpha = np.zeros((H, H, H // 2 + 1), dtype=np.complex128)
    beta = np.zeros_like(alpha)
    beta[0, 0, 0] = M0 / L ** 3
    astar = M0 / (L ** 3 * k ** 2)
    r = 1.0 / (1.0 + tau * k ** 2 / eps)
    for n in range(1, 201):
        alpha = O.update_alpha(alpha, beta, p)
        assert abs(alpha[0, 0, 0].real - astar * (1 - r ** n)) < 1e-13 * astar
    t = 200 * tau
    ode = astar * (1 - math.exp(-k ** 2 * t / eps))
    assert abs(alpha[0, 0, 0].real - ode) < 2 * tau * astar
    assert abs(alpha[0, 0, 0].real - ode) > 1e-6 * astar   # first-order, not exact


def test_mode_relaxes_to_pde_steady_state():
    """For a fixed source the update converges to the steady state of
    eps c_t = Lap c - k^2 c + rho, i.e. alpha_q = beta_q / (|y_q|^2 + k^2),
    at the implicit-Euler rate 1/(1 + tau/eps (|y|^2 + k^2))."""
    H, L = 8, 2.0
    p = O.Params(P=1, H=H, L=L, k=0.7, eps=0.3, dt=0.05)
    rng = np.random.default_rng(10)
    beta = rng.normal(size=(H, H, H // 2 + 1)) + 1j * rng.normal(size=(H, H, H // 2 + 1))
    alpha = np.zeros_like(beta)
    for _ in range(3000):
        alpha = O.update_alpha(alpha, beta, p)
    qx, qy, qz = O.mode_numbers(H)
    lam = (2 * np.pi / L) ** 2 * (qx ** 2 + qy ** 2 + qz ** 2) + p.k ** 2
    assert np.max(np.abs(alpha - beta / lam)) < 1e-10
    a1 = O.update_alpha(np.zeros_like(beta), beta, p)
    a2 = O.update_alpha(a1, beta, p)
    kappa = 1.0 / (1.0 + p.dt / p.eps * lam)
    assert np.max(np.abs((a2 - beta / lam) - kappa * (a1 - beta / lam))) < 1e-12


def test_exp_propagator_total_concentration():
    """Sec. 3.4 mass law for the exponential propagator (eps = 1):
    int c^n = e^{-k^2 n tau} int c^0 + tau M0 sum_{s=1}^n e^{-k^2 s tau}."""
    H, L, M0, k, tau = 8, 1.0, 3.0, 0.8, 0.01
    p = O.Params(P=1, H=H, L=L, mass=M0, k=k, eps=1.0, dt=tau)
    alpha = np.zeros((H, H, H // 2 + 1), dtype=np.complex128)
    alpha[0, 0, 0] = 0.25
    c0 = alpha[0, 0, 0].real * L ** 3
    beta = np.zeros_like(alpha)
    beta[0, 0, 0] = M0 / L ** 3
    for n in range(1, 51):
        alpha = O.update_alpha_exp(alpha, beta, p)
        law = math.exp(-k ** 2 * n * tau) * c0 + tau * M0 * sum(math.exp(-k ** 2 * s * tau) for s in range(1, n + 1))
        assert abs(alpha[0, 0, 0].real * L ** 3 - law) < 1e-12 * law


# ----------------------------------------------------------------- noise
def test_uniforms_are_uniform_and_distinct():
    u = O.uniforms(seed=123, step=7, P=20000)
    assert u.min() > 0 and u.max() < 1
    for c in range(8):
        assert stats.kstest(u[:, c], "uniform").pvalue > 1e-4
    assert abs(np.corrcoef(u[:, 0], u[:, 4])[0, 1]) < 0.03
    u2 = O.uniforms(seed=123, step=8, P=20000)
    u3 = O.uniforms(seed=124, step=7, P=20000)
    assert abs(np.corrcoef(u[:, 0], u2[:, 0])[0, 1]) < 0.03
    assert abs(np.corrcoef(u[:, 0], u3[:, 0])[0, 1]) < 0.03
    # counters are per particle: a sub-range reproduces the same numbers
    assert np.array_equal(O.uniforms(123, 7, 100, first=500), u[500:600])


def test_normals_distribution():
    z = O.normals(seed=5, step=1, P=50000)
    for c in range(6):
        assert stats.kstest(z[:, c], "norm").pvalue > 1e-4
        assert abs(z[:, c].mean()) < 0.03 and abs(z[:, c].var() - 1) < 0.03
    C = np.corrcoef(z.T)
    assert np.max(np.abs(C - np.eye(6))) < 0.03


def test_philox_is_a_bijection_on_a_sample_of_counters():
    """For a fixed key Philox is a permutation of counters: distinct counters
    never collide in a large sample."""
    n = 200000
    c = np.arange(n, dtype=np.uint64)
    out = O.philox4x32_10(c, 0, 0, 0, 0xDEADBEEF, 0x12345678)
    key = (out[0] << np.uint64(32)) | out[1]
    assert np.unique(key).size == n


# ----------------------------------------------------------------- whole step
def test_first_step_has_zero_drift_and_chi0_moves_are_pure_noise():
    """alpha^0 = 0 gives zero drift in step 1; with chi = 0 every step is
    X^n = X^{n-1} + W^- + W^+ (up to the periodic wrap)."""
    p = O.Params(P=500, H=8, L=1.0, chi=0.0, mu=0.7, dt=1e-3, seed=3)
    X0 = O.wrap(np.random.default_rng(11).normal(0, 0.1, size=(p.P, 3)), p.L)
    s = O.init_state(X0, p)
    disp = np.zeros_like(X0)
    for n in range(1, 6):
        s = O.step(s, p)
        z = O.normals(p.seed, n, p.P)
        disp += math.sqrt(p.mu * p.dt) * (z[:, 0:3] + z[:, 3:6])
    d = O.min_image(s.X - X0 - disp, p.L)
    assert np.max(np.abs(d)) < 1e-14
    p1 = O.Params(P=500, H=8, L=1.0, chi=1.0, mu=0.7, dt=1e-3, seed=3)
    s1 = O.step(O.init_state(X0, p1), p1)
    z = O.normals(p1.seed, 1, p1.P)
    expect = O.wrap(X0 + math.sqrt(p1.mu * p1.dt) * (z[:, :3] + z[:, 3:]), p1.L)
    assert np.max(np.abs(O.min_image(s1.X - expect, 1.0))) < 1e-15


def test_chi0_second_moment_grows_2_mu_t():
    """Free diffusion: E|Delta X_d|^2 = 2 mu t per dimension (the SDE with chi = 0)."""
    p = O.Params(P=20000, H=8, L=10.0, chi=0.0, mu=0.5, dt=2e-3, seed=21)
    X0 = np.zeros((p.P, 3))
    s = O.run(X0, p, 10)
    t = 10 * p.dt
    var = np.mean(O.min_image(s.X - X0, p.L) ** 2, axis=0)
    tol = 5 * 2 * p.mu * t * math.sqrt(2.0 / p.P)
    assert np.all(np.abs(var - 2 * p.mu * t) < tol)


def test_plain_em_uses_doubled_variance():
    p = O.Params(P=20000, H=8, L=10.0, chi=0.0, mu=0.5, dt=2e-3, seed=22, splitting="plain")
    s = O.run(np.zeros((p.P, 3)), p, 10)
    var = np.mean(O.min_image(s.X, p.L) ** 2, axis=0)
    assert np.all(np.abs(var - 2 * p.mu * 10 * p.dt) < 5 * 2 * p.mu * 10 * p.dt * math.sqrt(2.0 / p.P))


def test_pic_step_tracks_direct_sum_method():
    """SIPF-PIC vs the direct-sum method (Algorithm 1 operators, same noise,
    same filter and splitting): for a field the filter keeps smooth, the
    particle paths agree to the interpolation error, which falls at second
    order in h (Thm:G2P dominates; Thm:P2G is fourth order)."""
    errs = []
    for H in (8, 16, 32):
        p = O.Params(P=300, H=H, L=1.0, mass=20.0, chi=1.0, mu=1.0, eps=1.0, k=1.0,
                     dt=2e-3, H0=6.0, seed=2)
        X0 = O.wrap(np.random.default_rng(12).normal(0, 0.15, size=(p.P, 3)), p.L)
        s = O.init_state(X0, p)
        Xd, ad = X0.copy(), np.zeros((H, H, H), dtype=np.complex128)
        for n in range(1, 5):
            s = O.step(s, p)
            Xd, ad = O.direct_step(Xd, ad, p, n)
        da = np.max(np.abs(s.alpha - ad[:, :, : H // 2 + 1])) / np.max(np.abs(ad))
        dx = np.max(np.abs(O.min_image(s.X - Xd, p.L)))
        errs.append((da, dx))
    assert errs[-1][1] < 1e-4
    for (a0, x0), (a1, x1) in zip(errs, errs[1:]):
        assert x0 / x1 > 2.5 and a0 / a1 > 2.5


def test_diagnostics_consistency():
    p = O.Params(P=3000, H=16, L=1.0, mass=10.0, H0=0)
    X = O.wrap(np.random.default_rng(13).normal(0, 0.1, size=(p.P, 3)), p.L)
    s = O.init_state(X, p)
    d = O.diagnostics(s, p)
    assert abs(d["mass"] - 10.0) < 1e-12
    # with the filter off, rho_num is the deposited density phi / h^3
    phi = O.deposit(X, p.mass / p.P, p.H, p.L, 4)
    assert abs(d["peak"] - phi.max() / (p.L / p.H) ** 3) < 1e-9 * d["peak"]
    assert abs(d["m2"] - np.mean(np.sum(X ** 2, 1))) < 1e-15


def _curand_host():
    import ctypes
    import ctypes.util
    for name in ("libcurand.so", "libcurand.so.10", ctypes.util.find_library("curand")):
        if not name:
            continue
        for base in ("", "/usr/local/cuda/lib64/"):
            try:
                return ctypes.CDLL(base + name)
            except OSError:
                pass
    return None


def test_philox_matches_curand_host_generator():
    """Library pin: cuRAND's host-side PHILOX4_32_10 generator (default
    ordering) emits block i = Philox4x32-10(counter (0, 0, i, 0), key (seed lo,
    seed hi)); the oracle's Philox must reproduce those words exactly."""
    import ctypes
    lib = _curand_host()
    if lib is None:
        pytest.skip("libcurand not available")
    for seed in (0x123456789, 7, 0xFEDCBA9876543210):
        gen = ctypes.c_void_p()
        assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0   # PHILOX4_32_10
        try:
            assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            n = 4 * 512
            buf = (ctypes.c_uint32 * n)()
            assert lib.curandGenerate(gen, buf, n) == 0
        finally:
            lib.curandDestroyGenerator(gen)
        got = np.frombuffer(buf, dtype=np.uint32).reshape(-1, 4).astype(np.uint64)
        i = np.arange(got.shape[0], dtype=np.uint64)
        ref = np.stack(O.philox4x32_10(0, 0, i, 0, seed & 0xFFFFFFFF, seed >> 32), axis=1)
        assert np.array_equal(got, np.broadcast_to(ref, got.shape))


# ----------------------------------------------------------------- filter scale and HF-energy share
def test_auto_H0_exact_values():
    """H0 = ceil(8 H^(8/13) L^(5/13)) (Sec. 5.1).  Exact powers fix each
    exponent separately: H = 2^13, L = 1 gives 8 * 2^8 = 2048 (the H exponent),
    H = 1, L = 2^13 gives 8 * 2^5 = 256 (the L exponent); swapping or mistyping
    either fails.  H = L = 8 is the geometry of the Sec. 5.1 convergence study
    and gives exactly 8 * 8^(8/13) * 8^(5/13) = 64 (not 65)."""
    assert O.auto_H0(2 ** 13, 1.0) == 2048.0
    assert O.auto_H0(1, 2.0 ** 13) == 256.0
    assert O.auto_H0(8, 8.0) == 64.0
    assert O.auto_H0(2 ** 16, 8.0) == 8.0 * 2 ** 11      # 8 * 2^((8*16 + 15)/13)


@pytest.mark.parametrize("H,L", [(16, 1.0), (128, 1.0), (64, 2.0), (256, 8.0), (32, 0.7)])
def test_auto_H0_is_the_smallest_integer_above_the_rule(H, L):
    """Brute force on the definition: m = H0 satisfies m^13 >= 8^13 H^8 L^5 >
    (m-1)^13 in exact rational arithmetic."""
    from fractions import Fraction
    m = int(O.auto_H0(H, L))
    t = Fraction(8) ** 13 * Fraction(H) ** 8 * Fraction(L) ** 5
    assert Fraction(m) ** 13 >= t > Fraction(m - 1) ** 13


def _half(full):
    """Half layout (qz index 0..H/2) of a full H^3 spectrum."""
    H = full.shape[0]
    return full[:, :, : H // 2 + 1].copy()


def test_hf_energy_fraction_planted_modes():
    """Sec. 5.2 indicator: share of sum_q |alpha_q|^2 over the FULL spectrum in
    modes with ||q|| >= 4.  Planted Hermitian pairs with known energies:
    (+-3,0,0) amplitude 1 on the kz = 0 plane (both members stored), (0,0,+-3)
    amplitude 2 off it (only +3 stored), (+-4,0,0) amplitude 4 on the plane,
    (0,0,+-4) amplitude 3 off it, and (0,0,-8) amplitude 1 on the Nyquist
    plane (its own partner at H = 16).  Full energies: ||q|| = 3: 2 + 8 = 10;
    ||q|| >= 4: 32 + 18 + 1 = 51; share 51/61.  Counting the kz = 0 plane
    twice, the Nyquist plane twice, the off-plane modes once, or using
    ||q|| > 4, each gives another value."""
    H = 16
    full = np.zeros((H, H, H), dtype=complex)

    def plant(q, a):
        full[q[0] % H, q[1] % H, q[2] % H] = a
        full[-q[0] % H, -q[1] % H, -q[2] % H] = np.conj(a)

    plant((3, 0, 0), 1.0)
    plant((0, 0, 3), 2.0)
    plant((4, 0, 0), 4.0j)
    plant((0, 0, 4), 3.0)
    plant((0, 0, -8), 1.0)
    assert O.hf_energy_fraction(_half(full)) == pytest.approx(51.0 / 61.0, rel=1e-15)


def test_hf_energy_fraction_matches_full_spectrum_of_a_real_field():
    """Library special case: for a real field f, numpy's full complex FFT holds
    every mode once; the share of |F_q|^2 with ||q|| >= 4 from it must equal the
    oracle's share computed from the r2c half layout."""
    H = 16
    f = np.random.default_rng(5).normal(size=(H, H, H))
    F = np.fft.fftn(f)
    q = np.fft.fftfreq(H, 1.0 / H)
    qn = np.sqrt(q[:, None, None] ** 2 + q[None, :, None] ** 2 + q[None, None, :] ** 2)
    e = np.abs(F) ** 2
    ref = e[qn >= 4].sum() / e.sum()
    assert O.hf_energy_fraction(np.fft.rfftn(f)) == pytest.approx(ref, rel=1e-13)
