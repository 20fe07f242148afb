"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Operator by operator (noise, deposit, gather, forward and inverse F_H) and
for whole steps of Algorithm 4, at sizes the oracle finishes in seconds that
span several blocks and a ragged tail.  Tolerances:
  * FP64 path vs oracle: 1e-10 (relative to the largest value of the compared
    quantity; positions absolute, by minimum image);
  * FP32 path vs the FP64 oracle: 1e-4 on positions after 20 steps and on the
    relative L2 error of the fields, 1e-5 on single operators.
"""
import math

import numpy as np
import pytest

from oracle import sipf_oracle as O
from paper_2512_03452_gb300 import Simulation, _abi, build, make_params, params_from_workload, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TD = {32: torch.float32, 64: torch.float64}
OP_TOL = {32: 1e-5, 64: 1e-12}


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return _abi.load()


def _soa(X, prec):
    t = torch.tensor(np.ascontiguousarray(X.T), dtype=TD[prec], device="cuda").contiguous()
    return t, (t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr())


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _box_points(P, L, seed, edges=True):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-L / 2, L / 2, size=(P, 3))
    if edges and P >= 8:
        X[0] = [-L / 2, -L / 2, -L / 2]
        X[1] = [np.nextafter(L / 2, 0), 0.0, np.nextafter(-L / 2, 0) + L]
        X[2] = [0.0, 0.0, 0.0]
        X[3] = [L / 4, -L / 4, np.nextafter(L / 2, 0)]
    return O.wrap(X, L)


# ----------------------------------------------------------------- operators
@pytest.mark.parametrize("prec", [64, 32])
def test_noise_matches_oracle(prec):
    P, first, step, seed = 1000, 12345, 7, (1 << 40) + 3
    z = torch.empty((6, P), dtype=TD[prec], device="cuda")
    _abi.sipf_noise_dev(prec, seed, step, first, P, z.data_ptr())
    torch.cuda.synchronize()
    ref = O.normals(seed, step, P, first=first).T
    got = z.cpu().numpy()
    if prec == 64:
        assert np.max(np.abs(got - ref)) < 1e-12
    else:
        assert np.max(np.abs(got - ref) / (1 + np.abs(ref))) < 5e-5


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("order", [4, 2])
@pytest.mark.parametrize("H,P", [(8, 1), (16, 1000), (32, 4099), (64, 20000)])
def test_deposit_matches_oracle(prec, order, H, P):
    L, M0 = 1.3, 7.0
    X = _box_points(P, L, seed=H + P)
    t, (x, y, z) = _soa(X, prec)
    grid = torch.empty(H ** 3, dtype=TD[prec], device="cuda")
    _abi.sipf_deposit_dev(prec, x, y, z, P, H, L, M0 / P, order, grid.data_ptr())
    torch.cuda.synchronize()
    got = grid.cpu().numpy().reshape(H, H, H)
    ref = O.deposit(X, M0 / P, H, L, order)
    assert _rel(got, ref) < (1e-12 if prec == 64 else 1e-5)
    assert abs(got.sum() - M0) < (1e-12 if prec == 64 else 1e-4) * M0


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("H,P", [(8, 37), (32, 3001)])
def test_gather_matches_oracle(prec, order, H, P):
    L = 0.9
    X = _box_points(P, L, seed=7 * H + P)
    f = np.random.default_rng(1).normal(size=(3, H, H, H))
    t, (x, y, z) = _soa(X, prec)
    fd = torch.tensor(f.reshape(3, -1), dtype=TD[prec], device="cuda").contiguous()
    out = torch.empty((3, P), dtype=TD[prec], device="cuda")
    _abi.sipf_gather_dev(prec, x, y, z, P, H, L, fd.data_ptr(), 3, order, out.data_ptr())
    torch.cuda.synchronize()
    ref = O.gather(f, X, H, L, order)
    assert _rel(out.cpu().numpy(), ref) < OP_TOL[prec] * 10


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("H", [8, 16, 32, 64, 128, 256])
def test_forward_ft_matches_oracle(prec, H):
    L = 1.7
    phi = np.random.default_rng(H).normal(size=(H, H, H))
    g = torch.tensor(phi.ravel(), dtype=TD[prec], device="cuda")
    spec = torch.empty((H, H, H // 2 + 1, 2), dtype=TD[prec], device="cuda")
    _abi.sipf_forward_ft_dev(prec, H, L, g.data_ptr(), spec.data_ptr())
    torch.cuda.synchronize()
    s = spec.cpu().numpy()
    got = s[..., 0] + 1j * s[..., 1]
    ref = O.forward_ft(phi, L)
    assert _rel(got, ref) < (1e-13 if prec == 64 else 2e-6) * math.log2(H)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("H", [8, 16, 64, 128, 256])
def test_inverse_ft_matches_oracle(prec, H):
    field = np.random.default_rng(H + 1).normal(size=(H, H, H))
    G = O.forward_ft(field, 1.0)
    st = np.stack([G.real, G.imag], axis=-1)
    spec = torch.tensor(st, dtype=TD[prec], device="cuda").contiguous()
    out = torch.empty(H ** 3, dtype=TD[prec], device="cuda")
    _abi.sipf_inverse_ft_dev(prec, H, spec.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    ref = O.inverse_ft(G, H)
    assert _rel(out.cpu().numpy().reshape(H, H, H), ref) < (1e-13 if prec == 64 else 2e-6) * math.log2(H)


# ----------------------------------------------------------------- whole steps
def _oracle_run(w, X0, nsteps, **kw):
    p = O.Params.from_workload(w, **kw)
    s = O.init_state(X0, p)
    for _ in range(nsteps):
        s = O.step(s, p)
    return s, p


def _gpu_run(w, X0, nsteps, **kw):
    with Simulation(params_from_workload(w, **kw), X0) as sim:
        sim.step(nsteps)
        sim.sync()
        return sim.positions(), sim.spectrum(), sim.diagnostics(), sim.density(False)


_VARIANTS = {
    "paper": {},
    "plain_em": dict(splitting=1),
    "exp_propagator": dict(propagator=1),
    "orders_2_4": dict(p2g_order=2, g2p_order=4),
    "no_filter": dict(H0=0.0),
}


@pytest.mark.parametrize("variant", list(_VARIANTS))
def test_step_fp64_matches_oracle(variant):
    """Gaussian blob P=1e4, H=16, 20 steps: FP64 GPU path within 1e-10."""
    w = workloads.small_blob()
    X0 = workloads.sample_positions(w)
    gkw = dict(_VARIANTS[variant], precision=64)
    okw = {k: v for k, v in _VARIANTS[variant].items()}
    if "splitting" in okw:
        okw["splitting"] = "plain"
    if "propagator" in okw:
        okw["propagator"] = "exp"
    s, p = _oracle_run(w, X0, w.steps, **okw)
    X, alpha, diag, dens = _gpu_run(w, X0, w.steps, **gkw)
    assert np.max(np.abs(O.min_image(X - s.X, w.L))) < 1e-10
    assert _rel(alpha, s.alpha) < 1e-10
    phi = O.deposit(s.X, p.mass / p.P, p.H, p.L, p.p2g_order)
    assert _rel(dens * (p.L / p.H) ** 3, phi) < 1e-10


def test_step_fp32_matches_fp64_oracle():
    """FP32 form: positions within 1e-4 over 20 steps, field relative L2 within 1e-4."""
    w = workloads.small_blob()
    X0 = workloads.sample_positions(w)
    s, p = _oracle_run(w, X0, w.steps)
    X, alpha, diag, dens = _gpu_run(w, X0, w.steps, precision=32)
    assert np.max(np.abs(O.min_image(X - s.X, w.L))) < 1e-4
    assert np.linalg.norm(alpha - s.alpha) / np.linalg.norm(s.alpha) < 1e-4
    phi = O.deposit(s.X, p.mass / p.P, p.H, p.L, 4)
    d = dens * (p.L / p.H) ** 3
    assert np.linalg.norm(d - phi) / np.linalg.norm(phi) < 1e-4
    assert abs(diag["mass"] - w.mass) < 1e-5 * w.mass


def test_ragged_and_tiny_runs():
    """P = 1 and P = 257 (one block plus one), H = 8; particles on the box faces."""
    for P, H in [(1, 8), (257, 8), (300, 32)]:
        w = workloads.Workload("t", P=P, H=H, L=2.0, mass=3.0, dt=1e-3, steps=6, seed=5, sigma=0.3)
        X0 = _box_points(P, w.L, seed=P)
        s, _ = _oracle_run(w, X0, w.steps)
        X, alpha, _, _ = _gpu_run(w, X0, w.steps, precision=64)
        assert np.max(np.abs(O.min_image(X - s.X, w.L))) < 1e-10
        assert _rel(alpha, s.alpha) < 1e-10


def test_zero_steps_and_positions_roundtrip():
    w = workloads.small_blob()
    X0 = workloads.sample_positions(w)
    with Simulation(params_from_workload(w, precision=64), X0) as sim:
        assert sim.n == 0
        sim.step(0)
        assert np.array_equal(sim.positions(), X0)
        assert np.all(sim.spectrum() == 0)


def test_deterministic_deposit_is_bitwise_reproducible():
    w = workloads.small_blob()
    X0 = workloads.sample_positions(w)
    runs = []
    for _ in range(2):
        X, alpha, _, dens = _gpu_run(w, X0, 10, precision=32, deposit_mode=1)
        runs.append((X, alpha, dens))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])
    assert np.array_equal(runs[0][2], runs[1][2])
    s, _ = _oracle_run(w, X0, 10)
    assert np.max(np.abs(O.min_image(runs[0][0] - s.X, w.L))) < 1e-4
    X64, a64, _, _ = _gpu_run(w, X0, 10, precision=64, deposit_mode=1)
    assert np.max(np.abs(O.min_image(X64 - s.X, w.L))) < 1e-10
    assert _rel(a64, s.alpha) < 1e-9


def test_diagnostics_match_oracle():
    w = workloads.small_blob()
    X0 = workloads.sample_positions(w)
    s, p = _oracle_run(w, X0, 5)
    _, _, d, _ = _gpu_run(w, X0, 5, precision=64)
    ref = O.diagnostics(s, p)
    for key in ("mass", "m2", "ring_radius", "peak", "hf_frac"):
        assert abs(d[key] - ref[key]) <= 1e-10 * max(1.0, abs(ref[key])), key
    # the FP64 zero-mode shadow follows alpha0^n = a*(1 - r^n), a* = M0/(L^3 k^2)
    astar = w.mass / (w.L ** 3 * w.k ** 2)
    r = 1.0 / (1.0 + w.dt * w.k ** 2 / w.eps)
    assert abs(d["alpha0"] - astar * (1 - r ** 5)) < 1e-12 * astar
    assert d["step"] == 5


def test_field_and_gradient_outputs_match_oracle():
    w = workloads.small_blob()
    X0 = workloads.sample_positions(w)
    s, p = _oracle_run(w, X0, 4)
    with Simulation(params_from_workload(w, precision=64), X0) as sim:
        sim.step(4)
        c = sim.field()
        g = sim.gradient()
    assert _rel(c, O.inverse_ft(s.alpha, p.H)) < 1e-10
    assert _rel(g, O.gradient_grids(s.alpha, p)) < 1e-10


def test_chi0_free_diffusion_on_gpu():
    """chi = 0: the FP64 GPU path moves particles by exactly sum (W^- + W^+)."""
    w = workloads.Workload("free", P=5000, H=16, L=1.0, mass=1.0, chi=0.0, mu=0.4, dt=1e-3, steps=8, seed=9)
    X0 = workloads.sample_positions(w)
    X, _, _, _ = _gpu_run(w, X0, w.steps, precision=64)
    disp = np.zeros_like(X0)
    for n in range(1, w.steps + 1):
        z = O.normals(w.seed, n, w.P)
        disp += math.sqrt(w.mu * w.dt) * (z[:, :3] + z[:, 3:])
    assert np.max(np.abs(O.min_image(X - X0 - disp, w.L))) < 1e-12


# ----------------------------------------------------------------- larger grids
@pytest.mark.parametrize("H,prec", [(256, 64), (256, 32), (128, 64)])
def test_step_large_grid_matches_oracle(H, prec):
    """Torus data, P = 2e4, 5 whole steps at H = 128 (plane FFT kernels, as the
    benchmark runs them) and H = 256 (the pencil passes of the field solve):
    FP64 within 1e-10; FP32 positions within 1e-4 and the fields' relative L2
    within 1e-4 of the FP64 oracle."""
    w = workloads.torus_ring(H=H, P=20_000)
    X0 = workloads.sample_positions(w)
    n = 5
    s, p = _oracle_run(w, X0, n)
    X, alpha, diag, dens = _gpu_run(w, X0, n, precision=prec)
    phi = O.deposit(s.X, p.mass / p.P, p.H, p.L, p.p2g_order)
    d = dens * (p.L / p.H) ** 3
    dx = np.max(np.abs(O.min_image(X - s.X, w.L)))
    if prec == 64:
        assert dx < 1e-10
        assert _rel(alpha, s.alpha) < 1e-10
        assert _rel(d, phi) < 1e-10
    else:
        assert dx < 1e-4
        assert np.linalg.norm(alpha - s.alpha) / np.linalg.norm(s.alpha) < 1e-4
        assert np.linalg.norm(d - phi) / np.linalg.norm(phi) < 1e-4
    assert abs(diag["mass"] - w.mass) < (1e-12 if prec == 64 else 1e-5) * w.mass


@pytest.mark.parametrize("H", [8, 16])
def test_step_fp64_sec51_ball_geometry(H):
    """The Sec. 5.1 set-up (uniform unit ball, M0 = 80, L = 8, eps = 1e-4,
    k = 0.1, tau = 1e-5, automatic filter scale) at H = 8, where
    H0 = 8 * 8^(8/13) * 8^(5/13) = 64 exactly, and H = 16: 10 FP64 steps
    within 1e-10 of the oracle."""
    w = workloads.uniform_ball(P=4000, H=H)
    X0 = workloads.sample_positions(w)
    s, p = _oracle_run(w, X0, 10)
    assert p.H0_eff == (64.0 if H == 8 else O.auto_H0(H, w.L))
    assert _abi.sipf_filter_scale(params_from_workload(w, precision=64)) == p.H0_eff
    X, alpha, _, _ = _gpu_run(w, X0, 10, precision=64)
    assert np.max(np.abs(O.min_image(X - s.X, w.L))) < 1e-10
    assert _rel(alpha, s.alpha) < 1e-10


# ----------------------------------------------------------------- full-size deposit
K_MIN = 19           # smallest fixed-point exponent of any FP32 window (chunks of <= 4096 particles)
FP32_ROUNDINGS = 12  # roundings in one FP32 stencil weight, incl. the particle weight M0/P


def _stencil_counts(X, H, L, chunk=1 << 20):
    """Per node j: n_j, the number of Gamma_4 contributions, and S_j, the sum of
    their |F| (the oracle's stencil)."""
    n = np.zeros(H ** 3)
    S = np.zeros(H ** 3)
    for a in range(0, X.shape[0], chunk):
        cell, lam = O.cell_and_lambda(X[a:a + chunk], H, L)
        offs, F = O.stencil(lam, 4)
        idx = O.stencil_indices(cell, offs, H).ravel()
        n += np.bincount(idx, minlength=H ** 3)
        S += np.bincount(idx, weights=np.abs(F).ravel(), minlength=H ** 3)
    return n.reshape(H, H, H), S.reshape(H, H, H)


def _check_deposit(got, X, p):
    """Element by element against the oracle's deposit of the same positions.
    Bound per node j (w = M0/P, u = 2^-24):
      w n_j 2^-(K+1)            fixed-point rounding of each weight in the window,
    + w S_j (c + n_j) u         FP32 weights (c roundings each) and at most n_j
                                 floating-point additions into phi_j (Higham's
                                 bound for recursive summation);
    the relative L2 error must also stay 10x below the FP32 field bar."""
    w = p.mass / p.P
    ref = O.deposit(X, w, p.H, p.L, 4)
    n, S = _stencil_counts(X, p.H, p.L)
    u = 2.0 ** -24
    bound = w * n * 2.0 ** -(K_MIN + 1) + w * S * (FP32_ROUNDINGS + n) * u + 1e-300
    err = np.abs(got - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


def test_full_size_deposit_grid_matches_oracle():
    """P = 1e7, H = 128, FP32 torus workload in the benchmark's launch: the
    deposited mass grid I rho-hat of X^0 (initial deposit) and of X^1 (the
    deposit done by the step) against the oracle's Algorithm 2 of the same
    positions, node by node."""
    w = workloads.torus_ring()
    X0 = workloads.sample_positions(w)
    p = O.Params.from_workload(w)
    h3 = (p.L / p.H) ** 3
    with Simulation(params_from_workload(w, precision=32), X0) as sim:
        X0f = sim.positions()                     # the FP32 positions the GPU holds
        g0 = sim.density(False) * h3
        sim.step(1)
        X1 = sim.positions()
        g1 = sim.density(False) * h3
    _check_deposit(g0, X0f, p)
    _check_deposit(g1, X1, p)


# ----------------------------------------------------------------- full size, sampled
def test_torus_full_size_sampled_outputs():
    """P = 1e7, H = 128, FP32 (the benchmark workload and launch): the first
    step has zero drift, so every X^1_p is fixed by the noise alone; the second
    step's drift is checked on a sample of particles against the oracle's
    gradient grids of alpha^1, computed from the full deposit of X^0."""
    w = workloads.torus_ring()
    X0 = workloads.sample_positions(w)
    p = O.Params.from_workload(w)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(w.P, size=2000, replace=False))
    with Simulation(params_from_workload(w, precision=32), X0) as sim:
        d0 = sim.diagnostics()
        sim.step(1)
        X1 = sim.positions()
        sim.step(1)
        X2 = sim.positions()
        d2 = sim.diagnostics()
    assert abs(d0["mass"] - w.mass) < 1e-5 * w.mass and abs(d2["mass"] - w.mass) < 1e-5 * w.mass
    # step 1: zero drift
    s = math.sqrt(w.mu * w.dt)
    z1 = np.stack([O.normals(w.seed, 1, 1, first=int(i))[0] for i in idx])
    ref1 = O.wrap(X0[idx] + s * z1[:, :3] + s * z1[:, 3:], w.L)
    assert np.max(np.abs(O.min_image(X1[idx] - ref1, w.L))) < 2e-6
    # step 2: drift from alpha^1 = src * beta^0 (alpha^0 = 0)
    beta0 = O.forward_ft(O.deposit(X0, p.mass / p.P, p.H, p.L, 4), p.L)
    alpha1 = O.update_alpha(np.zeros_like(beta0), beta0, p)
    grads = O.gradient_grids(alpha1, p)
    z2 = np.stack([O.normals(w.seed, 2, 1, first=int(i))[0] for i in idx])
    Y = X1[idx].astype(np.float64) + s * z2[:, :3]
    drift = O.gather(grads, Y, p.H, p.L, 2).T
    ref2 = O.wrap(Y + p.chi * p.dt * drift + s * z2[:, 3:], w.L)
    assert np.max(np.abs(O.min_image(X2[idx] - ref2, w.L))) < 5e-6
