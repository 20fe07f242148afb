"""Adjoint form on the GPU (sipf_adjoint_*, the torch Function over it).

  * FP64: rho(T) and the gradients wrt chi, mu, X^0 against the FP64 CPU
    adjoint of the oracle (itself pinned by central differences), with
    checkpoint segments that do not divide N;
  * FP32 (the production precision): dJ/dchi and dJ/dmu against central
    differences of the FP32 forward (deterministic deposit, h = 1e-3 |theta|)
    and against the FP64 oracle adjoint;
  * the checkpoint interval does not change the result;
  * full size (P = 1e6, H = 64): with chi = 0 the positions move by the noise
    alone, so dJ/dX^0 equals the transpose of the deposit at X^N, checked on
    sampled particles.
"""
import math

import numpy as np
import pytest

from oracle import sipf_adjoint as OA
from oracle import sipf_oracle as O
from paper_2512_03452_gb300 import _abi, build, make_params, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return _abi.load()


from paper_2512_03452_gb300.adjoint import Adjoint, SipfDensity  # noqa: E402


def _case(P=2000, H=16, seed=3, **kw):
    d = dict(P=P, H=H, L=1.0, mass=10.0, chi=1.0, mu=0.7, eps=1.0, k=1.0, dt=1e-3, seed=seed)
    d.update(kw)
    w = workloads.Workload("adj", P=d["P"], H=d["H"], L=d["L"], mass=d["mass"], chi=d["chi"], mu=d["mu"],
                           eps=d["eps"], k=d["k"], dt=d["dt"], seed=seed, sigma=0.12)
    X0 = workloads.sample_positions(w)
    rng = np.random.default_rng(seed + 1)
    rho_star = rng.uniform(0, 2 * d["mass"] / d["L"] ** 3, size=(d["H"],) * 3)
    return d, X0, rho_star


_SPLIT = {"half": 0, "plain": 1}
_PROP = {"implicit": 0, "exp": 1}


def _gpu_params(d, prec, mode=0, splitting="half", propagator="implicit", p2g=4, g2p=2):
    return make_params(P=d["P"], H=d["H"], L=d["L"], mass=d["mass"], chi=d["chi"], mu=d["mu"], eps=d["eps"],
                       k=d["k"], dt=d["dt"], seed=d["seed"], precision=prec, deposit_mode=mode,
                       splitting=_SPLIT[splitting], propagator=_PROP[propagator], p2g_order=p2g, g2p_order=g2p)


def _oracle(d, X0, nsteps, rho_star, splitting="half", propagator="implicit", p2g=4, g2p=2):
    p = O.Params(P=d["P"], H=d["H"], L=d["L"], mass=d["mass"], chi=d["chi"], mu=d["mu"], eps=d["eps"], k=d["k"],
                 dt=d["dt"], seed=d["seed"], splitting=splitting, propagator=propagator, p2g_order=p2g,
                 g2p_order=g2p)
    traj = OA.forward(X0, p, nsteps)
    rho = OA.density(traj.X[-1], p)
    J, rhobar = OA.loss(rho, rho_star)
    return rho, J, rhobar, OA.adjoint(traj, p, rhobar)


@pytest.mark.parametrize("variant", [{}, dict(splitting="plain"), dict(propagator="exp"), dict(p2g=2, g2p=4)])
def test_adjoint_fp64_matches_oracle_adjoint(variant):
    d, X0, rho_star = _case()
    nsteps = 25
    rho_o, J, rhobar, g = _oracle(d, X0, nsteps, rho_star, **variant)
    with Adjoint(_gpu_params(d, 64, **variant), X0, nsteps, checkpoint_every=10) as eng:
        rho = eng.forward(d["chi"], d["mu"])
        assert np.max(np.abs(rho - rho_o)) <= 1e-10 * np.max(np.abs(rho_o))
        gc, gm, gX = eng.backward(2.0 * (rho - rho_star))
    assert abs(gc - g.chi) <= 1e-7 * abs(g.chi)
    assert abs(gm - g.mu) <= 1e-7 * abs(g.mu)
    assert np.max(np.abs(gX - g.X0)) <= 1e-7 * np.max(np.abs(g.X0))


def test_adjoint_fp32_matches_central_differences_and_oracle():
    d, X0, rho_star = _case(P=10_000, seed=5)
    nsteps = 20
    _, J, _, g = _oracle(d, X0, nsteps, rho_star)
    with Adjoint(_gpu_params(d, 32, mode=1), X0, nsteps) as eng:
        def loss(chi, mu):
            r = eng.forward(chi, mu)
            return float(np.sum((r - rho_star) ** 2)), r

        J32, rho = loss(d["chi"], d["mu"])
        gc, gm, gX = eng.backward(2.0 * (rho - rho_star))
        h = 1e-3
        fd_chi = (loss(d["chi"] * (1 + h), d["mu"])[0] - loss(d["chi"] * (1 - h), d["mu"])[0]) / (2 * h * d["chi"])
        fd_mu = (loss(d["chi"], d["mu"] * (1 + h))[0] - loss(d["chi"], d["mu"] * (1 - h))[0]) / (2 * h * d["mu"])
    assert abs(J32 - J) <= 1e-4 * J
    assert abs(gc - fd_chi) <= 1e-2 * abs(fd_chi)
    assert abs(gm - fd_mu) <= 1e-2 * abs(fd_mu)
    assert abs(gc - g.chi) <= 2e-3 * abs(g.chi)
    assert abs(gm - g.mu) <= 2e-3 * abs(g.mu)
    assert np.linalg.norm(gX - g.X0) <= 2e-3 * np.linalg.norm(g.X0)


def test_adjoint_fp64_x0_central_differences():
    d, X0, rho_star = _case(P=500, H=16, seed=9)
    nsteps = 12
    with Adjoint(_gpu_params(d, 64), X0, nsteps, checkpoint_every=5) as eng:
        rho = eng.forward(d["chi"], d["mu"], X0)
        _, _, gX = eng.backward(2.0 * (rho - rho_star))
        hx = 1e-6
        for i, e in [(0, 0), (17, 1), (250, 2), (499, 0)]:
            Xp, Xm = X0.copy(), X0.copy()
            Xp[i, e] += hx
            Xm[i, e] -= hx
            Jp = np.sum((eng.forward(d["chi"], d["mu"], Xp) - rho_star) ** 2)
            Jm = np.sum((eng.forward(d["chi"], d["mu"], Xm) - rho_star) ** 2)
            fd = (Jp - Jm) / (2 * hx)
            assert abs(fd - gX[i, e]) <= 1e-5 * max(abs(fd), 1e-3 * np.max(np.abs(gX))), (i, e)


def test_checkpoint_interval_does_not_change_gradients():
    d, X0, rho_star = _case(P=3000, H=32, seed=2)
    nsteps = 23
    out = []
    for C in (0, 7, 23, 1):
        with Adjoint(_gpu_params(d, 64, mode=1), X0, nsteps, checkpoint_every=C) as eng:
            rho = eng.forward(d["chi"], d["mu"])
            out.append((rho,) + eng.backward(2.0 * (rho - rho_star)))
    for rho, gc, gm, gX in out[1:]:
        assert np.array_equal(rho, out[0][0])
        assert abs(gc - out[0][1]) <= 1e-12 * abs(out[0][1])
        assert abs(gm - out[0][2]) <= 1e-12 * abs(out[0][2])
        assert np.max(np.abs(gX - out[0][3])) <= 1e-12 * np.max(np.abs(out[0][3]))


def test_torch_function_backpropagates_a_torch_loss():
    d, X0, rho_star = _case(P=1000, H=16, seed=4)
    nsteps = 10
    with Adjoint(_gpu_params(d, 64), X0, nsteps) as eng:
        X0_t = torch.tensor(X0, dtype=torch.float64, requires_grad=True)
        chi_t = torch.tensor(d["chi"], dtype=torch.float64, requires_grad=True)
        mu_t = torch.tensor(d["mu"], dtype=torch.float64, requires_grad=True)
        rho = SipfDensity.apply(X0_t, chi_t, mu_t, eng)
        loss = ((rho - torch.from_numpy(rho_star)) ** 2).sum()
        loss.backward()
        rho2 = eng.forward(d["chi"], d["mu"], X0)
        gc, gm, gX = eng.backward(2.0 * (rho2 - rho_star))
    assert abs(chi_t.grad.item() - gc) <= 1e-9 * abs(gc)
    assert abs(mu_t.grad.item() - gm) <= 1e-9 * abs(gm)
    assert np.max(np.abs(X0_t.grad.numpy() - gX)) <= 1e-9 * np.max(np.abs(gX))


def test_adjoint_rejects_bad_use():
    d, X0, _ = _case(P=100, H=16)
    with pytest.raises(_abi.SipfError):
        Adjoint(_gpu_params({**d, "mu": 0.0}, 32), X0, 5)
    with Adjoint(_gpu_params(d, 32), X0, 5) as eng:
        with pytest.raises(_abi.SipfError):
            eng.backward(np.zeros((16,) * 3))
        with pytest.raises(_abi.SipfError):
            eng.forward(d["chi"], -1.0)


def test_full_size_free_diffusion_gradient_on_sampled_particles():
    """P = 1e6, H = 64, FP32, 40 steps with chi = 0: dJ/dX^0_p is the transpose of
    the deposit at X^N_p, for every p; 2000 particles against the oracle's deposit
    transpose at X^N = X^0 + sum of the oracle's noise."""
    w = workloads.adjoint_case()
    nsteps = 40
    X0 = workloads.sample_positions(w)
    rng = np.random.default_rng(0)
    rho_star = rng.uniform(0, 2 * w.mass / w.L ** 3, size=(w.H,) * 3)
    p = make_params(P=w.P, H=w.H, L=w.L, mass=w.mass, chi=0.0, mu=w.mu, eps=w.eps, k=w.k, dt=w.dt, seed=w.seed,
                    precision=32)
    with Adjoint(p, X0, nsteps) as eng:
        rho = eng.forward(0.0, w.mu)
        gc, gm, gX = eng.backward(2.0 * (rho - rho_star))
    assert np.all(np.isfinite(gX)) and math.isfinite(gc) and math.isfinite(gm)
    # X^N of the chi = 0 run: X^0 plus the summed noise (FP64 oracle normals)
    first, m = 123_457, 2000
    idx = np.arange(first, first + m)
    s = math.sqrt(w.mu * w.dt)
    XN = X0[idx].copy()
    for n in range(1, nsteps + 1):
        z = O.normals(w.seed, n, m, first=first)
        XN += s * (z[:, 0:3] + z[:, 3:6])
    XN = O.wrap(XN, w.L)
    h3 = (w.L / w.H) ** 3
    ref = OA.deposit_adjoint(XN, w.mass / w.P, 2.0 * (rho - rho_star) / h3, w.H, w.L, 4)
    assert np.max(np.abs(gX[idx] - ref)) <= 1e-3 * np.max(np.abs(ref))
