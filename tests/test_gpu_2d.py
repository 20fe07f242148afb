"""Parity of the 2D variant (Sec. 5.2; sipf2d_* through the C ABI) with the 2D
FP64 oracle, and the second-moment law of the parabolic-elliptic system.

Bars as for the 3D path: FP64 within 1e-10 of the oracle (positions by
minimum image, spectra and grids relative to their largest value); FP32
positions within 1e-4 over 20 steps and field relative L2 within 1e-4.
"""
import math

import numpy as np
import pytest

from oracle import sipf2d_oracle as O2
from paper_2512_03452_gb300 import Simulation2D, _abi, build, make_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return _abi.load()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _disk(P, seed, radius=1.0):
    rng = np.random.default_rng(seed)
    r = radius * np.sqrt(rng.uniform(size=P))
    th = rng.uniform(0, 2 * math.pi, size=P)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


_VARIANTS = {
    "elliptic": {},
    "plain_em": dict(splitting="plain"),
    "orders_2_4": dict(p2g_order=2, g2p_order=4),
    "no_filter": dict(H0=0.0),
    "screened": dict(k=0.5),
    "parabolic": dict(eps=1.0, k=1.0),
}


def _params(P, H, **kw):
    base = dict(P=P, H=H, L=8.0, mass=20.0, chi=1.0, mu=1.0, eps=0.0, k=0.0, dt=5e-4, H0=-1.0, seed=7,
                p2g_order=4, g2p_order=2, splitting="half")
    base.update(kw)
    op = O2.Params2D(**base)
    gkw = dict(base)
    gkw["splitting"] = 0 if base["splitting"] == "half" else 1
    return op, gkw


def _runs(P, H, nsteps, prec, X0, **kw):
    op, gkw = _params(P, H, **kw)
    s = O2.init_state(X0, op)
    for _ in range(nsteps):
        s = O2.step(s, op)
    with Simulation2D(make_params(precision=prec, **gkw), X0) as sim:
        sim.step(nsteps)
        sim.sync()
        return s, op, sim.positions(), sim.spectrum(), sim.density(False), sim.diagnostics()


@pytest.mark.parametrize("variant", list(_VARIANTS))
def test_2d_fp64_matches_oracle(variant):
    """Unit disk, M0 = 20, L = 8, H = 32, 20 steps of 5e-4: FP64 within 1e-10."""
    X0 = _disk(4000, 1)
    s, op, X, spec, dens, d = _runs(4000, 32, 20, 64, X0, **_VARIANTS[variant])
    assert np.max(np.abs(O2.min_image(X - s.X, op.L))) < 1e-10
    assert _rel(spec, s.alpha) < 1e-10
    phi = O2.deposit(s.X, op.mass / op.P, op.H, op.L, op.p2g_order)
    assert _rel(dens * (op.L / op.H) ** 2, phi) < 1e-10
    assert abs(d["mass"] - op.mass) < 1e-12 * op.mass
    assert abs(d["m2"] - O2.second_moment(s.X)) < 1e-12 * O2.second_moment(s.X)
    assert d["step"] == 20


def test_2d_fp32_matches_fp64_oracle():
    X0 = _disk(4000, 2)
    s, op, X, spec, dens, d = _runs(4000, 64, 20, 32, X0)
    assert np.max(np.abs(O2.min_image(X - s.X, op.L))) < 1e-4
    assert np.linalg.norm(spec - s.alpha) / np.linalg.norm(s.alpha) < 1e-4
    phi = O2.deposit(s.X, op.mass / op.P, op.H, op.L, 4)
    assert np.linalg.norm(dens * (op.L / op.H) ** 2 - phi) / np.linalg.norm(phi) < 1e-4


def test_2d_ragged_tiny_and_edges():
    """P = 1 and 257 at H = 8, particles on the box faces."""
    for P in (1, 257):
        rng = np.random.default_rng(P)
        X0 = rng.uniform(-4.0, 4.0, size=(P, 2))
        if P > 4:
            X0[0] = [-4.0, -4.0]
            X0[1] = [np.nextafter(4.0, 0), 0.0]
            X0[2] = [0.0, 0.0]
        s, op, X, spec, _, _ = _runs(P, 8, 6, 64, X0)
        assert np.max(np.abs(O2.min_image(X - s.X, op.L))) < 1e-10
        assert _rel(spec, s.alpha) < 1e-10


def test_2d_chi0_moves_are_the_summed_noise():
    X0 = _disk(3000, 3)
    op, gkw = _params(3000, 32, chi=0.0, mu=0.6)
    with Simulation2D(make_params(precision=64, **gkw), X0) as sim:
        sim.step(8)
        X = sim.positions()
    disp = np.zeros_like(X0)
    for n in range(1, 9):
        z = O2.normals2(op.seed, n, op.P)
        disp += math.sqrt(op.mu * op.dt) * (z[:, :2] + z[:, 2:])
    assert np.max(np.abs(O2.min_image(X - X0 - disp, op.L))) < 1e-12


def test_2d_rejects_what_it_does_not_support():
    for kw in (dict(deposit_mode=1), dict(propagator=1), dict(H=512), dict(eps=-1.0)):
        base = dict(P=10, H=16, L=8.0, mass=1.0, eps=0.0, k=0.0)
        base.update(kw)
        with pytest.raises(_abi.SipfError) as e:
            _abi.sipf2d_init(make_params(**base), np.zeros((10, 2)))
        assert e.value.code == _abi.SIPF_EINVAL


@pytest.mark.parametrize("M0", [10.0, 20.0, 30.0])
def test_2d_second_moment_law(M0):
    """Sec. 5.2, Eq. (second_moment): dm2/dt = 4 M0 (1 - M0/(8 pi)) for
    (k, eps, mu, chi) = (0, 0, 1, 1) on the plane, i.e. the particle second
    moment (1/P) sum |X|^2 of the unit disk grows at the rate
    4 (1 - M0/(8 pi)) (decays for M0 > 8 pi).  FP32, P = 2^18, box of side 12,
    H = 256, 400 steps of 5e-4: the fitted rate within 5% of 4."""
    P = 2 ** 18
    X0 = _disk(P, 11)
    op, gkw = _params(P, 256, L=12.0, mass=M0, seed=21)
    ts, m2 = [], []
    with Simulation2D(make_params(precision=32, **gkw), X0) as sim:
        for n in range(0, 401, 50):
            if n:
                sim.step(50)
            ts.append(n * op.dt)
            m2.append(sim.diagnostics()["m2"])
    rate = np.polyfit(ts, m2, 1)[0]
    law = 4.0 * (1.0 - M0 / (8.0 * math.pi))
    assert abs(rate - law) < 0.05 * 4.0, (rate, law)
