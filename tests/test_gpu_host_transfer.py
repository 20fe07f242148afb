"""Host copies of the positions through the C ABI (sipf_upload_soa,
sipf_download_soa): page-locked buffers (read and written by kernels through
their mapped device addresses) and pageable ones (the pieces pipeline of both
directions, for one piece (P < 2^20) and for eight ragged pieces).

* download equals sipf_positions of the same state, bit for bit;
* upload followed by download returns the uploaded positions, bit for bit;
* a run that re-uploads its own initial positions and then steps gives the
  same bits as a fresh run (deterministic deposit), so the upload's re-binning
  and re-deposit leave the state as sipf_init made it.
"""
import numpy as np
import pytest

from paper_2512_03452_gb300 import DEPOSIT_DETERMINISTIC, Simulation, _abi, build, make_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return _abi.load()


def _blob(P, seed, L=1.0):
    rng = np.random.default_rng(seed)
    X = rng.normal(0.0, 0.12 * L, size=(P, 3))
    return (X + L / 2) % L - L / 2


def _params(P, prec, **kw):
    base = dict(P=P, H=64, L=1.0, mass=50.0, chi=1.0, mu=0.5, eps=1.0, k=1.0, dt=1e-4, seed=5, precision=prec)
    base.update(kw)
    return make_params(**base)


def _host_soa(P, dtype, pinned):
    if pinned:
        tdt = torch.float32 if dtype == np.float32 else torch.float64
        ts = [torch.empty(P, dtype=tdt).pin_memory() for _ in range(3)]
        return ts, [t.numpy() for t in ts], [t.data_ptr() for t in ts]
    arrs = [np.empty(P, dtype=dtype) for _ in range(3)]
    return arrs, arrs, [a.ctypes.data for a in arrs]


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("P,pinned", [(1000, False), (1000, True), ((1 << 20) + 37, True), ((1 << 20) + 37, False)])
def test_download_matches_positions(prec, P, pinned):
    dtype = np.float32 if prec == 32 else np.float64
    with Simulation(_params(P, prec), _blob(P, 1)) as sim:
        sim.step(3)
        keep, views, ptrs = _host_soa(P, dtype, pinned)
        _abi.sipf_download_soa(sim.ctx, *ptrs)
        sim.sync()
        got = np.stack(views, axis=1).astype(np.float64)
        assert np.array_equal(got, sim.positions())
        # again after more steps (the other bin buffer holds the read-back's records)
        sim.step(2)
        _abi.sipf_download_soa(sim.ctx, *ptrs)
        sim.sync()
        got = np.stack(views, axis=1).astype(np.float64)
        assert np.array_equal(got, sim.positions())
        del keep


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("P", [1000, (1 << 20) + 37])
@pytest.mark.parametrize("pinned_src", [False, True])
def test_upload_download_round_trip(prec, P, pinned_src):
    dtype = np.float32 if prec == 32 else np.float64
    Y = _blob(P, 2).astype(dtype)
    Y[::97, 0] += 3.0          # outside the box: the upload wraps them back in
    with Simulation(_params(P, prec), _blob(P, 3)) as sim:
        skeep, src, sptrs = _host_soa(P, dtype, pinned_src)
        for d in range(3):
            src[d][:] = Y[:, d]
        _abi.sipf_upload_soa(sim.ctx, *sptrs)
        keep, views, ptrs = _host_soa(P, dtype, True)
        _abi.sipf_download_soa(sim.ctx, *ptrs)
        sim.sync()
        # the periodic wrap of x + 3 L gives back x (x in [-L/2, L/2), exact in binary)
        Yw = Y.copy()
        Yw[::97, 0] -= 3.0
        assert np.array_equal(np.stack(views, axis=1), Yw)
        assert np.array_equal(sim.positions(), Yw.astype(np.float64))
        del keep, skeep


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("pinned_src", [False, True])
def test_reupload_then_steps_equal_a_fresh_run(prec, pinned_src):
    P = (1 << 20) + 37
    dtype = np.float32 if prec == 32 else np.float64
    X0 = _blob(P, 4).astype(dtype).astype(np.float64)
    prm = _params(P, prec, deposit_mode=DEPOSIT_DETERMINISTIC)
    with Simulation(prm, X0) as a, Simulation(prm, X0) as b:
        skeep, src, sptrs = _host_soa(P, dtype, pinned_src)
        for d in range(3):
            src[d][:] = X0[:, d]
        _abi.sipf_upload_soa(a.ctx, *sptrs)
        a.step(4)
        b.step(4)
        a.sync()
        b.sync()
        assert np.array_equal(a.positions(), b.positions())
        assert np.array_equal(a.spectrum(), b.spectrum())
