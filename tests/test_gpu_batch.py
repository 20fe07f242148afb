"""Batched runs (sipf_batch_*): many independent runs of Algorithm 4 in the
same launches.  Every run must compute what a single-run context with the same
parameters computes:
  * deterministic deposit: bit for bit (the grid sums are exact integers, the
    move of a particle depends only on its id, the step and the field);
  * atomic deposit, FP64: within 1e-10 (only the order of the floating-point
    additions of the deposit differs);
and, through the single-run parity, the FP64 oracle.  The 40-step runs cover
one replayed 32-step graph, 8 directly issued steps and 2 capacity rebuilds.
"""
import numpy as np
import pytest

from oracle import sipf_oracle as O
from paper_2512_03452_gb300 import Batch, Simulation, _abi, build, params_from_workload, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return _abi.load()


def _runs(prec, mode, n=4, seed=3, mild=False):
    """Uneven runs: P from 1 to ~2e4 (ragged), H in {32, 64}, varied chi, seed, dt.
    mild: small M0 chi and tau, so that no run aggregates within the test and
    rounding differences stay at rounding level."""
    rng = np.random.default_rng(seed)
    mass_hi, chi_hi, dts = (15.0, 1.0, [1e-4]) if mild else (80.0, 2.0, [1e-4, 5e-4])
    ws = []
    for i in range(n):
        P = [20_000, 1, 4099, 777, 12_345, 300][i % 6]
        H = [32, 64][i % 2]
        ws.append(workloads.Workload(f"b{i}", P=P, H=H, L=1.0 + 0.25 * i, mass=float(rng.uniform(5, mass_hi)),
                                     chi=float(rng.uniform(0.5, chi_hi)), dt=float(rng.choice(dts)),
                                     steps=40, seed=100 + i, sigma=0.12))
    params = [params_from_workload(w, precision=prec, deposit_mode=mode) for w in ws]
    X0s = [workloads.sample_positions(w) for w in ws]
    return ws, params, X0s


def _single(p, X0, nsteps):
    with Simulation(p, X0) as sim:
        sim.step(nsteps)
        sim.sync()
        return sim.positions(), sim.spectrum(), sim.diagnostics()


def _batch(params, X0s, nsteps, graph=True):
    with Batch(params, X0s) as b:
        b.use_graph(graph)
        b.step(nsteps)
        b.sync()
        assert b.n == nsteps
        return [(b.positions(r), b.spectrum(r), b.diagnostics(r)) for r in range(len(params))]


@pytest.mark.parametrize("prec", [64, 32])
def test_batch_deterministic_is_bitwise_single_run(prec):
    ws, params, X0s = _runs(prec, mode=1)
    got = _batch(params, X0s, 40)
    for r, (p, X0) in enumerate(zip(params, X0s)):
        X, a, d = _single(p, X0, 40)
        assert np.array_equal(got[r][0], X), r
        assert np.array_equal(got[r][1], a), r
        assert got[r][2]["step"] == 40


def test_batch_graph_and_direct_issue_agree():
    _, params, X0s = _runs(32, mode=1, n=3, seed=8)
    a = _batch(params, X0s, 70, graph=True)      # 2 graph replays + 6 direct steps
    b = _batch(params, X0s, 70, graph=False)
    for r in range(len(params)):
        assert np.array_equal(a[r][0], b[r][0]), r
        assert np.array_equal(a[r][1], b[r][1]), r


def test_batch_atomic_fp64_matches_single_run():
    """Atomic deposit: the order of the floating-point additions differs from
    the single run's; on mild runs that stays within 1e-10 over 40 steps."""
    _, params, X0s = _runs(64, mode=0, n=5, seed=4, mild=True)
    got = _batch(params, X0s, 40)
    for r, (p, X0) in enumerate(zip(params, X0s)):
        X, a, _ = _single(p, X0, 40)
        assert np.max(np.abs(O.min_image(got[r][0] - X, p.L))) < 1e-10, r
        assert np.max(np.abs(got[r][1] - a)) <= 1e-10 * max(np.max(np.abs(a)), 1e-300), r


def test_batch_fp64_matches_oracle():
    """Runs of H = 32 and H = 64 against the FP64 oracle, 36 steps (one graph
    replay).  The P = 1 run is left out here: a lone particle carrying the whole
    mass sits in its own steep field, and rounding differences of any two
    implementations grow exponentially there (it is compared bit for bit
    against the single-run path above instead)."""
    ws, params, X0s = _runs(64, mode=0, n=4, seed=6, mild=True)
    keep = [0, 2, 3]
    ws, params, X0s = [ws[i] for i in keep], [params[i] for i in keep], [X0s[i] for i in keep]
    nsteps = 36
    got = _batch(params, X0s, nsteps)
    for r, w in enumerate(ws):
        if w.P > 5000:
            continue                                   # present for the batching, oracle too slow
        p = O.Params.from_workload(w)
        s = O.init_state(X0s[r], p)
        for _ in range(nsteps):
            s = O.step(s, p)
        assert np.max(np.abs(O.min_image(got[r][0] - s.X, w.L))) < 1e-10, r
        assert np.max(np.abs(got[r][1] - s.alpha)) <= 1e-10 * np.max(np.abs(s.alpha)), r


def test_batch_launches_do_not_grow_with_runs():
    counts = []
    for n in (2, 6):
        _, params, X0s = _runs(32, mode=0, n=n, seed=9)
        with Batch(params, X0s) as b:
            k0 = _abi.sipf_batch_kernel_launches(b.handle)
            b.step(32)
            b.sync()
            counts.append(_abi.sipf_batch_kernel_launches(b.handle) - k0)
    # both batches hold H = 32 and H = 64 runs: same launches per step (the
    # plane kernels do each H's field solve in 3 launches)
    assert counts[0] == counts[1]
    assert counts[0] == 32 * (2 * 3 + 5) + 2 * 5


def test_batch_rejects_bad_parameter_sets():
    _, params, X0s = _runs(32, mode=0, n=2, seed=1)
    bad = [params[0], params_from_workload(workloads.small_blob(), precision=32)]   # H = 16
    with pytest.raises(_abi.SipfError) as e:
        Batch(bad, [X0s[0], workloads.sample_positions(workloads.small_blob())])
    assert e.value.code == _abi.SIPF_EINVAL and "run 1" in _abi.sipf_last_error()
    mixed = [params[0], params_from_workload(workloads.Workload("m", P=100, H=32), precision=64)]
    with pytest.raises(_abi.SipfError):
        Batch(mixed, [X0s[0], workloads.sample_positions(workloads.Workload("m", P=100, H=32))])
    det = [params[0], params_from_workload(workloads.Workload("d", P=100, H=32), precision=32, deposit_mode=1)]
    with pytest.raises(_abi.SipfError):
        Batch(det, [X0s[0], workloads.sample_positions(workloads.Workload("d", P=100, H=32))])


def test_autotune_changes_shapes_not_results():
    """Deterministic deposit: a batch that autotunes and one that does not give
    the same bits after the same number of steps."""
    _, params, X0s = _runs(32, mode=1, n=4, seed=12)
    with Batch(params, X0s) as a:
        t = a.autotune(2)
        assert t["steps_used"] > 0 and len(t["groups"]) == 2
        for g in t["groups"]:
            assert g["cols_tile"] in (8, 16, 32) and g["xpass_tile"] in (4, 8, 16) and g["field_ms"] > 0
        a.step(40)
        a.sync()
        n = a.n
        got = [(a.positions(r), a.spectrum(r)) for r in range(len(params))]
    with Batch(params, X0s) as b:
        b.step(n)
        b.sync()
        for r in range(len(params)):
            assert np.array_equal(b.positions(r), got[r][0]), r
            assert np.array_equal(b.spectrum(r), got[r][1]), r


def _tuning(H, **kw):
    t = _abi.sipf_batch_tuning()
    t.ngroups = len(H)
    for g, h in enumerate(H):
        t.H[g] = h
        t.plane_kernels[g] = 1
    for k, v in kw.items():
        if k in ("move_blocks_per_sm", "deposit_blocks_per_sm"):
            setattr(t, k, v)
        else:
            g, name = k.split("_", 1)
            getattr(t, name)[int(g[1:])] = v
    return t


@pytest.mark.parametrize("shape", [dict(g1_plane_kernels=0), dict(g0_plane_kernels=0, g0_cols_tile=32),
                                   dict(g1_plane_kernels=0, g1_cols_tile=8, g1_rows_blocks_per_sm=4),
                                   dict(g1_xpass_tile=4), dict(move_blocks_per_sm=1, deposit_blocks_per_sm=1),
                                   dict(g0_inverse_all_components=1, g1_inverse_all_components=1),
                                   dict(g1_inverse_all_components=1, g1_plane_warps=16),
                                   dict(g1_plane_kernels=2), dict(g1_plane_kernels=2, g1_plane_warps=8)])
def test_launch_shapes_give_identical_bits(shape):
    """Plane, cluster-plane or pencil FFT kernels, tile widths, grid sizes and
    the inverse plane kernel over one or all three gradient components: the same bits
    (deterministic deposit; the lone-particle run amplifies any difference)."""
    _, params, X0s = _runs(32, mode=1, n=4, seed=12)

    def run(t):
        with Batch(params, X0s) as b:
            if t is not None:
                _abi.sipf_batch_set_tuning(b.handle, t)
            b.step(60)
            b.sync()
            return [(b.positions(r), b.spectrum(r)) for r in range(len(params))]

    ref, got = run(None), run(_tuning([32, 64], **shape))
    for r in range(len(params)):
        assert np.array_equal(got[r][0], ref[r][0]), r
        assert np.array_equal(got[r][1], ref[r][1]), r


def test_inverse_over_all_components_in_fp64_gives_identical_bits():
    """The three-component inverse plane kernel in double precision (chosen
    only by tuning there): the same bits as the default shapes."""
    _, params, X0s = _runs(64, mode=1, n=4, seed=12)

    def run(t):
        with Batch(params, X0s) as b:
            if t is not None:
                _abi.sipf_batch_set_tuning(b.handle, t)
            b.step(40)
            b.sync()
            return [(b.positions(r), b.spectrum(r)) for r in range(len(params))]

    ref = run(None)
    got = run(_tuning([32, 64], g0_inverse_all_components=1, g1_inverse_all_components=1))
    for r in range(len(params)):
        assert np.array_equal(got[r][0], ref[r][0]), r
        assert np.array_equal(got[r][1], ref[r][1]), r


def test_set_tuning_rejects_bad_shapes():
    _, params, X0s = _runs(32, mode=0, n=2, seed=1)
    with Batch(params, X0s) as b:
        with pytest.raises(_abi.SipfError):
            _abi.sipf_batch_set_tuning(b.handle, _tuning([32, 64], g0_cols_tile=12))
        with pytest.raises(_abi.SipfError):
            _abi.sipf_batch_set_tuning(b.handle, _tuning([64, 32]))
        with pytest.raises(_abi.SipfError):
            _abi.sipf_batch_set_tuning(b.handle, _tuning([32, 64], g1_inverse_all_components=3))
