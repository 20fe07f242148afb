"""The benchmark's all-core oracle baseline (bench.ParallelOracle) is the
oracle's own step with its particle loops split over processes: it must
reproduce the serial oracle's trajectory (up to the summation order of the
partial deposits)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import sipf_oracle as O  # noqa: E402
from paper_2512_03452_gb300 import workloads  # noqa: E402


def test_parallel_oracle_matches_serial_steps():
    w = workloads.torus_ring(H=32, P=20_000)
    X = workloads.sample_positions(w)
    p = O.Params.from_workload(w)
    s = O.init_state(X, p)
    for _ in range(3):
        s = O.step(s, p)
    with bench.ParallelOracle(X, p, 2) as po:
        for _ in range(3):
            po.step()
        assert po.n == 3
        assert np.max(np.abs(O.min_image(po.X - s.X, p.L))) < 1e-13
        assert np.max(np.abs(po.alpha - s.alpha)) <= 1e-12 * np.max(np.abs(s.alpha))


def test_oracle_move_of_a_slice_uses_its_own_particle_indices():
    w = workloads.small_blob()
    X = workloads.sample_positions(w)[:300]
    p = O.Params.from_workload(w, P=300)
    grads = O.gradient_grids(np.zeros((p.H, p.H, p.H // 2 + 1), dtype=complex), p)
    whole = O.move(X, grads, p, 4)
    parts = np.concatenate([O.move(X[:100], grads, p, 4), O.move(X[100:], grads, p, 4, first=100)])
    assert np.array_equal(whole, parts)
