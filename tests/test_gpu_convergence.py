"""The Sec. 5.1 convergence study on the GPU: SIPF-PIC runs of the uniform-ball
set-up (FP32, Gamma_4 deposit, Gamma_2 gather, automatic filter scale, 2000
steps to T = 0.02) against the radial finite-volume reference, with the
paper's truncated quantile W1 discrepancy averaged over independent seeds.

The paper prints the fitted slopes of log2 E: -0.512 against log2 P (theory
-1/2) and -1.327 against log2 H (theory -16/13), measured over P = 2^11..2^20
and H = 8..256 with 30 seeds.  These tests run smaller sweeps (8 seeds) in
the same regime and check the slopes against bands around the printed values,
and that the error falls monotonically.
"""
import json
import os

import numpy as np
import pytest

from oracle import radial_fv as R
from paper_2512_03452_gb300 import _abi, build
from paper_2512_03452_gb300 import convergence as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLD_DIR = os.path.join(os.path.dirname(__file__), "golden")
PAPER = json.load(open(os.path.join(GOLD_DIR, "paper_constants.json")))["convergence_slopes"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return _abi.load()


@pytest.fixture(scope="module")
def reference():
    g = json.load(open(os.path.join(GOLD_DIR, "sec51_reference_quantiles.json")))
    return np.array(g["levels"]), np.array(g["quantiles"])


def _mean_error(P, H, seeds, reference):
    levels, q_ref = reference
    errs = [R.truncated_w1(q_ref, R.empirical_quantiles(r, levels)) for r in C.final_radii(P, H, seeds)]
    return float(np.mean(errs)), float(np.std(errs))


def test_study_quantile_conventions_agree_with_the_oracle(reference):
    """The library's quantile helper and the oracle's agree on GPU output."""
    levels, _ = reference
    r = C.final_radii(2 ** 12, 32, [3, 4])[0]
    assert np.array_equal(C.radial_quantiles(r, levels), R.empirical_quantiles(r, levels))


def test_particle_number_slope(reference):
    """H = 128 fixed, P = 2^11, 2^13, 2^15, 2^17: the slope of log2 E against
    log2 P within [-0.75, -0.35] (paper: -0.512, theory -1/2)."""
    Ps = [2 ** 11, 2 ** 13, 2 ** 15, 2 ** 17]
    E = [_mean_error(P, 128, range(8), reference)[0] for P in Ps]
    assert all(a > b for a, b in zip(E, E[1:])), E
    slope = C.fitted_slope(Ps, E)
    assert -0.75 < slope < -0.35, (slope, PAPER["P"], E)


def test_grid_slope(reference):
    """P = 2^19 fixed, H = 16, 32, 64, 128: the error falls with H at least at
    about the theory's order 16/13 (slope of log2 E against log2 H within
    [-2.3, -1.1]; paper: -1.327 over H = 8..256 at P = 2^20, theory -1.231).
    Over this sub-range the decay is steeper than the paper's fit over the
    whole range (about -1.7 measured): at small H the error is dominated by the
    grid, at large H the P^-1/2 floor flattens the curve."""
    Hs = [16, 32, 64, 128]
    E = [_mean_error(2 ** 19, H, range(8), reference)[0] for H in Hs]
    assert all(a > b for a, b in zip(E, E[1:])), E
    slope = C.fitted_slope(Hs, E)
    assert -2.3 < slope < -1.1, (slope, PAPER["H"], E)
