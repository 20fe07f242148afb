"""Writes sec51_reference_quantiles.json: the radial quantiles at T = 0.02 of
the finite-volume reference of the Sec. 5.1 convergence study (uniform unit
ball, M0 = 80, L = 8, mu = chi = 1, eps = 1e-4, k = 0.1, tau = 1e-5, 2000
steps, N = 4e5 cells as in the paper), at the study's levels j/1000,
j = 0..749.  Calls only the oracle (oracle/radial_fv.py).

    python tests/golden/make_sec51_reference.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import radial_fv as R  # noqa: E402

P = dict(L=8.0, mass=80.0, mu=1.0, chi=1.0, eps=1e-4, k=0.1, dt=1e-5, T=0.02, ball_radius=1.0)
N = 400_000


def main():
    g, rho, c = R.solve(P, N=N)
    levels = R.study_alphas(1000)
    q = R.cdf_quantiles(g, rho, levels)
    out = {"_about": "Radial quantiles q_{j/1000}, j = 0..749, at T = 0.02 of the implicit finite-volume "
                     "reference of Sec. 5.1 (Eq. (1D) on the ball of the box's volume, N = 4e5 cells); "
                     "written by make_sec51_reference.py from oracle/radial_fv.py",
           "params": P, "cells": N, "levels": levels.tolist(), "quantiles": q.tolist(),
           "r_0999": float(R.cdf_quantiles(g, rho, [0.999])[0]), "mass": R.mass(g, rho)}
    with open(os.path.join(HERE, "sec51_reference_quantiles.json"), "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")


if __name__ == "__main__":
    main()
