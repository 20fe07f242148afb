"""Radially symmetric reference solution of the Sec. 5.1 convergence study.

TEST INFRASTRUCTURE, like sipf_oracle: only the tests and the benchmark's
convergence leg may import it; the library never does.

Sec. 5.1 reduces the 3D Keller-Segel system with radial data to the 1D
problem of Eq. (1D),
    rho_t     = (1/r^2) d_r [ r^2 (mu rho_r - chi rho c_r) ],
    eps c_t   = (1/r^2) d_r ( r^2 c_r ) - k^2 c + rho,
with rho_r = c_r = 0 at r = 0, on the ball of radius R_ball whose volume equals
the periodic box's, (4 pi / 3) R_ball^3 = L^3, and states that it computes the
reference with an implicit finite-volume method on N = 4e5 points.  The paper
gives no further detail; this module takes the following readings:
  * cells [i dr, (i+1) dr], i = 0..N-1, dr = R_ball / N, unknowns are cell
    averages; fluxes through a face of area 4 pi r_f^2, no flux at r = 0 (zero
    area) and at r = R_ball;
  * time levels follow Algorithm 4: c^n is advanced implicitly with the source
    rho^(n-1), rho^n implicitly (diffusion and drift) with the drift velocity
    chi grad c^(n-1) -- both from the previous level, as the particles' move
    uses grad c^(n-1) and the update of alpha uses beta^(n-1);
  * the drift flux through a face is chi c_r(face) times the mean of the two
    cell averages (central; second order for the fine grids used here);
  * c^0 = 0 (alpha^(0) = 0 in Algorithm 4); rho^0 the exact cell averages of
    the initial density.
The discrepancy measure is the truncated quantile W1 of Sec. 5.1.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_banded


def ball_radius(L):
    """R_ball with (4 pi / 3) R_ball^3 = L^3 (Sec. 5.1)."""
    return (3.0 * L ** 3 / (4.0 * math.pi)) ** (1.0 / 3.0)


class RadialGrid:
    def __init__(self, R, N):
        self.R, self.N = float(R), int(N)
        self.dr = self.R / self.N
        self.rf = np.arange(self.N + 1) * self.dr                  # faces
        self.rc = (np.arange(self.N) + 0.5) * self.dr              # centres
        self.V = (4.0 * math.pi / 3.0) * (self.rf[1:] ** 3 - self.rf[:-1] ** 3)
        self.A = 4.0 * math.pi * self.rf ** 2                      # face areas


def cell_averages_of_ball(g, radius, density):
    """Exact cell averages of density * 1{|x| <= radius}."""
    lo, hi = g.rf[:-1], g.rf[1:]
    inside = np.clip(np.minimum(hi, radius) ** 3 - lo ** 3, 0.0, None) * (4.0 * math.pi / 3.0)
    return density * inside / g.V


def _diffusion_bands(g, coef):
    """Banded form of the FV operator  u -> -(1/V_i) sum_f A_f coef (u_nb - u_i)/dr
    (positive semi-definite, no-flux at both ends)."""
    w = g.A[1:-1] * coef / g.dr            # interior faces 1..N-1
    lower = np.zeros(g.N)                  # coefficient of u_{i-1} in row i
    upper = np.zeros(g.N)                  # coefficient of u_{i+1} in row i
    diag = np.zeros(g.N)
    diag[:-1] += w
    diag[1:] += w
    upper[:-1] = -w
    lower[1:] = -w
    return lower / g.V, diag / g.V, upper / g.V


def step_c(g, c, rho, p):
    """eps (c^n - c^(n-1)) / tau = Lap_h c^n - k^2 c^n + rho^(n-1)."""
    lo, d, up = _diffusion_bands(g, 1.0)
    a = p["eps"] / p["dt"]
    ab = np.zeros((3, g.N))
    ab[0, 1:] = up[:-1]
    ab[1] = a + d + p["k"] ** 2
    ab[2, :-1] = lo[1:]
    return solve_banded((1, 1), ab, a * c + rho)


def step_rho(g, rho, c, p):
    """(rho^n - rho^(n-1)) / tau = -(1/V) sum_f A_f F_f,
    F_f = -mu (rho_R - rho_L)/dr + chi c_r(f) (rho_L + rho_R)/2, with c = c^(n-1)."""
    lo, d, up = _diffusion_bands(g, p["mu"])
    v = p["chi"] * (c[1:] - c[:-1]) / g.dr          # drift velocity at interior faces
    af = g.A[1:-1] * v * 0.5                        # A_f v_f / 2
    # row i gets + (A_{i+1/2} F_{i+1/2} - A_{i-1/2} F_{i-1/2}) / V_i on the left-hand side
    d_adv = np.zeros(g.N)
    up_adv = np.zeros(g.N)
    lo_adv = np.zeros(g.N)
    d_adv[:-1] += af                                 # face i+1/2, rho_L = rho_i
    up_adv[:-1] += af                                # face i+1/2, rho_R = rho_{i+1}
    d_adv[1:] -= af                                  # face i-1/2, rho_R = rho_i
    lo_adv[1:] -= af                                 # face i-1/2, rho_L = rho_{i-1}
    inv_dt = 1.0 / p["dt"]
    ab = np.zeros((3, g.N))
    ab[0, 1:] = (up + up_adv / g.V)[:-1]
    ab[1] = inv_dt + d + d_adv / g.V
    ab[2, :-1] = (lo + lo_adv / g.V)[1:]
    return solve_banded((1, 1), ab, inv_dt * rho)


def solve(p, N=400_000, steps=None, rho0=None, c0=None, freeze_rho=False):
    """Run the scheme to step `steps` (default ceil(T/dt)).  p: dict with L, mass,
    mu, chi, eps, k, dt, T, ball_radius.  Returns (grid, rho, c)."""
    g = RadialGrid(ball_radius(p["L"]), N)
    if rho0 is None:
        r0 = p.get("ball_radius", 1.0)
        rho0 = cell_averages_of_ball(g, r0, p["mass"] / (4.0 * math.pi / 3.0 * r0 ** 3))
    rho = np.array(rho0, dtype=np.float64)
    c = np.zeros(g.N) if c0 is None else np.array(c0, dtype=np.float64)
    n = int(math.ceil(p["T"] / p["dt"] - 1e-9)) if steps is None else int(steps)
    for _ in range(n):
        c_new = step_c(g, c, rho, p)
        if not freeze_rho:
            rho = step_rho(g, rho, c, p)
        c = c_new
    return g, rho, c


def mass(g, rho):
    return float(np.sum(g.V * rho))


def cdf_quantiles(g, rho, alphas, total=None):
    """Quantiles q_a = inf{r : m(r) >= a} of m(r) = (4 pi / M0) int_0^r psi s^2 ds
    for the piecewise-constant cell averages (m is exact and increasing in r^3
    inside a cell)."""
    total = mass(g, rho) if total is None else total
    cum = np.concatenate([[0.0], np.cumsum(g.V * rho)]) / total
    alphas = np.asarray(alphas, dtype=np.float64)
    q = np.zeros_like(alphas)
    for j, a in enumerate(alphas):
        if a <= 0.0:
            q[j] = 0.0
            continue
        i = int(np.searchsorted(cum, a, side="left")) - 1     # cum[i] < a <= cum[i+1]
        i = min(max(i, 0), g.N - 1)
        dm = cum[i + 1] - cum[i]
        frac = 0.0 if dm <= 0.0 else (a - cum[i]) / dm
        lo3, hi3 = g.rf[i] ** 3, g.rf[i + 1] ** 3
        q[j] = (lo3 + frac * (hi3 - lo3)) ** (1.0 / 3.0)
    return q


def empirical_quantiles(radii, alphas):
    """q_a = inf{r : (1/P) #{|X_p| <= r} >= a}: the ceil(a P)-th smallest radius
    (0 at a = 0)."""
    r = np.sort(np.asarray(radii, dtype=np.float64))
    P = r.shape[0]
    out = np.zeros(len(alphas))
    for j, a in enumerate(alphas):
        k = int(math.ceil(a * P - 1e-12))
        out[j] = 0.0 if k <= 0 else r[min(k, P) - 1]
    return out


def truncated_w1(q_ref, q_hat):
    """Sec. 5.1: E = (1/(m+1)) sum_{j=0}^{m} |q_{j/n} - qhat_{j/n}| over the
    quantiles j = 0..m, m = ceil(3n/4) - 1 (the upper quartile left out)."""
    q_ref, q_hat = np.asarray(q_ref), np.asarray(q_hat)
    return float(np.mean(np.abs(q_ref - q_hat)))


def study_alphas(n=1000):
    """The quantile levels j/n, j = 0..m, m = ceil(3n/4) - 1, of Sec. 5.1."""
    m = int(math.ceil(3 * n / 4)) - 1
    return np.arange(m + 1) / n
