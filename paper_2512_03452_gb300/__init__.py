"""GB300-native SIPF-PIC (Algorithm 4 of arXiv 2512.03452) for the 3D
parabolic-parabolic Keller-Segel system.

The compute path lives in libsipf.so (hand-written CUDA for sm_103a behind the
C ABI of include/sipf.h).  `_abi` forwards to it by name; `Simulation` is a
small convenience wrapper that marshals numpy arrays.
"""
from __future__ import annotations

import numpy as np

from . import _abi
from ._abi import (DEPOSIT_ATOMIC, DEPOSIT_DETERMINISTIC, PROP_EXP, PROP_IMPLICIT, SPLIT_HALF,
                   SPLIT_PLAIN, SipfError)

__all__ = ["Simulation", "Simulation2D", "Batch", "make_params", "SipfError", "SPLIT_HALF", "SPLIT_PLAIN",
           "DEPOSIT_ATOMIC", "DEPOSIT_DETERMINISTIC", "PROP_IMPLICIT", "PROP_EXP"]


def make_params(P, H, L=1.0, mass=1.0, chi=1.0, mu=1.0, eps=1.0, k=1.0, dt=1e-3, T=0.0, H0=-1.0,
                seed=0, precision=32, p2g_order=4, g2p_order=2, splitting=SPLIT_HALF,
                deposit_mode=DEPOSIT_ATOMIC, propagator=PROP_IMPLICIT, resort_every=0):
    """Build a sipf_params struct (field names of include/sipf.h)."""
    p = _abi.sipf_params_default()
    for name, val in dict(P=P, H=H, L=L, mass=mass, chi=chi, mu=mu, eps=eps, k=k, dt=dt, T=T, H0=H0,
                          seed=seed, precision=precision, p2g_order=p2g_order, g2p_order=g2p_order,
                          splitting=splitting, deposit_mode=deposit_mode, propagator=propagator,
                          resort_every=resort_every).items():
        setattr(p, name, val)
    return p


def params_from_workload(w, **overrides):
    """sipf_params of a workloads.Workload (overrides win)."""
    d = dict(P=w.P, H=w.H, L=w.L, mass=w.mass, chi=w.chi, mu=w.mu, eps=w.eps, k=w.k, dt=w.dt,
             T=w.dt * w.steps, H0=w.H0, seed=w.seed)
    d.update(overrides)
    return make_params(**d)


class Simulation:
    """One SIPF-PIC run on the current CUDA device (state owned by libsipf)."""

    def __init__(self, params, X0, stream: int | None = None):
        self.params = params
        self.P = int(params.P)
        self.H = int(params.H)
        self.ctx = _abi.sipf_init(params, X0, stream)

    def step(self, n: int = 1):
        _abi.sipf_step(self.ctx, n)

    def run(self):
        _abi.sipf_run(self.ctx)

    @property
    def n(self) -> int:
        return _abi.sipf_current_step(self.ctx)

    def sync(self):
        _abi.sipf_sync(self.ctx)

    def positions(self) -> np.ndarray:
        out = np.empty((self.P, 3), dtype=np.float64)
        _abi.sipf_positions(self.ctx, out)
        return out

    def set_positions(self, X):
        _abi.sipf_set_positions(self.ctx, np.ascontiguousarray(X, dtype=np.float64))

    def density(self, filtered: bool = False) -> np.ndarray:
        out = np.empty((self.H,) * 3, dtype=np.float64)
        _abi.sipf_density(self.ctx, out, int(filtered))
        return out

    def field(self) -> np.ndarray:
        out = np.empty((self.H,) * 3, dtype=np.float64)
        _abi.sipf_field(self.ctx, out)
        return out

    def spectrum(self) -> np.ndarray:
        out = np.empty((self.H, self.H, self.H // 2 + 1, 2), dtype=np.float64)
        _abi.sipf_spectrum(self.ctx, out)
        return out[..., 0] + 1j * out[..., 1]

    def gradient(self) -> np.ndarray:
        out = np.empty((3,) + (self.H,) * 3, dtype=np.float64)
        _abi.sipf_gradient(self.ctx, out)
        return out

    def diagnostics(self) -> dict:
        d = _abi.sipf_diagnostics(self.ctx)
        return {name: getattr(d, name) for name, _ in d._fields_}

    def positions_dev(self, x: int, y: int, z: int):
        """Write X in particle order into device arrays (pointers) x, y, z."""
        _abi.sipf_positions_dev(self.ctx, x, y, z)

    def close(self):
        if self.ctx:
            _abi.sipf_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation2D:
    """One run of the 2D variant (Sec. 5.2: eps = 0 is the parabolic-elliptic
    system) on the current CUDA device; X0 is (P, 2)."""

    def __init__(self, params, X0, stream: int | None = None):
        self.params = params
        self.P = int(params.P)
        self.H = int(params.H)
        self.ctx = _abi.sipf2d_init(params, X0, stream)

    def step(self, n: int = 1):
        _abi.sipf2d_step(self.ctx, n)

    @property
    def n(self) -> int:
        return _abi.sipf2d_current_step(self.ctx)

    def sync(self):
        _abi.sipf2d_sync(self.ctx)

    def positions(self) -> np.ndarray:
        out = np.empty((self.P, 2), dtype=np.float64)
        _abi.sipf2d_positions(self.ctx, out)
        return out

    def spectrum(self) -> np.ndarray:
        out = np.empty((self.H, self.H // 2 + 1, 2), dtype=np.float64)
        _abi.sipf2d_spectrum(self.ctx, out)
        return out[..., 0] + 1j * out[..., 1]

    def density(self, filtered: bool = False) -> np.ndarray:
        out = np.empty((self.H, self.H), dtype=np.float64)
        _abi.sipf2d_density(self.ctx, out, int(filtered))
        return out

    def diagnostics(self) -> dict:
        d = _abi.sipf2d_diagnostics(self.ctx)
        return {name: getattr(d, name) for name in ("mass", "peak", "hf_frac", "m2", "step")}

    def close(self):
        if self.ctx:
            _abi.sipf2d_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent runs advanced together (one launch per kernel for all runs,
    steps replayed from a CUDA graph).  Run r behaves like
    Simulation(params[r], X0s[r])."""

    def __init__(self, params, X0s, stream: int | None = None):
        self.params = list(params)
        self.P = [int(p.P) for p in self.params]
        self.H = [int(p.H) for p in self.params]
        self.handle = _abi.sipf_batch_init(self.params, X0s, stream)

    def __len__(self):
        return len(self.params)

    def step(self, n: int = 1):
        _abi.sipf_batch_step(self.handle, n)

    def use_graph(self, enable: bool):
        _abi.sipf_batch_use_graph(self.handle, int(enable))

    def autotune(self, steps_per_trial: int = 3) -> dict:
        """Choose tile and block shapes by timing real steps (the runs advance by
        the returned steps_used); returns the choices and best times."""
        t = _abi.sipf_batch_autotune(self.handle, steps_per_trial)
        g = t.ngroups
        return {"groups": [{"H": t.H[i], "cols_tile": t.cols_tile[i], "xpass_tile": t.xpass_tile[i],
                            "rows_blocks_per_sm": t.rows_blocks_per_sm[i], "plane_kernels": t.plane_kernels[i],
                            "plane_warps": t.plane_warps[i], "xpass_warps": t.xpass_warps[i],
                            "inverse_all_components": t.inverse_all_components[i],
                            "field_ms": t.field_ms[i]}
                           for i in range(g)],
                "move_blocks_per_sm": t.move_blocks_per_sm, "deposit_blocks_per_sm": t.deposit_blocks_per_sm,
                "move_ms": t.move_ms, "deposit_ms": t.deposit_ms, "steps_used": t.steps_used}

    @property
    def n(self) -> int:
        return _abi.sipf_batch_current_step(self.handle)

    def sync(self):
        _abi.sipf_batch_sync(self.handle)

    def positions(self, run: int) -> np.ndarray:
        out = np.empty((self.P[run], 3), dtype=np.float64)
        _abi.sipf_batch_positions(self.handle, run, out)
        return out

    def spectrum(self, run: int) -> np.ndarray:
        H = self.H[run]
        out = np.empty((H, H, H // 2 + 1, 2), dtype=np.float64)
        _abi.sipf_batch_spectrum(self.handle, run, out)
        return out[..., 0] + 1j * out[..., 1]

    def diagnostics(self, run: int) -> dict:
        d = _abi.sipf_batch_diagnostics(self.handle, run)
        return {name: getattr(d, name) for name, _ in d._fields_}

    def close(self):
        if self.handle:
            _abi.sipf_batch_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
