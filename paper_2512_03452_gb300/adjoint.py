"""Adjoint form: gradients of a function of the final density rho(T) with
respect to chi, mu and X^0 through N steps of Algorithm 4 with fixed noise.

`Adjoint` marshals numpy arrays to the C entry points sipf_adjoint_* (all the
arithmetic runs in libsipf's kernels); `SipfDensity` is a
torch.autograd.Function over it, so that a loss written in torch (FP64 on the
host) back-propagates into chi, mu and X0:

    engine = Adjoint(params, X0, nsteps=200)
    rho = SipfDensity.apply(X0_t, chi_t, mu_t, engine)      # (H, H, H) float64
    loss = ((rho - rho_star) ** 2).sum()
    loss.backward()                                         # X0_t.grad, chi_t.grad, mu_t.grad
"""
from __future__ import annotations

import numpy as np
import torch

from . import _abi


class Adjoint:
    """Forward with checkpoints every `checkpoint_every` steps, reverse sweep
    on request (state owned by libsipf)."""

    def __init__(self, params, X0, nsteps: int, checkpoint_every: int = 0, stream: int | None = None):
        self.params = params
        self.P = int(params.P)
        self.H = int(params.H)
        self.nsteps = int(nsteps)
        self.handle = _abi.sipf_adjoint_init(params, X0, nsteps, checkpoint_every, stream)

    def forward(self, chi: float, mu: float, X0=None) -> np.ndarray:
        """rho(T) on the grid (H^3 float64) for these chi, mu and X0 (None: the last X0)."""
        rho = np.empty((self.H,) * 3, dtype=np.float64)
        _abi.sipf_adjoint_forward(self.handle, chi, mu, X0, rho)
        return rho

    def backward(self, rho_bar):
        """(dJ/dchi, dJ/dmu, dJ/dX0) for dJ/drho(T) = rho_bar."""
        gX = np.empty((self.P, 3), dtype=np.float64)
        gc, gm = _abi.sipf_adjoint_backward(self.handle, rho_bar, gX)
        return gc, gm, gX

    def timing(self):
        """Device ms of the last forward and backward calls."""
        return _abi.sipf_adjoint_timing(self.handle)

    def close(self):
        if self.handle:
            _abi.sipf_adjoint_destroy(self.handle)
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


class SipfDensity(torch.autograd.Function):
    """rho(T) = SipfDensity.apply(X0, chi, mu, engine): X0 (P, 3), chi and mu
    0-d tensors; returns the (H, H, H) float64 density on X0's device."""

    @staticmethod
    def forward(ctx, X0, chi, mu, engine):
        X = X0.detach().to("cpu", torch.float64).numpy()
        rho = engine.forward(float(chi), float(mu), X)
        ctx.engine = engine
        ctx.meta = (X0.dtype, X0.device, chi.dtype, chi.device, mu.dtype, mu.device)
        return torch.from_numpy(rho).to(X0.device)

    @staticmethod
    def backward(ctx, rho_bar):
        xd, xdev, cd, cdev, md, mdev = ctx.meta
        gc, gm, gX = ctx.engine.backward(rho_bar.detach().to("cpu", torch.float64).numpy())
        return (torch.from_numpy(gX).to(xdev, xd), torch.tensor(gc, dtype=cd, device=cdev),
                torch.tensor(gm, dtype=md, device=mdev), None)
