"""The inverse transform for callers that cannot allocate device memory.

sipf_inverse_ft_noalloc_dev works in the library's built-in device work space
instead of overwriting (or asking for) caller memory, so it can serve code
that must not call cudaMalloc / cudaFree (for example inside another library's
callback or under a fixed memory budget).  It must give the oracle's inverse
transform within the usual operator tolerance and the same grid as the
ordinary entry point sipf_inverse_ft_dev, bit for bit, call after call, and
leave its input spectrum untouched.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest

from oracle import sipf_oracle as O
from paper_2512_03452_gb300 import _abi, build

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TD = {32: torch.float32, 64: torch.float64}
TOL = {32: 2e-6, 64: 1e-13}     # relative to the largest value, per log2(H)


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return _abi.load()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("H", [16, 64])
def test_noalloc_inverse_matches_oracle_and_allocating_entry_point(prec, H):
    """Two calls in a row (they share the work space): each result matches the
    oracle's inverse transform F_H^-1 of the same spectrum within the operator
    bar of the inverse-transform parity test, and equals the allocating entry
    point's result bit for bit (the same kernels on the same input, so any
    difference would mean the work space was stale or aliased)."""
    for call, seed in enumerate((11, 12)):
        field = np.random.default_rng(seed + H).normal(size=(H, H, H))
        G = O.forward_ft(field, 1.0)
        spec = torch.tensor(np.stack([G.real, G.imag], axis=-1), dtype=TD[prec], device="cuda").contiguous()
        spec_before = spec.clone()
        work = spec.clone()                          # the ordinary entry point overwrites its input
        ref = torch.empty(H ** 3, dtype=TD[prec], device="cuda")
        out = torch.full((H ** 3,), float("nan"), dtype=TD[prec], device="cuda")
        _abi.sipf_inverse_ft_dev(prec, H, work.data_ptr(), ref.data_ptr())
        _abi.sipf_inverse_ft_noalloc_dev(prec, H, spec.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.all(np.isfinite(o)), call
        exact = O.inverse_ft(G, H).ravel()
        assert np.max(np.abs(o - exact)) <= TOL[prec] * math.log2(H) * np.max(np.abs(exact)), call
        assert torch.equal(out, ref), call
        assert torch.equal(spec, spec_before), "input spectrum must be left unchanged"


def test_noalloc_rejects_spectra_beyond_its_work_space():
    H = 128
    spec = torch.zeros((H, H, H // 2 + 1, 2), dtype=torch.float32, device="cuda")
    out = torch.empty(H ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(_abi.SipfError) as e:
        _abi.sipf_inverse_ft_noalloc_dev(32, H, spec.data_ptr(), out.data_ptr())
    assert e.value.code == _abi.SIPF_EINVAL
    assert "work space" in _abi.sipf_last_error()
