"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every entry point include/sipf.h declares; parameter validation and
error reporting work without touching a device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2512_03452_gb300 import _abi, build, make_params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sipf.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.load()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sipf[a-z0-9]*_[a-z_0-9]+)\s*\(", text)))


def test_header_declarations_match_binding():
    assert declared_symbols() == _abi.exported_symbols()


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sipf\w+)", out))
    for name in declared_symbols():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_defaults_and_validation(lib):
    p = _abi.sipf_params_default()
    assert (p.H, p.precision, p.p2g_order, p.g2p_order, p.H0) == (64, 32, 4, 2, -1.0)
    with pytest.raises(_abi.SipfError) as e:
        _abi.sipf_validate(p)                  # P = 0
    assert e.value.code == _abi.SIPF_EINVAL and "P" in _abi.sipf_last_error()
    good = make_params(P=10, H=16)
    _abi.sipf_validate(good)
    for field, val in [("H", 12), ("H", 512), ("H", 4), ("precision", 16), ("dt", 0.0), ("eps", -1.0),
                       ("p2g_order", 3), ("g2p_order", 1), ("splitting", 2), ("deposit_mode", 5),
                       ("L", float("nan")), ("mass", 0.0), ("resort_every", -1)]:
        p = make_params(P=10, H=16)
        setattr(p, field, val)
        with pytest.raises(_abi.SipfError) as e:
            _abi.sipf_validate(p)
        assert e.value.code == _abi.SIPF_EINVAL, field


def test_strerror(lib):
    assert _abi.sipf_strerror(0) == "ok"
    assert "invalid" in _abi.sipf_strerror(_abi.SIPF_EINVAL)
    assert _abi.sipf_strerror(12345) == "unknown error"


def test_stateless_entry_points_reject_bad_sizes(lib):
    with pytest.raises(_abi.SipfError):
        _abi.sipf_deposit_dev(32, 0, 0, 0, 10, 12, 1.0, 1.0, 4, 0)       # H not a power of two
    with pytest.raises(_abi.SipfError):
        _abi.sipf_forward_ft_dev(16, 16, 1.0, 0, 0)                     # bad precision
    with pytest.raises(_abi.SipfError):
        _abi.sipf_noise_dev(32, 0, -1, 0, 10, 0)                         # negative step


def test_init_rejects_nonfinite_positions_before_touching_a_device(lib):
    p = make_params(P=4, H=8)
    X = np.zeros((4, 3))
    X[2, 1] = np.nan
    with pytest.raises(_abi.SipfError) as e:
        _abi.sipf_init(p, X)
    assert e.value.code == _abi.SIPF_ENONFINITE


def test_filter_scale_matches_the_exact_rule(lib):
    """The library's automatic H0 equals the oracle's exact ceil(8 H^(8/13)
    L^(5/13)) (Sec. 5.1) over the supported H and a spread of box sides,
    including H = L = 8 where the value is an exact integer (64)."""
    from oracle import sipf_oracle as O
    for H in (8, 16, 32, 64, 128, 256):
        for L in (1.0, 2.0, 8.0, 0.7, 3.3, 10.0, 40.0, 2.0 ** -13, 2.0 ** 13):
            assert _abi.sipf_filter_scale(make_params(P=10, H=H, L=L)) == O.auto_H0(H, L), (H, L)
    assert _abi.sipf_filter_scale(make_params(P=10, H=8, L=8.0)) == 64.0
    assert _abi.sipf_filter_scale(make_params(P=10, H=64, L=1.0, H0=12.5)) == 12.5
    assert _abi.sipf_filter_scale(make_params(P=10, H=64, L=1.0, H0=0.0)) == 0.0
    with pytest.raises(_abi.SipfError):
        _abi.sipf_filter_scale(make_params(P=10, H=12))
