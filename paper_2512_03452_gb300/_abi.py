"""ctypes binding of libsipf.so (include/sipf.h): argument marshalling only.

Every function here has the name of the C entry point it forwards to; all
computation happens in the library's CUDA kernels.  Loading fails loudly when
the compiled library is missing: there is no Python or CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsipf.so")

SIPF_OK = 0
SIPF_EINVAL = -1
SIPF_ENOMEM = -2
SIPF_ECUDA = -3
SIPF_ENONFINITE = -4
SIPF_ETIMEOUT = -5
SIPF_ENODEV = -6

SPLIT_HALF, SPLIT_PLAIN = 0, 1
DEPOSIT_ATOMIC, DEPOSIT_DETERMINISTIC = 0, 1
PROP_IMPLICIT, PROP_EXP = 0, 1


class sipf_params(ctypes.Structure):
    _fields_ = [
        ("chi", ctypes.c_double), ("mu", ctypes.c_double), ("eps", ctypes.c_double),
        ("k", ctypes.c_double), ("L", ctypes.c_double), ("mass", ctypes.c_double),
        ("dt", ctypes.c_double), ("T", ctypes.c_double), ("H0", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("P", ctypes.c_int64), ("H", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("p2g_order", ctypes.c_int32),
        ("g2p_order", ctypes.c_int32), ("splitting", ctypes.c_int32),
        ("deposit_mode", ctypes.c_int32), ("propagator", ctypes.c_int32),
        ("resort_every", ctypes.c_int32),
    ]


class sipf_diag(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double), ("alpha0", ctypes.c_double), ("peak", ctypes.c_double),
        ("hf_frac", ctypes.c_double), ("m2", ctypes.c_double), ("ring_radius", ctypes.c_double),
        ("step", ctypes.c_int64),
    ]


class sipf_timing(ctypes.Structure):
    _fields_ = [
        ("forward_ms", ctypes.c_double), ("spectral_ms", ctypes.c_double), ("inverse_ms", ctypes.c_double),
        ("move_ms", ctypes.c_double), ("bookkeeping_ms", ctypes.c_double), ("deposit_ms", ctypes.c_double),
        ("steps", ctypes.c_int64),
        ("kernels", ctypes.c_int64), ("overflow", ctypes.c_int64),
    ]


class sipf_batch_tuning(ctypes.Structure):
    _fields_ = [("ngroups", ctypes.c_int32), ("H", ctypes.c_int32 * 4), ("cols_tile", ctypes.c_int32 * 4),
                ("xpass_tile", ctypes.c_int32 * 4), ("rows_blocks_per_sm", ctypes.c_int32 * 4),
                ("plane_kernels", ctypes.c_int32 * 4), ("plane_warps", ctypes.c_int32 * 4),
                ("xpass_warps", ctypes.c_int32 * 4), ("inverse_all_components", ctypes.c_int32 * 4),
                ("move_blocks_per_sm", ctypes.c_int32), ("deposit_blocks_per_sm", ctypes.c_int32),
                ("field_ms", ctypes.c_double * 4), ("move_ms", ctypes.c_double), ("deposit_ms", ctypes.c_double),
                ("steps_used", ctypes.c_int64)]


class SipfError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed ({code}: {msg})")
        self.code = code


_lib = None

_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "sipf_params_default": (ctypes.c_int, [ctypes.POINTER(sipf_params)]),
    "sipf_validate": (ctypes.c_int, [ctypes.POINTER(sipf_params)]),
    "sipf_filter_scale": (ctypes.c_int, [ctypes.POINTER(sipf_params), _D]),
    "sipf_init": (ctypes.c_int, [ctypes.POINTER(sipf_params), _D, _P, ctypes.POINTER(_P)]),
    "sipf_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "sipf_run": (ctypes.c_int, [_P]),
    "sipf_current_step": (ctypes.c_int64, [_P]),
    "sipf_positions": (ctypes.c_int, [_P, _D]),
    "sipf_set_positions": (ctypes.c_int, [_P, _D]),
    "sipf_upload_soa": (ctypes.c_int, [_P, _P, _P, _P]),
    "sipf_download_soa": (ctypes.c_int, [_P, _P, _P, _P]),
    "sipf_positions_dev": (ctypes.c_int, [_P, _P, _P, _P]),
    "sipf_density": (ctypes.c_int, [_P, _D, ctypes.c_int]),
    "sipf_field": (ctypes.c_int, [_P, _D]),
    "sipf_spectrum": (ctypes.c_int, [_P, _D]),
    "sipf_gradient": (ctypes.c_int, [_P, _D]),
    "sipf_diagnostics": (ctypes.c_int, [_P, ctypes.POINTER(sipf_diag)]),
    "sipf_sync": (ctypes.c_int, [_P]),
    "sipf_timing_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "sipf_timing_read": (ctypes.c_int, [_P, ctypes.POINTER(sipf_timing)]),
    "sipf_kernel_launches": (ctypes.c_int64, [_P]),
    "sipf_destroy": (None, [_P]),
    "sipf_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sipf_last_error": (ctypes.c_char_p, []),
    "sipf_noise_dev": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_int64, _P, _P]),
    "sipf_deposit_dev": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int32, _P, _P]),
    "sipf_gather_dev": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_double, _P, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "sipf_forward_ft_dev": (ctypes.c_int, [ctypes.c_int, ctypes.c_int32, ctypes.c_double, _P, _P, _P]),
    "sipf_inverse_ft_dev": (ctypes.c_int, [ctypes.c_int, ctypes.c_int32, _P, _P, _P]),
    "sipf_inverse_ft_noalloc_dev": (ctypes.c_int, [ctypes.c_int, ctypes.c_int32, _P, _P, _P]),
    "sipf_batch_init": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(sipf_params), ctypes.POINTER(_D), _P,
                                       ctypes.POINTER(_P)]),
    "sipf_batch_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "sipf_batch_use_graph": (ctypes.c_int, [_P, ctypes.c_int]),
    "sipf_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(sipf_batch_tuning)]),
    "sipf_batch_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(sipf_batch_tuning)]),
    "sipf_batch_current_step": (ctypes.c_int64, [_P]),
    "sipf_batch_kernel_launches": (ctypes.c_int64, [_P]),
    "sipf_batch_positions": (ctypes.c_int, [_P, ctypes.c_int32, _D]),
    "sipf_batch_diagnostics": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(sipf_diag)]),
    "sipf_batch_spectrum": (ctypes.c_int, [_P, ctypes.c_int32, _D]),
    "sipf_batch_sync": (ctypes.c_int, [_P]),
    "sipf_batch_destroy": (None, [_P]),
    "sipf_adjoint_init": (ctypes.c_int, [ctypes.POINTER(sipf_params), _D, ctypes.c_int64, ctypes.c_int32, _P,
                                         ctypes.POINTER(_P)]),
    "sipf_adjoint_forward": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, _D, _D]),
    "sipf_adjoint_backward": (ctypes.c_int, [_P, _D, _D, _D, _D]),
    "sipf_adjoint_timing": (ctypes.c_int, [_P, _D, _D]),
    "sipf_adjoint_kernel_launches": (ctypes.c_int64, [_P]),
    "sipf_adjoint_destroy": (None, [_P]),
    "sipf_measure_fp64_fma": (ctypes.c_int, [_P, _D]),
    "sipf2d_init": (ctypes.c_int, [ctypes.POINTER(sipf_params), _D, _P, ctypes.POINTER(_P)]),
    "sipf2d_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "sipf2d_current_step": (ctypes.c_int64, [_P]),
    "sipf2d_positions": (ctypes.c_int, [_P, _D]),
    "sipf2d_spectrum": (ctypes.c_int, [_P, _D]),
    "sipf2d_density": (ctypes.c_int, [_P, _D, ctypes.c_int]),
    "sipf2d_diagnostics": (ctypes.c_int, [_P, ctypes.POINTER(sipf_diag)]),
    "sipf2d_sync": (ctypes.c_int, [_P]),
    "sipf2d_destroy": (None, [_P]),
}


def exported_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return sorted(_SIGS)


def load(path: str = LIB_PATH):
    """Load libsipf.so (once) and attach the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libsipf.so not built at {path}: run paper_2512_03452_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != SIPF_OK:
        lib = load()
        raise SipfError(code, where, (lib.sipf_last_error() or b"").decode() or lib.sipf_strerror(code).decode())


def _dptr(a):
    """ctypes double* of a contiguous float64 numpy array."""
    return a.ctypes.data_as(_D)


# ---- same-name wrappers ------------------------------------------------------
def sipf_params_default() -> sipf_params:
    p = sipf_params()
    _check(load().sipf_params_default(ctypes.byref(p)), "sipf_params_default")
    return p


def sipf_validate(p: sipf_params) -> None:
    _check(load().sipf_validate(ctypes.byref(p)), "sipf_validate")


def sipf_filter_scale(p: sipf_params) -> float:
    out = ctypes.c_double()
    _check(load().sipf_filter_scale(ctypes.byref(p), ctypes.byref(out)), "sipf_filter_scale")
    return out.value


def sipf_init(p: sipf_params, X0, stream: int | None = None) -> int:
    """X0: contiguous (P, 3) float64 numpy array.  Returns the context handle."""
    import numpy as np
    X0 = np.ascontiguousarray(X0, dtype=np.float64)
    h = _P()
    _check(load().sipf_init(ctypes.byref(p), _dptr(X0), _P(stream or 0), ctypes.byref(h)), "sipf_init")
    return h.value


def sipf_step(ctx: int, nsteps: int) -> None:
    _check(load().sipf_step(_P(ctx), int(nsteps)), "sipf_step")


def sipf_run(ctx: int) -> None:
    _check(load().sipf_run(_P(ctx)), "sipf_run")


def sipf_current_step(ctx: int) -> int:
    return int(load().sipf_current_step(_P(ctx)))


def sipf_positions(ctx: int, out) -> None:
    _check(load().sipf_positions(_P(ctx), _dptr(out)), "sipf_positions")


def sipf_set_positions(ctx: int, X) -> None:
    _check(load().sipf_set_positions(_P(ctx), _dptr(X)), "sipf_set_positions")


def sipf_upload_soa(ctx: int, x: int, y: int, z: int) -> None:
    _check(load().sipf_upload_soa(_P(ctx), _P(x), _P(y), _P(z)), "sipf_upload_soa")


def sipf_download_soa(ctx: int, x: int, y: int, z: int) -> None:
    _check(load().sipf_download_soa(_P(ctx), _P(x), _P(y), _P(z)), "sipf_download_soa")


def sipf_positions_dev(ctx: int, x: int, y: int, z: int) -> None:
    _check(load().sipf_positions_dev(_P(ctx), _P(x), _P(y), _P(z)), "sipf_positions_dev")


def sipf_density(ctx: int, out, filtered: int) -> None:
    _check(load().sipf_density(_P(ctx), _dptr(out), int(filtered)), "sipf_density")


def sipf_field(ctx: int, out) -> None:
    _check(load().sipf_field(_P(ctx), _dptr(out)), "sipf_field")


def sipf_spectrum(ctx: int, out) -> None:
    _check(load().sipf_spectrum(_P(ctx), _dptr(out)), "sipf_spectrum")


def sipf_gradient(ctx: int, out) -> None:
    _check(load().sipf_gradient(_P(ctx), _dptr(out)), "sipf_gradient")


def sipf_diagnostics(ctx: int) -> sipf_diag:
    d = sipf_diag()
    _check(load().sipf_diagnostics(_P(ctx), ctypes.byref(d)), "sipf_diagnostics")
    return d


def sipf_sync(ctx: int) -> None:
    _check(load().sipf_sync(_P(ctx)), "sipf_sync")


def sipf_timing_enable(ctx: int, enable: int) -> None:
    _check(load().sipf_timing_enable(_P(ctx), int(enable)), "sipf_timing_enable")


def sipf_timing_read(ctx: int) -> sipf_timing:
    t = sipf_timing()
    _check(load().sipf_timing_read(_P(ctx), ctypes.byref(t)), "sipf_timing_read")
    return t


def sipf_kernel_launches(ctx: int) -> int:
    return int(load().sipf_kernel_launches(_P(ctx)))


def sipf_destroy(ctx: int) -> None:
    load().sipf_destroy(_P(ctx))


def sipf_strerror(code: int) -> str:
    return load().sipf_strerror(int(code)).decode()


def sipf_last_error() -> str:
    return (load().sipf_last_error() or b"").decode()


def sipf_noise_dev(precision, seed, step, first, P, z, stream=0) -> None:
    _check(load().sipf_noise_dev(precision, seed, step, first, P, _P(z), _P(stream)), "sipf_noise_dev")


def sipf_deposit_dev(precision, x, y, z, P, H, L, w, order, grid, stream=0) -> None:
    _check(load().sipf_deposit_dev(precision, _P(x), _P(y), _P(z), P, H, L, w, order, _P(grid), _P(stream)),
           "sipf_deposit_dev")


def sipf_gather_dev(precision, x, y, z, P, H, L, f, ncomp, order, out, stream=0) -> None:
    _check(load().sipf_gather_dev(precision, _P(x), _P(y), _P(z), P, H, L, _P(f), ncomp, order, _P(out),
                                  _P(stream)), "sipf_gather_dev")


def sipf_forward_ft_dev(precision, H, L, grid, spec, stream=0) -> None:
    _check(load().sipf_forward_ft_dev(precision, H, L, _P(grid), _P(spec), _P(stream)), "sipf_forward_ft_dev")


def sipf_inverse_ft_dev(precision, H, spec, grid, stream=0) -> None:
    _check(load().sipf_inverse_ft_dev(precision, H, _P(spec), _P(grid), _P(stream)), "sipf_inverse_ft_dev")


def sipf_inverse_ft_noalloc_dev(precision, H, spec, grid, stream=0) -> None:
    """Inverse transform with the library's built-in work space (no device
    allocation; `spec` is left unchanged; H <= 64)."""
    _check(load().sipf_inverse_ft_noalloc_dev(precision, H, _P(spec), _P(grid), _P(stream)),
           "sipf_inverse_ft_noalloc_dev")


# ---- batched runs --------------------------------------------------------------
def sipf_batch_init(params, X0s, stream: int | None = None) -> int:
    """params: sequence of sipf_params; X0s: matching (P_r, 3) float64 arrays.
    Returns the batch handle."""
    import numpy as np
    n = len(params)
    if len(X0s) != n:
        raise ValueError("one X0 per run")
    arr = (sipf_params * n)(*params)
    keep = [np.ascontiguousarray(X, dtype=np.float64) for X in X0s]
    ptrs = (_D * n)(*[_dptr(X) for X in keep])
    h = _P()
    _check(load().sipf_batch_init(n, arr, ptrs, _P(stream or 0), ctypes.byref(h)), "sipf_batch_init")
    return h.value


def sipf_batch_step(b: int, nsteps: int) -> None:
    _check(load().sipf_batch_step(_P(b), int(nsteps)), "sipf_batch_step")


def sipf_batch_autotune(b: int, steps_per_trial: int = 3) -> sipf_batch_tuning:
    t = sipf_batch_tuning()
    _check(load().sipf_batch_autotune(_P(b), int(steps_per_trial), ctypes.byref(t)), "sipf_batch_autotune")
    return t


def sipf_batch_set_tuning(b: int, t: sipf_batch_tuning) -> None:
    _check(load().sipf_batch_set_tuning(_P(b), ctypes.byref(t)), "sipf_batch_set_tuning")


def sipf_batch_use_graph(b: int, enable: int) -> None:
    _check(load().sipf_batch_use_graph(_P(b), int(enable)), "sipf_batch_use_graph")


def sipf_batch_current_step(b: int) -> int:
    return int(load().sipf_batch_current_step(_P(b)))


def sipf_batch_kernel_launches(b: int) -> int:
    return int(load().sipf_batch_kernel_launches(_P(b)))


def sipf_batch_positions(b: int, run: int, out) -> None:
    _check(load().sipf_batch_positions(_P(b), int(run), _dptr(out)), "sipf_batch_positions")


def sipf_batch_diagnostics(b: int, run: int) -> sipf_diag:
    d = sipf_diag()
    _check(load().sipf_batch_diagnostics(_P(b), int(run), ctypes.byref(d)), "sipf_batch_diagnostics")
    return d


def sipf_batch_spectrum(b: int, run: int, out) -> None:
    _check(load().sipf_batch_spectrum(_P(b), int(run), _dptr(out)), "sipf_batch_spectrum")


def sipf_batch_sync(b: int) -> None:
    _check(load().sipf_batch_sync(_P(b)), "sipf_batch_sync")


def sipf_batch_destroy(b: int) -> None:
    load().sipf_batch_destroy(_P(b))


# ---- adjoint ---------------------------------------------------------------------
def sipf_adjoint_init(p: sipf_params, X0, nsteps: int, checkpoint_every: int = 0, stream: int | None = None) -> int:
    import numpy as np
    X0 = np.ascontiguousarray(X0, dtype=np.float64)
    h = _P()
    _check(load().sipf_adjoint_init(ctypes.byref(p), _dptr(X0), int(nsteps), int(checkpoint_every), _P(stream or 0),
                                    ctypes.byref(h)), "sipf_adjoint_init")
    return h.value


def sipf_adjoint_forward(a: int, chi: float, mu: float, X0, rho_out) -> None:
    """X0: (P, 3) float64 array or None; rho_out: (H, H, H) float64 array or None."""
    import numpy as np
    x = None if X0 is None else _dptr(np.ascontiguousarray(X0, dtype=np.float64))
    r = None if rho_out is None else _dptr(rho_out)
    _check(load().sipf_adjoint_forward(_P(a), float(chi), float(mu), x, r), "sipf_adjoint_forward")


def sipf_adjoint_backward(a: int, rho_bar, grad_X0=None):
    """Returns (dJ/dchi, dJ/dmu); fills grad_X0 ((P, 3) float64) if given."""
    import numpy as np
    rb = np.ascontiguousarray(rho_bar, dtype=np.float64)
    gc, gm = ctypes.c_double(), ctypes.c_double()
    gx = None if grad_X0 is None else _dptr(grad_X0)
    _check(load().sipf_adjoint_backward(_P(a), _dptr(rb), ctypes.byref(gc), ctypes.byref(gm), gx),
           "sipf_adjoint_backward")
    return gc.value, gm.value


def sipf_adjoint_timing(a: int):
    f, b = ctypes.c_double(), ctypes.c_double()
    _check(load().sipf_adjoint_timing(_P(a), ctypes.byref(f), ctypes.byref(b)), "sipf_adjoint_timing")
    return f.value, b.value


def sipf_adjoint_kernel_launches(a: int) -> int:
    return int(load().sipf_adjoint_kernel_launches(_P(a)))


def sipf_adjoint_destroy(a: int) -> None:
    load().sipf_adjoint_destroy(_P(a))


def sipf_measure_fp64_fma(stream: int = 0) -> float:
    g = ctypes.c_double()
    _check(load().sipf_measure_fp64_fma(_P(stream), ctypes.byref(g)), "sipf_measure_fp64_fma")
    return g.value


# ---- 2D variant (Sec. 5.2) ----------------------------------------------------
def sipf2d_init(p: sipf_params, X0, stream: int | None = None) -> int:
    """X0: contiguous (P, 2) float64 numpy array.  Returns the 2D context handle."""
    import numpy as np
    X0 = np.ascontiguousarray(X0, dtype=np.float64)
    h = _P()
    _check(load().sipf2d_init(ctypes.byref(p), _dptr(X0), _P(stream or 0), ctypes.byref(h)), "sipf2d_init")
    return h.value


def sipf2d_step(ctx: int, nsteps: int) -> None:
    _check(load().sipf2d_step(_P(ctx), int(nsteps)), "sipf2d_step")


def sipf2d_current_step(ctx: int) -> int:
    return int(load().sipf2d_current_step(_P(ctx)))


def sipf2d_positions(ctx: int, out) -> None:
    _check(load().sipf2d_positions(_P(ctx), _dptr(out)), "sipf2d_positions")


def sipf2d_spectrum(ctx: int, out) -> None:
    _check(load().sipf2d_spectrum(_P(ctx), _dptr(out)), "sipf2d_spectrum")


def sipf2d_density(ctx: int, out, filtered: int) -> None:
    _check(load().sipf2d_density(_P(ctx), _dptr(out), int(filtered)), "sipf2d_density")


def sipf2d_diagnostics(ctx: int) -> sipf_diag:
    d = sipf_diag()
    _check(load().sipf2d_diagnostics(_P(ctx), ctypes.byref(d)), "sipf2d_diagnostics")
    return d


def sipf2d_sync(ctx: int) -> None:
    _check(load().sipf2d_sync(_P(ctx)), "sipf2d_sync")


def sipf2d_destroy(ctx: int) -> None:
    load().sipf2d_destroy(_P(ctx))
