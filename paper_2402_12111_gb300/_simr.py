"""ctypes binding of libsimr.so (include/simr.h): argument marshalling only.

Every step of the pricing path runs in the CUDA library; this module turns
torch tensors (device memory and streams) or host arrays into the C ABI's plain
pointers, allocates outputs, and raises SimrError on a non-zero status.  There
is no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SIMR_OK, SIMR_EINVAL, SIMR_ENOMEM, SIMR_ECUDA, SIMR_ETIMEOUT, SIMR_EUNSUPPORTED = 0, -1, -2, -3, -4, -5

G_DELTA, G_GAMMA, G_VEGA, G_THETA, G_RHO = 1, 2, 4, 8, 16
G_KAPPA, G_LRVAR, G_VOLVOL, G_CORR = 32, 64, 128, 256
G_ALL = 0x1FF
GREEK_BITS = {"delta": G_DELTA, "gamma": G_GAMMA, "vega": G_VEGA, "theta": G_THETA, "rho": G_RHO,
              "kappa": G_KAPPA, "lrvar": G_LRVAR, "volvol": G_VOLVOL, "corr": G_CORR}

MODEL_FIELDS = ("S0", "r", "T", "v0", "kappa", "theta", "sigma", "rho")


class SimrError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"simr error {code}: {message}")
        self.code = code


class Heston(ctypes.Structure):
    """simr_heston: spot, rate, maturity, v0, kappa, theta, sigma, rho (FP64)."""

    _fields_ = [(n, ctypes.c_double) for n in MODEL_FIELDS]


class Option(ctypes.Structure):
    """simr_option: model, strike, put flag, steps, paths."""

    _fields_ = [("m", Heston), ("K", ctypes.c_double), ("is_put", ctypes.c_int32), ("steps", ctypes.c_uint32),
                ("paths", ctypes.c_uint64)]


BATCH_ADJOINT, BATCH_GRAPH, BATCH_NO_AUTOTUNE = 1, 2, 4
FAULT_ALLOC, FAULT_LAUNCH, FAULT_BARRIER = 1, 2, 3


def batch_variant_flag(v: int) -> int:
    """SIMR_BATCH_VARIANT(v): run kernel shape v (0-7) of the book kernel."""
    return ((int(v) & 7) + 1) << 8


SCHEMES = {"qe": 0, "qem": 1}


def as_heston(model) -> Heston:
    if isinstance(model, Heston):
        return model
    return Heston(**{k: float(model[k]) for k in MODEL_FIELDS})


def greek_mask(greeks) -> int:
    if isinstance(greeks, int):
        return greeks
    m = 0
    for g in greeks:
        m |= GREEK_BITS[g]
    return m


_lock = threading.Lock()
_lib = None
_ctx = {}


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libsimr.so (building it first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise SimrError(SIMR_EUNSUPPORTED, f"{path} is missing: run paper_2402_12111_gb300.build.build()")
        L = ctypes.CDLL(path)
        H = ctypes.POINTER(Heston)
        dp = ctypes.c_void_p
        u32, u64, c_int, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        L.simr_create.argtypes = [ctypes.POINTER(vp), c_int]
        L.simr_destroy.argtypes = [vp]
        L.simr_destroy.restype = None
        L.simr_last_error.restype = ctypes.c_char_p
        L.simr_version.restype = c_int
        L.simr_price.argtypes = [vp, H, dp, c_int, c_int, u32, u64, u64, u32, dp, dp, vp]
        L.simr_greeks_fd.argtypes = [vp, H, dp, c_int, c_int, u32, u64, u64, u32, ctypes.c_double, u32, dp, dp, vp]
        L.simr_paths_terminal.argtypes = [vp, H, u32, u64, u64, u64, u32, dp, dp, vp]
        L.simr_path_sums.argtypes = [vp, H, dp, c_int, c_int, u32, u64, u64, u64, u32, ctypes.c_double, u32, dp, vp]
        L.simr_finalize_sums.argtypes = [vp, H, dp, c_int, c_int, u32, u64, ctypes.c_double, u32, dp, dp, dp, dp,
                                         vp]
        L.simr_greeks_adjoint.argtypes = [vp, H, dp, c_int, c_int, u32, u64, u64, u32, u32, dp, dp, dp, vp]
        L.simr_paths_adjoint.argtypes = [vp, H, u32, u64, u64, u64, u32, u32, dp, dp, vp]
        L.simr_adjoint_interval.argtypes = [vp, c_int, u32, ctypes.POINTER(u32)]
        L.simr_inject_fault.argtypes = [c_int, c_int]
        L.simr_batch_submit.argtypes = [vp, ctypes.POINTER(Option), c_int, u64, u32, dp, dp, dp, vp]
        L.simr_lsm_price.argtypes = [vp, H, ctypes.c_double, c_int, u32, u32, u64, u64, u32, dp, dp, dp, dp, vp]
        L.simr_set_scheme.argtypes = [vp, c_int]
        L.simr_basket_price.argtypes = [vp, H, c_int, dp, dp, dp, c_int, c_int, u32, u64, u64, dp, dp, vp]
        L.simr_sync.argtypes = [vp, vp]
        L.simr_price_noalloc.argtypes = [H, dp, c_int, c_int, u32, u64, u64, u32, dp, dp, vp]
        L.simr_philox_words.argtypes = [vp, u64, u32, u64, u64, u32, u32, dp, vp]
        L.simr_normals.argtypes = [vp, dp, u64, dp, dp, vp]
        L.simr_unit_rates.argtypes = [vp, dp, vp]
        _lib = L
        return L


def check(rc: int) -> None:
    if rc != SIMR_OK:
        msg = load().simr_last_error().decode(errors="replace")
        raise SimrError(rc, msg)


def context(device: int = 0):
    """The library context of a CUDA device (created once per process)."""
    L = load()
    with _lock:
        if device not in _ctx:
            h = ctypes.c_void_p()
            rc = L.simr_create(ctypes.byref(h), int(device))
            if rc != SIMR_OK:
                raise SimrError(rc, L.simr_last_error().decode(errors="replace"))
            _ctx[device] = h
        return _ctx[device]
