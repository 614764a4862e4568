"""FP64 CPU oracle for Heston QE Monte Carlo pricing -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline and
reference legs may import this package.  The product path (``include/simr.h``,
the CUDA library and its Python binding) never imports it, and the two share no
code: this package compiles its own plain C file, ``simr_oracle.c``, with gcc.

Functions follow the SIMR stages named in the paper (Sec. 4-5: VariancePathQE,
LogPricePathQE, AssetPathExponential, and the reduction over paths of Sec. 6)
with the formulas of Andersen's QE scheme (2008) for the Heston (1993) model;
``simr_oracle.c`` states each formula beside its code.  ``analytic.py`` holds
the closed forms and semi-analytic prices that pin the oracle in the tests.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "simr_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Greek selection bits (same meaning as the oracle's C enum).
G_DELTA, G_GAMMA, G_VEGA, G_THETA, G_RHO = 1, 2, 4, 8, 16
G_KAPPA, G_LRVAR, G_VOLVOL, G_CORR = 32, 64, 128, 256


class Heston(ctypes.Structure):
    """Model and market inputs: spot, rate, maturity and the Heston parameters."""

    _fields_ = [(n, ctypes.c_double) for n in ("S0", "r", "T", "v0", "kappa", "theta", "sigma", "rho")]


def build(force: bool = False) -> str:
    """Compile simr_oracle.c into _build/liboracle.so (plain IEEE FP64, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", "-std=c11"]
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            H = ctypes.POINTER(Heston)
            dp = ctypes.POINTER(ctypes.c_double)
            u32, u64, i64, c_int = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int
            L.oracle_philox4x32_10.argtypes = [ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)]
            L.oracle_uniform.argtypes = [u32]
            L.oracle_uniform.restype = ctypes.c_double
            L.oracle_norminv.argtypes = [ctypes.c_double]
            L.oracle_norminv.restype = ctypes.c_double
            L.oracle_norminv_array.argtypes = [dp, dp, i64]
            L.oracle_step_uniforms.argtypes = [u64, u32, u64, u32, dp, dp]
            L.oracle_qe_constants.argtypes = [H, u32, dp]
            L.oracle_qe_step.argtypes = [H, u32, ctypes.c_double, ctypes.c_double, ctypes.POINTER(c_int)]
            L.oracle_qe_step.restype = ctypes.c_double
            L.oracle_qe_step_array.argtypes = [H, u32, ctypes.c_double, dp, dp, i64]
            L.oracle_terminal.argtypes = [H, u32, u64, u32, u64, i64, dp, dp, dp]
            L.oracle_terminal_diag.argtypes = [H, u32, u64, u32, u64, i64, dp, dp, dp, dp]
            L.oracle_price.argtypes = [H, dp, c_int, c_int, u32, i64, u64, u32, dp, dp]
            L.oracle_greeks_fd.argtypes = [H, dp, c_int, c_int, u32, i64, u64, u32, ctypes.c_double, u32, dp, dp]
            L.oracle_path_grad_reverse.argtypes = [H, u32, u64, u32, u64, i64, dp, dp]
            L.oracle_path_grad_forward.argtypes = [H, u32, u64, u32, u64, i64, dp, dp]
            L.oracle_adjoint.argtypes = [H, dp, c_int, c_int, u32, i64, u64, u32, dp, dp]
            L.oracle_path_grad_flip.argtypes = [H, u32, u64, u32, u64, i64, ctypes.c_double, dp, dp,
                                                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                                ctypes.POINTER(ctypes.c_int32)]
            L.oracle_terminal_forced.argtypes = [H, u32, u64, u32, u64, ctypes.c_int64, c_int, c_int]
            L.oracle_terminal_forced.restype = ctypes.c_double
            L.oracle_states.argtypes = [H, u32, u32, u64, u32, u64, i64, dp, dp]
            L.oracle_basket_terminal.argtypes = [H, c_int, dp, u32, u64, u64, i64, dp, dp]
            L.oracle_set_scheme.argtypes = [c_int]
            L.oracle_set_scheme.restype = None
            L.oracle_step_exp_mean.argtypes = [H, u32, ctypes.c_double]
            L.oracle_step_exp_mean.restype = ctypes.c_double
            L.oracle_max_threads.restype = c_int
            L.oracle_set_threads.argtypes = [c_int]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _model(model) -> Heston:
    if isinstance(model, Heston):
        return model
    return Heston(**{k: float(model[k]) for k in ("S0", "r", "T", "v0", "kappa", "theta", "sigma", "rho")})


SCHEMES = {"qe": 0, "qem": 1}


class scheme:
    """Context manager selecting the log-spot scheme of every oracle call inside:
    "qe" (Andersen's QE) or "qem" (QE with Andersen's martingale correction)."""

    def __init__(self, name: str):
        self.code = SCHEMES[name]

    def __enter__(self):
        lib().oracle_set_scheme(self.code)
        return self

    def __exit__(self, *exc):
        lib().oracle_set_scheme(0)
        return False


def step_exp_mean(model, steps: int, v: float) -> float:
    """E[exp(x(t+dt) - x(t) - r dt) | v(t) = v] of one step, exact over the uniform
    lattice (1 for a martingale scheme), under the current scheme."""
    return float(lib().oracle_step_exp_mean(ctypes.byref(_model(model)), int(steps), float(v)))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 128-bit counter (4 words) under a 64-bit key (2 words)."""
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform(w: int) -> float:
    return float(lib().oracle_uniform(int(w) & 0xFFFFFFFF))


def norminv(u) -> np.ndarray:
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).ravel())
    z = np.empty_like(u)
    lib().oracle_norminv_array(_dp(u), _dp(z), u.size)
    return z


def step_uniforms(seed: int, option_index: int, path: int, step: int):
    a, b = ctypes.c_double(), ctypes.c_double()
    lib().oracle_step_uniforms(seed, option_index, path, step, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def qe_constants(model, steps: int) -> dict:
    out = np.empty(9)
    lib().oracle_qe_constants(ctypes.byref(_model(model)), steps, _dp(out))
    return dict(zip(("dt", "E", "c1", "c2", "K0", "K1", "K2", "K3", "K4"), out.tolist()))


def qe_step(model, steps: int, v: float, u_v: float):
    """One QE variance step: returns (v_next, branch) with branch 0 quadratic,
    1 exponential (v' > 0), 2 exponential (v' = 0), 3 zero mean."""
    br = ctypes.c_int()
    vn = lib().oracle_qe_step(ctypes.byref(_model(model)), steps, float(v), float(u_v), ctypes.byref(br))
    return float(vn), int(br.value)


def qe_step_array(model, steps: int, v: float, u_v) -> np.ndarray:
    """The QE variance step from one v over an array of variance uniforms."""
    u = np.ascontiguousarray(np.asarray(u_v, dtype=np.float64).ravel())
    out = np.empty_like(u)
    lib().oracle_qe_step_array(ctypes.byref(_model(model)), steps, float(v), _dp(u), _dp(out), u.size)
    return out


def terminal(model, steps: int, seed: int, path_begin: int, n_paths: int, option_index: int = 0):
    """(x_T, v_T, margin) per path; x_T = ln(S_T/S0)."""
    x = np.empty(n_paths)
    v = np.empty(n_paths)
    mg = np.empty(n_paths)
    rc = lib().oracle_terminal(ctypes.byref(_model(model)), steps, seed, option_index, path_begin, n_paths,
                               _dp(x), _dp(v), _dp(mg))
    if rc != 0:
        raise ValueError(f"oracle_terminal failed ({rc})")
    return x, v, mg


def terminal_diag(model, steps: int, seed: int, path_begin: int, n_paths: int, option_index: int = 0):
    """(x_T, v_T, margin, cond) per path; cond = min |b + Z_V| / (1 + b) over quadratic steps."""
    x, v, mg, cd = (np.empty(n_paths) for _ in range(4))
    rc = lib().oracle_terminal_diag(ctypes.byref(_model(model)), steps, seed, option_index, path_begin, n_paths,
                                    _dp(x), _dp(v), _dp(mg), _dp(cd))
    if rc != 0:
        raise ValueError(f"oracle_terminal_diag failed ({rc})")
    return x, v, mg, cd


def states(model, steps: int, every: int, seed: int, path_begin: int, n_paths: int, option_index: int = 0):
    """(S, v) of shape [n_paths, steps // every]: spot and variance after steps
    every, 2 every, ..., steps (the exercise dates of a Bermudan option)."""
    if every < 1 or steps % every:
        raise ValueError("every must divide steps")
    n_ex = steps // every
    S = np.empty((n_paths, n_ex))
    v = np.empty((n_paths, n_ex))
    rc = lib().oracle_states(ctypes.byref(_model(model)), steps, every, seed, option_index, path_begin, n_paths,
                             _dp(S), _dp(v))
    if rc != 0:
        raise ValueError(f"oracle_states failed ({rc})")
    return S, v


def basket_terminal(models, corr, steps: int, seed: int, path_begin: int, n_paths: int, with_margin: bool = False):
    """x[n_paths, A] = ln(S_T/S0) of A assets whose log-spot normals have correlation
    `corr` (via numpy's Cholesky factor); asset k uses the counters of option index k.
    With with_margin, also each path's smallest branch-decision margin."""
    A = len(models)
    arr = (Heston * A)(*[_model(m) for m in models])
    Lc = np.ascontiguousarray(np.linalg.cholesky(np.asarray(corr, dtype=np.float64)))
    x = np.empty((n_paths, A))
    mg = np.empty(n_paths)
    rc = lib().oracle_basket_terminal(arr, A, _dp(Lc), steps, seed, path_begin, n_paths, _dp(x), _dp(mg))
    if rc != 0:
        raise ValueError(f"oracle_basket_terminal failed ({rc})")
    return (x, mg) if with_margin else x


def basket_price(models, corr, weights, strikes, is_put: bool, steps: int, paths: int, seed: int):
    """(price[n_K], stderr[n_K]) of the basket option on B_T = sum_k w_k S_T,k:
    e^{-rT} mean max(+-(B_T - K), 0), serial sums in path order."""
    x = basket_terminal(models, corr, steps, seed, 0, paths)
    S0 = np.array([float(m["S0"]) for m in models])
    B = (np.exp(x) * S0[None, :]) @ np.asarray(weights, dtype=np.float64)
    K = np.atleast_1d(np.asarray(strikes, dtype=np.float64))
    disc = math.exp(-float(models[0]["r"]) * float(models[0]["T"]))
    price, se = np.empty(K.size), np.empty(K.size)
    for j, k in enumerate(K):
        f = np.maximum(k - B, 0.0) if is_put else np.maximum(B - k, 0.0)
        s1, s2 = 0.0, 0.0
        for val in f:
            s1 += val
            s2 += val * val
        mean = s1 / paths
        price[j] = disc * mean
        var = (s2 / paths - mean * mean) / (paths - 1) if paths > 1 else 0.0
        se[j] = disc * math.sqrt(max(var, 0.0))
    return price, se


def price(model, strikes, is_put: bool, steps: int, paths: int, seed: int, option_index: int = 0):
    K = np.ascontiguousarray(np.atleast_1d(np.asarray(strikes, dtype=np.float64)))
    p = np.empty(K.size)
    se = np.empty(K.size)
    rc = lib().oracle_price(ctypes.byref(_model(model)), _dp(K), K.size, int(bool(is_put)), steps, paths, seed,
                            option_index, _dp(p), _dp(se))
    if rc != 0:
        raise ValueError(f"oracle_price failed ({rc})")
    return p, se


def greeks_fd(model, strikes, is_put: bool, steps: int, paths: int, seed: int, rel_bump: float,
              greek_mask: int, option_index: int = 0):
    """(price[n_K], greeks[n_K, n_greeks]); greeks in bit order of greek_mask."""
    K = np.ascontiguousarray(np.atleast_1d(np.asarray(strikes, dtype=np.float64)))
    n_g = bin(greek_mask & 0x1FF).count("1")
    p = np.empty(K.size)
    g = np.empty(K.size * n_g)
    rc = lib().oracle_greeks_fd(ctypes.byref(_model(model)), _dp(K), K.size, int(bool(is_put)), steps, paths,
                                seed, option_index, float(rel_bump), greek_mask, _dp(p), _dp(g))
    if rc < 0:
        raise ValueError(f"oracle_greeks_fd failed ({rc})")
    return p, g.reshape(K.size, n_g)


def path_grad(model, steps: int, seed: int, path_begin: int, n_paths: int, mode: str = "reverse",
              option_index: int = 0):
    """(x_T, dx_T/d(v0, kappa, theta, sigma, rho)) per path, by reverse or forward mode."""
    x = np.empty(n_paths)
    g = np.empty(n_paths * 5)
    fn = lib().oracle_path_grad_reverse if mode == "reverse" else lib().oracle_path_grad_forward
    rc = fn(ctypes.byref(_model(model)), steps, seed, option_index, path_begin, n_paths, _dp(x), _dp(g))
    if rc != 0:
        raise ValueError(f"oracle path gradient failed ({rc})")
    return x, g.reshape(n_paths, 5)


def path_grad_flip(model, steps: int, seed: int, path_begin: int, n_paths: int, margin_below: float,
                   option_index: int = 0):
    """Per path, (x_T, dx_T/d(v0, kappa, theta, sigma, rho), flip_step, flip_kind, flip_value) of the path with
    its branch decision closest to its threshold taken the other way, where that decision's margin
    is below margin_below (flip_step -1 and the plain reverse-mode result elsewhere): the pathwise
    derivative a lower-precision evaluation computes when it decides that step the other way.
    flip_kind 1: the QE branch (psi against psi_c; value 1 quadratic); 2: the exponential branch's atom
    (U_V against p; value 1 the logarithm's side).  Under QE-M an imposed branch is also the branch whose
    ln M the step's martingale correction takes."""
    x = np.empty(n_paths)
    g = np.empty(n_paths * 5)
    st = np.empty(n_paths, dtype=np.int64)
    kd = np.empty(n_paths, dtype=np.int32)
    fv = np.empty(n_paths, dtype=np.int32)
    rc = lib().oracle_path_grad_flip(ctypes.byref(_model(model)), steps, seed, option_index, path_begin, n_paths,
                                     float(margin_below), _dp(x), _dp(g),
                                     st.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                     kd.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     fv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc != 0:
        raise ValueError(f"oracle_path_grad_flip failed ({rc})")
    return x, g.reshape(n_paths, 5), st, kd, fv


def terminal_forced(model, steps: int, seed: int, path: int, f_step: int, f_kind: int, f_value: int,
                    option_index: int = 0) -> float:
    """x_T of one path with the decision of kind f_kind at step f_step imposed as f_value
    (f_step -1: none)."""
    return float(lib().oracle_terminal_forced(ctypes.byref(_model(model)), steps, seed, option_index, path,
                                              int(f_step), int(f_kind), int(f_value)))


def adjoint(model, strikes, is_put: bool, steps: int, paths: int, seed: int, option_index: int = 0):
    """(price[n_K], grad[n_K, 7]) with columns d/d{S0, v0, kappa, theta, sigma, rho, r}."""
    K = np.ascontiguousarray(np.atleast_1d(np.asarray(strikes, dtype=np.float64)))
    p = np.empty(K.size)
    g = np.empty(K.size * 7)
    rc = lib().oracle_adjoint(ctypes.byref(_model(model)), _dp(K), K.size, int(bool(is_put)), steps, paths, seed,
                              option_index, _dp(p), _dp(g))
    if rc != 0:
        raise ValueError(f"oracle_adjoint failed ({rc})")
    return p, g.reshape(K.size, 7)
