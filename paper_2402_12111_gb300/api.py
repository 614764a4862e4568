"""Tensor-level entry points: one C-ABI call each, no arithmetic of the method here."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _simr as S


def _as_f64(x, device=None) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        t = x.to(dtype=torch.float64)
        if device is not None:
            t = t.to(device)
        return t.contiguous()
    t = torch.as_tensor(np.ascontiguousarray(np.atleast_1d(np.asarray(x, dtype=np.float64))))
    return t if device is None else t.to(device)


def _device_index(t: torch.Tensor, device) -> int:
    if t.is_cuda:
        return t.device.index if t.device.index is not None else torch.cuda.current_device()
    if device is not None:
        d = torch.device(device)
        if d.type == "cuda":
            return d.index if d.index is not None else torch.cuda.current_device()
    return 0


def _stream(t: torch.Tensor, stream):
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    if t.is_cuda:
        return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    return ctypes.c_void_p(None)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(None)


def price(model, strikes, is_put: bool = False, steps: int = 64, paths: int = 65536, seed: int = 1,
          option_index: int = 0, stderr: bool = True, device=None, stream=None):
    """simr_price: (price[n_K], stderr[n_K] or None), FP64, on the strikes' device."""
    K = _as_f64(strikes)
    p = torch.empty(K.numel(), dtype=torch.float64, device=K.device)
    se = torch.empty_like(p) if stderr else None
    L = S.load()
    ctx = S.context(_device_index(K, device))
    S.check(L.simr_price(ctx, ctypes.byref(S.as_heston(model)), _ptr(K), K.numel(), int(bool(is_put)), int(steps),
                         int(paths), int(seed), int(option_index), _ptr(p), _ptr(se), _stream(K, stream)))
    return p, se


def greeks_fd(model, strikes, is_put: bool = False, steps: int = 64, paths: int = 65536, seed: int = 1,
              greeks=("delta", "gamma", "vega"), rel_bump: float = 1e-4, option_index: int = 0, device=None,
              stream=None):
    """simr_greeks_fd: (price[n_K], greeks[n_K, n_greeks]) with columns in bit order of the mask."""
    K = _as_f64(strikes)
    mask = S.greek_mask(greeks)
    ng = bin(mask & S.G_ALL).count("1")
    p = torch.empty(K.numel(), dtype=torch.float64, device=K.device)
    g = torch.empty(K.numel(), max(ng, 1), dtype=torch.float64, device=K.device)
    L = S.load()
    ctx = S.context(_device_index(K, device))
    S.check(L.simr_greeks_fd(ctx, ctypes.byref(S.as_heston(model)), _ptr(K), K.numel(), int(bool(is_put)),
                             int(steps), int(paths), int(seed), int(option_index), float(rel_bump), int(mask), _ptr(p),
                             _ptr(g), _stream(K, stream)))
    return p, g


ADJOINT_COLUMNS = ("S0", "v0", "kappa", "theta", "sigma", "rho", "r")


def greeks_adjoint(model, strikes, is_put: bool = False, steps: int = 64, paths: int = 65536, seed: int = 1,
                   ckpt_every: int = 0, option_index: int = 0, stderr: bool = True, device=None, stream=None):
    """simr_greeks_adjoint: (price[n_K], stderr[n_K] or None, grad[n_K, 7]) with grad columns
    d/d(S0, v0, kappa, theta, sigma, rho, r), from one pathwise reverse-mode launch."""
    K = _as_f64(strikes)
    p = torch.empty(K.numel(), dtype=torch.float64, device=K.device)
    se = torch.empty_like(p) if stderr else None
    g = torch.empty(K.numel(), 7, dtype=torch.float64, device=K.device)
    L = S.load()
    ctx = S.context(_device_index(K, device))
    S.check(L.simr_greeks_adjoint(ctx, ctypes.byref(S.as_heston(model)), _ptr(K), K.numel(), int(bool(is_put)),
                                  int(steps), int(paths), int(seed), int(option_index), int(ckpt_every), _ptr(p),
                                  _ptr(se), _ptr(g), _stream(K, stream)))
    return p, se, g


def adjoint_interval(n_strikes: int, steps: int, device: int = 0) -> int:
    """simr_adjoint_interval: the checkpoint interval greeks_adjoint takes for ckpt_every=0."""
    k = ctypes.c_uint32()
    S.check(S.load().simr_adjoint_interval(S.context(device), int(n_strikes), int(steps), ctypes.byref(k)))
    return int(k.value)


def inject_fault(what: str, after: int = 1) -> None:
    """simr_inject_fault: the after-th next scratch request ("alloc") or kernel launch
    ("launch") of this process fails on the host; "barrier": the after-th next
    Longstaff-Schwartz sweep's first grid barrier waits until its bounded wait runs
    out (SIMR_ETIMEOUT, the context stays usable); "off" disarms."""
    kinds = {"off": 0, "alloc": S.FAULT_ALLOC, "launch": S.FAULT_LAUNCH, "barrier": S.FAULT_BARRIER}
    S.check(S.load().simr_inject_fault(kinds[what], int(after)))


class HestonAdjoint(torch.autograd.Function):
    """Monte Carlo price as a differentiable function of the model parameters.

    forward(params, strikes, T, is_put, steps, paths, seed, ckpt_every) with
    params = (S0, v0, kappa, theta, sigma, rho, r) returns the price per strike;
    the same launch computes the pathwise adjoint Jacobian d price / d params,
    so backward is grad_out @ J (no second pass over the paths).
    """

    @staticmethod
    def forward(ctx, params, strikes, T, is_put=False, steps=64, paths=65536, seed=1, ckpt_every=0):
        vals = params.detach().double().cpu().tolist()
        model = dict(zip(ADJOINT_COLUMNS, vals))
        model["T"] = float(T)
        price, _, jac = greeks_adjoint(model, strikes, is_put, steps, paths, seed, ckpt_every, stderr=False)
        ctx.save_for_backward(jac)
        ctx.params_meta = (params.dtype, params.device)
        return price

    @staticmethod
    def backward(ctx, grad_out):
        (jac,) = ctx.saved_tensors
        g = grad_out.to(jac.dtype).to(jac.device) @ jac
        dtype, device = ctx.params_meta
        return g.to(device=device, dtype=dtype), None, None, None, None, None, None, None


def heston_price(params, strikes, T, is_put=False, steps=64, paths=65536, seed=1, ckpt_every=0):
    """Differentiable price per strike (see HestonAdjoint)."""
    return HestonAdjoint.apply(params, strikes, T, is_put, steps, paths, seed, ckpt_every)


def batch(options, seed: int = 1, adjoint: bool = False, graph: bool = False, autotune: bool = True,
          device=None, stream=None, out_device=None, variant=None):
    """simr_batch_submit over a book: options is a sequence of dicts with keys
    model (dict), K, is_put, steps, paths.  Returns (price[n], stderr[n], grad[n, 7] or None)
    in the book's order, on `out_device` (default: the CUDA device).  `variant` (0-7, or
    None for the tuned one) forces the kernel shape of SIMR_BATCH_VARIANT."""
    n = len(options)
    arr = (S.Option * n)()
    for i, o in enumerate(options):
        arr[i].m = S.as_heston(o["model"])
        arr[i].K = float(o["K"])
        arr[i].is_put = int(bool(o["is_put"]))
        arr[i].steps = int(o["steps"])
        arr[i].paths = int(o["paths"])
    dev_index = torch.cuda.current_device() if device is None else torch.device(device).index or 0
    odev = torch.device("cuda", dev_index) if out_device is None else torch.device(out_device)
    p = torch.empty(n, dtype=torch.float64, device=odev)
    se = torch.empty_like(p)
    g = torch.empty(n, 7, dtype=torch.float64, device=odev) if adjoint else None
    flags = (S.BATCH_ADJOINT if adjoint else 0) | (S.BATCH_GRAPH if graph else 0) | \
        (0 if autotune else S.BATCH_NO_AUTOTUNE) | (0 if variant is None else S.batch_variant_flag(variant))
    L = S.load()
    ctx = S.context(dev_index)
    st = _stream(p, stream) if p.is_cuda else ctypes.c_void_p(None)
    S.check(L.simr_batch_submit(ctx, arr, n, int(seed), flags, _ptr(p), _ptr(se), _ptr(g), st))
    return p, se, g


def lsm_price(model, K: float, is_put: bool = True, steps: int = 64, exercise_every: int = 1, paths: int = 65536,
              seed: int = 1, option_index: int = 0, with_beta: bool = False, with_stop: bool = False,
              device="cuda", stream=None):
    """simr_lsm_price: Longstaff-Schwartz Bermudan price on the paths of simr_price.
    Returns (price, stderr, beta[n_ex, 6] or None, stop[paths] int32 or None), on `device`."""
    dev = torch.device(device)
    n_ex = int(steps) // max(int(exercise_every), 1)
    p = torch.empty(1, dtype=torch.float64, device=dev)
    se = torch.empty_like(p)
    b = torch.empty(max(n_ex, 1), 6, dtype=torch.float64, device=dev) if with_beta else None
    st = torch.empty(int(paths), dtype=torch.int32, device=dev) if with_stop else None
    L = S.load()
    ctx = S.context(_device_index(p, device))
    S.check(L.simr_lsm_price(ctx, ctypes.byref(S.as_heston(model)), float(K), int(bool(is_put)), int(steps),
                             int(exercise_every), int(paths), int(seed), int(option_index), _ptr(p), _ptr(se), _ptr(b),
                             _ptr(st), _stream(p, stream)))
    return p, se, b, st


def paths_adjoint(model, steps: int, path_begin: int, n_paths: int, seed: int = 1, ckpt_every: int = 0,
                  option_index: int = 0, device="cuda", stream=None):
    """simr_paths_adjoint: (x_T[n], grad[n, 5]) FP32, grad = d x_T / d(v0, kappa, theta, sigma, rho)."""
    dev = torch.device(device)
    x = torch.empty(int(n_paths), dtype=torch.float32, device=dev)
    g = torch.empty(int(n_paths), 5, dtype=torch.float32, device=dev)
    L = S.load()
    ctx = S.context(_device_index(x, device))
    S.check(L.simr_paths_adjoint(ctx, ctypes.byref(S.as_heston(model)), int(steps), int(path_begin), int(n_paths),
                                 int(seed), int(option_index), int(ckpt_every), _ptr(x), _ptr(g), _stream(x, stream)))
    return x, g


def paths_terminal(model, steps: int, path_begin: int, n_paths: int, seed: int = 1, option_index: int = 0,
                   device="cuda", with_variance: bool = True, stream=None):
    """simr_paths_terminal: (x_T, v_T) FP32 per path, x_T = ln(S_T/S0)."""
    dev = torch.device(device)
    x = torch.empty(int(n_paths), dtype=torch.float32, device=dev)
    v = torch.empty_like(x) if with_variance else None
    L = S.load()
    ctx = S.context(_device_index(x, device))
    S.check(L.simr_paths_terminal(ctx, ctypes.byref(S.as_heston(model)), int(steps), int(path_begin), int(n_paths),
                                  int(seed), int(option_index), _ptr(x), _ptr(v), _stream(x, stream)))
    return x, v


def path_sums(model, strikes, is_put: bool, steps: int, path_begin: int, path_count: int, seed: int = 1,
              greeks=(), rel_bump: float = 1e-4, option_index: int = 0, device=None, stream=None):
    """simr_path_sums: raw FP64 sums [n_K, 2 + n_greeks] over a path range (for sharded runs)."""
    K = _as_f64(strikes)
    mask = S.greek_mask(greeks)
    n_acc = 2 + bin(mask & S.G_ALL).count("1")
    out = torch.empty(K.numel(), n_acc, dtype=torch.float64, device=K.device)
    L = S.load()
    ctx = S.context(_device_index(K, device))
    S.check(L.simr_path_sums(ctx, ctypes.byref(S.as_heston(model)), _ptr(K), K.numel(), int(bool(is_put)),
                             int(steps), int(path_begin), int(path_count), int(seed), int(option_index),
                             float(rel_bump), int(mask), _ptr(out), _stream(K, stream)))
    return out


def finalize_sums(model, strikes, is_put: bool, steps: int, paths: int, sums: torch.Tensor, greeks=(),
                  rel_bump: float = 1e-4, device=None, stream=None):
    """simr_finalize_sums: (price, stderr, greeks) from combined sums over `paths` paths."""
    K = _as_f64(strikes, device=sums.device)
    mask = S.greek_mask(greeks)
    ng = bin(mask & S.G_ALL).count("1")
    sums = sums.to(torch.float64).contiguous()
    p = torch.empty(K.numel(), dtype=torch.float64, device=sums.device)
    se = torch.empty_like(p)
    g = torch.empty(K.numel(), max(ng, 1), dtype=torch.float64, device=sums.device) if ng else None
    L = S.load()
    ctx = S.context(_device_index(sums, device))
    S.check(L.simr_finalize_sums(ctx, ctypes.byref(S.as_heston(model)), _ptr(K), K.numel(), int(bool(is_put)),
                                 int(steps), int(paths), float(rel_bump), int(mask), _ptr(sums), _ptr(p), _ptr(se),
                                 _ptr(g), _stream(sums, stream)))
    return p, se, g


def basket_price(models, corr, weights, strikes, is_put: bool = False, steps: int = 64, paths: int = 65536,
                 seed: int = 1, device=None, stream=None):
    """simr_basket_price: (price[n_K], stderr[n_K]) of the basket option on
    sum_k w_k S_T,k of correlated assets (`corr`: correlation of the spot drivers)."""
    n = len(models)
    arr = (S.Heston * n)(*[S.as_heston(m) for m in models])
    C = np.ascontiguousarray(np.asarray(corr, dtype=np.float64).reshape(n, n))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(n))
    K = _as_f64(strikes)
    p = torch.empty(K.numel(), dtype=torch.float64, device=K.device)
    se = torch.empty_like(p)
    L = S.load()
    ctx = S.context(_device_index(K, device))
    S.check(L.simr_basket_price(ctx, arr, n, C.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p),
                                _ptr(K), K.numel(), int(bool(is_put)), int(steps), int(paths), int(seed), _ptr(p),
                                _ptr(se), _stream(K, stream)))
    return p, se


def set_scheme(name: str, device: int = 0):
    """simr_set_scheme: "qe" (Andersen's QE) or "qem" (QE with the martingale correction)
    for the device context's later path simulations."""
    L = S.load()
    S.check(L.simr_set_scheme(S.context(device), S.SCHEMES[name]))


class scheme:
    """Context manager: the simulations inside use the given scheme on `device`."""

    def __init__(self, name: str, device: int = 0):
        self.name, self.device = name, device

    def __enter__(self):
        set_scheme(self.name, self.device)
        return self

    def __exit__(self, *exc):
        set_scheme("qe", self.device)
        return False


def sync(device: int = 0, stream=None):
    """simr_sync on a device's current (or given) stream."""
    L = S.load()
    st = stream if stream is not None else torch.cuda.current_stream(device)
    S.check(L.simr_sync(S.context(device), ctypes.c_void_p(st.cuda_stream)))


def philox_words(seed: int, option_index: int, path_begin: int, n_paths: int, pair_begin: int, n_pairs: int,
                 device="cuda", stream=None):
    """simr_philox_words: int32 tensor [n_paths, n_pairs, 4] holding the uint32 words the path
    kernels draw for those counters (view as uint32 on the host: ``.cpu().numpy().view(np.uint32)``)."""
    dev = torch.device(device)
    w = torch.empty((int(n_paths), int(n_pairs), 4), dtype=torch.int32, device=dev)
    L = S.load()
    ctx = S.context(_device_index(w, device))
    S.check(L.simr_philox_words(ctx, int(seed), int(option_index), int(path_begin), int(n_paths), int(pair_begin),
                                int(n_pairs), _ptr(w), _stream(w, stream)))
    return w


def normals(words: torch.Tensor, paired: bool = True, stream=None):
    """simr_normals: (z, z_paired or None), FP32, the path kernels' standard normals of int32/uint32
    words on a CUDA device (one at a time, and two at a time in the packed form)."""
    w = words.contiguous().view(-1)
    if w.dtype not in (torch.int32,):
        w = w.to(torch.int32)
    z = torch.empty(w.numel(), dtype=torch.float32, device=w.device)
    zp = torch.empty_like(z) if paired else None
    L = S.load()
    ctx = S.context(_device_index(w, None))
    S.check(L.simr_normals(ctx, _ptr(w), w.numel(), _ptr(z), _ptr(zp), _stream(w, stream)))
    return z, zp


UNIT_RATES = ("fp32_fma_tflops", "fp32_fma2_tflops", "mufu_rsqrt_tops", "mul_wide_tops", "fp64_fma_tflops", "ms")


def unit_rates(device: int = 0, stream=None) -> dict:
    """simr_unit_rates: the measured throughput of the units the path kernels use, keyed as UNIT_RATES."""
    out = (ctypes.c_double * 6)()
    L = S.load()
    st = stream if stream is not None else torch.cuda.current_stream(device)
    S.check(L.simr_unit_rates(S.context(device), out, ctypes.c_void_p(st.cuda_stream)))
    return dict(zip(UNIT_RATES, list(out)))
