"""The Python binding against the C header, and its marshalling (no GPU).

* Every declaration in include/simr.h has the same parameter list, type by
  type, as the ctypes argtypes the binding gives it.
* The tensor-level functions pass the right sizes, flags and pointers and
  return what the library writes: each is called with host tensors against a
  stand-in for the library that records its arguments and fills the outputs.
* HestonAdjoint's backward is grad_out @ J of the Jacobian the forward launch
  returned.
"""
import ctypes
import glob
import os
import re

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_TYPES = {"double": ctypes.c_double, "int": ctypes.c_int, "int32_t": ctypes.c_int32, "uint32_t": ctypes.c_uint32,
           "uint64_t": ctypes.c_uint64}


def _declarations():
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", " ", open(h).read(), flags=re.S)
        for m in re.finditer(r"SIMR_API\s+([\w\s\*]+?)\b(simr_\w+)\s*\(([^)]*)\)\s*;", text):
            params = [p.strip() for p in m.group(3).split(",") if p.strip() and p.strip() != "void"]
            out[m.group(2)] = params
    return out


def _ctype_of(param: str):
    """ctypes type a C parameter declaration maps to: pointers by pointee, scalars by name."""
    p = re.sub(r"\bconst\b", " ", param)
    if "*" in p:
        base = p.split("*")[0].split()[-1]
        return ("ptr", base, p.count("*"))
    toks = p.split()
    return ("val", toks[-2] if len(toks) > 1 else toks[0])


def test_binding_argtypes_match_the_header():
    from paper_2402_12111_gb300 import _simr as S, build

    try:
        build.build()
    except RuntimeError as e:
        if "nvcc not found" in str(e):
            pytest.skip("no CUDA toolkit")
        raise
    L = S.load(build_if_missing=False)
    decls = _declarations()
    assert {"simr_price", "simr_greeks_fd", "simr_greeks_adjoint", "simr_batch_submit", "simr_sync"} <= set(decls)
    for name, params in decls.items():
        argtypes = getattr(L, name).argtypes
        if argtypes is None:
            assert not params, name  # functions without parameters keep ctypes' default
            continue
        assert len(argtypes) == len(params), (name, params, argtypes)
        for decl, at in zip(params, argtypes):
            kind = _ctype_of(decl)
            if kind[0] == "val":
                assert at is C_TYPES[kind[1]], (name, decl, at)
            elif kind[1] == "simr_heston":
                assert at is ctypes.POINTER(S.Heston), (name, decl, at)
            elif kind[1] == "simr_option":
                assert at is ctypes.POINTER(S.Option), (name, decl, at)
            elif kind[1] == "uint32_t" and name == "simr_adjoint_interval":
                assert at is ctypes.POINTER(ctypes.c_uint32), (name, decl, at)
            else:  # data pointers, the context, streams and out-handles travel as void pointers
                assert at is ctypes.c_void_p or at is ctypes.POINTER(ctypes.c_void_p), (name, decl, at)


class FakeLib:
    """Records each call; `fill[name](args)` may write outputs through the pointers."""

    def __init__(self, fill=None, rc=0):
        self.calls, self.fill, self.rc = [], fill or {}, rc

    def simr_last_error(self):
        return b"planted failure"

    def __getattr__(self, name):
        def call(*args):
            self.calls.append((name, args))
            if name in self.fill:
                self.fill[name](args)
            return self.rc

        return call


def _write(ptr, values):
    """Write FP64 values where the call's output pointer points (nothing for a NULL output)."""
    if ptr.value is None:
        return
    arr = np.ascontiguousarray(values, dtype=np.float64)
    ctypes.memmove(ptr.value, arr.ctypes.data, arr.nbytes)


@pytest.fixture
def fake(monkeypatch):
    from paper_2402_12111_gb300 import _simr as S

    lib = FakeLib()
    monkeypatch.setattr(S, "load", lambda build_if_missing=True: lib)
    monkeypatch.setattr(S, "context", lambda device=0: ctypes.c_void_p(0x1234))
    return lib


MODEL = dict(S0=100.0, r=0.05, T=1.0, v0=0.04, kappa=1.5, theta=0.04, sigma=0.3, rho=-0.7)


def test_price_marshals_sizes_flags_and_outputs(fake):
    from paper_2402_12111_gb300 import api

    # outputs: price = 1, 2, ... and stderr = 0.1, 0.2, ... over the call's n_strikes
    fake.fill["simr_price"] = lambda a: (_write(a[9], np.arange(1, a[3] + 1)),
                                         _write(a[10], np.arange(1, a[3] + 1) / 10))
    p, se = api.price(MODEL, [90.0, 100.0, 110.0], True, 252, 1 << 20, 7, option_index=3)
    name, a = fake.calls[-1]
    assert name == "simr_price"
    assert a[0].value == 0x1234 and a[1]._obj.S0 == 100.0 and a[1]._obj.rho == -0.7
    assert a[3:9] == (3, 1, 252, 1 << 20, 7, 3)
    assert a[11].value is None  # host tensors: no stream
    assert p.tolist() == [1.0, 2.0, 3.0] and se.tolist() == [0.1, 0.2, 0.3]
    p1, se1 = api.price(MODEL, [100.0], stderr=False)
    assert fake.calls[-1][1][10].value is None and se1 is None and p1.tolist() == [1.0]  # no stderr: NULL


def test_greeks_fd_mask_and_output_shape(fake):
    from paper_2402_12111_gb300 import api

    _, g = api.greeks_fd(MODEL, [90.0, 100.0], greeks=("rho", "delta", "vega"), rel_bump=1e-3)
    name, a = fake.calls[-1]
    assert name == "simr_greeks_fd" and a[9] == 1e-3 and a[10] == 1 | 4 | 16
    assert tuple(g.shape) == (2, 3)


def test_batch_flags_and_option_records(fake):
    from paper_2402_12111_gb300 import api

    book = [dict(model=MODEL, K=95.0, is_put=True, steps=64, paths=4096),
            dict(model=dict(MODEL, S0=80.0), K=85.0, is_put=False, steps=128, paths=8192)]
    p, se, g = api.batch(book, seed=5, adjoint=True, graph=True, autotune=False, device="cuda:0", out_device="cpu",
                         variant=6)
    name, a = fake.calls[-1]
    assert name == "simr_batch_submit" and a[2] == 2 and a[3] == 5
    assert a[4] == 1 | 2 | 4 | ((6 + 1) << 8)
    opts = a[1]
    assert opts[0].K == 95.0 and opts[0].is_put == 1 and opts[0].steps == 64 and opts[0].paths == 4096
    assert opts[1].m.S0 == 80.0 and opts[1].is_put == 0 and opts[1].steps == 128
    assert tuple(g.shape) == (2, 7) and p.device.type == "cpu"
    api.batch(book, device="cuda:0", out_device="cpu")
    assert fake.calls[-1][1][4] == 0 and fake.calls[-1][1][7].value is None  # prices only: no grad buffer


def test_path_sums_accumulator_count(fake):
    from paper_2402_12111_gb300 import api

    out = api.path_sums(MODEL, [100.0, 110.0], False, 16, 1000, 96, greeks=("delta", "gamma"))
    name, a = fake.calls[-1]
    assert name == "simr_path_sums" and a[6:9] == (1000, 96, 1) and a[11] == 3
    assert tuple(out.shape) == (2, 4)


def test_a_failed_call_raises_with_the_library_message(monkeypatch):
    from paper_2402_12111_gb300 import _simr as S, api

    lib = FakeLib(rc=S.SIMR_EINVAL)
    monkeypatch.setattr(S, "load", lambda build_if_missing=True: lib)
    monkeypatch.setattr(S, "context", lambda device=0: ctypes.c_void_p(0x1234))
    with pytest.raises(S.SimrError) as e:
        api.price(MODEL, [100.0])
    assert e.value.code == S.SIMR_EINVAL and "planted failure" in str(e.value)


def test_heston_adjoint_backward_is_grad_out_times_the_jacobian(fake):
    from paper_2402_12111_gb300 import api

    J = np.arange(21, dtype=np.float64).reshape(3, 7) / 10.0
    fake.fill["simr_greeks_adjoint"] = lambda a: (_write(a[10], [5.0, 6.0, 7.0]), _write(a[12], J))
    params = torch.tensor([100.0, 0.04, 1.5, 0.04, 0.3, -0.7, 0.05], dtype=torch.float64, requires_grad=True)
    price = api.heston_price(params, torch.tensor([90.0, 100.0, 110.0]), 1.0, False, 64, 4096, 3, 0)
    assert price.tolist() == [5.0, 6.0, 7.0]
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    (price * w).sum().backward()
    np.testing.assert_allclose(params.grad.numpy(), w.numpy() @ J, rtol=0, atol=1e-15)
    name, a = fake.calls[-1]
    # the model the forward call passed: (S0, v0, kappa, theta, sigma, rho, r) from params, T given
    m = a[1]._obj
    assert (m.S0, m.v0, m.kappa, m.theta, m.sigma, m.rho, m.r, m.T) == (100.0, 0.04, 1.5, 0.04, 0.3, -0.7, 0.05, 1.0)
    assert a[11].value is None  # the forward pass asks for no standard error
