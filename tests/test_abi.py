"""The C ABI library builds for sm_103a, loads, and exports every symbol include/*.h declares (no GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"^SIMR_API\s+[\w\s\*]+?\b(simr_\w+)\s*\(", text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2402_12111_gb300 import build

    try:
        return build.build()
    except RuntimeError as e:
        if "nvcc not found" in str(e):
            pytest.skip("no CUDA toolkit")
        raise


def test_header_declares_entry_points():
    names = _declared()
    for required in ("simr_price", "simr_greeks_fd", "simr_create", "simr_destroy", "simr_last_error", "simr_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in sorted(_declared()):
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (simr_\w+)", out))
    assert _declared() <= exported
    # nothing but the declared C entry points leaks out of the library
    assert exported == _declared()


def test_binding_loads_without_gpu(libpath):
    import paper_2402_12111_gb300 as simr

    L = simr.load(build_if_missing=False)
    assert L.simr_version() >= 100
    assert L.simr_last_error() == b""


def test_no_context_without_gpu(libpath):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2402_12111_gb300 as simr
    from paper_2402_12111_gb300 import _simr

    with pytest.raises(simr.SimrError):
        _simr.context(0)


def test_product_path_does_not_import_oracle():
    # The package must not reach the CPU oracle (no fallback); only tests, smoke and bench may.
    for path in glob.glob(os.path.join(ROOT, "paper_2402_12111_gb300", "**", "*.py"), recursive=True):
        src = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), path
    for path in glob.glob(os.path.join(ROOT, "paper_2402_12111_gb300", "csrc", "*")):
        assert "simr_oracle" not in open(path).read(), path


def test_bench_source_hash_ignores_comments_only():
    # the profiled-traffic lookup in bench.py keys on the path kernel's code: a
    # comment edit keeps the key, a code edit changes it
    import sys

    sys.path.insert(0, ROOT)
    import bench

    code = 'int f(int a) { return a + 1; }  // one\n/* two\n three */ const char* s = "x // y /* z";\n'
    same = 'int f(int a) { return a + 1; }\n// a different comment\nconst char* s = "x // y /* z";\n'
    other = 'int f(int a) { return a + 2; }\nconst char* s = "x // y /* z";\n'
    assert bench._code_only(code) == bench._code_only(same)
    assert bench._code_only(code) != bench._code_only(other)
    assert '"x // y /* z"' in bench._code_only(code)


def test_fault_injection_hook_arguments(libpath):
    # arming and disarming needs no GPU; bad arguments are refused
    lib = ctypes.CDLL(libpath)
    lib.simr_inject_fault.argtypes = [ctypes.c_int, ctypes.c_int]
    assert lib.simr_inject_fault(1, 3) == 0
    assert lib.simr_inject_fault(0, 0) == 0
    assert lib.simr_inject_fault(2, 1) == 0
    assert lib.simr_inject_fault(0, 0) == 0
    assert lib.simr_inject_fault(3, 1) == 0
    assert lib.simr_inject_fault(0, 0) == 0
    assert lib.simr_inject_fault(4, 1) != 0
    assert lib.simr_inject_fault(1, 0) != 0


def test_host_validation_of_the_problem_statement(libpath):
    # The argument rules are checked on the host before any CUDA call; simr_price_noalloc
    # needs no context, so they can be exercised here without a GPU.
    import numpy as np

    from paper_2402_12111_gb300 import _simr as S

    L = S.load(build_if_missing=False)
    good = dict(S0=100.0, r=0.05, T=1.0, v0=0.04, kappa=1.5, theta=0.04, sigma=0.3, rho=-0.7)
    K = np.array([100.0] * 33)
    out = np.zeros(33)
    kp, op = K.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p)

    def call(model=good, strikes=kp, n=1, steps=64, paths=1024, price=op):
        rc = L.simr_price_noalloc(ctypes.byref(S.as_heston(model)), strikes, n, 0, steps, paths, 1, 0, price, None,
                                  None)
        return rc, L.simr_last_error().decode()

    bad_models = {"S0": 0.0, "T": -1.0, "v0": -1e-3, "theta": -1e-3, "kappa": 0.0, "sigma": 0.0, "rho": 1.5}
    for field, value in bad_models.items():
        rc, msg = call(model=dict(good, **{field: value}))
        assert rc == S.SIMR_EINVAL and msg.startswith(field), (field, msg)
    rc, msg = call(model=dict(good, r=float("nan")))
    assert rc == S.SIMR_EINVAL and "non-finite" in msg
    assert call(steps=0)[0] == S.SIMR_EINVAL and "steps" in call(steps=0)[1]
    assert call(paths=0)[0] == S.SIMR_EINVAL and "paths" in call(paths=0)[1]
    assert call(strikes=None)[1] == "strikes is NULL"
    assert "n_strikes" in call(n=0)[1] and "n_strikes" in call(n=33)[1]
    assert call(price=None)[1] == "price is NULL"
    # the edge cases the rules admit: v0 = theta = 0, rho = +-1, r < 0 -- they pass every
    # model check and stop only at the rule that this entry point takes device memory
    for edge in (dict(v0=0.0, theta=0.0), dict(rho=1.0), dict(rho=-1.0), dict(r=-0.02)):
        rc, msg = call(model=dict(good, **edge))
        assert rc == S.SIMR_EINVAL and "device pointers only" in msg, (edge, msg)
    # a NULL context is refused by every context call
    rc = L.simr_price(None, ctypes.byref(S.as_heston(good)), kp, 1, 0, 64, 1024, 1, 0, op, None, None)
    assert rc == S.SIMR_EINVAL and L.simr_last_error() == b"context is NULL"


def test_the_c_abi_from_plain_c(libpath, tmp_path):
    # include/simr.h compiles as strict C99 and a C program links against libsimr.so;
    # without a GPU the program reports the library's message for the failed context
    src = os.path.join(ROOT, "tests", "c", "price_from_c.c")
    exe = str(tmp_path / "price_from_c")
    libdir = os.path.dirname(libpath)
    cc = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", f"-I{ROOT}/include", src, "-o",
                         exe, f"-L{libdir}", "-lsimr", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    if run.returncode == 2:
        assert run.stdout.startswith("no context: -3 "), run.stdout
    else:
        assert run.returncode == 0, run.stdout + run.stderr
        prices = [float(line.split("price=")[1].split()[0]) for line in run.stdout.splitlines()]
        assert len(prices) == 3 and all(p > 0 for p in prices) and prices[0] > prices[1] > prices[2]
