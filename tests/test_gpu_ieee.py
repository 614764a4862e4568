"""The build for error studies (SIMR_IEEE=1: correctly rounded division, square
roots and log2f in place of the special-function unit's approximations) against
the FP64 oracle, beside the default build, on the same Philox counters."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CFG = dict(workloads.BASE_MODEL)
K = [80.0, 90.0, 100.0, 110.0, 120.0]


def test_ieee_build_prices_match_the_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    code = ("import json, sys; sys.path.insert(0, '.'); "
            "from paper_2402_12111_gb300 import build; build.build(); "
            "import paper_2402_12111_gb300 as simr, workloads; "
            f"p, _ = simr.price(workloads.BASE_MODEL, {K!r}, False, 64, 65536, 1); "
            f"q, _, g = simr.greeks_adjoint(workloads.BASE_MODEL, {K!r}, False, 64, 16384, 1); "
            "print(json.dumps([p.tolist(), q.tolist(), g.tolist()]))")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT,
                         env=dict(os.environ, SIMR_IEEE="1"), timeout=1200)
    assert out.returncode == 0, out.stderr[-3000:]
    p, q, g = (np.array(a) for a in json.loads(out.stdout.strip().splitlines()[-1]))
    po, _ = oracle.price(CFG, K, False, 64, 65536, 1)
    assert np.all(np.abs(p - po) <= 1e-5 * po), (p - po) / po
    qo, go = oracle.adjoint(CFG, K, False, 64, 16384, 1)
    assert np.all(np.abs(q - qo) <= 1e-5 * qo), (q - qo) / qo
    assert np.all(np.abs(g - go) <= 1e-4 * np.abs(go).max(axis=0)), (g - go)
