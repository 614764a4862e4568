"""The measured error of every result against the FP64 oracle, on the same Philox counters.

For each result the GPU returns -- the price and each bump-and-revalue Greek of the
single-option case (64 steps, 65,536 paths), the price and five Greeks of the
32-strike grid at its full size (252 steps, 2^20 paths), and the seven pathwise
adjoint sensitivities of the same grid (2^18 paths) -- this computes two numbers:
"rel", max over strikes of |GPU - oracle| / |oracle| (strikes whose oracle value is
below 1e-3 of the column's largest left out: relative error there measures
nothing), and "rel_col", max over strikes of |GPU - oracle| / max |oracle column|.
Set SIMR_ERROR_REPORT to a file name to have them written there as JSON.  The
per-result tolerances themselves, with their derivations (the FP32 resolution of
S_T in gamma and the re-simulated Greeks, branch decisions at FP32 distance from
a threshold), are enforced in test_gpu_parity.py and test_gpu_adjoint.py; this test
bounds the report loosely: prices 1e-5, every Greek 1e-3 of its column.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

CFG = dict(workloads.BASE_MODEL)
G5 = ("delta", "gamma", "vega", "theta", "rho")
MASK = {"delta": 1, "gamma": 2, "vega": 4, "theta": 8, "rho": 16}


@pytest.fixture(scope="module")
def simr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_12111_gb300 as simr

    simr.load()
    return simr


def _rel(gpu, ref):
    gpu, ref = np.asarray(gpu, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    keep = np.abs(ref) >= 1e-3 * scale
    err = np.abs(gpu - ref)
    return {"rel": float(np.max(err[keep] / np.abs(ref[keep]))), "rel_col": float(err.max() / scale)}


def test_error_of_every_result(simr):
    report = {}
    # the single call: 64 steps, 65,536 paths, delta / gamma / vega
    K1 = np.array([100.0])
    g3 = ("delta", "gamma", "vega")
    p, g = simr.greeks_fd(CFG, torch.as_tensor(K1, device="cuda"), False, 64, 65536, 1, greeks=list(g3))
    po, go = oracle.greeks_fd(CFG, K1, False, 64, 65536, 1, 1e-4, sum(MASK[n] for n in g3))
    single = {"price": _rel(p.cpu(), po)}
    for j, n in enumerate(g3):
        single[n] = _rel(g.cpu()[:, j], go[:, j])
    report["single_64x65536"] = single

    # the 32-strike grid at full size: 252 steps, 2^20 paths
    K = workloads.strike_grid()
    paths = 1 << 20
    p, g = simr.greeks_fd(CFG, torch.as_tensor(K, device="cuda"), False, 252, paths, 1, greeks=list(G5))
    po, go = oracle.greeks_fd(CFG, K, False, 252, paths, 1, 1e-4, sum(MASK[n] for n in G5))
    grid = {"price": _rel(p.cpu(), po)}
    for j, n in enumerate(G5):
        grid[n] = _rel(g.cpu()[:, j], go[:, j])
    report["grid32_252x1048576_fd"] = grid

    # the pathwise adjoint on the grid: 2^18 paths, 7 sensitivities
    pa, _, ga = simr.greeks_adjoint(CFG, torch.as_tensor(K, device="cuda"), False, 252, 1 << 18, 1)
    pao, gao = oracle.adjoint(CFG, K, False, 252, 1 << 18, 1)
    adj = {"price": _rel(pa.cpu(), pao)}
    for j, n in enumerate(simr.ADJOINT_COLUMNS):
        adj["d/d" + n] = _rel(ga.cpu()[:, j], gao[:, j])
    report["grid32_252x262144_adjoint"] = adj

    path = os.environ.get("SIMR_ERROR_REPORT")
    if path:
        with open(path, "w") as f:
            json.dump(report, f, indent=1)
    for case in report.values():
        assert case["price"]["rel"] <= 1e-5, report
        for name, err in case.items():
            assert np.isfinite(err["rel"]) and np.isfinite(err["rel_col"]), report
            assert err["rel_col"] <= 1e-3, report
