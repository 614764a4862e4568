"""QE-M (Andersen's martingale correction) on the GPU against the FP64 oracle's QE-M.

The correction adds lam = ln M - A m per step (a small positive number, computed
without cancellation in FP32), so the per-path and price tolerances are those of
the plain scheme (tests/test_gpu_parity.py); the property the scheme exists for,
E[e^{-rT} S_T] = S0, is checked on the GPU's own paths.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import lsm as olsm
import workloads

pytestmark = pytest.mark.gpu

CFG = dict(workloads.BASE_MODEL)
HARD = dict(S0=100.0, r=0.05, T=1.0, v0=0.09, kappa=1.0, theta=0.04, sigma=0.9, rho=-0.3)
WILD = dict(CFG, sigma=1.0, rho=-0.9, kappa=0.5, T=2.0)  # coarse steps, strong leverage
FLIP_MARGIN = 1e-4


@pytest.fixture(scope="module")
def simr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_12111_gb300 as simr

    simr.load()
    return simr


def _dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("model,steps,n,xf", [(CFG, 64, 8192, 1), (WILD, 8, 8192, 1), (HARD, 64, 8192, 6),
                                              (CFG, 252, 4096, 1)], ids=["cfg", "wild", "hard", "cfg252"])
def test_terminal_states_per_path(simr, model, steps, n, xf):
    with simr.scheme("qem"):
        x, v = simr.paths_terminal(model, steps, 0, n, seed=7)
    x, v = x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    with oracle.scheme("qem"):
        xo, vo, mg = oracle.terminal(model, steps, 7, 0, n)
    ok = mg > FLIP_MARGIN
    dx = np.abs(x - xo)[ok]
    bound = xf * 1.5e-7 * math.sqrt(steps) + 1e-6
    assert np.quantile(dx, 0.999) < bound, (np.quantile(dx, 0.999), dx.max())
    assert np.mean(dx > bound) <= 0.005


def _flip_allowance(model, K, is_put, steps, paths, seed):
    with oracle.scheme("qem"):
        x, _, mg = oracle.terminal(model, steps, seed, 0, paths)
    S = model["S0"] * np.exp(x)
    close = mg < FLIP_MARGIN
    if not close.any():
        return np.zeros(len(K))
    fmax = (np.maximum(K, 0.0) if is_put else np.maximum(S.max() - K, 0.0))
    pay = np.maximum(K[:, None] - S[close][None, :], 0) if is_put else np.maximum(S[close][None, :] - K[:, None], 0)
    return math.exp(-model["r"] * model["T"]) * (pay.sum(axis=1) + close.sum() * fmax) / paths


PRICE_CASES = [
    ("cfg_call", CFG, [100.0], False, 64, 65536, 1),
    ("cfg_grid_put", CFG, workloads.strike_grid(), True, 252, 16384, 3),
    ("wild_grid", WILD, workloads.strike_grid(), False, 8, 65536, 2),
    ("hard", HARD, [80.0, 100.0, 120.0], False, 64, 32768, 5),
    ("ragged", CFG, [95.0, 105.0], True, 33, 1000, 9),
]


@pytest.mark.parametrize("name,model,K,is_put,steps,paths,seed", PRICE_CASES, ids=[c[0] for c in PRICE_CASES])
def test_price_parity(simr, name, model, K, is_put, steps, paths, seed):
    K = np.asarray(K, dtype=np.float64)
    with simr.scheme("qem"):
        p, se = simr.price(model, _dev(K), is_put, steps, paths, seed)
    with oracle.scheme("qem"):
        po, seo = oracle.price(model, K, is_put, steps, paths, seed)
    p, se = p.cpu().numpy(), se.cpu().numpy()
    tol = 1e-5 * np.abs(po) + _flip_allowance(model, K, is_put, steps, paths, seed) + 1e-12
    assert np.all(np.abs(p - po) <= tol), (p - po, tol)
    assert np.all(np.abs(se - seo) <= 1e-4 * seo + 1e-9)


def test_discounted_spot_is_a_martingale_on_the_gpu(simr):
    n = 1 << 21
    with simr.scheme("qem"):
        x, _ = simr.paths_terminal(WILD, 8, 0, n, seed=3, with_variance=False)
    d = math.exp(-WILD["r"] * WILD["T"]) * WILD["S0"] * torch.exp(x.double())
    mean, se = d.mean().item(), d.std().item() / math.sqrt(n)
    assert abs(mean - WILD["S0"]) < 3 * se, (mean, se)


def test_zero_correlation_agrees_with_plain_qe(simr):
    m = dict(CFG, rho=0.0)  # A = 0: the correction vanishes; FP32 evaluation order differs only
    x0, _ = simr.paths_terminal(m, 64, 0, 8192, seed=4)
    with simr.scheme("qem"):
        x1, _ = simr.paths_terminal(m, 64, 0, 8192, seed=4)
    assert (x1 - x0).abs().max().item() < 1e-5


def test_base_path_greeks_match_oracle(simr):
    K = np.array([90.0, 100.0, 110.0])
    with simr.scheme("qem"):
        p, g = simr.greeks_fd(WILD, _dev(K), False, 8, 65536, 6, greeks=("delta", "gamma", "rho"))
    bits = oracle.G_DELTA | oracle.G_GAMMA | oracle.G_RHO
    with oracle.scheme("qem"):
        po, go = oracle.greeks_fd(WILD, K, False, 8, 65536, 6, 1e-4, bits)
    np.testing.assert_allclose(p.cpu().numpy(), po, rtol=1e-5)
    g = g.cpu().numpy()
    np.testing.assert_allclose(g[:, 0], go[:, 0], rtol=1e-4, atol=1e-6)   # delta
    np.testing.assert_allclose(g[:, 2], go[:, 2], rtol=1e-4, atol=1e-5)   # rho
    # gamma: the tent difference of S_T at h = 1e-4 resolves FP32 S_T to ~1e-3 relative
    np.testing.assert_allclose(g[:, 1], go[:, 1], rtol=2e-2, atol=2e-4)


def test_lsm_under_qem_matches_oracle(simr):
    with simr.scheme("qem"):
        p, _, _, stop = simr.lsm_price(WILD, 100.0, True, 16, 2, 8192, 3, with_stop=True)
    with oracle.scheme("qem"):
        ref = olsm.lsm(WILD, 100.0, True, 16, 2, 8192, 3)
    diff = np.nonzero(stop.cpu().numpy() != ref.stop)[0]
    assert diff.size <= 3
    if diff.size == 0:
        assert p.item() == pytest.approx(ref.price, rel=1e-5)


def test_unsupported_calls_refuse_qem(simr):
    K = _dev([100.0])
    with simr.scheme("qem"):
        for call in (lambda: simr.greeks_fd(CFG, K, False, 16, 1024, 1, greeks=("vega",)),
                     lambda: simr.greeks_adjoint(CFG, K, False, 16, 1024, 1),
                     lambda: simr.paths_adjoint(CFG, 16, 0, 1024),
                     lambda: simr.batch([dict(model=CFG, K=100.0, is_put=False, steps=16, paths=1024)])):
            with pytest.raises(simr.SimrError):
                call()
    # the scheme is back to QE afterwards
    simr.greeks_fd(CFG, K, False, 16, 1024, 1, greeks=("vega",))
