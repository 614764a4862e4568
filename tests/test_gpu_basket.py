"""Basket options on correlated assets (simr_basket_price) on the GPU against the FP64 oracle.

Tolerance: prices relative 1e-5 plus, for paths where some asset's branch
decision lies within 1e-4 of its threshold (FP32 may take the other branch),
the oracle's bound on those paths' payoffs -- as for single-asset prices.
"""
import math

import numpy as np
import pytest
import torch
from scipy.stats import norm

import oracle
import workloads

pytestmark = pytest.mark.gpu

BASE = dict(workloads.BASE_MODEL)
FLIP_MARGIN = 1e-4


@pytest.fixture(scope="module")
def simr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_12111_gb300 as simr

    simr.load()
    return simr


def _models(n, seed):
    ms = workloads.random_models(n, seed)
    for k, m in enumerate(ms):
        m["T"] = 1.0
        m["r"] = 0.03
        m["S0"] = 80.0 + 5.0 * k
    return ms


def _corr(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n + 2))
    C = G @ G.T
    d = np.sqrt(np.diag(C))
    C = C / d[:, None] / d[None, :]
    C = 0.5 * (C + C.T)
    np.fill_diagonal(C, 1.0)
    return C


def _allowance(models, corr, w, K, is_put, steps, paths, seed):
    x, mg = oracle.basket_terminal(models, corr, steps, seed, 0, paths, with_margin=True)
    close = mg < FLIP_MARGIN
    if not close.any():
        return np.zeros(len(K))
    S0 = np.array([m["S0"] for m in models])
    B = (np.exp(x) * S0[None, :]) @ np.asarray(w)
    span = np.abs(np.asarray(w)) @ (S0 * np.exp(x).max(axis=0))  # bound on |B| over the paths
    pay = np.abs(B[close][None, :] - np.asarray(K)[:, None]) + span
    disc = math.exp(-models[0]["r"] * models[0]["T"])
    return disc * pay.sum(axis=1) / paths


CASES = [
    ("two_assets", 2, [100.0, 160.0], False, 32, 65536, 1),
    ("three_put_grid", 3, list(np.linspace(150.0, 300.0, 32)), True, 64, 16384, 2),
    ("five_call", 5, [400.0, 450.0, 500.0], False, 48, 32768, 3),
    ("eight_ragged", 8, [700.0], True, 33, 5003, 4),
    ("sixteen", 16, [1500.0, 1700.0], False, 16, 8192, 5),
]


@pytest.mark.parametrize("name,n,K,is_put,steps,paths,seed", CASES, ids=[c[0] for c in CASES])
def test_basket_price_parity(simr, name, n, K, is_put, steps, paths, seed):
    models = _models(n, 10 + seed)
    corr = _corr(n, seed)
    w = np.linspace(1.0, 0.5, n)
    K = np.asarray(K)
    p, se = simr.basket_price(models, corr, w, torch.as_tensor(K, device="cuda"), is_put, steps, paths, seed)
    po, seo = oracle.basket_price(models, corr, w, K, is_put, steps, paths, seed)
    p, se = p.cpu().numpy(), se.cpu().numpy()
    tol = 1e-5 * np.abs(po) + _allowance(models, corr, w, K, is_put, steps, paths, seed) + 1e-12
    assert np.all(np.abs(p - po) <= tol), (p - po, tol)
    assert np.all(np.abs(se - seo) <= 1e-4 * seo + 1e-9)


def test_identity_correlation_reproduces_single_asset_prices(simr):
    models = _models(3, 21)
    K = np.array([70.0, 90.0, 110.0])
    for k in range(3):
        w = np.eye(3)[k]
        p, se = simr.basket_price(models, np.eye(3), w, K, False, 40, 30000, 6)
        pk, sek = simr.price(models[k], K, False, 40, 30000, 6, option_index=k)
        # the same per-path values; the two kernels group the FP32 partial sums differently
        np.testing.assert_allclose(p.numpy(), pk.numpy(), rtol=1e-8, atol=1e-10)
        np.testing.assert_allclose(se.numpy(), sek.numpy(), rtol=1e-6, atol=1e-10)


def test_exchange_option_matches_margrabe(simr):
    m1 = dict(S0=100.0, r=0.07, T=1.5, v0=0.04, kappa=1.0, theta=0.04, sigma=1e-4, rho=0.0)
    m2 = dict(m1, S0=95.0, v0=0.09, theta=0.09)
    c = 0.6
    p, se = simr.basket_price([m1, m2], [[1.0, c], [c, 1.0]], [1.0, -1.0], [0.0], False, 32, 1 << 20, 3)
    s = math.sqrt(0.04 + 0.09 - 2 * c * 0.2 * 0.3)
    d1 = (math.log(100.0 / 95.0) + 0.5 * s * s * 1.5) / (s * math.sqrt(1.5))
    ref = 100.0 * norm.cdf(d1) - 95.0 * norm.cdf(d1 - s * math.sqrt(1.5))
    assert abs(p.item() - ref) < 3 * se.item() + 1e-3 * ref


def test_basket_rejects_bad_inputs(simr):
    m = [BASE, BASE]
    with pytest.raises(simr.SimrError):
        simr.basket_price(m, [[1.0, 1.2], [1.2, 1.0]], [1, 1], [100.0])        # |corr| > 1
    with pytest.raises(simr.SimrError):
        simr.basket_price(m, [[1.0, 1.0], [1.0, 1.0]], [1, 1], [100.0])        # not positive definite
    with pytest.raises(simr.SimrError):
        simr.basket_price([BASE, dict(BASE, T=2.0)], np.eye(2), [1, 1], [100.0])  # T differs
    with pytest.raises(simr.SimrError):
        simr.basket_price([BASE] * 17, np.eye(17), np.ones(17), [100.0])       # too many assets


# QE-M: each asset takes its own martingale correction (its log-spot normal is
# independent of its own variance path); both sides under QE-M, the same
# tolerances.  Odd counts run their last asset alone (the scalar QE-M step).
QEM_CASES = [
    ("two_assets", 2, [100.0, 160.0], False, 32, 65536, 1),
    ("five_call", 5, [400.0, 450.0, 500.0], False, 48, 32768, 3),
    ("eight_ragged_put_grid", 8, list(np.linspace(500.0, 800.0, 40)), True, 33, 5003, 4),
]


@pytest.mark.parametrize("name,n,K,is_put,steps,paths,seed", QEM_CASES, ids=[c[0] for c in QEM_CASES])
def test_basket_price_parity_under_qem(simr, name, n, K, is_put, steps, paths, seed):
    models = _models(n, 10 + seed)
    corr = _corr(n, seed)
    w = np.linspace(1.0, 0.5, n)
    K = np.asarray(K)
    with simr.scheme("qem"):
        p, se = simr.basket_price(models, corr, w, torch.as_tensor(K, device="cuda"), is_put, steps, paths, seed)
    p0, _ = simr.basket_price(models, corr, w, torch.as_tensor(K, device="cuda"), is_put, steps, paths, seed)
    with oracle.scheme("qem"):
        po, seo = oracle.basket_price(models, corr, w, K, is_put, steps, paths, seed)
        tol = 1e-5 * np.abs(po) + _allowance(models, corr, w, K, is_put, steps, paths, seed) + 1e-12
    p, se = p.cpu().numpy(), se.cpu().numpy()
    assert np.all(np.abs(p - po) <= tol), (p - po, tol)
    assert np.all(np.abs(se - seo) <= 1e-4 * seo + 1e-9)
    assert np.abs(p0.cpu().numpy() - p).max() > 0.0  # the correction reached the kernel


def test_identity_correlation_reproduces_single_asset_qem_prices(simr):
    models = _models(3, 21)
    K = np.array([70.0, 90.0, 110.0])
    with simr.scheme("qem"):
        for k in range(3):
            w = np.eye(3)[k]
            p, se = simr.basket_price(models, np.eye(3), w, K, False, 40, 30000, 6)
            pk, sek = simr.price(models[k], K, False, 40, 30000, 6, option_index=k)
            np.testing.assert_allclose(p.numpy(), pk.numpy(), rtol=1e-8, atol=1e-10)
            np.testing.assert_allclose(se.numpy(), sek.numpy(), rtol=1e-6, atol=1e-10)
