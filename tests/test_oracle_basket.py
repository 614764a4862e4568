"""Pins of the oracle's correlated multi-asset (basket) simulation.

The cross-asset correlation acts only on the log-spot normals, so: one asset is
the single-asset scheme bit for bit; with the identity correlation every asset
is the single-asset scheme of its own option index; in the Black-Scholes limit
(vol-of-vol -> 0, v0 = theta, spot-variance correlation 0) two correlated
assets make the exchange option max(S1 - S2, 0), whose price is Margrabe's
closed form (1978) -- independent of r, so it also checks that each asset's
drift is its own; and the discounted basket is a martingale.
"""
import math

import numpy as np
import pytest
from scipy.stats import norm

import oracle
import workloads

BASE = dict(workloads.BASE_MODEL)


def test_one_asset_is_the_single_asset_scheme():
    x = oracle.basket_terminal([BASE], [[1.0]], 24, 5, 0, 3000)
    xo, _, _ = oracle.terminal(BASE, 24, 5, 0, 3000)
    np.testing.assert_array_equal(x[:, 0], xo)
    p, se = oracle.basket_price([BASE], [[1.0]], [1.0], [95.0, 105.0], True, 24, 3000, 5)
    po, seo = oracle.price(BASE, [95.0, 105.0], True, 24, 3000, 5)
    np.testing.assert_allclose(p, po, rtol=1e-13)
    np.testing.assert_allclose(se, seo, rtol=1e-9)


def test_identity_correlation_gives_each_asset_its_own_paths():
    models = workloads.random_models(3, 12)
    for m in models:
        m["T"] = 1.0
        m["r"] = 0.03
    x = oracle.basket_terminal(models, np.eye(3), 16, 9, 100, 2000)
    for k, m in enumerate(models):
        xo, _, _ = oracle.terminal(m, 16, 9, 100, 2000, option_index=k)
        np.testing.assert_array_equal(x[:, k], xo)


def margrabe(S1, S2, vol1, vol2, c, T):
    s = math.sqrt(vol1 ** 2 + vol2 ** 2 - 2.0 * c * vol1 * vol2)
    d1 = (math.log(S1 / S2) + 0.5 * s * s * T) / (s * math.sqrt(T))
    return S1 * norm.cdf(d1) - S2 * norm.cdf(d1 - s * math.sqrt(T))


@pytest.mark.parametrize("c", [-0.5, 0.0, 0.6, 0.95])
def test_exchange_option_in_the_black_scholes_limit_is_margrabe(c):
    m1 = dict(S0=100.0, r=0.07, T=1.5, v0=0.04, kappa=1.0, theta=0.04, sigma=1e-4, rho=0.0)
    m2 = dict(m1, S0=95.0, v0=0.09, theta=0.09)
    p, se = oracle.basket_price([m1, m2], [[1.0, c], [c, 1.0]], [1.0, -1.0], [0.0], False, 32, 1 << 17, 3)
    ref = margrabe(100.0, 95.0, 0.2, 0.3, c, 1.5)
    assert abs(p[0] - ref) < 3 * se[0] + 1e-3 * ref, (p[0], ref, se[0])


def test_discounted_basket_is_a_martingale():
    models = [dict(BASE), dict(BASE, S0=80.0, v0=0.09, theta=0.06, rho=-0.3), dict(BASE, S0=120.0, sigma=0.6)]
    corr = np.array([[1.0, 0.3, -0.2], [0.3, 1.0, 0.5], [-0.2, 0.5, 1.0]])
    w = [0.5, 1.0, 0.25]
    p, se = oracle.basket_price(models, corr, w, [0.0], False, 32, 1 << 16, 4)
    fwd = sum(wk * m["S0"] for wk, m in zip(w, models))
    # QE without the martingale correction: a small drift bias on top of 3 SE
    assert abs(p[0] - fwd) < 3 * se[0] + 2e-3 * fwd


# QE-M: each asset's log-spot normal z_k is standard normal and independent of
# its own variance path, so each asset takes its single-asset correction.
def test_one_asset_is_the_single_asset_scheme_under_qem():
    with oracle.scheme("qem"):
        x = oracle.basket_terminal([BASE], [[1.0]], 24, 5, 0, 3000)
        xo, _, _ = oracle.terminal(BASE, 24, 5, 0, 3000)
    np.testing.assert_array_equal(x[:, 0], xo)
    x_qe = oracle.basket_terminal([BASE], [[1.0]], 24, 5, 0, 3000)
    assert np.abs(x_qe[:, 0] - xo).max() > 1e-7  # the correction is in there


def test_identity_correlation_gives_each_asset_its_qem_paths():
    models = workloads.random_models(3, 12)
    for m in models:
        m["T"] = 1.0
        m["r"] = 0.03
    with oracle.scheme("qem"):
        x = oracle.basket_terminal(models, np.eye(3), 16, 9, 100, 2000)
        for k, m in enumerate(models):
            xo, _, _ = oracle.terminal(m, 16, 9, 100, 2000, option_index=k)
            np.testing.assert_array_equal(x[:, k], xo)


def test_each_discounted_asset_is_a_martingale_under_qem():
    # a coarse, strongly correlated book: every asset's discounted spot within 3 SE
    # of its S0 (the scheme's exact one-step martingale is pinned in
    # test_oracle_qem.py; this checks that the correlated normals leave it intact)
    models = [dict(BASE, sigma=1.0, rho=-0.9, kappa=0.5, T=2.0), dict(BASE, S0=80.0, sigma=0.8, rho=-0.8, T=2.0)]
    corr = np.array([[1.0, 0.7], [0.7, 1.0]])
    n = 1 << 18
    with oracle.scheme("qem"):
        x = oracle.basket_terminal(models, corr, 8, 6, 0, n)
    for k, m in enumerate(models):
        d = math.exp(-m["r"] * m["T"]) * m["S0"] * np.exp(x[:, k])
        se = d.std(ddof=1) / math.sqrt(n)
        assert abs(d.mean() - m["S0"]) < 3 * se, (k, d.mean(), se)
