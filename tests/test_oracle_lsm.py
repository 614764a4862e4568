"""Pins of the oracle's Longstaff-Schwartz (least-squares Monte Carlo) Bermudan price.

Each test ties the oracle to something other than itself: the European price of
the same paths (one exercise date), numpy's least-squares routine (the solver),
the exact value of optimal stopping on deterministic paths (dates, stopping and
discounting), a Cox-Ross-Rubinstein lattice of the Bermudan put in the
Black-Scholes limit (the whole estimator), and the no-early-exercise property of
calls without dividends.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import lsm
import workloads

BASE = dict(workloads.BASE_MODEL)


def test_single_exercise_date_is_the_european_price():
    # every = steps: the only date is the maturity, so LSM is the European estimator
    for is_put in (False, True):
        r = lsm.lsm(BASE, 95.0, is_put, 48, 48, 6000, seed=3)
        p, se = oracle.price(BASE, [95.0], is_put, 48, 6000, 3)
        assert r.price == pytest.approx(p[0], rel=1e-13)
        assert r.stderr == pytest.approx(se[0], rel=1e-9)
        assert np.all(np.isnan(r.beta))


def test_normal_equation_solve_matches_lstsq():
    rng = np.random.default_rng(5)
    S = 100.0 * np.exp(0.2 * rng.standard_normal(400))
    v = 0.04 * rng.gamma(4.0, 0.25, 400)
    Phi = lsm.basis(S, v, 100.0, 0.04)
    Y = np.maximum(100.0 - S, 0.0) + rng.standard_normal(400)
    beta, keep = lsm.solve_normal(Phi.T @ Phi, Phi.T @ Y)
    ref = np.linalg.lstsq(Phi, Y, rcond=None)[0]
    assert all(keep)
    np.testing.assert_allclose(beta, ref, rtol=1e-8, atol=1e-10)
    # exactly collinear columns (v = w: y = 0): the fitted values are the projection
    # onto the span, whichever coefficients represent it
    Phi0 = lsm.basis(S, np.full(400, 0.04), 100.0, 0.04)
    beta0, keep0 = lsm.solve_normal(Phi0.T @ Phi0, Phi0.T @ Y)
    assert keep0 == [True, True, True, False, False, False]
    ref0 = np.linalg.lstsq(Phi0, Y, rcond=None)[0]
    np.testing.assert_allclose(Phi0 @ beta0, Phi0 @ ref0, rtol=1e-9, atol=1e-9)
    # constant v in standardised coordinates: ys is a constant, collinear with 1
    coef = lsm.standardise(dict(workloads.BASE_MODEL), 10, 4)
    Ps = lsm.basis_std(S, np.full(400, 0.05), coef)
    bs, keeps = lsm.solve_normal(Ps.T @ Ps, Ps.T @ Y)
    assert keeps == [True, True, True, False, False, False]
    np.testing.assert_allclose(Ps @ bs, Phi0 @ ref0, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("v0", [0.04, 0.09])
def test_standardised_and_reported_coefficients_are_the_same_quadratic(v0):
    # v0 = theta puts the variance's two centres (E v_t and w) on the same value, so
    # the coordinate shifts of y vanish; v0 != theta exercises every term of the map
    rng = np.random.default_rng(6)
    m = dict(workloads.BASE_MODEL, v0=v0)
    S = 100.0 * np.exp(0.2 * rng.standard_normal(50))
    v = 0.04 * rng.gamma(4.0, 0.25, 50)
    coef = lsm.standardise(m, 12, 3)
    bs = rng.standard_normal(6)
    br = lsm.reported(bs, coef, 95.0, lsm.basis_scale(m))
    np.testing.assert_allclose(lsm.basis(S, v, 95.0, lsm.basis_scale(m)) @ br, lsm.basis_std(S, v, coef) @ bs,
                               rtol=1e-9, atol=1e-9)


def test_regression_on_simulated_paths_matches_lstsq():
    r = lsm.lsm(BASE, 100.0, True, 32, 4, 5000, seed=7)
    n_ex = r.beta.shape[0]
    h = lsm.payoff(r.S, 100.0, True)
    j = n_ex - 2  # the first regression: targets are the maturity payoffs
    itm = h[:, j] > 0
    # the first regression's targets, rebuilt independently: only the maturity cash flow exists
    Y = h[itm, -1] * math.exp(-BASE["r"] * (r.t[-1] - r.t[j]))
    Phi = lsm.basis(r.S[itm, j], r.v[itm, j], 100.0, lsm.basis_scale(BASE))
    ref = np.linalg.lstsq(Phi, Y, rcond=None)[0]
    np.testing.assert_allclose(Phi @ r.beta[j], Phi @ ref, rtol=1e-8, atol=1e-8 * np.abs(Y).max())


DET = dict(S0=50.0, r=0.1, T=1.0, v0=1e-12, kappa=1.5, theta=1e-12, sigma=1e-4, rho=0.0)


def test_deterministic_paths_deep_put_exercises_at_the_first_date():
    # S_t = S0 e^{rt} (v ~ 1e-12): the discounted payoff e^{-rt} K - S0 falls with t,
    # so the optimal rule stops at the first date t_0 = T / n_ex (never at t = 0)
    r = lsm.lsm(DET, 100.0, True, 64, 8, 400, seed=1)
    t0 = DET["T"] / 8
    exact = 100.0 * math.exp(-DET["r"] * t0) - DET["S0"]
    assert np.all(r.stop == 0)
    assert r.price == pytest.approx(exact, rel=1e-6)


def test_deterministic_paths_negative_rate_put_waits_to_maturity():
    # r < 0: e^{-rt} K - S0 rises with t, so no path stops before the maturity
    m = dict(DET, S0=100.0, r=-0.02)
    r = lsm.lsm(m, 110.0, True, 64, 8, 400, seed=1)
    exact = 110.0 * math.exp(-m["r"] * m["T"]) - m["S0"]
    assert np.all(r.stop == 7)
    assert r.price == pytest.approx(exact, rel=1e-6)


def crr_bermudan_put(S0, K, r, vol, T, n_ex, per_date=40):
    """Cox-Ross-Rubinstein lattice, exercise allowed at the n_ex dates (j + 1) T / n_ex."""
    n = n_ex * per_date
    dt = T / n
    u = math.exp(vol * math.sqrt(dt))
    d = 1.0 / u
    q = (math.exp(r * dt) - d) / (u - d)
    disc = math.exp(-r * dt)
    S = S0 * u ** np.arange(n, -n - 1, -2)
    V = np.maximum(K - S, 0.0)
    for i in range(n - 1, -1, -1):
        S = S0 * u ** np.arange(i, -i - 1, -2)
        V = disc * (q * V[:-1] + (1.0 - q) * V[1:])
        if i > 0 and i % per_date == 0:
            V = np.maximum(V, K - S)
    return float(V[0])


def test_bermudan_put_black_scholes_limit_matches_lattice():
    # sigma -> 0 with v0 = theta, rho = 0: log-normal paths of volatility 0.2 (the
    # Longstaff-Schwartz paper's first example: S0 36, K 40, r 0.06, T 1, 50 dates)
    m = dict(S0=36.0, r=0.06, T=1.0, v0=0.04, kappa=1.5, theta=0.04, sigma=1e-4, rho=0.0)
    r = lsm.lsm(m, 40.0, True, 50, 1, 1 << 16, seed=11)
    ref = crr_bermudan_put(36.0, 40.0, 0.06, 0.2, 1.0, 50)
    assert 4.3 < ref < 4.6
    # Monte Carlo noise plus the estimator's own bias (regression on a finite basis)
    assert abs(r.price - ref) < 3 * r.stderr + 0.01 * ref
    euro, _ = oracle.price(m, [40.0], True, 50, 1 << 16, 11)
    assert r.price > euro[0] + 0.2  # a visible early-exercise premium


def test_call_without_dividends_has_no_early_exercise_premium():
    r = lsm.lsm(BASE, 100.0, False, 64, 4, 1 << 14, seed=2)
    p, se = oracle.price(BASE, [100.0], False, 64, 1 << 14, 2)
    early = (r.stop >= 0) & (r.stop < r.beta.shape[0] - 1)
    assert early.mean() < 0.02
    # same paths: the difference is confined to the few early-exercised paths
    assert abs(r.price - p[0]) < 3 * se[0]


def test_put_early_exercise_premium_is_positive():
    r = lsm.lsm(BASE, 100.0, True, 64, 4, 1 << 14, seed=2)
    p, _ = oracle.price(BASE, [100.0], True, 64, 1 << 14, 2)
    assert r.price > p[0] + 3 * r.stderr


# The cases the GPU parity test (test_gpu_lsm.py) runs, and a bench-shaped sample.
PIVOT_CASES = [
    (BASE, 100.0, True, 64, 4, 1 << 14, 1), (BASE, 110.0, True, 50, 1, 8192, 2),
    (BASE, 90.0, False, 32, 2, 8192, 3), (dict(BASE, sigma=0.9, rho=-0.3, kappa=0.5, v0=0.09), 100.0, True, 48, 3,
                                         1 << 14, 4),
    (BASE, 105.0, True, 33, 11, 5003, 5), (BASE, 130.0, True, 40, 2, 6000, 6), (BASE, 100.0, True, 252, 1, 1 << 13, 1),
]


@pytest.mark.parametrize("case", PIVOT_CASES)
def test_gpu_pivot_threshold_never_binds_on_the_parity_cases(case, monkeypatch):
    # The oracle leaves a basis function out below 1e-12 of its diagonal (FP64),
    # the GPU's FP32 Cholesky below 1e-5.  On every regression of these cases the
    # smallest pivot ratio is far above both, so both keep all six functions and
    # the thresholds cannot make the two sides' fits differ.
    pivots = []
    orig = lsm.solve_normal

    def recording(G, b, tol=lsm.PIVOT_TOL):
        beta, keep = orig(G, b, tol)
        n = len(b)
        d = np.linalg.cholesky(G)  # all kept: the plain factor
        pivots.append(min(d[k, k] ** 2 / G[k, k] for k in range(n)))
        assert all(keep)
        return beta, keep

    monkeypatch.setattr(lsm, "solve_normal", recording)
    lsm.lsm(*case)
    assert pivots and min(pivots) > 1e-3, min(pivots)
