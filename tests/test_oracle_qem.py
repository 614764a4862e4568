"""Pins of the oracle's QE-M scheme (QE with Andersen's martingale correction).

The correction is defined by one property: the discounted spot is an exact
martingale of the discrete scheme, E[exp(x(t+dt) - x(t) - r dt) | v(t)] = 1.
The oracle's one-step expectation sums the variance uniform over its whole
lattice (every value the generator can produce) and integrates the normal
exactly, so it is the scheme's exact expectation; a wrong term in ln M breaks
it.  Further pins: with rho = 0 the correction vanishes (A = 0, M = 1) and the
paths are plain QE's bit for bit; where the correction does not exist the step
falls back to QE; the multi-step martingale holds within Monte Carlo error.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

BASE = dict(workloads.BASE_MODEL)
WILD = dict(BASE, sigma=1.0, rho=-0.9, kappa=0.5, T=2.0)  # coarse steps, strong leverage


@pytest.mark.parametrize("model", [BASE, WILD], ids=["base", "wild"])
def test_one_step_expectation_is_a_martingale(model):
    for v in (0.0, 0.003, 0.04, 0.3):
        with oracle.scheme("qem"):
            assert abs(oracle.step_exp_mean(model, 8, v) - 1.0) < 5e-9
    # the plain scheme is off by far more on the coarse, strongly correlated model
    with oracle.scheme("qe"):
        assert max(abs(oracle.step_exp_mean(WILD, 8, v) - 1.0) for v in (0.0, 0.3)) > 1e-5


def test_zero_correlation_reduces_to_plain_qe():
    m = dict(BASE, rho=0.0)
    x0, v0, _ = oracle.terminal(m, 40, 3, 0, 2000)
    with oracle.scheme("qem"):
        x1, v1, _ = oracle.terminal(m, 40, 3, 0, 2000)
    np.testing.assert_array_equal(v0, v1)
    np.testing.assert_allclose(x1, x0, rtol=0, atol=1e-15)


def test_correction_falls_back_where_it_does_not_exist():
    # one 4-year step, rho = 0.99, sigma = 3, v = 2: the exponential branch with
    # A = K2 + K4/2 above beta = (1 - p)/m, where E[exp(A v')] is infinite
    m = dict(BASE, T=4.0, rho=0.99, sigma=3.0, kappa=5.0)
    k = oracle.qe_constants(m, 1)
    A = k["K2"] + 0.5 * k["K4"]
    v = 2.0
    mean = m["theta"] + (v - m["theta"]) * k["E"]
    s2 = v * k["c1"] + k["c2"]
    psi = s2 / mean ** 2
    p = (psi - 1) / (psi + 1)
    assert psi > 1.5 and A >= (1 - p) / mean
    with oracle.scheme("qe"):
        plain = oracle.step_exp_mean(m, 1, v)
    with oracle.scheme("qem"):
        assert oracle.step_exp_mean(m, 1, v) == plain


def test_multi_step_martingale_within_monte_carlo_error():
    n = 1 << 18
    with oracle.scheme("qem"):
        x, _, _ = oracle.terminal(WILD, 8, 5, 0, n)
    disc = np.exp(-WILD["r"] * WILD["T"]) * WILD["S0"] * np.exp(x)
    se = disc.std(ddof=1) / math.sqrt(n)
    assert abs(disc.mean() - WILD["S0"]) < 3 * se


HARD_Q = dict(S0=100.0, r=0.05, T=1.0, v0=0.09, kappa=1.0, theta=0.04, sigma=0.9, rho=-0.3)


@pytest.mark.parametrize("model", [BASE, WILD, HARD_Q], ids=["base", "wild", "hard"])
def test_qem_reverse_mode_matches_forward_mode_duals(model):
    # the reverse mode's adjoint of ln M (oracle C: qem_log_m_adjoint) against the
    # dual-number forward mode, which differentiates ln M's formula as written --
    # independent code; and the reverse sweep's x_T is the QE-M simulation's
    with oracle.scheme("qem"):
        xr, gr = oracle.path_grad(model, 48, 5, 0, 4096, mode="reverse")
        xf, gf = oracle.path_grad(model, 48, 5, 0, 4096, mode="forward")
        xs, _, _ = oracle.terminal(model, 48, 5, 0, 4096)
    np.testing.assert_allclose(xr, xf, rtol=0, atol=1e-12)
    np.testing.assert_allclose(xr, xs, rtol=0, atol=1e-12)
    scale = np.maximum(np.abs(gf), 1e-3)
    assert np.max(np.abs(gr - gf) / scale) < 1e-9
    # and the correction is in there: the QE-M gradient differs from QE's
    xq, gq = oracle.path_grad(model, 48, 5, 0, 4096, mode="reverse")
    assert np.max(np.abs(gq - gr)) > 1e-6


def test_qem_adjoint_matches_its_finite_differences():
    # pathwise Greeks of the QE-M estimator against central differences of the same
    # estimator (common draws, relative bump 1e-5): only the QE map's rare branch
    # switches separate them, as for plain QE
    P = 1 << 17
    K = np.array([90.0, 100.0, 110.0])
    mask = oracle.G_DELTA | oracle.G_VEGA | oracle.G_RHO | oracle.G_KAPPA | oracle.G_LRVAR | oracle.G_VOLVOL | \
        oracle.G_CORR
    with oracle.scheme("qem"):
        pa, ga = oracle.adjoint(BASE, K, False, 64, P, 13)
        pf, gf = oracle.greeks_fd(BASE, K, False, 64, P, 13, 1e-5, mask)
    np.testing.assert_allclose(pa, pf, rtol=1e-13)
    for ca, cf in [(0, 0), (1, 1), (6, 2), (2, 3), (3, 4), (4, 5), (5, 6)]:
        tol = 2e-3 * max(abs(gf[:, cf]).max(), 1.0)
        np.testing.assert_allclose(ga[:, ca], gf[:, cf], rtol=2e-2, atol=tol)


@pytest.mark.parametrize("model", [
    dict(S0=100.0, r=0.03, T=7.6, v0=1.85, kappa=3.8, theta=0.75, sigma=1.64, rho=0.89),  # quadratic, 2Aa = 1.30
    dict(S0=100.0, r=0.05, T=4.0, v0=2.0, kappa=5.0, theta=0.04, sigma=3.0, rho=0.99),    # exponential, A > beta
], ids=["quadratic", "exponential"])
def test_qem_reverse_mode_where_the_correction_does_not_exist(model):
    # one long step from a large v0: M does not exist on any path, so QE-M takes the
    # plain step -- its reverse mode (the plain derivatives) against the dual
    # numbers' fallback branch, and both equal plain QE's
    with oracle.scheme("qem"):
        xr, gr = oracle.path_grad(model, 1, 5, 0, 2048, mode="reverse")
        xf, gf = oracle.path_grad(model, 1, 5, 0, 2048, mode="forward")
    xq, gq = oracle.path_grad(model, 1, 5, 0, 2048, mode="reverse")
    np.testing.assert_allclose(xr, xf, rtol=0, atol=1e-12)
    scale = np.maximum(np.abs(gf), 1e-3)
    assert np.max(np.abs(gr - gf) / scale) < 1e-9
    np.testing.assert_array_equal(xr, xq)
    np.testing.assert_allclose(gr, gq, rtol=1e-13, atol=1e-14)
