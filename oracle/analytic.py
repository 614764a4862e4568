"""Closed forms and semi-analytic prices that pin the Monte Carlo oracle (test infrastructure only).

None of these is the method: the paper's path (Sec. 4-5) is a time-discretised
Monte Carlo estimator.  These are the exact quantities that estimator must
reproduce within its statistical error and discretisation bias:

* ``heston_call_p1p2`` / ``heston_call_lewis``: European call under Heston
  (1993), by two independent Fourier inversions of the same characteristic
  function (Heston's P1/P2 form; Lewis's single-integral form).  The
  characteristic function uses the "little trap" branch of Albrecher, Mayer,
  Schoutens and Tistaert (2007).
* ``bs_call`` / ``bs_put``: Black-Scholes (1973) closed form (the Heston model
  with a vanishing vol-of-vol and v0 = theta).
* ``cir_mean`` / ``cir_var``: exact mean and variance of the CIR variance
  process at a horizon t (the QE step matches the first two conditional
  moments, so these hold exactly after any number of steps).
* ``heston_log_mean``: E[ln(S_T/S0)] = rT - 1/2 * integral of E[v_t] dt.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate
from scipy.special import ndtr


def _cf_log_spot(u, S0, r, T, v0, kappa, theta, sigma, rho):
    """E[exp(i u ln S_T)] under Heston, little-trap form (complex u allowed)."""
    iu = 1j * u
    b = kappa - rho * sigma * iu
    d = np.sqrt(b * b + sigma * sigma * (iu + u * u))
    g = (b - d) / (b + d)
    edt = np.exp(-d * T)
    C = (kappa * theta / sigma ** 2) * ((b - d) * T - 2.0 * np.log((1.0 - g * edt) / (1.0 - g)))
    D = (v0 / sigma ** 2) * (b - d) * (1.0 - edt) / (1.0 - g * edt)
    return np.exp(iu * (math.log(S0) + r * T) + C + D)


def heston_call_p1p2(K, S0, r, T, v0, kappa, theta, sigma, rho):
    """C = S0 P1 - K e^{-rT} P2 with the two exercise probabilities by Gil-Pelaez inversion."""
    lnK = math.log(K)
    phi_mi = _cf_log_spot(-1j, S0, r, T, v0, kappa, theta, sigma, rho)  # = E[S_T]

    def f1(u):
        return (np.exp(-1j * u * lnK) * _cf_log_spot(u - 1j, S0, r, T, v0, kappa, theta, sigma, rho)
                / (1j * u * phi_mi)).real

    def f2(u):
        return (np.exp(-1j * u * lnK) * _cf_log_spot(u, S0, r, T, v0, kappa, theta, sigma, rho) / (1j * u)).real

    opts = dict(limit=2000, epsabs=1e-12, epsrel=1e-11)
    P1 = 0.5 + integrate.quad(f1, 0.0, np.inf, **opts)[0] / math.pi
    P2 = 0.5 + integrate.quad(f2, 0.0, np.inf, **opts)[0] / math.pi
    return S0 * P1 - K * math.exp(-r * T) * P2, P1, P2


def heston_call_lewis(K, S0, r, T, v0, kappa, theta, sigma, rho):
    """Lewis (2001), forward form: C = e^{-rT} (F - sqrt(F K)/pi * int_0^inf Re[e^{iuk} phi(u - i/2)] / (u^2 + 1/4) du)
    with F = S0 e^{rT}, phi the characteristic function of ln(S_T/F) and k = ln(F/K)."""
    k = math.log(S0 / K) + r * T
    shift = math.log(S0) + r * T

    def f(u):
        z = u - 0.5j
        phi = _cf_log_spot(z, S0, r, T, v0, kappa, theta, sigma, rho) * np.exp(-1j * z * shift)
        return (np.exp(1j * u * k) * phi).real / (u * u + 0.25)

    val = integrate.quad(f, 0.0, np.inf, limit=2000, epsabs=1e-12, epsrel=1e-11)[0]
    F = S0 * math.exp(r * T)
    return math.exp(-r * T) * (F - math.sqrt(F * K) * val / math.pi)


def heston_put_from_call(call, K, S0, r, T):
    return call - S0 + K * math.exp(-r * T)


def bs_call(S0, K, r, T, vol):
    sd = vol * math.sqrt(T)
    d1 = (math.log(S0 / K) + (r + 0.5 * vol * vol) * T) / sd
    return S0 * ndtr(d1) - K * math.exp(-r * T) * ndtr(d1 - sd)


def bs_put(S0, K, r, T, vol):
    return bs_call(S0, K, r, T, vol) - S0 + K * math.exp(-r * T)


def cir_mean(t, v0, kappa, theta):
    return theta + (v0 - theta) * math.exp(-kappa * t)


def cir_var(t, v0, kappa, theta, sigma):
    e = math.exp(-kappa * t)
    return v0 * sigma ** 2 * e * (1.0 - e) / kappa + theta * sigma ** 2 * (1.0 - e) ** 2 / (2.0 * kappa)


def heston_log_mean(r, T, v0, kappa, theta):
    """E[ln(S_T/S0)] = rT - 1/2 (theta T + (v0 - theta)(1 - e^{-kappa T}) / kappa)."""
    return r * T - 0.5 * (theta * T + (v0 - theta) * (1.0 - math.exp(-kappa * T)) / kappa)
