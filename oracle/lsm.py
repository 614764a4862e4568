"""Longstaff-Schwartz least-squares Monte Carlo of a Bermudan option on the Heston
QE paths -- TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's dataflow ends in the stages longstaffSchwartzPathReduction and
writeLongstaffSchwartzPath (Sec. 5, Fig. 1) and prints no formula for them; the
method is F. Longstaff and E. Schwartz, "Valuing American options by simulation:
a simple least-squares approach", Review of Financial Studies 14(1), 2001.
Backwards over the exercise dates, the discounted cash flows that the paths
realise under the exercise decisions already taken are regressed, over the
in-the-money paths, on basis functions of the state at the date; a path
exercises where its immediate payoff exceeds the fitted continuation value.

Readings of what neither source fixes for this model (stated once here):
  * exercise dates t_j = (j + 1) every dt, j = 0 .. n_ex - 1, n_ex = steps / every;
    none at t = 0; the last is the maturity, where a positive payoff is taken;
  * basis 1, x, x^2, y, x y, y^2 with x = S/K - 1, y = v/w - 1, w = (v0 + theta)/2
    (w = 1 when that is 0): the quadratic polynomials in spot and variance;
  * only paths with a positive payoff enter the regression or may exercise;
  * least squares through the normal equations, written in the date's
    standardised coordinates xs = (S - F)/sd_S, ys = (v - E v)/sd_v (F = S0 e^{rt},
    sd_S = F sqrt(vbar t) with vbar the mean expected variance over [0, t],
    E v and sd_v the CIR mean and standard deviation of v_t): the same
    quadratics as in x, y, with order-one Gram entries.  Cholesky in basis
    order, a basis function left out (coefficient 0) when its pivot is not
    above 1e-12 of its diagonal entry: least squares fixes the projection onto
    the span of the basis, not the coefficients of dependent functions, and in
    FP64 a Gram matrix of order-one entries summed over at most 2^31 paths
    carries relative rounding far below 1e-12, so a pivot under that threshold
    is a function in the span of the earlier ones (exact collinearity) and
    leaving it out leaves the projection unchanged; with fewer than 12
    in-the-money paths there is no regression and no exercise at that date
    (coefficients NaN).  Coefficients are reported in x, y;
  * exercise when payoff > continuation (strict);
  * price = mean over paths of e^{-r t_stop} x cash flow (0 if never exercised),
    standard error as for the European estimator.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import states

N_BASIS = 6
MIN_ITM = 12
PIVOT_TOL = 1e-12


def basis_scale(model) -> float:
    w = 0.5 * (float(model["v0"]) + float(model["theta"]))
    return w if w > 0.0 else 1.0


def basis(S, v, K: float, w: float) -> np.ndarray:
    """Rows (1, x, x^2, y, x y, y^2), x = S/K - 1, y = v/w - 1."""
    x = np.asarray(S, dtype=np.float64) / K - 1.0
    y = np.asarray(v, dtype=np.float64) / w - 1.0
    return np.stack([np.ones_like(x), x, x * x, y, x * y, y * y], axis=-1)


def standardise(model, n_ex: int, j: int):
    """(a, b, p, q) of date j: xs = a S + b, ys = p v + q (see the module docstring)."""
    T, r, S0 = float(model["T"]), float(model["r"]), float(model["S0"])
    kap, th, v0, s2 = float(model["kappa"]), float(model["theta"]), float(model["v0"]), float(model["sigma"]) ** 2
    t = T * (j + 1) / n_ex
    E = math.exp(-kap * t)
    omE = -math.expm1(-kap * t)
    F = S0 * math.exp(r * t)
    vbar = th + (v0 - th) * omE / (kap * t)
    sdS = F * math.sqrt(max(vbar * t, 1e-12))
    Ev = th + (v0 - th) * E
    varv = v0 * s2 * E * omE / kap + th * s2 * omE * omE / (2.0 * kap)
    sdv = math.sqrt(max(varv, 1e-24))
    return 1.0 / sdS, -F / sdS, 1.0 / sdv, -Ev / sdv


def basis_std(S, v, coef) -> np.ndarray:
    """Rows (1, xs, xs^2, ys, xs ys, ys^2) with xs = a S + b, ys = p v + q."""
    a, b, p, q = coef
    xs = a * np.asarray(S, dtype=np.float64) + b
    ys = p * np.asarray(v, dtype=np.float64) + q
    return np.stack([np.ones_like(xs), xs, xs * xs, ys, xs * ys, ys * ys], axis=-1)


def reported(beta_s, coef, K: float, w: float) -> np.ndarray:
    """Coefficients in (1, x, x^2, y, xy, y^2), x = S/K - 1, y = v/w - 1, of the
    quadratic with coefficients beta_s in (1, xs, xs^2, ys, xs ys, ys^2):
    S = K (1 + x) gives xs = kx (x - cx), kx = aK, cx = -(aK + b)/(aK); likewise ys."""
    a, b, p, q = coef
    kx, ky = a * K, p * w
    cx, cy = -(kx + b) / kx, -(ky + q) / ky
    b0, b1, b2, b3, b4, b5 = beta_s
    return np.array([
        b0 - b1 * kx * cx + b2 * kx * kx * cx * cx - b3 * ky * cy + b4 * kx * ky * cx * cy + b5 * ky * ky * cy * cy,
        b1 * kx - 2.0 * b2 * kx * kx * cx - b4 * kx * ky * cy,
        b2 * kx * kx,
        b3 * ky - b4 * kx * ky * cx - 2.0 * b5 * ky * ky * cy,
        b4 * kx * ky,
        b5 * ky * ky,
    ])


def solve_normal(G, b, tol: float = PIVOT_TOL):
    """beta with G beta = b over the kept basis functions: Cholesky G = L L^T in
    basis order, function k left out when its pivot d_k <= tol G_kk; then the
    two triangular solves.  Returns (beta, kept)."""
    n = len(b)
    L = np.zeros((n, n))
    keep = [False] * n
    for k in range(n):
        d = G[k][k] - sum(L[k][i] ** 2 for i in range(k) if keep[i])
        if not (G[k][k] > 0.0 and d > tol * G[k][k]):
            continue
        keep[k] = True
        L[k][k] = math.sqrt(d)
        for r in range(k + 1, n):
            L[r][k] = (G[r][k] - sum(L[r][i] * L[k][i] for i in range(k) if keep[i])) / L[k][k]
    z = np.zeros(n)
    for k in range(n):
        if keep[k]:
            z[k] = (b[k] - sum(L[k][i] * z[i] for i in range(k) if keep[i])) / L[k][k]
    beta = np.zeros(n)
    for k in reversed(range(n)):
        if keep[k]:
            beta[k] = (z[k] - sum(L[i][k] * beta[i] for i in range(k + 1, n) if keep[i])) / L[k][k]
    return beta, keep


def payoff(S, K: float, is_put: bool) -> np.ndarray:
    return np.maximum(K - S, 0.0) if is_put else np.maximum(S - K, 0.0)


@dataclass
class LsmResult:
    price: float
    stderr: float
    beta: np.ndarray     # [n_ex, 6]; NaN rows: no regression at that date
    stop: np.ndarray     # [paths] exercise date index, -1 = never
    cash: np.ndarray     # [paths] payoff at the exercise date (0 if never)
    margin: np.ndarray   # [paths, n_ex] |payoff - continuation| where a regression decided
    t: np.ndarray        # [n_ex] exercise times
    S: np.ndarray        # [paths, n_ex]
    v: np.ndarray
    Y: np.ndarray | None = None  # [paths, n_ex] regression targets at each date (keep_targets)


def lsm(model, K: float, is_put: bool, steps: int, every: int, paths: int, seed: int = 1,
        option_index: int = 0, path_begin: int = 0, keep_targets: bool = False) -> LsmResult:
    """Longstaff-Schwartz price of the Bermudan option over paths
    [path_begin, path_begin + paths) of the simulation of simr_price.  With
    keep_targets, Y[:, j] holds every path's cash flow discounted to t_j as the
    regression of date j saw it (NaN at the maturity)."""
    S, v = states(model, steps, every, seed, path_begin, paths, option_index)
    n_ex = steps // every
    r = float(model["r"])
    t = (np.arange(n_ex) + 1.0) * (float(model["T"]) / n_ex)
    w = basis_scale(model)
    h = payoff(S, K, is_put)
    cash = h[:, -1].copy()
    stop = np.where(cash > 0.0, n_ex - 1, -1)
    beta = np.full((n_ex, N_BASIS), np.nan)
    margin = np.full((paths, n_ex), np.inf)
    Yall = np.full((paths, n_ex), np.nan) if keep_targets else None
    for j in range(n_ex - 2, -1, -1):
        if keep_targets:
            Yall[:, j] = np.where(stop >= 0, cash * np.exp(-r * (t[np.maximum(stop, 0)] - t[j])), 0.0)
        itm = np.nonzero(h[:, j] > 0.0)[0]
        if itm.size < MIN_ITM:
            continue
        st = stop[itm]
        Y = np.where(st >= 0, cash[itm] * np.exp(-r * (t[np.maximum(st, 0)] - t[j])), 0.0)
        coef = standardise(model, n_ex, j)
        Phi = basis_std(S[itm, j], v[itm, j], coef)
        beta_s, _ = solve_normal(Phi.T @ Phi, Phi.T @ Y)
        beta[j] = reported(beta_s, coef, K, w)
        C = Phi @ beta_s
        hj = h[itm, j]
        margin[itm, j] = np.abs(hj - C)
        ex = hj > C
        cash[itm[ex]] = hj[ex]
        stop[itm[ex]] = j
    dcf = np.where(stop >= 0, cash * np.exp(-r * t[np.maximum(stop, 0)]), 0.0)
    s1 = float(np.sum(dcf))
    s2 = float(np.sum(dcf * dcf))
    mean = s1 / paths
    var = (s2 / paths - mean * mean) / (paths - 1) if paths > 1 else 0.0
    return LsmResult(mean, math.sqrt(max(var, 0.0)), beta, stop, cash, margin, t, S, v, Yall)
