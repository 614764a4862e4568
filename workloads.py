"""Seeded synthetic workloads shared by the tests, the bench and the oracle runs.

This module only produces inputs (model parameters, strike grids, option books)
and counts work units; it holds none of the pricing arithmetic, so both the
CUDA path and the CPU oracle can be fed from it without sharing any method code.

Shapes follow the paper's problem statement -- assets x timesteps x paths, one
element per (asset, timestep, path) (Sec. 3, Table 1) -- and the Heston /
bump-and-revalue workloads used to measure the GPU path:

  single   : one European call, 64 steps, 65,536 paths, price + delta/gamma/vega
  grid     : one underlying, 252 steps, 2^20 paths, 32 strikes K/S0 in [0.7, 1.3],
             price + delta/gamma/vega/theta/rho with relative bump 1e-4
  adjoint  : as grid, pathwise adjoint Greeks, checkpoint every 16 steps
  book     : 1,024 heterogeneous European calls/puts (log-uniform steps and paths)
  headline : 8 underlyings x 32 strikes, 1,024 steps, 2^26 paths each
  paper_*  : the paper's Tiny/Small/Medium/Large sizes (Table 1) with the
             single-option model, for context
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_MODEL = dict(S0=100.0, r=0.05, T=1.0, v0=0.04, kappa=1.5, theta=0.04, sigma=0.3, rho=-0.7)

GREEKS_SINGLE = ("delta", "gamma", "vega")
GREEKS_GRID = ("delta", "gamma", "vega", "theta", "rho")
ADJOINT_COLUMNS = ("S0", "v0", "kappa", "theta", "sigma", "rho", "r")


def strike_grid(S0: float = 100.0, n: int = 32, lo: float = 0.7, hi: float = 1.3) -> np.ndarray:
    """n strikes with K/S0 evenly spaced on [lo, hi], both ends included."""
    return S0 * (lo + (hi - lo) * np.arange(n, dtype=np.float64) / (n - 1))


@dataclass
class Workload:
    name: str
    model: dict
    strikes: np.ndarray
    steps: int
    paths: int
    seed: int = 1
    is_put: bool = False
    greeks: tuple = ()
    rel_bump: float = 1e-4
    ckpt_every: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def path_steps(self) -> int:
        """Elements in the paper's sense (Table 1): one per (path, timestep)."""
        return self.steps * self.paths


def single() -> Workload:
    return Workload("heston_call_64x65536", dict(BASE_MODEL), np.array([100.0]), 64, 65536,
                    greeks=GREEKS_SINGLE)


def grid() -> Workload:
    return Workload("heston_grid32_252x1048576", dict(BASE_MODEL), strike_grid(), 252, 1 << 20,
                    greeks=GREEKS_GRID)


def adjoint() -> Workload:
    return Workload("heston_adjoint_grid32_252x1048576", dict(BASE_MODEL), strike_grid(), 252, 1 << 20)


def lsm() -> Workload:
    """Bermudan put, exercisable after every one of 252 steps (a daily-exercise
    proxy for the American option), 2^20 paths: the Longstaff-Schwartz workload."""
    return Workload("heston_lsm_put_252x1048576_daily", dict(BASE_MODEL), np.array([100.0]), 252, 1 << 20,
                    is_put=True, extra={"exercise_every": 1})


def _draw_params(rng: np.random.Generator) -> dict:
    """One option's parameters, in a fixed draw order."""
    v0 = rng.uniform(0.01, 0.09)
    theta = rng.uniform(0.01, 0.09)
    kappa = rng.uniform(0.5, 5.0)
    sigma = rng.uniform(0.1, 1.0)
    rho = rng.uniform(-0.95, 0.0)
    r = rng.uniform(0.0, 0.06)
    T = rng.uniform(0.1, 3.0)
    return dict(S0=100.0, r=r, T=T, v0=v0, kappa=kappa, theta=theta, sigma=sigma, rho=rho)


def book(n_options: int = 1024, seed: int = 1, steps_range=(16, 512), paths_range=(16384, 1 << 20)):
    """Heterogeneous book: per option steps = round(exp(U[ln a, ln b])), likewise paths,
    model parameters uniform on the stated ranges, K/S0 ~ U[0.7, 1.3], call/put 50:50.
    Returns a list of dicts with keys model, K, is_put, steps, paths."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_options):
        steps = int(round(math.exp(rng.uniform(math.log(steps_range[0]), math.log(steps_range[1])))))
        paths = int(round(math.exp(rng.uniform(math.log(paths_range[0]), math.log(paths_range[1])))))
        model = _draw_params(rng)
        K = 100.0 * rng.uniform(0.7, 1.3)
        is_put = bool(rng.uniform() < 0.5)
        out.append(dict(model=model, K=K, is_put=is_put, steps=steps, paths=paths))
    return out


def basket(n_assets: int = 8, seed: int = 31):
    """Correlated basket: n_assets book-style models (T = 1, r = 0.03), a random
    correlation (normalised Gram matrix of Gaussian rows), equal weights, the
    32-strike grid, 252 steps, 2^20 paths.  Returns (models, corr, weights,
    strikes, steps, paths)."""
    models = random_models(n_assets, seed)
    for m in models:
        m["T"], m["r"] = 1.0, 0.03
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n_assets, n_assets + 2))
    C = G @ G.T
    C = C / np.sqrt(np.outer(np.diag(C), np.diag(C)))
    C = 0.5 * (C + C.T)
    np.fill_diagonal(C, 1.0)
    return models, C, np.full(n_assets, 1.0 / n_assets), strike_grid(), 252, 1 << 20


def headline(n_underlyings: int = 8, seed: int = 4):
    """8 underlyings with book-style parameters, each on the 32-strike grid,
    1,024 steps and 2^26 paths, the adjoint at the library's checkpoint interval."""
    rng = np.random.default_rng(seed)
    return [Workload(f"headline_u{i}", _draw_params(rng), strike_grid(), 1024, 1 << 26)
            for i in range(n_underlyings)]


# The paper's problem sizes (Table 1): assets A, timesteps T, paths P.
PAPER_SIZES = {"Tiny": (5, 126, 25_000), "Small": (10, 126, 25_000),
               "Medium": (20, 252, 25_000), "Large": (30, 504, 25_000)}


def paper_elements(size: str) -> int:
    A, T, P = PAPER_SIZES[size]
    return A * T * P


def paper_datapoint_bytes(size: str) -> int:
    """Two FP32 data points (V and Z) per element, as in the paper's Table 1."""
    return 2 * 4 * paper_elements(size)


def paper_book(size: str, seed: int = 7):
    """The paper's problem size as a book: A independent assets (options analysed),
    each with T time steps and P paths; models drawn like the book's parameters
    with T fixed to T/252 years, strikes at the money.  Elements = A T P."""
    A, T, P = PAPER_SIZES[size]
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(A):
        model = _draw_params(rng)
        model["T"] = T / 252.0
        out.append(dict(model=model, K=100.0, is_put=False, steps=T, paths=P))
    return out


def random_models(n: int, seed: int):
    """n model dicts drawn like the book's parameters (for parity sweeps)."""
    rng = np.random.default_rng(seed)
    return [_draw_params(rng) for _ in range(n)]
