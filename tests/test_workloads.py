"""The seeded input generators follow their stated recipes (no GPU): the strike
grid, the 1,024-option book's distributions, the headline underlyings, the
paper-shaped books and the basket's correlation matrix."""
import numpy as np

import workloads


def test_strike_grid_spans_the_stated_range():
    K = workloads.strike_grid()
    assert K.shape == (32,)
    assert K[0] == 70.0 and abs(K[-1] - 130.0) < 1e-12
    assert np.allclose(np.diff(K), 60.0 / 31)


def test_book_draws_follow_the_recipe_and_repeat():
    book = workloads.book()
    assert len(book) == 1024
    steps = np.array([o["steps"] for o in book])
    paths = np.array([o["paths"] for o in book])
    assert steps.min() >= 16 and steps.max() <= 512
    assert paths.min() >= 16384 and paths.max() <= 1 << 20
    # log-uniform: the log of the draws spreads evenly over its range
    u = (np.log(steps) - np.log(16)) / (np.log(512) - np.log(16))
    assert 0.4 < np.median(u) < 0.6
    m = {k: np.array([o["model"][k] for o in book]) for k in ("v0", "theta", "kappa", "sigma", "rho", "r", "T")}
    for k, (lo, hi) in {"v0": (0.01, 0.09), "theta": (0.01, 0.09), "kappa": (0.5, 5.0), "sigma": (0.1, 1.0),
                        "rho": (-0.95, 0.0), "r": (0.0, 0.06), "T": (0.1, 3.0)}.items():
        assert m[k].min() >= lo and m[k].max() <= hi, k
    kr = np.array([o["K"] / o["model"]["S0"] for o in book])
    assert kr.min() >= 0.7 and kr.max() <= 1.3
    puts = np.mean([o["is_put"] for o in book])
    assert 0.45 < puts < 0.55
    again = workloads.book()
    assert all(a["K"] == b["K"] and a["model"] == b["model"] and a["steps"] == b["steps"] for a, b in zip(book, again))


def test_headline_and_paper_shapes():
    hw = workloads.headline()
    assert len(hw) == 8 and all(u.steps == 1024 and u.paths == 1 << 26 and len(u.strikes) == 32 for u in hw)
    for size, (A, T, P) in workloads.PAPER_SIZES.items():
        opts = workloads.paper_book(size)
        assert len(opts) == A and all(o["steps"] == T and o["paths"] == P for o in opts)
        assert workloads.paper_elements(size) == A * T * P


def test_basket_correlation_is_a_valid_correlation():
    models, C, w, K, steps, paths = workloads.basket()
    assert len(models) == 8 and C.shape == (8, 8) and steps == 252 and paths == 1 << 20
    assert np.allclose(C, C.T) and np.allclose(np.diag(C), 1.0)
    assert np.linalg.eigvalsh(C).min() > 0
    assert abs(w.sum() - 1.0) < 1e-12
