"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same Philox counters.

Tolerances (stated per quantity, from the arithmetic of the FP32 path):
  * per path, x_T = ln(S_T/S0): the FP32 state v is rounded every step and the
    log-spot step carries its changes with weight rho/sigma, so x_T drifts from
    the FP64 path like a random walk: rms ~2.5e-8 sqrt(N) measured on GB300.
    99.9% of the paths whose oracle branch decisions are not within 1e-4 of a
    threshold must agree to 1.5e-7 sqrt(N) + 1e-6; at most 0.5% may differ more
    (a branch taken differently near v = 0, where FP32 has few digits);
  * prices: relative 1e-5 (the target for prices), plus the effect of the
    flip-capable paths bounded by the oracle's own per-path payoffs;
  * FD Greeks: relative 1e-4 (the target for Greeks) plus, for the Greeks whose
    per-path term depends on the FP32 resolution of S_T, that resolution's
    5-sigma effect on the estimator (see _greek_tol).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

CFG = dict(workloads.BASE_MODEL)
HARD = dict(S0=100.0, r=0.05, T=1.0, v0=0.09, kappa=1.0, theta=0.04, sigma=0.9, rho=-0.3)
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


def _flip_allowance(model, K, is_put, steps, paths, seed):
    """Bound on |price difference| from paths that FP32 could send down another branch:
    each such path moves the mean by at most (its oracle payoff + the payoff at the
    largest S_T seen) / paths; zero when no path is within FLIP_MARGIN."""
    x, _, mg = oracle.terminal(model, steps, seed, 0, paths)
    S = model["S0"] * np.exp(x)
    close = mg < FLIP_MARGIN
    if not close.any():
        return np.zeros(len(K))
    fmax = (np.maximum(K - 0.0, 0.0) if is_put else np.maximum(S.max() - K, 0.0))
    pay = np.maximum(K[:, None] - S[close][None, :], 0) if is_put else np.maximum(S[close][None, :] - K[:, None], 0)
    return math.exp(-model["r"] * model["T"]) * (pay.sum(axis=1) + close.sum() * fmax) / paths


# ------------------------------------------------------------- per path ----
# xf: per-case scale of the per-path bound (the vol-of-vol 0.9 model spends many
# steps near v = 0, where the FP32 state has fewer correct digits).
@pytest.mark.parametrize("model,steps,n,begin,xf", [
    (CFG, 1, 1000, 0, 1), (CFG, 2, 4096, 5, 1), (CFG, 7, 4099, 12345, 1), (CFG, 64, 8192, 0, 1),
    (HARD, 64, 8192, 77, 6), (CFG, 252, 4096, 1 << 33, 1), (dict(CFG, rho=1.0), 16, 2048, 0, 1),
    (dict(CFG, v0=0.0), 16, 2048, 0, 1), (dict(CFG, theta=0.0, v0=0.0), 8, 512, 0, 1)])
def test_terminal_states_per_path(simr, model, steps, n, begin, xf):
    x, v = simr.paths_terminal(model, steps, begin, n, seed=7)
    x, v = x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    xo, vo, mg = oracle.terminal(model, steps, 7, begin, n)
    ok = mg > FLIP_MARGIN
    assert ok.mean() > 0.98
    assert np.all(np.isfinite(x)) and np.all(v >= 0)
    dx = np.abs(x - xo)[ok]
    bound = xf * 1.5e-7 * math.sqrt(steps) + 1e-6
    assert np.quantile(dx, 0.999) < bound, (np.quantile(dx, 0.999), dx.max())
    assert np.mean(dx > bound) <= 0.005
    dv = (np.abs(v - vo) / np.maximum(vo, 0.1 * max(model["theta"], 1e-3)))[ok]
    assert np.quantile(dv, 0.999) < 1e-4, dv.max()


@pytest.mark.parametrize("k", [0, 6])
def test_headline_paths_at_the_end_of_the_range(simr, k):
    # the headline book's shape at its sampled outputs: 1,024 steps, the last
    # 2,048 of an underlying's 2^26 paths, one by one against the oracle
    u = workloads.headline()[k]
    n, begin = 2048, (1 << 26) - 2048
    x, v = simr.paths_terminal(u.model, u.steps, begin, n, seed=u.seed)
    x, v = x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    xo, vo, mg = oracle.terminal(u.model, u.steps, u.seed, begin, n)
    ok = mg > FLIP_MARGIN
    assert ok.mean() > 0.95
    assert np.all(np.isfinite(x)) and np.all(v >= 0)
    dx = np.abs(x - xo)[ok]
    bound = 1.5e-7 * math.sqrt(u.steps) + 1e-6
    assert np.quantile(dx, 0.999) < bound, (np.quantile(dx, 0.999), dx.max())
    assert np.mean(dx > bound) <= 0.005


# --------------------------------------------------------------- prices ----
PRICE_CASES = [
    ("cfg_single", CFG, [100.0], False, 64, 65536, 1),
    ("cfg_single_put", CFG, [100.0], True, 64, 65536, 1),
    ("grid32_small", CFG, workloads.strike_grid(), False, 252, 16384, 3),
    ("grid32_put", CFG, workloads.strike_grid(), True, 252, 16384, 3),
    ("hard_exp_branch", HARD, [80.0, 100.0, 120.0], False, 64, 32768, 5),
    ("ragged_paths", CFG, [95.0, 105.0], False, 33, 1000, 9),
    ("one_path", CFG, [100.0], False, 8, 1, 9),
    ("one_step", CFG, [90.0, 100.0, 110.0], True, 1, 4097, 2),
    ("strikes_40", CFG, np.linspace(60, 140, 40), False, 16, 8192, 4),
    ("seed_hi_word", CFG, [100.0], False, 16, 8192, (0xABCDEF << 32) | 12345),
    # the largest strike count simr_price takes: 32 tiles of 32 strikes
    ("strikes_1024_max", CFG, np.linspace(50.0, 150.0, 1024), True, 16, 8192, 12),
]


@pytest.mark.parametrize("name,model,K,is_put,steps,paths,seed", PRICE_CASES, ids=[c[0] for c in PRICE_CASES])
def test_price_parity(simr, name, model, K, is_put, steps, paths, seed):
    K = np.asarray(K, dtype=np.float64)
    p, se = simr.price(model, _dev(K), is_put, steps, paths, seed)
    p, se = p.cpu().numpy(), se.cpu().numpy()
    po, seo = oracle.price(model, K, is_put, steps, paths, seed)
    tol = 1e-5 * np.abs(po) + _flip_allowance(model, K, is_put, steps, paths, seed) + 1e-12
    assert np.all(np.abs(p - po) <= tol), (p - po, tol)
    if paths > 1:
        assert np.all(np.abs(se - seo) <= 1e-4 * seo + 1e-9)


def test_host_and_device_pointers_agree(simr):
    K = workloads.strike_grid()
    pd, sd = simr.price(CFG, _dev(K), False, 32, 20000, 11)
    ph, sh = simr.price(CFG, K, False, 32, 20000, 11)  # host buffers
    assert torch.equal(pd.cpu(), ph) and torch.equal(sd.cpu(), sh)


def test_deterministic(simr):
    K = _dev(workloads.strike_grid())
    a = simr.greeks_fd(CFG, K, False, 40, 50000, 3, greeks=("delta", "gamma", "vega", "theta", "rho"))
    b = simr.greeks_fd(CFG, K, False, 40, 50000, 3, greeks=("delta", "gamma", "vega", "theta", "rho"))
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


# --------------------------------------------------------------- Greeks ----
EPS_X = 3e-8  # rms FP32 error of x_T per sqrt(step), measured on GB300 against the oracle

# bump denominators (one-sided where the down-bump leaves the domain)
BUMPS = {"vega": lambda m, h: 2 * h * m["v0"] if m["v0"] > 0 else h,
         "theta": lambda m, h: 2 * h * m["T"], "kappa": lambda m, h: 2 * h * m["kappa"],
         "lrvar": lambda m, h: 2 * h * m["theta"] if m["theta"] > 0 else h,
         "volvol": lambda m, h: 2 * h * m["sigma"],
         "corr": lambda m, h: 2 * h if abs(m["rho"]) + h <= 1 else h}


def _greek_tol(name, og, h, steps, paths, model):
    """Tolerance of each FD Greek column vs the FP64 oracle.

    delta and rho are same-path revaluations whose per-path terms are bands of
    width O(h S) around each strike, exact in FP32 except at their edges: 1e-4.
    gamma's tent terms have height h S and carry the FP32 error of S_T
    (S0 EPS_X sqrt(N) rms); ~paths * f * 2hS0 paths fall in the tent with a
    density f <= 0.05 per unit S: 1e-4 + 5 S0 EPS_X sqrt(N) sqrt(n_tent) / (paths (h S0)^2).
    Re-simulated Greeks difference two independently rounded FP32 paths: per path
    sqrt(2) S0 EPS_X sqrt(N) of noise, averaged over the paths and divided by the
    bump: 1e-4 + 5 sqrt(2) S0 EPS_X sqrt(N) / (sqrt(paths) |bump denominator|)."""
    S0 = model["S0"]
    ex = EPS_X * math.sqrt(steps)
    base = 1e-4 * np.abs(og) + 1e-9
    if name == "gamma":
        n_tent = max(paths * 0.05 * 2 * h * S0, 1.0)
        return base + 5 * S0 * ex * math.sqrt(n_tent) / (paths * (h * S0) ** 2)
    if name in BUMPS:
        den = BUMPS[name](model, h)
        return base + 5 * math.sqrt(2) * S0 * ex / (math.sqrt(paths) * den)
    return base


GREEK_CASES = [
    ("cfg_single", CFG, [100.0], False, 64, 65536, 1, ("delta", "gamma", "vega")),
    ("grid_small", CFG, workloads.strike_grid(), False, 252, 1 << 15, 1, ("delta", "gamma", "vega", "theta", "rho")),
    ("grid_put", CFG, workloads.strike_grid(n=8), True, 64, 1 << 15, 2, ("delta", "gamma", "vega", "theta", "rho")),
    ("all_nine", CFG, [90.0, 100.0, 110.0], False, 32, 1 << 15, 4, tuple(oracle_name for oracle_name in
                                                                          ("delta", "gamma", "vega", "theta", "rho",
                                                                           "kappa", "lrvar", "volvol", "corr"))),
    ("one_sided_v0_zero", dict(CFG, v0=0.0), [100.0], False, 16, 1 << 14, 5, ("vega",)),
    ("one_sided_rho_edge", dict(CFG, rho=-1.0), [100.0], False, 16, 1 << 14, 5, ("corr", "delta")),
    # parameter edges: vol-of-vol near the Black-Scholes limit, mean reversion near zero
    ("small_vol_of_vol", dict(CFG, sigma=0.01), [90.0, 100.0, 110.0], False, 32, 1 << 15, 7,
     ("delta", "gamma", "vega", "theta", "rho", "corr")),
    ("small_kappa", dict(CFG, kappa=1e-3), [90.0, 100.0, 110.0], True, 32, 1 << 15, 8,
     ("delta", "gamma", "vega", "theta", "rho", "lrvar")),
    # the largest strike count the bump-and-revalue kernels take: 8 tiles of 32
    ("strikes_256_max", CFG, np.linspace(60.0, 140.0, 256), False, 16, 1 << 14, 13, ("delta", "gamma", "vega", "rho")),
]

ORACLE_BITS = {"delta": oracle.G_DELTA, "gamma": oracle.G_GAMMA, "vega": oracle.G_VEGA, "theta": oracle.G_THETA,
               "rho": oracle.G_RHO, "kappa": oracle.G_KAPPA, "lrvar": oracle.G_LRVAR, "volvol": oracle.G_VOLVOL,
               "corr": oracle.G_CORR}


@pytest.mark.parametrize("name,model,K,is_put,steps,paths,seed,greeks", GREEK_CASES, ids=[c[0] for c in GREEK_CASES])
def test_fd_greeks_parity(simr, name, model, K, is_put, steps, paths, seed, greeks):
    K = np.asarray(K, dtype=np.float64)
    h = 1e-4
    p, g = simr.greeks_fd(model, _dev(K), is_put, steps, paths, seed, greeks=greeks, rel_bump=h)
    p, g = p.cpu().numpy(), g.cpu().numpy()
    mask = sum(ORACLE_BITS[x] for x in greeks)
    po, go = oracle.greeks_fd(model, K, is_put, steps, paths, seed, h, mask)
    assert np.all(np.abs(p - po) <= 1e-5 * np.abs(po) + _flip_allowance(model, K, is_put, steps, paths, seed) + 1e-12)
    order = sorted(greeks, key=lambda x: ORACLE_BITS[x])
    for j, gname in enumerate(order):
        tol = _greek_tol(gname, go[:, j], h, steps, paths, model)
        err = np.abs(g[:, j] - go[:, j])
        assert np.all(err <= tol), (gname, err.max(), (err / np.maximum(np.abs(go[:, j]), 1e-300)).max())


# ----------------------------------------------------------- sharding ----
def test_path_sums_shards_add_up(simr):
    K = workloads.strike_grid(n=16)
    greeks = ("delta", "gamma", "vega", "rho")
    whole = simr.path_sums(CFG, _dev(K), False, 24, 0, 30000, seed=8, greeks=greeks)
    parts = [simr.path_sums(CFG, _dev(K), False, 24, b, n, seed=8, greeks=greeks)
             for b, n in ((0, 10000), (10000, 7777), (17777, 12223))]
    tot = sum(parts)
    assert torch.allclose(tot, whole, rtol=1e-5, atol=1e-9)
    p, se, g = simr.finalize_sums(CFG, K, False, 24, 30000, tot, greeks=greeks)
    pf, gf = simr.greeks_fd(CFG, _dev(K), False, 24, 30000, 8, greeks=greeks)
    assert torch.allclose(p.cpu(), pf.cpu(), rtol=1e-5) and torch.allclose(g.cpu(), gf.cpu(), rtol=1e-4, atol=1e-9)


# ----------------------------------------------------- full-size sample ----
def test_full_size_grid_price_parity(simr):
    w = workloads.grid()
    p, se = simr.price(w.model, _dev(w.strikes), False, w.steps, w.paths, w.seed)
    p = p.cpu().numpy()
    po, _ = oracle.price(w.model, w.strikes, False, w.steps, w.paths, w.seed)
    tol = 1e-5 * np.abs(po) + _flip_allowance(w.model, w.strikes, False, w.steps, w.paths, w.seed)
    assert np.all(np.abs(p - po) <= tol), np.max(np.abs(p - po) / np.abs(po))


# ---------------------------------------------------------------- errors ----
@pytest.mark.parametrize("bad", [dict(sigma=0.0), dict(T=0.0), dict(S0=-1.0), dict(rho=1.5), dict(kappa=0.0),
                                 dict(v0=-0.01), dict(theta=float("nan"))])
def test_invalid_model_rejected(simr, bad):
    with pytest.raises(simr.SimrError) as e:
        simr.price(dict(CFG, **bad), [100.0], False, 8, 100, 1)
    assert e.value.code == -1


def test_invalid_sizes_rejected(simr):
    for kw in (dict(steps=0), dict(paths=0)):
        args = dict(steps=8, paths=100)
        args.update(kw)
        with pytest.raises(simr.SimrError):
            simr.price(CFG, [100.0], False, args["steps"], args["paths"], 1)
    with pytest.raises(simr.SimrError):
        simr.price(CFG, [100.0, -5.0], False, 8, 100, 1)        # host strike checked on the host
    with pytest.raises(simr.SimrError):
        simr.greeks_fd(CFG, [100.0], False, 8, 100, 1, greeks=0)
    # one strike past each entry point's maximum
    for call, n in ((lambda K: simr.price(CFG, K, False, 8, 100, 1), 1025),
                    (lambda K: simr.greeks_fd(CFG, K, False, 8, 100, 1), 257),
                    (lambda K: simr.greeks_adjoint(CFG, K, False, 8, 100, 1), 257)):
        with pytest.raises(simr.SimrError) as e:
            call(_dev(np.full(n, 100.0)))
        assert e.value.code == -1


def test_device_strike_error_reported_by_sync(simr):
    K = _dev([100.0, -1.0])
    p, _ = simr.price(CFG, K, False, 8, 256, 1)
    with pytest.raises(simr.SimrError) as e:
        simr.sync(0)
    assert e.value.code == -1
    assert math.isnan(p[1].item()) and math.isfinite(p[0].item())
    simr.sync(0)  # status was cleared


def test_injected_faults_are_reported_and_the_context_survives(simr):
    # host-side fault injection: the call that meets the fault fails with its
    # status, nothing reaches the GPU for it, and the next call is unaffected
    K = _dev([90.0, 100.0, 110.0])
    ref = simr.price(CFG, K, False, 32, 4096, 3)[0]
    simr.inject_fault("launch")
    with pytest.raises(simr.SimrError) as e:
        simr.price(CFG, K, False, 32, 4096, 3)
    assert e.value.code == -3  # SIMR_ECUDA
    torch.testing.assert_close(simr.price(CFG, K, False, 32, 4096, 3)[0], ref, rtol=0, atol=0)
    simr.inject_fault("alloc")
    with pytest.raises(simr.SimrError) as e:
        simr.greeks_adjoint(CFG, K, False, 32, 4096, 3)
    assert e.value.code == -2  # SIMR_ENOMEM
    a = simr.greeks_adjoint(CFG, K, False, 32, 4096, 3)
    torch.testing.assert_close(a[0], ref, rtol=1e-6, atol=1e-9)
    for name, call in (("launch", lambda: simr.batch([dict(model=CFG, K=100.0, is_put=False, steps=8, paths=999)])),
                       ("launch", lambda: simr.lsm_price(CFG, 100.0, True, 16, 4, 999, 1)),
                       ("alloc", lambda: simr.basket_price([CFG, CFG], np.eye(2), [0.5, 0.5], [100.0]))):
        simr.inject_fault(name)
        with pytest.raises(simr.SimrError):
            call()
        call()
    simr.inject_fault("off")


def test_tiny_paths_reproduce_the_oracle_fixture(simr):
    # the oracle's stored terminal states at 1 and 2 steps, 8 paths
    # (tests/golden/tiny_paths.txt): the GPU's per-path states within FP32 rounding
    import os

    models = {"standard": CFG, "vol_of_vol_0.9": HARD}
    bound = {"standard": 2e-6, "vol_of_vol_0.9": 8e-6}  # xf x (1.5e-7 sqrt(N) + 1e-6) of the per-path test
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "tiny_paths.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, steps, p, x, v = line.split()
                rows.setdefault((name, int(steps)), []).append((int(p), float(x), float(v)))
    assert len(rows) == 4
    for (name, steps), vals in rows.items():
        x, v = simr.paths_terminal(models[name], steps, 0, 8, seed=7)
        x, v = x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
        for p, xe, ve in vals:
            assert abs(x[p] - xe) <= bound[name], (name, steps, p, x[p], xe)
            assert abs(v[p] - ve) <= 1e-6 * max(ve, 0.01), (name, steps, p, v[p], ve)
