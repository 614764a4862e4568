"""Longstaff-Schwartz (simr_lsm_price) on the GPU against the FP64 oracle (oracle/lsm.py).

The GPU's path states are FP32 and the oracle's FP64, so an exercise decision
(payoff > fitted continuation) can go the other way where the two are nearly
equal; such a flip changes that path's cash flow, and through the later
regressions the fits a little.  The checks therefore are:
  * exercise dates: equal on all but a small fraction of paths, and every path
    that differs had an oracle decision margin |h - C| below MARGIN_TOL x K at
    the first date where the two sides parted;
  * price: after the exact (signed) effect of the differing paths -- their
    oracle cash flows at the GPU's exercise date minus at the oracle's -- the
    difference is within 1e-5 of the price;
  * regressions: the fitted continuation values of the two sides' coefficients,
    on the oracle's in-the-money states, agree to FIT_TOL x K, plus the exact
    effect of the paths whose spot lies within AMBIGUOUS x K of the strike (in
    the money on one side only, so in one side's regression only): the oracle's
    fit with those paths' membership toggled, against its own.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import lsm as olsm
import workloads

pytestmark = pytest.mark.gpu

BASE = dict(workloads.BASE_MODEL)
HARD = dict(BASE, sigma=0.9, rho=-0.3, kappa=0.5, v0=0.09, theta=0.04)
# x K: a flip needs |h - C| within the two sides' difference in h - C, i.e. the
# FP32 path error of S (~1e-6 S after a few hundred steps) plus the fit difference
MARGIN_TOL = 1e-4
# x K, median over a date's in-the-money states: the fits differ by the FP32 error
# of the 21 regression sums (~1e-7 relative each, order-one Gram entries in the
# kernel's scaled coordinates) times the fit's sensitivity (measured ~4e-8)
FIT_TOL = 1e-6
FLIP_FRACTION = 1e-3
# x K: spots this close to the strike may be in the money on one side only (FP32
# path error ~1e-6 relative after a few hundred steps)
AMBIGUOUS = 1e-5


@pytest.fixture(scope="module")
def simr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_12111_gb300 as simr

    simr.load()
    return simr


CASES = [
    # name, model, K, is_put, steps, every, paths, seed
    ("put_atm_16_dates", BASE, 100.0, True, 64, 4, 1 << 14, 1),
    ("put_itm_every_step", BASE, 110.0, True, 50, 1, 8192, 2),
    ("call_otm", BASE, 90.0, False, 32, 2, 8192, 3),
    ("put_feller_violated", HARD, 100.0, True, 48, 3, 1 << 14, 4),
    ("ragged_tail_odd_steps", BASE, 105.0, True, 33, 11, 5003, 5),
    ("deep_itm_put", BASE, 130.0, True, 40, 2, 6000, 6),
]


def _check_against_oracle(simr, model, K, is_put, steps, every, paths, seed):
    p, se, beta, stop = simr.lsm_price(model, K, is_put, steps, every, paths, seed, with_beta=True, with_stop=True)
    p, se = float(p.item()), float(se.item())
    beta = beta.cpu().numpy()
    g = stop.cpu().numpy().astype(np.int64)
    ref = olsm.lsm(model, K, is_put, steps, every, paths, seed, keep_targets=True)
    o = ref.stop
    n_ex = steps // every

    # regressions ran at the same dates
    np.testing.assert_array_equal(np.isnan(beta[:, 0]), np.isnan(ref.beta[:, 0]))

    # exercise dates
    diff = np.nonzero(g != o)[0]
    assert diff.size <= max(3, FLIP_FRACTION * paths), f"{diff.size} of {paths} paths stop elsewhere"
    for i in diff:
        d = min(x for x in (g[i], o[i]) if x >= 0)
        ambiguous = np.any(np.abs(ref.S[i, d:] - K) <= AMBIGUOUS * K)
        assert ref.margin[i, d] < MARGIN_TOL * K or ambiguous, (i, g[i], o[i], ref.margin[i, d])

    # price: the differing paths' exact effect, then 1e-5
    disc = np.exp(-model["r"] * ref.t)
    h = olsm.payoff(ref.S, K, is_put)
    cf_g = np.where(g >= 0, h[np.arange(paths), np.maximum(g, 0)] * disc[np.maximum(g, 0)], 0.0)
    cf_o = np.where(o >= 0, ref.cash * disc[np.maximum(o, 0)], 0.0)
    shift = float(np.sum(cf_g[diff] - cf_o[diff])) / paths
    assert abs(p - ref.price - shift) <= 1e-5 * ref.price + 1e-12, (p, ref.price, shift)
    assert se == pytest.approx(ref.stderr, rel=1e-3, abs=1e-9)

    # fitted continuation values on the oracle's in-the-money states
    w = olsm.basis_scale(model)
    for j in range(n_ex - 1):
        if np.isnan(ref.beta[j, 0]):
            continue
        itm = h[:, j] > 0
        Phi = olsm.basis(ref.S[itm, j], ref.v[itm, j], K, w)
        dC = np.abs(Phi @ (beta[j] - ref.beta[j]))
        allow = 0.0
        amb = np.abs(ref.S[:, j] - K) <= AMBIGUOUS * K
        if diff.size == 0 and amb.any():
            alt = itm ^ amb
            Pa = olsm.basis(ref.S[alt, j], ref.v[alt, j], K, w)
            ba, _ = olsm.solve_normal(Pa.T @ Pa, Pa.T @ ref.Y[alt, j])
            allow = float(np.median(np.abs(Phi @ (ba - ref.beta[j]))))
        elif diff.size:
            # targets of the differing paths moved by at most their cash-flow change (at t_j)
            allow = 10 * math.exp(model["r"] * model["T"]) * np.sum(np.abs(cf_g[diff] - cf_o[diff])) / itm.sum()
        assert np.median(dC) <= FIT_TOL * K + 2 * allow, (j, np.median(dC), allow)
    return p, ref


@pytest.mark.parametrize("name,model,K,is_put,steps,every,paths,seed", CASES, ids=[c[0] for c in CASES])
def test_lsm_matches_oracle(simr, name, model, K, is_put, steps, every, paths, seed):
    _check_against_oracle(simr, model, K, is_put, steps, every, paths, seed)


def test_single_exercise_date_equals_price_kernel(simr):
    # one date (the maturity): the same per-path payoffs as simr_price; the two
    # kernels group the FP32 partial sums differently (per-thread runs and 32-lane
    # warp sums here, 64-path warp sums there), which moves the FP64 total by
    # ~1e-7 / sqrt(groups) relative
    K = torch.tensor([97.0], dtype=torch.float64, device="cuda")
    for is_put in (False, True):
        p, se, beta, stop = simr.lsm_price(BASE, 97.0, is_put, 64, 64, 30000, 9, with_beta=True, with_stop=True)
        pe, see = simr.price(BASE, K, is_put, 64, 30000, 9)
        torch.testing.assert_close(p, pe, rtol=1e-8, atol=1e-12)
        torch.testing.assert_close(se, see, rtol=1e-7, atol=1e-12)
        assert torch.isnan(beta).all()
        assert set(np.unique(stop.cpu().numpy())) <= {-1, 0}


def test_lsm_deterministic_and_host_outputs(simr):
    a = simr.lsm_price(BASE, 100.0, True, 32, 2, 10000, 3, with_beta=True, with_stop=True)
    b = simr.lsm_price(BASE, 100.0, True, 32, 2, 10000, 3, with_beta=True, with_stop=True, device="cpu")
    assert a[0].item() == b[0].item() and a[1].item() == b[1].item()
    np.testing.assert_array_equal(a[2].cpu().numpy(), b[2].numpy())
    np.testing.assert_array_equal(a[3].cpu().numpy(), b[3].numpy())


def test_lsm_full_size_properties(simr):
    # 2^20 paths, 252 steps, an exercise date every step: consistency properties
    m = dict(BASE)
    p, se, beta, stop = simr.lsm_price(m, 100.0, True, 252, 1, 1 << 20, 1, with_beta=True, with_stop=True)
    pe, see = simr.price(m, torch.tensor([100.0], dtype=torch.float64, device="cuda"), True, 252, 1 << 20, 1)
    assert p.item() > pe.item() + 5 * se.item()             # early-exercise premium
    assert 0 < se.item() < 0.02
    st = stop.cpu().numpy()
    assert st.min() >= -1 and st.max() <= 251
    assert np.isnan(beta[-1].cpu().numpy()).all() and not np.isnan(beta[:-1].cpu().numpy()).any()
    # a sample of paths against the oracle's states: the exercise rule applied to the
    # oracle's own states with the GPU's coefficients reproduces the GPU's stops
    n = 2000
    S, v = oracle.states(m, 252, 1, 1, 0, n)
    h = olsm.payoff(S, 100.0, True)
    w = olsm.basis_scale(m)
    b = beta.cpu().numpy()
    stop_cpu = np.where(h[:, -1] > 0, 251, -1)
    for j in range(250, -1, -1):
        C = olsm.basis(S[:, j], v[:, j], 100.0, w) @ b[j]
        ex = (h[:, j] > 0) & (h[:, j] > C)
        stop_cpu[ex] = j
    agree = np.mean(stop_cpu == st[:n])
    assert agree > 0.995, agree


def _perturbed_oracle_spread(model, K, is_put, steps, every, paths, seed, n=3, eps=1e-7):
    """The oracle's own sensitivity: its price and exercise dates with S and v
    perturbed by eps relative (the size of the FP32 path error), n draws.
    Returns (the unperturbed result, max |price change|, max fraction of paths
    whose date changed)."""
    base = olsm.lsm(model, K, is_put, steps, every, paths, seed)
    orig = olsm.states
    dp, ds = 0.0, 0.0
    for k in range(n):
        rng = np.random.default_rng(100 + k)

        def noisy(*a, **kw):
            S, v = orig(*a, **kw)
            return S * (1 + eps * rng.standard_normal(S.shape)), v * (1 + eps * rng.standard_normal(v.shape))

        olsm.states = noisy
        try:
            r = olsm.lsm(model, K, is_put, steps, every, paths, seed)
        finally:
            olsm.states = orig
        dp = max(dp, abs(r.price - base.price))
        ds = max(ds, float(np.mean(r.stop != base.stop)))
    return base, dp, ds


def test_lsm_large_matches_oracle_within_its_own_sensitivity(simr):
    # With tens of thousands of paths a decision somewhere sits within rounding of
    # its boundary; its flip moves every earlier fit a little and flips more
    # near-boundary decisions (the oracle does the same under 1e-7 noise: ~1e-4 of
    # the price at 2^16 paths).  The GPU must stay within a few times that spread.
    args = (BASE, 100.0, True, 64, 2, 1 << 16, 4)
    ref, dp, ds = _perturbed_oracle_spread(*args)
    p, _, _, stop = simr.lsm_price(*args, with_stop=True)
    assert abs(p.item() - ref.price) <= 4 * dp + 1e-5 * ref.price, (p.item(), ref.price, dp)
    assert np.mean(stop.cpu().numpy() != ref.stop) <= 4 * ds + 1e-4


@pytest.mark.parametrize("paths", [5003, 1 << 18, 400_000, 1 << 20])
def test_cooperative_sweep_and_per_date_launches_agree(simr, paths, monkeypatch):
    # the backward induction runs as one cooperative launch or as one kernel per
    # date; they group the FP32 partial sums differently, so their fits differ at
    # ~1e-7 -- below the estimator's own sensitivity at large path counts (see
    # above), hence a bound of a small fraction of the standard error there
    args = (BASE, 100.0, True, 64, 2, paths, 4)
    a = simr.lsm_price(*args, with_beta=True, with_stop=True)
    monkeypatch.setenv("SIMR_LSM_SWEEP", "0")
    b = simr.lsm_price(*args, with_beta=True, with_stop=True)
    sa, sb = a[3].cpu().numpy(), b[3].cpu().numpy()
    if paths < 10000:
        assert a[0].item() == pytest.approx(b[0].item(), rel=1e-6)
        assert np.mean(sa != sb) <= 1e-3
    else:
        assert abs(a[0].item() - b[0].item()) <= 0.1 * a[1].item()
        assert np.mean(sa != sb) <= 2e-2
    ba, bb = a[2].cpu().numpy(), b[2].cpu().numpy()
    np.testing.assert_array_equal(np.isnan(ba), np.isnan(bb))


def test_lsm_at_the_maximum_date_count(simr, monkeypatch):
    # 8,192 exercise dates (the limit): the sweep's discount table fills 32 KB of
    # shared memory and its grid barrier runs 8,192 times.  With dates this close
    # most paths stay near the exercise boundary for many dates, and the estimator
    # is chaotic at the FP32 path error (3e-8 sqrt(N) relative after N steps): the
    # oracle itself, its states perturbed that much, moves the exercise date of
    # about a third of the paths (measured 0.33-0.36) and the price by up to 0.07.
    # The GPU must stay within that spread, and the sweep agree with the per-date
    # launches.
    args = (dict(BASE, T=2.0), 100.0, True, 8192, 1, 2048, 15)
    ref, dp, ds = _perturbed_oracle_spread(*args, eps=3e-8 * math.sqrt(8192))
    p, se, _, stop = simr.lsm_price(*args, with_stop=True)
    assert abs(p.item() - ref.price) <= 2 * dp + 1e-5 * ref.price, (p.item(), ref.price, dp)
    assert abs(p.item() - ref.price) <= 0.5 * se.item()
    assert np.mean(stop.cpu().numpy() != ref.stop) <= 1.5 * ds + 0.02, ds
    monkeypatch.setenv("SIMR_LSM_SWEEP", "0")
    q = simr.lsm_price(*args)[0].item()
    assert q == pytest.approx(p.item(), rel=1e-6)
    with pytest.raises(simr.SimrError):
        simr.lsm_price(BASE, 100.0, True, 8193, 1, 2048, 15)  # one date past it


def test_lsm_rejects_bad_arguments(simr):
    with pytest.raises(simr.SimrError):
        simr.lsm_price(BASE, 100.0, True, 64, 5, 1000, 1)   # 5 does not divide 64
    with pytest.raises(simr.SimrError):
        simr.lsm_price(BASE, -1.0, True, 64, 4, 1000, 1)
    with pytest.raises(simr.SimrError):
        simr.lsm_price(BASE, 100.0, True, 64, 4, 1, 1)      # one path


def test_barrier_wait_runs_out_and_the_context_survives(simr):
    # fault injection: the next sweep's first grid barrier waits for one block more
    # than the grid holds, so its bounded wait runs out (0.25 s); the blocks leave,
    # the status reports SIMR_ETIMEOUT, and the next valuation on the same context
    # is the normal one
    import time

    args = (BASE, 100.0, True, 32, 2, 1 << 14, 3)
    ref = simr.lsm_price(*args)[0].item()
    simr.sync()
    simr.inject_fault("barrier")
    t0 = time.perf_counter()
    simr.lsm_price(*args)
    with pytest.raises(simr.SimrError) as e:
        simr.sync()
    assert e.value.code == -4, e.value
    assert time.perf_counter() - t0 < 10.0
    assert simr.lsm_price(*args)[0].item() == ref
    simr.sync()  # the status word was cleared
