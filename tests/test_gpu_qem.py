"""QE-M (Andersen's martingale correction) on the GPU against the FP64 oracle's QE-M.

The correction adds lam = ln M - A m per step (a small positive number, computed
without cancellation in FP32), so the per-path and price tolerances are those of
the plain scheme (tests/test_gpu_parity.py); the property the scheme exists for,
E[e^{-rT} S_T] = S0, is checked on the GPU's own paths.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import lsm as olsm
import workloads

pytestmark = pytest.mark.gpu

CFG = dict(workloads.BASE_MODEL)
HARD = dict(S0=100.0, r=0.05, T=1.0, v0=0.09, kappa=1.0, theta=0.04, sigma=0.9, rho=-0.3)
WILD = dict(CFG, sigma=1.0, rho=-0.9, kappa=0.5, T=2.0)  # coarse steps, strong leverage
POS_RHO = dict(CFG, rho=0.5)  # A = K2 + qa > 0
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


@pytest.mark.parametrize("model,steps,n,xf", [(CFG, 64, 8192, 1), (WILD, 8, 8192, 1), (HARD, 64, 8192, 6),
                                              (CFG, 252, 4096, 1)], ids=["cfg", "wild", "hard", "cfg252"])
def test_terminal_states_per_path(simr, model, steps, n, xf):
    with simr.scheme("qem"):
        x, v = simr.paths_terminal(model, steps, 0, n, seed=7)
    x, v = x.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    with oracle.scheme("qem"):
        xo, vo, mg = oracle.terminal(model, steps, 7, 0, n)
    ok = mg > FLIP_MARGIN
    dx = np.abs(x - xo)[ok]
    bound = xf * 1.5e-7 * math.sqrt(steps) + 1e-6
    assert np.quantile(dx, 0.999) < bound, (np.quantile(dx, 0.999), dx.max())
    assert np.mean(dx > bound) <= 0.005


def _flip_allowance(model, K, is_put, steps, paths, seed, option_index=0):
    with oracle.scheme("qem"):
        x, _, mg = oracle.terminal(model, steps, seed, 0, paths, option_index=option_index)
    S = model["S0"] * np.exp(x)
    close = mg < FLIP_MARGIN
    if not close.any():
        return np.zeros(len(K))
    fmax = (np.maximum(K, 0.0) if is_put else np.maximum(S.max() - K, 0.0))
    pay = np.maximum(K[:, None] - S[close][None, :], 0) if is_put else np.maximum(S[close][None, :] - K[:, None], 0)
    return math.exp(-model["r"] * model["T"]) * (pay.sum(axis=1) + close.sum() * fmax) / paths


PRICE_CASES = [
    ("cfg_call", CFG, [100.0], False, 64, 65536, 1),
    ("cfg_grid_put", CFG, workloads.strike_grid(), True, 252, 16384, 3),
    ("wild_grid", WILD, workloads.strike_grid(), False, 8, 65536, 2),
    ("hard", HARD, [80.0, 100.0, 120.0], False, 64, 32768, 5),
    ("ragged", CFG, [95.0, 105.0], True, 33, 1000, 9),
]


@pytest.mark.parametrize("name,model,K,is_put,steps,paths,seed", PRICE_CASES, ids=[c[0] for c in PRICE_CASES])
def test_price_parity(simr, name, model, K, is_put, steps, paths, seed):
    K = np.asarray(K, dtype=np.float64)
    with simr.scheme("qem"):
        p, se = simr.price(model, _dev(K), is_put, steps, paths, seed)
    with oracle.scheme("qem"):
        po, seo = oracle.price(model, K, is_put, steps, paths, seed)
    p, se = p.cpu().numpy(), se.cpu().numpy()
    tol = 1e-5 * np.abs(po) + _flip_allowance(model, K, is_put, steps, paths, seed) + 1e-12
    assert np.all(np.abs(p - po) <= tol), (p - po, tol)
    assert np.all(np.abs(se - seo) <= 1e-4 * seo + 1e-9)


def test_discounted_spot_is_a_martingale_on_the_gpu(simr):
    n = 1 << 21
    with simr.scheme("qem"):
        x, _ = simr.paths_terminal(WILD, 8, 0, n, seed=3, with_variance=False)
    d = math.exp(-WILD["r"] * WILD["T"]) * WILD["S0"] * torch.exp(x.double())
    mean, se = d.mean().item(), d.std().item() / math.sqrt(n)
    assert abs(mean - WILD["S0"]) < 3 * se, (mean, se)


def test_zero_correlation_agrees_with_plain_qe(simr):
    m = dict(CFG, rho=0.0)  # A = 0: the correction vanishes; FP32 evaluation order differs only
    x0, _ = simr.paths_terminal(m, 64, 0, 8192, seed=4)
    with simr.scheme("qem"):
        x1, _ = simr.paths_terminal(m, 64, 0, 8192, seed=4)
    assert (x1 - x0).abs().max().item() < 1e-5


def test_base_path_greeks_match_oracle(simr):
    K = np.array([90.0, 100.0, 110.0])
    with simr.scheme("qem"):
        p, g = simr.greeks_fd(WILD, _dev(K), False, 8, 65536, 6, greeks=("delta", "gamma", "rho"))
    bits = oracle.G_DELTA | oracle.G_GAMMA | oracle.G_RHO
    with oracle.scheme("qem"):
        po, go = oracle.greeks_fd(WILD, K, False, 8, 65536, 6, 1e-4, bits)
    np.testing.assert_allclose(p.cpu().numpy(), po, rtol=1e-5)
    g = g.cpu().numpy()
    np.testing.assert_allclose(g[:, 0], go[:, 0], rtol=1e-4, atol=1e-6)   # delta
    np.testing.assert_allclose(g[:, 2], go[:, 2], rtol=1e-4, atol=1e-5)   # rho
    # gamma: the tent difference of S_T at h = 1e-4 resolves FP32 S_T to ~1e-3 relative
    np.testing.assert_allclose(g[:, 1], go[:, 1], rtol=2e-2, atol=2e-4)


def test_lsm_under_qem_matches_oracle(simr):
    with simr.scheme("qem"):
        p, _, _, stop = simr.lsm_price(WILD, 100.0, True, 16, 2, 8192, 3, with_stop=True)
    with oracle.scheme("qem"):
        ref = olsm.lsm(WILD, 100.0, True, 16, 2, 8192, 3)
    diff = np.nonzero(stop.cpu().numpy() != ref.stop)[0]
    assert diff.size <= 3
    if diff.size == 0:
        assert p.item() == pytest.approx(ref.price, rel=1e-5)


def test_scheme_context_restores_qe(simr):
    # every entry point runs QE-M inside the context and QE again after it
    K = _dev([100.0])
    p_qe, _ = simr.price(CFG, K, False, 16, 4096, 1)
    with simr.scheme("qem"):
        p_qem, _ = simr.price(CFG, K, False, 16, 4096, 1)
    p_after, _ = simr.price(CFG, K, False, 16, 4096, 1)
    assert torch.equal(p_after, p_qe) and not torch.equal(p_qem, p_qe)


# ---------------------------------------------------------------------------
# Re-simulated bump-and-revalue Greeks under QE-M: every bumped scenario runs the
# QE-M step on its own moments and A, with the deltas of its constants (r dt, qa,
# K2, A and the plain QE ones) to the base scenario's entering as separate FP64-
# derived sums, and step 0 on FP64 first-step constants (r dt - qa (v0 + m0) -
# lam(v0)) -- the plain scheme's common-random-number construction.  Against the
# QE-M oracle's bump-and-revalue (each bumped model simulated in FP64), with the
# plain scheme's per-Greek tolerances (tests/test_gpu_parity.py).
# ---------------------------------------------------------------------------
# The 8-step coarse case keeps the Feller condition (2 kappa theta >= sigma^2):
# with vol-of-vol 1 (WILD) a bumped scenario's paths cross QE branch and atom
# thresholds that the FP64 oracle's do not, and each such path moves a
# difference quotient by its payoff change over the bump (measured: 0.6% on
# d/dkappa), which no rounding bound covers -- the adjoint tests above flag and
# bound such paths instead.
COARSE = dict(CFG, rho=-0.9, T=2.0)
ALL_NINE = ("delta", "gamma", "vega", "theta", "rho", "kappa", "lrvar", "volvol", "corr")
QEM_FD_CASES = [
    ("cfg_all_nine", CFG, [90.0, 100.0, 110.0], False, 32, 1 << 15, 4, ALL_NINE),
    ("grid_put_252", CFG, workloads.strike_grid(n=8), True, 252, 1 << 15, 2,
     ("delta", "gamma", "vega", "theta", "rho")),
    ("coarse_all_nine", COARSE, [90.0, 100.0, 110.0], False, 8, 1 << 15, 3, ALL_NINE),
    ("positive_rho_grid", POS_RHO, workloads.strike_grid(), False, 64, 1 << 15, 5,
     ("vega", "theta", "kappa", "lrvar", "volvol", "corr")),
    ("one_sided_v0_zero", dict(CFG, v0=0.0), [100.0], False, 16, 1 << 14, 5, ("vega", "corr")),
    ("seven_in_pairs", COARSE, [90.0, 100.0, 110.0], True, 16, 1 << 15, 6,
     ("delta", "vega", "rho", "kappa", "lrvar", "volvol", "corr")),
    ("one_step_ragged_all_nine", CFG, [95.0, 100.5, 105.0], True, 1, 999, 7, ALL_NINE),
    ("one_step_in_pairs", CFG, [100.0], False, 1, 4097, 8, ("delta", "gamma", "vega", "theta", "rho")),
]


@pytest.mark.parametrize("name,model,K,is_put,steps,paths,seed,greeks", QEM_FD_CASES,
                         ids=[c[0] for c in QEM_FD_CASES])
def test_fd_greeks_match_qem_oracle(simr, name, model, K, is_put, steps, paths, seed, greeks):
    from test_gpu_parity import ORACLE_BITS, _greek_tol

    K = np.asarray(K, dtype=np.float64)
    h = 1e-4
    with simr.scheme("qem"):
        p, g = simr.greeks_fd(model, _dev(K), is_put, steps, paths, seed, greeks=greeks, rel_bump=h)
    p, g = p.cpu().numpy(), g.cpu().numpy()
    mask = sum(ORACLE_BITS[x] for x in greeks)
    with oracle.scheme("qem"):
        po, go = oracle.greeks_fd(model, K, is_put, steps, paths, seed, h, mask)
    assert np.all(np.abs(p - po) <= 1e-5 * np.abs(po) + _flip_allowance(model, K, is_put, steps, paths, seed)
                  + 1e-12)
    order = sorted(greeks, key=lambda x: ORACLE_BITS[x])
    for j, gname in enumerate(order):
        tol = _greek_tol(gname, go[:, j], h, steps, paths, model)
        err = np.abs(g[:, j] - go[:, j])
        assert np.all(err <= tol), (gname, err.max(), (err / np.maximum(np.abs(go[:, j]), 1e-300)).max())


def test_qem_scenario_pairs_equal_single_scenarios(simr):
    # 5 and 11 scenarios run in packed pairs, other counts one scenario at a time
    # (the dynamic kernel): lane for lane the same operations, so the Greeks both
    # kernels compute are equal bit for bit
    K = _dev([90.0, 100.0, 110.0])
    with simr.scheme("qem"):
        _, g5 = simr.greeks_fd(COARSE, K, False, 16, 20000, 3, greeks=("vega", "theta"))        # 5: pairs
        _, g7 = simr.greeks_fd(COARSE, K, False, 16, 20000, 3, greeks=("vega", "theta", "corr"))  # 7: dynamic
        _, g11 = simr.greeks_fd(COARSE, K, False, 16, 20000, 3,
                                greeks=("vega", "theta", "kappa", "lrvar", "volvol"))             # 11: pairs
        _, g13 = simr.greeks_fd(COARSE, K, False, 16, 20000, 3,
                                greeks=("vega", "theta", "kappa", "lrvar", "volvol", "corr"))     # 13: dynamic
    torch.testing.assert_close(g5, g7[:, :2], rtol=0, atol=0)
    torch.testing.assert_close(g11, g13[:, :5], rtol=0, atol=0)


def test_qem_fd_differs_from_qe_fd(simr):
    # the bumped scenarios took the QE-M step: their Greeks move with the scheme
    K = _dev([90.0, 100.0, 110.0])
    greeks = ("vega", "kappa", "corr")
    _, g0 = simr.greeks_fd(WILD, K, False, 8, 1 << 15, 3, greeks=greeks)
    with simr.scheme("qem"):
        _, g1 = simr.greeks_fd(WILD, K, False, 8, 1 << 15, 3, greeks=greeks)
    assert (g1 - g0).abs().max().item() > 1e-3 * g0.abs().max().item()


def test_qem_adjoint_agrees_with_qem_bump_and_revalue(simr):
    # pathwise vs CRN finite differences, both under QE-M on the GPU (the plain
    # scheme's test of the same name): differences only from branch switches
    K = _dev([90.0, 100.0, 110.0])
    with simr.scheme("qem"):
        _, _, g = simr.greeks_adjoint(CFG, K, False, 64, 1 << 17, 11, ckpt_every=16)
        _, f = simr.greeks_fd(CFG, K, False, 64, 1 << 17, 11,
                              greeks=("delta", "vega", "rho", "kappa", "lrvar", "volvol", "corr"), rel_bump=1e-4)
    g, f = g.cpu().numpy(), f.cpu().numpy()
    for ca, cf in [(0, 0), (1, 1), (6, 2), (2, 3), (3, 4), (4, 5), (5, 6)]:
        np.testing.assert_allclose(g[:, ca], f[:, cf], rtol=2e-2, atol=2e-3 * max(np.abs(f[:, cf]).max(), 1.0))


def test_qem_path_sums_shards_add_up(simr):
    K = workloads.strike_grid(n=16)
    greeks = ("delta", "gamma", "vega", "rho", "corr")
    with simr.scheme("qem"):
        whole = simr.path_sums(CFG, _dev(K), False, 24, 0, 30000, seed=8, greeks=greeks)
        parts = [simr.path_sums(CFG, _dev(K), False, 24, b, n, seed=8, greeks=greeks)
                 for b, n in ((0, 10000), (10000, 7777), (17777, 12223))]
        _, gf = simr.greeks_fd(CFG, _dev(K), False, 24, 30000, 8, greeks=greeks)
    tot = sum(parts)
    assert torch.allclose(tot, whole, rtol=1e-5, atol=1e-9)
    _, _, g = simr.finalize_sums(CFG, K, False, 24, 30000, tot, greeks=greeks)
    assert torch.allclose(g.cpu(), gf.cpu(), rtol=1e-4, atol=1e-9)


# ---------------------------------------------------------------------------
# The pathwise adjoint under QE-M: the reverse step adds the derivatives of the
# correction lam = ln M - A m (through m, s^2 and A) and of the constants qa, K2
# and A = K2 + qa in rho, kappa and sigma; steps where M does not exist take the
# plain step's derivatives.  The checker is the plain scheme's
# (tests/test_gpu_adjoint.py: oracle-only kink and decision allowances, the
# unflagged bulk strictly, the per-path quantile), run with both sides under QE-M.
# A positive rho makes A positive (the correction's M then grows with A); the
# coarse 8-step case with rho = -0.9 is where the correction is largest.  Bounds
# as in the plain scheme's cases; measured on a GB300: the Greeks' errors reach
# at most 0.08 of their tolerance (the stress case with vol-of-vol 0.9: 0.004),
# the positive-rho grid's kink allowance 3.5e-3 of a column (its far strikes'
# columns are small), the 8-step case flags 1.6% of its paths (allowance 0.30
# of a column) and its unflagged bulk meets the strict 1e-4.
# ---------------------------------------------------------------------------
QEM_ADJ_CASES = [
    ("single", CFG, [100.0], False, 64, 65536, 1, 16, 1e-3, 0.0, 2e-3),
    ("grid_put_252", CFG, workloads.strike_grid(n=8), True, 252, 16384, 2, 0, 1e-3, 0.0, 2e-3),
    ("positive_rho_grid", POS_RHO, workloads.strike_grid(), False, 64, 16384, 3, 8, 1e-3, 0.0, 5e-3),
    ("wild_coarse", WILD, [90.0, 100.0, 110.0], False, 8, 65536, 4, 2, 1e-3, 0.03, 0.5),
    ("hard_exp_branch", HARD, [90.0, 100.0, 110.0], False, 64, 16384, 5, 8, 5e-3, 0.08, 2.5, 1e-3),
    ("odd_steps_one_segment", CFG, [95.0, 105.0], True, 33, 4097, 6, 34, 1e-3, 0.0, 2e-3),
    # 40 strikes (a ragged second 32-strike tile), 7 steps, 1,000 paths (a ragged last warp)
    ("ragged_40_strikes", CFG, workloads.strike_grid(n=40), True, 7, 1000, 9, 2, 1e-3, 0.0, 2e-2),
    ("one_step", COARSE, [100.0], False, 1, 2048, 10, 2, 1e-3, 0.0, 2e-3),
]


@pytest.mark.parametrize("case", QEM_ADJ_CASES, ids=[c[0] for c in QEM_ADJ_CASES])
def test_adjoint_matches_qem_oracle(simr, case):
    from test_gpu_adjoint import check_adjoint

    with simr.scheme("qem"), oracle.scheme("qem"):
        check_adjoint(simr, *case[1:])


@pytest.mark.parametrize("case_id", ["small_vol_of_vol", "small_kappa", "zero_variance"])
def test_adjoint_at_parameter_edges_under_qem(simr, case_id):
    # the plain scheme's parameter edges (tests/test_gpu_adjoint.py) under QE-M; at
    # v0 = theta = 0 every step has a zero mean, where M = 1 and only -A m of lam moves
    from test_gpu_adjoint import EDGE_CASES, check_adjoint

    case = next(c for c in EDGE_CASES if c[0] == case_id)
    with simr.scheme("qem"), oracle.scheme("qem"):
        check_adjoint(simr, *case[1:])


def test_adjoint_price_is_the_qem_price(simr):
    K = _dev(workloads.strike_grid())
    with simr.scheme("qem"):
        p1, _ = simr.price(CFG, K, False, 100, 30000, 9)
        p2, _, _ = simr.greeks_adjoint(CFG, K, False, 100, 30000, 9, ckpt_every=10)
    torch.testing.assert_close(p1, p2, rtol=1e-6, atol=1e-9)
    p0, _, _ = simr.greeks_adjoint(CFG, K, False, 100, 30000, 9, ckpt_every=10)
    assert not torch.equal(p0, p2)  # the scheme reached the adjoint kernel


def test_qem_checkpoints_and_segments_do_not_change_results(simr):
    # shared-memory segments at several intervals and global-memory segments
    # (one segment of 200 steps) give the same results bit for bit
    K = _dev(workloads.strike_grid())
    with simr.scheme("qem"):
        ref = simr.greeks_adjoint(WILD, K, False, 200, 5003, 11, ckpt_every=16)
        for k in (2, 50, 150, 200, 0):
            got = simr.greeks_adjoint(WILD, K, False, 200, 5003, 11, ckpt_every=k)
            for a, b in zip(got, ref):
                torch.testing.assert_close(a, b, rtol=0, atol=0)
        K1 = _dev([100.0])
        r1 = simr.greeks_adjoint(WILD, K1, True, 64, 4096, 2, ckpt_every=4)
        g1 = simr.greeks_adjoint(WILD, K1, True, 64, 4096, 2, ckpt_every=64)
    for a, b in zip(g1, r1):
        torch.testing.assert_close(a, b, rtol=0, atol=0)


def test_qem_autograd_function_backward(simr):
    params = torch.tensor([100.0, 0.04, 1.5, 0.04, 0.3, -0.7, 0.05], dtype=torch.float64, requires_grad=True)
    K = _dev(workloads.strike_grid(n=8))
    with simr.scheme("qem"):
        price = simr.heston_price(params, K, 1.0, False, 64, 20000, 3, 16)
        w = torch.linspace(1.0, 2.0, 8, dtype=torch.float64, device="cuda")
        (price * w).sum().backward()
        _, _, jac = simr.greeks_adjoint(dict(CFG), K, False, 64, 20000, 3, ckpt_every=16)
    torch.testing.assert_close(params.grad, (w @ jac).cpu(), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------
# The batched book under QE-M: every option's log-spot steps take the correction
# (price books through the paired QE-M step, adjoint books through the QE-M
# reverse step), so option i equals simr_price / simr_greeks_adjoint under QE-M
# with option_index i up to the order of the FP64 additions.
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_book():
    return workloads.book(n_options=40, seed=5, steps_range=(1, 96), paths_range=(1, 20000))


def _k(o):
    return torch.tensor([o["K"]], dtype=torch.float64, device="cuda")


def test_qem_book_prices_equal_per_option_calls(simr, small_book):
    with simr.scheme("qem"):
        p, se, _ = simr.batch(small_book, seed=9)
        for i, o in enumerate(small_book):
            pi, si = simr.price(o["model"], _k(o), o["is_put"], o["steps"], o["paths"], 9, option_index=i)
            torch.testing.assert_close(p[i:i + 1], pi, rtol=1e-12, atol=1e-12)
            torch.testing.assert_close(se[i:i + 1], si, rtol=1e-9, atol=1e-12)
    p0, _, _ = simr.batch(small_book, seed=9)
    assert not torch.equal(p0, p)  # the plain scheme's book differs


def test_qem_book_adjoint_equals_per_option_calls(simr, small_book):
    with simr.scheme("qem"):
        p, _, g = simr.batch(small_book, seed=4, adjoint=True)
        for i, o in enumerate(small_book):
            pi, _, gi = simr.greeks_adjoint(o["model"], _k(o), o["is_put"], o["steps"], o["paths"], 4, ckpt_every=0,
                                            option_index=i)
            torch.testing.assert_close(p[i:i + 1], pi, rtol=1e-12, atol=1e-12)
            torch.testing.assert_close(g[i:i + 1], gi, rtol=1e-9, atol=1e-9)


def test_qem_book_long_options_use_shared_segments(simr):
    book = workloads.book(n_options=5, seed=8, steps_range=(1100, 1300), paths_range=(300, 2000))
    with simr.scheme("qem"):
        p, _, g = simr.batch(book, seed=2, adjoint=True)
        for i, o in enumerate(book):
            pi, _, gi = simr.greeks_adjoint(o["model"], _k(o), o["is_put"], o["steps"], o["paths"], 2, ckpt_every=0,
                                            option_index=i)
            torch.testing.assert_close(p[i:i + 1], pi, rtol=1e-12, atol=1e-12)
            torch.testing.assert_close(g[i:i + 1], gi, rtol=1e-9, atol=1e-9)


def test_qem_book_kernel_shapes_agree(simr, small_book):
    with simr.scheme("qem"):
        for adjoint in (False, True):
            ref = simr.batch(small_book, seed=6, adjoint=adjoint, variant=0)
            got = simr.batch(small_book, seed=6, adjoint=adjoint, variant=1)
            for a, b in zip(got, ref):
                if a is not None:
                    torch.testing.assert_close(a, b, rtol=0, atol=0)
        with pytest.raises(simr.SimrError):
            simr.batch(small_book, seed=6, variant=2)  # price books under QE-M have two shapes


def test_qem_book_sample_matches_oracle(simr, small_book):
    with simr.scheme("qem"):
        p, _, g = simr.batch(small_book, seed=7, adjoint=True)
    p, g = p.cpu().numpy(), g.cpu().numpy()
    for i in (0, 7, 19, 33):
        o = small_book[i]
        K = np.array([o["K"]])
        with oracle.scheme("qem"):
            po, _ = oracle.price(o["model"], K, o["is_put"], o["steps"], o["paths"], 7, option_index=i)
            _, go = oracle.adjoint(o["model"], K, o["is_put"], o["steps"], o["paths"], 7, option_index=i)
        tol = 1e-5 * abs(po[0]) + _flip_allowance(o["model"], K, o["is_put"], o["steps"], o["paths"], 7, i)[0] + 1e-9
        assert abs(p[i] - po[0]) <= tol, (i, p[i], po[0])
        # the Greeks to 1e-3 of the option's largest sensitivity (paths near a strike
        # or a branch threshold can move a few paths' terms: the full parity is the
        # adjoint tests' above)
        assert np.all(np.abs(g[i] - go[0]) <= 1e-3 * np.abs(go[0]).max() + 1e-4 * np.abs(go[0])), (i, g[i], go[0])


def test_full_size_grid_price_parity_under_qem(simr):
    # the bench workload's size (252 steps x 2^20 paths x 32 strikes) under QE-M
    w = workloads.grid()
    with simr.scheme("qem"):
        p, se = simr.price(w.model, _dev(w.strikes), False, w.steps, w.paths, w.seed)
    with oracle.scheme("qem"):
        po, seo = oracle.price(w.model, w.strikes, False, w.steps, w.paths, w.seed)
    p, se = p.cpu().numpy(), se.cpu().numpy()
    tol = 1e-5 * np.abs(po) + _flip_allowance(w.model, w.strikes, False, w.steps, w.paths, w.seed) + 1e-12
    assert np.all(np.abs(p - po) <= tol), (np.abs(p - po) / np.abs(po)).max()
    assert np.all(np.abs(se - seo) <= 1e-4 * seo + 1e-9)


def test_full_size_adjoint_under_qem_checkpoint_every_16(simr):
    # config 2's adjoint workload (252 x 2^20 x 32 strikes, a checkpoint every 16
    # steps) under QE-M, every column against the QE-M oracle's reverse mode
    from test_gpu_adjoint import check_adjoint

    with simr.scheme("qem"), oracle.scheme("qem"):
        check_adjoint(simr, CFG, workloads.strike_grid(), False, 252, 1 << 20, 1, 16, 1e-3, 0.0, 1e-3)


# Where the correction does not exist (2 A a >= 1 in the quadratic branch, A >= beta
# in the exponential one) the QE-M step takes the plain increment.  One long step
# from a large v0 reaches it on every path: NOEXIST_QUAD in the quadratic branch
# (psi = 0.47, 2 A a = 1.30), NOEXIST_EXP in the exponential branch (the oracle's
# fallback pin).
NOEXIST_QUAD = dict(S0=100.0, r=0.03, T=7.6, v0=1.85, kappa=3.8, theta=0.75, sigma=1.64, rho=0.89)
NOEXIST_EXP = dict(S0=100.0, r=0.05, T=4.0, v0=2.0, kappa=5.0, theta=0.04, sigma=3.0, rho=0.99)


@pytest.mark.parametrize("model", [NOEXIST_QUAD, NOEXIST_EXP], ids=["quadratic", "exponential"])
def test_absent_correction_takes_the_plain_step(simr, model):
    K = _dev([60.0, 100.0, 160.0])
    p0, se0 = simr.price(model, K, False, 1, 40000, 5)
    _, _, g0 = simr.greeks_adjoint(model, K, False, 1, 40000, 5)
    with simr.scheme("qem"):
        p1, se1 = simr.price(model, K, False, 1, 40000, 5)
        _, _, g1 = simr.greeks_adjoint(model, K, False, 1, 40000, 5)
    # the plain step's arithmetic on every path: the same prices bit for bit; the
    # reverse steps differ from the plain ones only in the order of their roundings
    assert torch.equal(p1, p0) and torch.equal(se1, se0)
    torch.testing.assert_close(g1, g0, rtol=1e-6, atol=0.0)
    with oracle.scheme("qem"):
        po, _ = oracle.price(model, K.cpu().numpy(), False, 1, 40000, 5)
    np.testing.assert_allclose(p1.cpu().numpy(), po, rtol=1e-5)


@pytest.mark.parametrize("model", [NOEXIST_QUAD, NOEXIST_EXP], ids=["quadratic", "exponential"])
def test_absent_correction_adjoint_matches_qem_oracle(simr, model):
    from test_gpu_adjoint import check_adjoint

    with simr.scheme("qem"), oracle.scheme("qem"):
        check_adjoint(simr, model, [60.0, 100.0, 160.0], False, 1, 40000, 5, 2, 1e-3, 0.05, 2.5, 1e-3)
