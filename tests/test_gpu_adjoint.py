"""GPU pathwise adjoint vs the FP64 oracle's reverse-mode adjoint on the same Philox counters.

Both differentiate the same discretised path with the branches held fixed, so on
every path where both take the same branches and the same side of the payoff
kink they agree up to FP32 rounding.  Every flag and allowance below comes from
the oracle alone (its states, decision margins and derivatives); the GPU is only
ever the quantity under test.

  * Kink flags: (strike k, path p) with |x_T,p - ln(K_k/S0)| < DX, where the FP32
    path can end on the other side of the strike (DX is 3 times the per-path
    x_T bound of the parity tests, 1.5e-7 sqrt(N) + 1e-6, which the measured
    largest errors -- 0.9e-6 at 64 steps, 3.1e-6 at 252 -- stay within; for
    vol-of-vol far outside the Feller condition, where paths restart from v = 0,
    1e-4).  If the indicator flips, the path's term jumps by its whole value, so
    the allowance is e^{-rT} sum |f'(S_T) S_T dx_T/dq| / P over the flagged
    pairs.  The test also checks that no unflagged pair's GPU indicator differs.
  * Decision flags: paths whose branch decision closest to its threshold (the QE
    branch, or the exponential branch's atom) has a margin below 1e-3.  FP32 can
    take the other side there, and short of that it resolves the step poorly (a
    small logarithm just above the atom, whose inputs an FP32 state knows to
    ~1e-6); the oracle computes the derivative of the path with that decision
    taken the other way (oracle.path_grad_flip, pinned by finite differences in
    the CPU suite), and the allowance is e^{-rT} sum |term(flipped) - term| / P
    over those paths.  No decision of the standard model comes within 1e-2 of
    its threshold.
  * Greeks: |GPU - oracle| <= 1e-4 |oracle| + 1e-4 max|column| (columns that
    change sign across the strikes) + the two allowances; the flagged fractions
    and the allowances themselves are bounded per case.
  * The unflagged bulk, strictly: the GPU's per-path terms (simr_paths_adjoint,
    the same device code as the reduction) summed over the paths no flag
    touches equal the oracle's to 1e-4 (standard model; 1e-3 in the stress case
    with vol-of-vol 0.9, whose FP32 state resolves its many near-zero variances
    to ~1e-6 relative), plus 1e-5 of the column's largest sum.
  * Per path: 99.9% of the unflagged paths' derivatives agree to pq relative.
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
DECISION_MARGIN = 1e-3


@pytest.fixture(scope="module")
def simr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_12111_gb300 as simr

    simr.load()
    return simr


def _dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


def _kink_dx(model, steps):
    feller = 2.0 * model["kappa"] * model["theta"] >= model["sigma"] ** 2
    return 3.0 * (1.5e-7 * math.sqrt(steps) + 1e-6) if feller else 1e-4


def _strike_terms(model, K, is_put, x, g):
    """Per-path adjoint terms of one strike, [n_paths, 7] (before the discount and the -T P of r)."""
    S = model["S0"] * np.exp(x)
    fp = np.where(S < K, -1.0, 0.0) if is_put else np.where(S > K, 1.0, 0.0)
    w = fp * S
    return np.concatenate([(w / model["S0"])[:, None], w[:, None] * g, (w * model["T"])[:, None]], axis=1)


def oracle_allowances(model, K, is_put, steps, paths, seed, option_index=0):
    """Oracle-only flags and allowances (see the module docstring): per strike the
    kink and decision allowances [n_K, 7], the kink flags [n_K, paths] and the
    decision flags [paths], plus the oracle's per-path (x_T, gradient)."""
    disc = math.exp(-model["r"] * model["T"])
    xo, go = oracle.path_grad(model, steps, seed, 0, paths, option_index=option_index)
    xf, gf, st, _, _ = oracle.path_grad_flip(model, steps, seed, 0, paths, DECISION_MARGIN,
                                             option_index=option_index)
    dec = st >= 0
    dx = _kink_dx(model, steps)
    kink = np.abs(xo[None, :] - np.log(np.asarray(K)[:, None] / model["S0"])) < dx
    a_kink = np.zeros((len(K), 7))
    a_dec = np.zeros((len(K), 7))
    for k, Kk in enumerate(K):
        to = _strike_terms(model, Kk, is_put, xo, go)
        a_kink[k] = disc * np.abs(to[kink[k]]).sum(axis=0) / paths
        if dec.any():
            tf = _strike_terms(model, Kk, is_put, xf[dec], gf[dec])
            a_dec[k] = disc * np.abs(tf - to[dec]).sum(axis=0) / paths
    return a_kink, a_dec, kink, dec, xo, go


def check_adjoint(simr, model, K, is_put, steps, paths, seed, ckpt, pq, dec_frac_max, allow_max, bulk_tol=1e-4):
    K = np.asarray(K, dtype=np.float64)
    p, se, g = simr.greeks_adjoint(model, _dev(K), is_put, steps, paths, seed, ckpt_every=ckpt)
    p, g = p.cpu().numpy(), g.cpu().numpy()
    po, go = oracle.adjoint(model, K, is_put, steps, paths, seed)
    a_kink, a_dec, kink, dec, xo, gro = oracle_allowances(model, K, is_put, steps, paths, seed)
    colmax = np.abs(go).max(axis=0, keepdims=True)
    # the flags and allowances stay small
    assert dec.mean() <= dec_frac_max, dec.mean()
    assert kink.mean() <= 1e-3, kink.mean()
    assert np.all(a_kink + a_dec <= allow_max * colmax), (a_kink + a_dec) / colmax
    # prices: 1e-5
    assert np.all(np.abs(p - po) <= 1e-5 * np.abs(po) + 1e-9), (p, po)
    # Greeks, with the oracle's allowances
    err = np.abs(g - go)
    # (+ a floor at rounding size for columns the oracle gives as exactly zero)
    tol = 1e-4 * np.abs(go) + 1e-4 * colmax + a_kink + a_dec + 1e-9 * np.abs(go).max()
    bad = err > tol
    assert not bad.any(), (np.argwhere(bad), (err / colmax)[bad], ((a_kink + a_dec) / colmax)[bad])
    # the unflagged bulk, strictly, and per path
    xg, gg = simr.paths_adjoint(model, steps, 0, paths, seed, ckpt_every=ckpt)
    xg, gg = xg.cpu().double().numpy(), gg.cpu().double().numpy()
    # the kink band covers every side the GPU took differently
    lnk = np.log(K[:, None] / model["S0"])
    assert not np.any(((xg[None, :] > lnk) != (xo[None, :] > lnk)) & ~kink), "an unflagged strike side differs"
    clean = ~dec & ~kink.any(axis=0)
    scale = np.abs(gro[clean]).max(axis=0, keepdims=True)
    live = scale[0] > 0  # columns the oracle gives as exactly zero on every path: zero on the GPU too
    assert np.abs(gg[clean][:, ~live]).max(initial=0.0) <= 1e-9 * scale.max(), "a zero column is not zero"
    rel = np.abs(gg[clean][:, live] - gro[clean][:, live]) / (np.abs(gro[clean][:, live]) + 1e-3 * scale[:, live])
    assert np.quantile(rel, 0.999) < pq
    sg = np.array([_strike_terms(model, Kk, is_put, xg[clean], gg[clean]).sum(axis=0) for Kk in K])
    so = np.array([_strike_terms(model, Kk, is_put, xo[clean], gro[clean]).sum(axis=0) for Kk in K])
    tol_c = bulk_tol * np.abs(so).max(axis=0, keepdims=True) if bulk_tol > 1e-4 else \
        1e-4 * np.abs(so) + 1e-5 * np.abs(so).max(axis=0, keepdims=True)
    tol_c = tol_c + 1e-12 * np.abs(so).max()
    bad_c = np.abs(sg - so) > tol_c
    assert not bad_c.any(), (np.argwhere(bad_c), (np.abs(sg - so) / np.abs(so).max(axis=0))[bad_c])
    return err / colmax, (a_kink + a_dec) / colmax


# pq: bound on the 99.9% quantile of unflagged paths' relative derivative errors.
# With vol-of-vol 0.9 many steps end near v = 0 through v' = a (b + Z_V)^2 with
# Z_V close to -b, or through a small logarithm just above the exponential
# branch's atom, where FP32 keeps few digits of v' and of its derivatives.
# dec_frac_max, allow_max: bounds on the decision-flagged fraction of the paths
# and on the allowances (x the column's largest magnitude).  The standard model's
# decisions all sit far from their thresholds (no flags) and its allowances are
# the kink terms alone, at most 1.05e-3 of a column (the rho column, whose
# per-path derivatives largely cancel in the mean).  With vol-of-vol 0.9 (Feller
# ratio 0.1) 6.9% of the paths have a decision within 1e-3 of its threshold,
# mostly the exponential branch's atom, and the other side's derivative moves
# dP/dkappa (a column near zero across these strikes), dP/dtheta and dP/dsigma by
# up to 2.2, 0.35 and 0.74 of their largest values: that case's Greek-level
# check is loose on those three columns, and its strict check is the bulk's
# (the other 93% of the paths).
CASES = [
    ("single", CFG, [100.0], False, 64, 65536, 1, 16, 1e-3, 0.0, 2e-3),
    ("grid", CFG, workloads.strike_grid(), False, 252, 16384, 1, 16, 1e-3, 0.0, 2e-3),
    ("grid_put", CFG, workloads.strike_grid(n=8), True, 252, 16384, 2, 0, 1e-3, 0.0, 2e-3),
    ("odd_steps_small_ckpt", CFG, [90.0, 110.0], False, 33, 8192, 3, 2, 1e-3, 0.0, 2e-3),
    ("ckpt_beyond_steps", CFG, [100.0], True, 10, 4097, 4, 64, 1e-3, 0.0, 2e-3),
    ("hard_exp_branch", HARD, [90.0, 100.0, 110.0], False, 64, 16384, 5, 8, 5e-3, 0.08, 2.5, 1e-3),
    ("one_step", CFG, [100.0], False, 1, 2048, 6, 2, 1e-3, 0.0, 2e-3),
    # a long path with the library's own interval (checkpoints past one segment
    # of 1,024 steps: shared-memory segments and a forward pass); the per-path
    # derivatives carry FP32 rounding over 4,096 steps (measured 99.9% quantile
    # 1.03e-3, against ~4e-4 at 252; the unflagged bulk's kappa and sigma sums
    # within 6.2e-5 of their columns' largest values)
    ("long_path_4096", dict(CFG, T=4.0), [90.0, 100.0, 120.0], False, 4096, 4096, 16, 0, 2e-3, 0.0, 2e-3, 2e-4),
    # the largest strike count the adjoint takes: 8 tiles of 32 strikes
    ("strikes_256_max", CFG, np.linspace(60.0, 140.0, 256), False, 16, 65536, 14, 4, 1e-3, 0.0, 2e-3),
]

# Parameter edges: vol-of-vol near the Black-Scholes limit (the constants divide
# by sigma: K1, K2 ~ rho/sigma = 70, so the kappa and sigma columns come out of
# sums of terms far larger than themselves: 1e-4 of a column on the bulk, and the
# per-path quantile at 2.2e-3), mean reversion near zero (Feller ratio 0.001:
# 2.3% of the paths flagged, allowances up to 0.9 of a column), and a degenerate
# variance (v0 = theta = 0: every step at the atom, S_T = S0 e^{rT}; the kappa,
# sigma and rho columns exactly zero).
EDGE_CASES = [
    ("small_vol_of_vol", dict(CFG, sigma=0.01), [90.0, 100.0, 110.0], False, 64, 16384, 7, 16, 5e-3, 0.0, 2e-3,
     5e-4),
    ("small_kappa", dict(CFG, kappa=1e-3), [90.0, 100.0, 110.0], True, 64, 16384, 8, 16, 5e-3, 0.05, 1.5, 2e-2),
    ("zero_variance", dict(CFG, v0=0.0, theta=0.0), [90.0, 110.0], False, 16, 4096, 9, 4, 1e-3, 0.0, 2e-3),
]


@pytest.mark.parametrize("case", EDGE_CASES, ids=[c[0] for c in EDGE_CASES])
def test_adjoint_at_parameter_edges(simr, case):
    check_adjoint(simr, *case[1:])


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_adjoint_matches_oracle(simr, case):
    check_adjoint(simr, *case[1:])


def test_adjoint_full_size_grid_checkpoint_every_16(simr):
    # the adjoint workload at full size: 252 steps x 2^20 paths x 32 strikes, a
    # checkpoint every 16 steps; every column against the oracle's FP64 reverse
    # mode, with the oracle-only kink allowance (no decision of this model comes
    # within 1e-3 of its threshold; the allowance is at most 3.9e-4 of a column,
    # the rho column's)
    check_adjoint(simr, CFG, workloads.strike_grid(), False, 252, 1 << 20, 1, 16, 1e-3, 0.0, 1e-3)


def test_adjoint_price_equals_price_kernel(simr):
    K = _dev(workloads.strike_grid())
    p1, se1 = simr.price(CFG, K, False, 100, 30000, 9)
    p2, se2, _ = simr.greeks_adjoint(CFG, K, False, 100, 30000, 9, ckpt_every=10)
    torch.testing.assert_close(p1, p2, rtol=1e-6, atol=1e-9)


def test_checkpoint_interval_does_not_change_results(simr):
    K = _dev([95.0, 105.0])
    ref = simr.greeks_adjoint(CFG, K, False, 48, 8192, 7, ckpt_every=2)[2]
    for k in (4, 8, 16, 48, 0):
        torch.testing.assert_close(simr.greeks_adjoint(CFG, K, False, 48, 8192, 7, ckpt_every=k)[2], ref,
                                   rtol=0, atol=0)


def test_segments_in_global_memory(simr):
    # intervals whose segment (3 k floats per thread) exceeds shared memory keep
    # their segments in global memory: one segment of the whole path (no forward
    # pass) or a few long ones; the same results bit for bit
    K = _dev(workloads.strike_grid())
    for steps, ks in ((200, (200, 150)), (301, (302, 160))):
        ref = simr.greeks_adjoint(CFG, K, False, steps, 5003, 11, ckpt_every=16)
        for k in ks:
            got = simr.greeks_adjoint(CFG, K, False, steps, 5003, 11, ckpt_every=k)
            for a, b in zip(got, ref):
                torch.testing.assert_close(a, b, rtol=0, atol=0)
    K1 = _dev([100.0])
    ref = simr.greeks_adjoint(CFG, K1, True, 256, 4096, 2, ckpt_every=8)
    got = simr.greeks_adjoint(CFG, K1, True, 256, 4096, 2, ckpt_every=256)
    for a, b in zip(got, ref):
        torch.testing.assert_close(a, b, rtol=0, atol=0)


def test_automatic_interval(simr):
    # the interval taken for ckpt_every=0: even, one segment when it fits, the
    # same results as any explicit interval
    for nk, steps in ((1, 252), (32, 252), (33, 100), (32, 7), (1, 1000)):
        k = simr.adjoint_interval(nk, steps)
        assert k % 2 == 0 and 2 <= k <= steps + (steps & 1), (nk, steps, k)
    assert simr.adjoint_interval(32, 7) == 8
    k = simr.adjoint_interval(32, 252)
    assert k == 252  # one segment of the whole path, no forward pass
    k2 = simr.adjoint_interval(32, 3000)  # longer than one segment may be: shared-memory segments
    assert k2 % 2 == 0 and 2 <= k2 <= 200
    K = _dev(workloads.strike_grid())
    a = simr.greeks_adjoint(CFG, K, False, 252, 4096, 5, ckpt_every=0)
    b = simr.greeks_adjoint(CFG, K, False, 252, 4096, 5, ckpt_every=k)
    c = simr.greeks_adjoint(CFG, K, False, 252, 4096, 5, ckpt_every=2)
    for x, y, z in zip(a, b, c):
        torch.testing.assert_close(x, y, rtol=0, atol=0)
        torch.testing.assert_close(x, z, rtol=0, atol=0)
    with pytest.raises(simr.SimrError):
        simr.adjoint_interval(0, 10)


def test_autograd_function_backward(simr):
    params = torch.tensor([100.0, 0.04, 1.5, 0.04, 0.3, -0.7, 0.05], dtype=torch.float64, requires_grad=True)
    K = _dev(workloads.strike_grid(n=8))
    price = simr.heston_price(params, K, 1.0, False, 64, 20000, 3, 16)
    w = torch.linspace(1.0, 2.0, 8, dtype=torch.float64, device="cuda")
    (price * w).sum().backward()
    _, _, jac = simr.greeks_adjoint(dict(workloads.BASE_MODEL), K, False, 64, 20000, 3, ckpt_every=16)
    torch.testing.assert_close(params.grad, (w @ jac).cpu(), rtol=1e-12, atol=1e-12)


def test_adjoint_agrees_with_bump_and_revalue(simr):
    # pathwise vs CRN finite differences on the GPU: same paths, differences only from
    # branch switches of the QE map (c.f. the oracle's own adjoint-vs-FD pin).
    K = _dev([90.0, 100.0, 110.0])
    _, _, g = simr.greeks_adjoint(CFG, K, False, 64, 1 << 17, 11, ckpt_every=16)
    _, f = simr.greeks_fd(CFG, K, False, 64, 1 << 17, 11,
                          greeks=("delta", "vega", "rho", "kappa", "lrvar", "volvol", "corr"), rel_bump=1e-4)
    g, f = g.cpu().numpy(), f.cpu().numpy()
    # columns: adjoint (S0, v0, kappa, theta, sigma, rho, r); FD bit order (delta, vega, rho_r, kappa, lrvar, volvol, corr)
    for ca, cf in [(0, 0), (1, 1), (6, 2), (2, 3), (3, 4), (4, 5), (5, 6)]:
        np.testing.assert_allclose(g[:, ca], f[:, cf], rtol=2e-2, atol=2e-3 * max(np.abs(f[:, cf]).max(), 1.0))


def test_adjoint_rejects_bad_checkpoint(simr):
    with pytest.raises(simr.SimrError):
        simr.greeks_adjoint(CFG, [100.0], False, 16, 100, 1, ckpt_every=3)
