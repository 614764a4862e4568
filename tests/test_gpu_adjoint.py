"""GPU pathwise adjoint vs the FP64 oracle's reverse-mode adjoint on the same Philox counters.

Both differentiate the same discretised path with branches held fixed, so on
every path where both take the same QE branches they agree up to FP32 rounding.
Tolerance per Greek: relative 1e-4 (the target for Greeks), an absolute floor of
1e-4 x the column's largest magnitude (columns that pass through zero across the
strike grid), plus the exact effect of the paths whose oracle branch decisions
sit within 1e-3 of a threshold or whose payoff indicator differs: for those the
GPU's own per-path terms (simr_paths_adjoint, the same device code as the
reduction) are compared with the oracle's, and their difference / paths is
allowed -- on such a path FP32 may take the other branch of the QE map, whose
derivative belongs to the other branch, and near the exponential branch's
U_V = p boundary v' = (m/q) ln(q/(1 - U_V)) is a small logarithm that FP32
resolves with relative error ~1e-7 / |U_V - p|.  The same accounting covers paths
that pass a quadratic step with |b + Z_V| < 1e-2 (1 + b): there v' = a (b + Z_V)^2
is a cancellation that FP32 resolves to a few digits only.  Both are common only
far outside the Feller condition (vol-of-vol 0.9: 9% of the paths; none of the
64-step single-option model's).
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


@pytest.fixture(scope="module")
def simr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_12111_gb300 as simr

    simr.load()
    return simr


def _dev(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")


# pq: bound on the 99.9% quantile of per-path relative derivative errors.  With
# vol-of-vol 0.9 many steps end near v = 0 through v' = a (b + Z_V)^2 with
# Z_V close to -b, where FP32 keeps few digits of v' and of its derivatives.
CASES = [
    ("single", CFG, [100.0], False, 64, 65536, 1, 16, 1e-3),
    ("grid", CFG, workloads.strike_grid(), False, 252, 16384, 1, 16, 1e-3),
    ("grid_put", CFG, workloads.strike_grid(n=8), True, 252, 16384, 2, 0, 1e-3),
    ("odd_steps_small_ckpt", CFG, [90.0, 110.0], False, 33, 8192, 3, 2, 1e-3),
    ("ckpt_beyond_steps", CFG, [100.0], True, 10, 4097, 4, 64, 1e-3),
    ("hard_exp_branch", HARD, [90.0, 100.0, 110.0], False, 64, 16384, 5, 8, 5e-3),
    ("one_step", CFG, [100.0], False, 1, 2048, 6, 2, 1e-3),
]


def _terms(model, K, is_put, S, g):
    """Per-path, per-strike adjoint terms [n_K, n_paths, 7] (before the discount and the -T P of r)."""
    fp = np.where(S[None, :] < K[:, None], -1.0, 0.0) if is_put else np.where(S[None, :] > K[:, None], 1.0, 0.0)
    w = fp * S[None, :]
    cols = [w / model["S0"]] + [w * g[None, :, j] for j in range(5)] + [w * model["T"]]
    return np.stack(cols, axis=2)


@pytest.mark.parametrize("name,model,K,is_put,steps,paths,seed,ckpt,pq", CASES, ids=[c[0] for c in CASES])
def test_adjoint_matches_oracle(simr, name, model, K, is_put, steps, paths, seed, ckpt, pq):
    K = np.asarray(K, dtype=np.float64)
    p, se, g = simr.greeks_adjoint(model, _dev(K), is_put, steps, paths, seed, ckpt_every=ckpt)
    p, g = p.cpu().numpy(), g.cpu().numpy()
    po, go = oracle.adjoint(model, K, is_put, steps, paths, seed)
    # per path: GPU and oracle
    xg, gg = simr.paths_adjoint(model, steps, 0, paths, seed, ckpt_every=ckpt)
    xg, gg = xg.cpu().double().numpy(), gg.cpu().double().numpy()
    xo, gro = oracle.path_grad(model, steps, seed, 0, paths)
    _, _, mg, cond = oracle.terminal_diag(model, steps, seed, 0, paths)
    Sg, So = model["S0"] * np.exp(xg), model["S0"] * np.exp(xo)
    ind_g = (Sg < K[:, None]) if is_put else (Sg > K[:, None])
    ind_o = (So < K[:, None]) if is_put else (So > K[:, None])
    ill = (mg < 1e-3) | (cond < 1e-2)
    flagged = ill[None, :] | (ind_g != ind_o)                               # [n_K, n_paths]
    ok = ~ill
    # paths with the same branches: per-path derivatives agree to FP32 accuracy
    scale = np.abs(gro[ok]).max(axis=0, keepdims=True)
    assert np.quantile(np.abs(gg[ok] - gro[ok]) / (np.abs(gro[ok]) + 1e-3 * scale), 0.999) < pq
    diff = np.abs(_terms(model, K, is_put, Sg, gg) - _terms(model, K, is_put, So, gro))
    allowance = math.exp(-model["r"] * model["T"]) * (diff * flagged[:, :, None]).sum(axis=1) / paths
    assert np.all(np.abs(p - po) <= 1e-5 * np.abs(po) + 1e-9), (p, po)
    floor = 1e-4 * np.max(np.abs(go), axis=0, keepdims=True)
    err = np.abs(g - go)
    tol = 1e-4 * np.abs(go) + floor + allowance
    bad = err > tol
    assert not bad.any(), (np.argwhere(bad), (err / np.maximum(np.abs(go), 1e-300))[bad])


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
