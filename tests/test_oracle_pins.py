"""Pins of the FP64 oracle against what mathematics and libraries fix (no GPU).

Each test compares the oracle with something other than itself:
  * Philox4x32-10 against Triton's library implementation run on the CPU
    interpreter (Salmon et al. SC'11 definition, 10 rounds);
  * the inverse normal against scipy.special.ndtri and the normal CDF;
  * the QE variance step against the exact CIR conditional mean and variance
    (the moments the QE scheme of Andersen 2008 is built to match), evaluated
    over the full 2^23-point uniform lattice the method samples from;
  * after many steps: exact CIR marginal moments, the exact Heston E[ln S_T],
    the martingale E[e^{-rT} S_T] = S0;
  * European prices against the Heston semi-analytic price (two Fourier forms
    that agree to 1e-10) and the Black-Scholes limit;
  * the standard error against the spread of prices over independent seeds;
  * FD and adjoint Greeks against the semi-analytic delta/gamma/vega/theta/rho and
    against each other, and reverse-mode against forward-mode (dual number)
    per-path tangents.
The paper itself (Sec. 3-6) prints no option value, so parity with the paper's
own numbers is unpinned; the harness accounting is pinned to its Tables 1-2.
"""
import json
import math
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
from scipy.special import ndtr, ndtri

import oracle
import workloads
from oracle import analytic as A

CFG = dict(workloads.BASE_MODEL)
HARD = dict(S0=100.0, r=0.05, T=1.0, v0=0.09, kappa=1.0, theta=0.04, sigma=0.9, rho=-0.3)


# ---------------------------------------------------------------- Philox ----
def _triton_philox(ctrs, seeds):
    """Run Triton's Philox4x32-10 (tl.random.philox, 10 rounds) on the CPU interpreter."""
    code = textwrap.dedent("""
        import json, sys
        import torch, triton, triton.language as tl
        data = json.loads(sys.stdin.read())
        @triton.jit
        def k(out_ptr, c_ptr, seed, N: tl.constexpr):
            i = tl.arange(0, N)
            c0 = tl.load(c_ptr + 4 * i + 0); c1 = tl.load(c_ptr + 4 * i + 1)
            c2 = tl.load(c_ptr + 4 * i + 2); c3 = tl.load(c_ptr + 4 * i + 3)
            a, b, c, d = tl.random.philox(seed, c0, c1, c2, c3, 10)
            tl.store(out_ptr + 4 * i + 0, a); tl.store(out_ptr + 4 * i + 1, b)
            tl.store(out_ptr + 4 * i + 2, c); tl.store(out_ptr + 4 * i + 3, d)
        res = []
        for seed in data["seeds"]:
            c = torch.tensor(data["ctrs"], dtype=torch.int64).to(torch.int32).view(torch.uint32).reshape(-1).contiguous()
            out = torch.zeros_like(c)
            k[(1,)](out, c, seed, N=len(data["ctrs"]))
            res.append([int(x) & 0xFFFFFFFF for x in out.view(torch.int32).tolist()])
        print(json.dumps(res))
    """)
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", code], input=json.dumps({"ctrs": ctrs, "seeds": seeds}),
                       capture_output=True, text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip(f"Triton CPU interpreter unavailable: {p.stderr.strip().splitlines()[-1:]}")
    return json.loads(p.stdout.strip().splitlines()[-1])


def test_philox_matches_triton_library():
    pytest.importorskip("triton")
    rng = np.random.default_rng(2024)
    ctrs = [[0, 0, 0, 0], [0xFFFFFFFF] * 4] + rng.integers(0, 2 ** 32, size=(30, 4)).tolist()
    # counters as the method uses them: (step/2, path lo, path hi, option)
    ctrs += [[n, p, 0, o] for n, p, o in [(0, 0, 0), (1, 5, 0), (127, 65535, 3), (511, (1 << 20) - 1, 7)]]
    ctrs += rng.integers(0, 2 ** 32, size=(64 - len(ctrs), 4)).tolist()  # power-of-two batch
    ctrs = [[int(x) if x < 2 ** 31 else int(x) - 2 ** 32 for x in c] for c in ctrs]  # int32 view
    seeds = [0, 1, 0xDEADBEEF, 0x123456789ABCDEF]
    ref = _triton_philox(ctrs, seeds)
    for s, row in zip(seeds, ref):
        for i, c in enumerate(ctrs):
            got = oracle.philox4x32_10([x & 0xFFFFFFFF for x in c], [s & 0xFFFFFFFF, s >> 32])
            assert got.tolist() == row[4 * i:4 * i + 4], (s, c)


def test_philox_counter_bijective_and_uniform():
    # For a fixed key the map is a bijection of the counter space: no collisions
    # among many distinct counters; output words are uniform (chi-square on bytes).
    outs = np.array([oracle.philox4x32_10([i, 7, 0, 0], [1, 0]) for i in range(20000)], dtype=np.uint64)
    packed = (outs[:, 0] << 32) | outs[:, 1]
    assert len(np.unique(packed)) == len(packed)
    top = (outs.ravel() >> np.uint64(24)).astype(np.int64)
    counts = np.bincount(top, minlength=256)
    exp = top.size / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 255 + 5 * math.sqrt(2 * 255)


def test_step_uniform_mapping():
    # u = ((w >> 9) + 1/2) 2^-23: extremes, exactness in FP32, counter/word layout.
    assert oracle.uniform(0) == 2.0 ** -24
    assert oracle.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    for w in (0, 511, 512, 0x80000000, 0xFFFFFE00, 0xFFFFFFFF):
        u = oracle.uniform(w)
        assert float(np.float32(u)) == u
        assert u == ((w >> 9) + 0.5) / 2 ** 23
    seed, path, opt = 0x1234ABCD5678, (1 << 33) + 17, 3
    w = oracle.philox4x32_10([2, path & 0xFFFFFFFF, path >> 32, opt], [seed & 0xFFFFFFFF, seed >> 32])
    assert oracle.step_uniforms(seed, opt, path, 4) == (oracle.uniform(w[0]), oracle.uniform(w[1]))
    assert oracle.step_uniforms(seed, opt, path, 5) == (oracle.uniform(w[2]), oracle.uniform(w[3]))


# ---------------------------------------------------------- inverse normal ----
def test_norminv_against_scipy_and_cdf():
    k = np.concatenate([np.arange(0, 4096), np.arange(0, 1 << 23, 613), (1 << 23) - 1 - np.arange(0, 4096)])
    u = (k + 0.5) * 2.0 ** -23
    z = oracle.norminv(u)
    ref = ndtri(u)
    assert np.max(np.abs(z - ref) / np.abs(ref)) < 5e-15
    assert np.max(np.abs(ndtr(z) - u) / np.minimum(u, 1 - u)) < 1e-13
    # symmetry Phi^-1(1-u) = -Phi^-1(u) (1-u is exact on the lattice)
    assert np.max(np.abs(oracle.norminv(1.0 - u) + z)) < 1e-14
    assert oracle.norminv([0.5])[0] == 0.0


# ------------------------------------------------------ the closed forms ----
@pytest.mark.parametrize("m", [CFG, HARD, dict(CFG, v0=0.0, kappa=4.0, sigma=1.0)])
def test_closed_form_moments_solve_their_moment_equations(m):
    # Ito's lemma on dv = kappa (theta - v) dt + sigma sqrt(v) dW gives the moment
    # equations d/dt E v = kappa (theta - E v) and d/dt Var v = -2 kappa Var v +
    # sigma^2 E v, and d/dt E ln S = r - E v / 2; integrated numerically here,
    # they must reproduce the closed forms the oracle is checked against.
    from scipy.integrate import solve_ivp

    k, th, s = m["kappa"], m["theta"], m["sigma"]

    def rhs(t, y):
        mean, var, logs = y
        return [k * (th - mean), -2.0 * k * var + s * s * mean, m["r"] - 0.5 * mean]

    ts = np.linspace(0.0, 2.0, 9)[1:]
    sol = solve_ivp(rhs, (0.0, 2.0), [m["v0"], 0.0, 0.0], t_eval=ts, rtol=1e-11, atol=1e-14)
    for j, t in enumerate(ts):
        assert abs(sol.y[0, j] - A.cir_mean(t, m["v0"], k, th)) < 1e-10
        assert abs(sol.y[1, j] - A.cir_var(t, m["v0"], k, th, s)) < 1e-10
        assert abs(sol.y[2, j] - A.heston_log_mean(m["r"], t, m["v0"], k, th)) < 1e-10


def test_black_scholes_closed_form_is_the_lognormal_expectation():
    # e^{-rT} E[(S_T - K)+] with ln S_T ~ N(ln S0 + (r - vol^2/2) T, vol^2 T), by quadrature
    from scipy import integrate

    for S0, K, r, T, vol in [(100.0, 80.0, 0.05, 1.0, 0.2), (100.0, 120.0, 0.0, 0.25, 0.5), (36.0, 40.0, 0.06, 2.0, 0.3)]:
        mu, sd = math.log(S0) + (r - 0.5 * vol * vol) * T, vol * math.sqrt(T)

        def density(z, pay):
            return pay(math.exp(mu + sd * z)) * math.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)

        zk = (math.log(K) - mu) / sd
        # the normal density beyond |z| = 14 is below 1e-42
        call = math.exp(-r * T) * integrate.quad(density, zk, 14.0, args=(lambda s: s - K,), epsabs=1e-13)[0]
        put = math.exp(-r * T) * integrate.quad(density, -14.0, zk, args=(lambda s: K - s,), epsabs=1e-13)[0]
        assert abs(A.bs_call(S0, K, r, T, vol) - call) < 1e-9
        assert abs(A.bs_put(S0, K, r, T, vol) - put) < 1e-9


# --------------------------------------------------------------- QE step ----
LATTICE = (np.arange(1 << 23, dtype=np.float64) + 0.5) * 2.0 ** -23


@pytest.mark.parametrize("v", [0.0, 0.001, 0.005, 0.0085, 0.02, 0.04, 0.2])
def test_qe_step_matches_cir_conditional_moments(v):
    # The QE step is constructed so that E[v'|v] and Var[v'|v] equal the exact CIR
    # conditional moments over one step (Andersen 2008); the small v values take
    # the exponential branch (psi > 1.5), the large ones the quadratic branch.
    dt = HARD["T"] / 64
    vn = oracle.qe_step_array(HARD, 64, v, LATTICE)
    mu = A.cir_mean(dt, v, HARD["kappa"], HARD["theta"])
    var = A.cir_var(dt, v, HARD["kappa"], HARD["theta"], HARD["sigma"])
    assert abs(vn.mean() / mu - 1) < 1e-6
    assert abs(vn.var() / var - 1) < 2e-5
    assert vn.min() >= 0.0


def test_qe_step_branches_and_degenerate_cases():
    _, br = oracle.qe_step(HARD, 64, 0.2, 0.3)
    assert br == 0
    v0, br = oracle.qe_step(HARD, 64, 0.001, 1e-3)
    assert br == 2 and v0 == 0.0          # U_V <= p gives an atom at zero
    v1, br = oracle.qe_step(HARD, 64, 0.001, 0.999)
    assert br == 1 and v1 > 0.0
    z = dict(HARD, theta=0.0)
    v2, br = oracle.qe_step(z, 64, 0.0, 0.7)  # zero mean and variance: stays at zero
    assert br == 3 and v2 == 0.0


# ------------------------------------------------------- multi-step pins ----
def hard_paths():
    """2^19 paths of 64 steps of the hard model (coarse steps, both QE branches)."""
    return oracle.terminal(HARD, 64, 7, 0, 1 << 19)


def cfg_paths():
    """2^19 paths of 64 steps of the base model started away from theta (v0 = 0.09)."""
    return oracle.terminal(dict(CFG, v0=0.09), 64, 11, 0, 1 << 19)


@pytest.fixture(scope="module")
def terminal_hard():
    return hard_paths()


@pytest.fixture(scope="module")
def terminal_cfg():
    return cfg_paths()


@pytest.mark.parametrize("which", ["hard", "cfg"])
def test_variance_marginal_moments(which, terminal_hard, terminal_cfg):
    x, v, _ = terminal_hard if which == "hard" else terminal_cfg
    m = HARD if which == "hard" else dict(CFG, v0=0.09)
    n = v.size
    mu = A.cir_mean(m["T"], m["v0"], m["kappa"], m["theta"])
    var = A.cir_var(m["T"], m["v0"], m["kappa"], m["theta"], m["sigma"])
    assert abs(v.mean() - mu) < 4 * v.std() / math.sqrt(n)
    d2 = (v - v.mean()) ** 2
    assert abs(d2.mean() - var) < 4 * d2.std() / math.sqrt(n)


@pytest.mark.parametrize("which", ["hard", "cfg"])
def test_log_spot_mean_and_martingale(which, terminal_hard, terminal_cfg):
    # E[x_T] = rT - 1/2 int E[v_t] dt for the exact model; the scheme's own mean
    # differs only by a trapezoid error far below the MC error at 64 steps.
    # v0 != theta makes the rho/sigma terms of K1, K2 contribute.
    x, _, _ = terminal_hard if which == "hard" else terminal_cfg
    m = HARD if which == "hard" else dict(CFG, v0=0.09)
    n = x.size
    ref = A.heston_log_mean(m["r"], m["T"], m["v0"], m["kappa"], m["theta"])
    assert abs(x.mean() - ref) < 4 * x.std() / math.sqrt(n) + 1e-5
    disc_s = np.exp(x - m["r"] * m["T"])  # e^{-rT} S_T / S0
    assert abs(disc_s.mean() - 1.0) < 4 * disc_s.std() / math.sqrt(n) + 2e-4


@pytest.mark.parametrize("model,steps", [(CFG, 64), (HARD, 128)])
@pytest.mark.parametrize("is_put", [False, True])
def test_price_matches_heston_semi_analytic(model, steps, is_put):
    K = np.array([70.0, 100.0, 130.0])
    p, se = oracle.price(model, K, is_put, steps, 1 << 20, 3)
    for j, k in enumerate(K):
        c = A.heston_call_p1p2(k, **model)[0]
        ref = A.heston_put_from_call(c, k, model["S0"], model["r"], model["T"]) if is_put else c
        assert abs(p[j] - ref) < 4 * se[j] + 5e-3, (k, p[j], ref, se[j])


def test_semi_analytic_forms_agree_and_bs_limit():
    for m in (CFG, HARD, dict(CFG, rho=0.5, r=0.0, T=0.25)):
        for k in (70.0, 100.0, 130.0):
            assert abs(A.heston_call_p1p2(k, **m)[0] - A.heston_call_lewis(k, **m)) < 1e-9
    # vanishing vol-of-vol with v0 = theta, rho = 0: the price approaches Black-Scholes
    # with vol sqrt(theta) as BS + c sigma^2 + O(sigma^4); Richardson-extrapolate sigma -> 0.
    for k in (80.0, 100.0, 120.0):
        p1, p2 = (A.heston_call_lewis(k, **dict(CFG, sigma=s, rho=0.0)) for s in (0.01, 0.005))
        bs = A.bs_call(100.0, k, 0.05, 1.0, 0.2)
        assert abs(p2 - bs) < abs(p1 - bs) / 3.5          # second-order convergence
        assert abs((4 * p2 - p1) / 3 - bs) < 1e-7


def test_oracle_bs_limit():
    m = dict(CFG, sigma=1e-4)
    K = np.array([80.0, 100.0, 120.0])
    for is_put in (False, True):
        p, se = oracle.price(m, K, is_put, 64, 1 << 19, 5)
        for j, k in enumerate(K):
            ref = (A.bs_put if is_put else A.bs_call)(100.0, k, 0.05, 1.0, 0.2)
            assert abs(p[j] - ref) < 4 * se[j] + 1e-3


def test_put_call_parity_on_common_paths():
    K = workloads.strike_grid(n=8)
    c, _ = oracle.price(CFG, K, False, 32, 1 << 16, 9)
    p, _ = oracle.price(CFG, K, True, 32, 1 << 16, 9)
    x, _, _ = oracle.terminal(CFG, 32, 9, 0, 1 << 16)
    fwd = math.exp(-CFG["r"] * CFG["T"]) * (100.0 * np.exp(x)).mean()
    np.testing.assert_allclose(c - p, fwd - K * math.exp(-CFG["r"] * CFG["T"]), rtol=0, atol=1e-10)


def test_standard_error_matches_the_spread_over_seeds():
    # stderr estimates the standard deviation of the price estimator itself: over
    # 128 independent seeds the prices spread by that much.  The sample standard
    # deviation of 128 draws has a relative error near 1/sqrt(254) = 6%, so the
    # band [0.8, 1.25] holds comfortably and a factor sqrt(2) falls outside it.
    K = np.array([80.0, 100.0, 120.0])
    for is_put in (False, True):
        runs = [oracle.price(CFG, K, is_put, 16, 8192, s) for s in range(1, 129)]
        prices = np.array([p for p, _ in runs])
        errs = np.array([e for _, e in runs])
        ratio = prices.std(axis=0, ddof=1) / errs.mean(axis=0)
        assert np.all((ratio > 0.8) & (ratio < 1.25)), ratio


def test_counter_independence_of_path_ranges():
    # A path's result depends only on (seed, option, path index): shards agree with the whole.
    xa, va, _ = oracle.terminal(CFG, 16, 3, 0, 4096)
    xb, vb, _ = oracle.terminal(CFG, 16, 3, 1000, 96)
    np.testing.assert_array_equal(xa[1000:1096], xb)
    np.testing.assert_array_equal(va[1000:1096], vb)
    xo, _, _ = oracle.terminal(CFG, 16, 3, 0, 64, option_index=1)
    assert not np.array_equal(xo, xa[:64])


# ------------------------------------------------------------- Greeks ----
def _cf_call(m):
    return A.heston_call_p1p2(100.0, **m)[0]


def test_fd_greeks_against_semi_analytic():
    P = 1 << 20
    mask = oracle.G_DELTA | oracle.G_GAMMA | oracle.G_VEGA | oracle.G_RHO
    price, g = oracle.greeks_fd(CFG, [100.0], False, 64, P, 1, 1e-4, mask)
    _, P1, _ = A.heston_call_p1p2(100.0, **CFG)
    # delta = P1 (Heston price is homogeneous of degree one in (S0, K))
    assert abs(g[0, 0] - P1) < 4 * 0.6 / math.sqrt(P) + 2e-3
    h = 1e-4
    vega = (_cf_call(dict(CFG, v0=CFG["v0"] + h)) - _cf_call(dict(CFG, v0=CFG["v0"] - h))) / (2 * h)
    assert abs(g[0, 2] / vega - 1) < 0.02
    rho = (_cf_call(dict(CFG, r=CFG["r"] + h)) - _cf_call(dict(CFG, r=CFG["r"] - h))) / (2 * h)
    assert abs(g[0, 3] / rho - 1) < 0.01
    gam = (_cf_call(dict(CFG, S0=100.5)) - 2 * _cf_call(CFG) + _cf_call(dict(CFG, S0=99.5))) / 0.25
    assert abs(g[0, 1] / gam - 1) < 0.25   # FD gamma with a 1e-4 bump is noisy


def test_fd_theta_against_semi_analytic():
    # theta = -dP/dT: the oracle bumps T (and with it dt) on common random numbers
    K = np.array([90.0, 100.0, 110.0])
    _, g = oracle.greeks_fd(CFG, K, False, 64, 1 << 18, 1, 1e-4, oracle.G_THETA)
    h = 1e-4
    for j, k in enumerate(K):
        up = A.heston_call_p1p2(k, **dict(CFG, T=CFG["T"] + h))[0]
        dn = A.heston_call_p1p2(k, **dict(CFG, T=CFG["T"] - h))[0]
        ref = -(up - dn) / (2 * h)
        assert abs(g[j, 0] / ref - 1) < 0.015, (k, g[j, 0], ref)


def test_reverse_mode_matches_forward_mode_duals():
    for m in (CFG, HARD):
        xr, gr = oracle.path_grad(m, 48, 5, 0, 4096, mode="reverse")
        xf, gf = oracle.path_grad(m, 48, 5, 0, 4096, mode="forward")
        np.testing.assert_allclose(xr, xf, rtol=0, atol=1e-12)
        scale = np.maximum(np.abs(gf), 1e-3)
        assert np.max(np.abs(gr - gf) / scale) < 1e-9


def test_adjoint_matches_fd_and_closed_form_delta():
    P = 1 << 18
    K = np.array([90.0, 100.0, 110.0])
    mask = oracle.G_DELTA | oracle.G_VEGA | oracle.G_RHO | oracle.G_KAPPA | oracle.G_LRVAR | oracle.G_VOLVOL | oracle.G_CORR
    for is_put in (False, True):
        pa, ga = oracle.adjoint(CFG, K, is_put, 64, P, 13)
        pf, gf = oracle.greeks_fd(CFG, K, is_put, 64, P, 13, 1e-5, mask)
        np.testing.assert_allclose(pa, pf, rtol=1e-13)
        # columns: adjoint (S0, v0, kappa, theta, sigma, rho, r); FD in mask bit order
        # (delta, vega, rho_r, kappa, theta, sigma, rho)
        pairs = [(0, 0), (1, 1), (6, 2), (2, 3), (3, 4), (4, 5), (5, 6)]
        for ca, cf in pairs:
            # pathwise misses only the rare branch-switch jumps of the QE map
            tol = 2e-3 * max(abs(gf[:, cf]).max(), 1.0)
            np.testing.assert_allclose(ga[:, ca], gf[:, cf], rtol=2e-2, atol=tol)
        # delta = e^{-rT} E[1{S_T > K} S_T] / S0 for calls, on the same paths
        x, _, _ = oracle.terminal(CFG, 64, 13, 0, P)
        S = 100.0 * np.exp(x)
        ind = (S < K[:, None]) * -1.0 if is_put else (S > K[:, None]) * 1.0
        d = math.exp(-CFG["r"] * CFG["T"]) * (ind * S).mean(axis=1) / 100.0
        np.testing.assert_allclose(ga[:, 0], d, rtol=1e-12)


# ------------------------------------------------------- paper's tables ----
def _read_golden(name):
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_paper_table1_element_accounting():
    for name, A_, T_, P_, el_m, dp_m, mb in _read_golden("paper_table1_sizes.txt"):
        assert workloads.PAPER_SIZES[name] == (int(A_), int(T_), int(P_))
        assert workloads.paper_elements(name) == round(float(el_m) * 1e6)
        assert workloads.paper_datapoint_bytes(name) == round(float(mb) * 1e6)
        assert 2 * workloads.paper_elements(name) == round(float(dp_m) * 1e6)


def test_paper_table2_ops_per_cycle():
    ops = 36 * 504
    assert ops == 18144
    for _, _, cycles, opc, eff in _read_golden("paper_table2_ops.txt"):
        assert round(ops / int(cycles), 2) == float(opc)
        assert abs(100 * ops / int(cycles) / 8 - float(eff)) < 0.06


# ------------------------------------------------ branch decision taken the other way ----
HARD_FLIP = dict(S0=100.0, r=0.05, T=1.0, v0=0.09, kappa=1.0, theta=0.04, sigma=0.9, rho=-0.3)


# Under QE-M the two branches' ln M agree to second order in A (both match the
# step's mean and variance), so the branch ln M takes shows in the gradient only
# with a large |A| and coarse steps: rho = -0.9 over 8 steps (up to 2.4e-3 of a
# path's largest derivative there, against 6e-5 at rho = -0.3).
FLIP_CASES = {"qe": (HARD_FLIP, 64, 4096), "qem": (dict(HARD_FLIP, rho=-0.9), 8, 16384)}


@pytest.mark.parametrize("scheme", ["qe", "qem"])
def test_flipped_decision_gradient_matches_finite_differences(scheme):
    # oracle.path_grad_flip: the reverse-mode gradient of the path whose decision
    # closest to its threshold is taken the other way.  Central differences of that
    # forced path's x_T (oracle.terminal_forced, the decision imposed at the same
    # step, every other decision left to the path) must agree with it, and paths
    # without a flip must equal the plain reverse mode bit for bit.  A path whose
    # atom (v' = 0) is forced to the logarithm's side keeps v' = 0 there (the
    # continuation below the boundary is negative) and takes that side's
    # one-sided derivative, which no difference of the held value can show: those
    # flips are left out of the check.  Under QE-M a flipped branch also takes the
    # other branch's ln M in the step's correction, on both sides of the check.
    with oracle.scheme(scheme):
        _check_flipped_decision_gradient(*FLIP_CASES[scheme])


def _check_flipped_decision_gradient(model, steps, n):
    seed = 5
    x, g, st, kd, fv = oracle.path_grad_flip(model, steps, seed, 0, n, 1e-3)
    x0, g0 = oracle.path_grad(model, steps, seed, 0, n)
    nf = st < 0
    assert 0.01 < (~nf).mean() < 0.2 and set(np.unique(kd[~nf])) <= {1, 2}
    np.testing.assert_array_equal(g[nf], g0[nf])
    np.testing.assert_array_equal(x[nf], x0[nf])
    assert np.all(np.isfinite(g)) and np.all(np.isfinite(x))
    fields = ("v0", "kappa", "theta", "sigma", "rho")
    checked = {1: 0, 2: 0}
    # every branch flip (up to 40) and the first 80 atom flips
    pick = np.concatenate([np.flatnonzero(~nf & (kd == 1))[:40], np.flatnonzero(~nf & (kd == 2))[:80]])
    for i in pick:
        i = int(i)
        value = int(fv[i])
        assert oracle.terminal_forced(model, steps, seed, i, int(st[i]), int(kd[i]), value) == x[i]
        if kd[i] == 2 and value == 1:
            continue  # the atom forced to the logarithm's side: held at v' = 0
        fd, clean = np.empty(5), True
        for j, f in enumerate(fields):
            vals = []
            for h in (1e-6, 5e-7):
                hh = h * max(abs(model[f]), 1.0)
                up, dn = dict(model), dict(model)
                up[f] += hh
                dn[f] -= hh
                xu = oracle.terminal_forced(up, steps, seed, i, int(st[i]), int(kd[i]), value)
                xd = oracle.terminal_forced(dn, steps, seed, i, int(st[i]), int(kd[i]), value)
                vals.append((xu - xd) / (2 * hh))
            # another decision of the path within the bump makes the difference meaningless
            clean = clean and abs(vals[0] - vals[1]) <= 1e-4 * max(abs(vals[0]), 1e-2)
            fd[j] = vals[0]
        if not clean:
            continue
        np.testing.assert_allclose(g[i], fd, rtol=1e-4, atol=1e-6 * np.abs(g[i]).max(), err_msg=f"path {i}")
        checked[int(kd[i])] += 1
    assert checked[1] >= 3 and checked[2] >= 5, checked


def _tiny_paths():
    rows = {}
    for name, steps, p, x, v in _read_golden("tiny_paths.txt"):
        rows.setdefault((name, int(steps)), []).append((int(p), float(x), float(v)))
    return rows


TINY_MODELS = {"standard": dict(workloads.BASE_MODEL),
               "vol_of_vol_0.9": dict(S0=100.0, r=0.05, T=1.0, v0=0.09, kappa=1.0, theta=0.04, sigma=0.9, rho=-0.3)}


def test_oracle_reproduces_its_tiny_path_fixture():
    # a regression fixture (tests/golden/make_tiny_paths.py): the oracle's terminal
    # states at 1 and 2 steps, 8 paths; a change of the oracle's path arithmetic
    # shows here and must come with a regenerated fixture
    rows = _tiny_paths()
    assert len(rows) == 4
    for (name, steps), vals in rows.items():
        x, v, _ = oracle.terminal(TINY_MODELS[name], steps, 7, 0, 8)
        for p, xe, ve in vals:
            assert x[p] == pytest.approx(xe, rel=1e-15, abs=1e-17) and v[p] == pytest.approx(ve, rel=1e-15, abs=1e-17)


@pytest.mark.parametrize("scheme", ["qe", "qem"])
def test_adjoint_at_zero_variance_in_closed_form(scheme):
    # v0 = theta = 0: m = s^2 = 0 at every step, every v' = 0 and x_T = r T on
    # every path, so S_T = S0 e^{rT} and e^{-rT} S_T = S0.  With v' held at 0 the
    # only dependence on v0 is the first step's v0 term of the log-spot step
    # (the sqrt term's derivative at zero variance taken as 0): under QE
    # K1 = dt (kappa rho / sigma - 1/2) / 2 - rho / sigma (Andersen's gamma1 = 1/2), so
    # dP/dv0 = S0 K1 for a strike below S_T; under QE-M the step is
    # r dt - ln M - (K1 + K3/2) v + K1 v + K2 v' with M = 1 at a zero mean, so
    # dP/dv0 = -S0 K3 / 2, K3 = dt (1 - rho^2) / 2.  dP/dtheta: theta enters QE's
    # K0 = -rho kappa theta dt / sigma + r dt at every step (S0 (-rho kappa T / sigma));
    # QE-M replaces K0 by r dt - ln M, so 0.  kappa, sigma, rho: every term they
    # enter multiplies theta or a variance, so 0.  dP/dS0 = 1, dP/dr = e^{-rT} T K.
    # A strike above S_T: every column 0.
    model = dict(CFG, v0=0.0, theta=0.0)
    steps, S0, T, r = 16, model["S0"], model["T"], model["r"]
    dt = T / steps
    kap, sig, rho = model["kappa"], model["sigma"], model["rho"]
    K = np.array([90.0, 110.0])
    with oracle.scheme(scheme):
        p, g = oracle.adjoint(model, K, False, steps, 64, 9)
    K1 = 0.5 * dt * (kap * rho / sig - 0.5) - rho / sig
    K3 = 0.5 * dt * (1.0 - rho * rho)
    if scheme == "qe":
        v0_col, theta_col = S0 * K1, -S0 * rho * kap * T / sig
    else:
        v0_col, theta_col = -0.5 * S0 * K3, 0.0
    np.testing.assert_allclose(p, [S0 - math.exp(-r * T) * 90.0, 0.0], rtol=1e-13, atol=1e-13)
    want = [1.0, v0_col, 0.0, theta_col, 0.0, 0.0, math.exp(-r * T) * T * 90.0]
    np.testing.assert_allclose(g[0], want, rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(g[1], np.zeros(7))
