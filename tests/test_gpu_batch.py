"""Batched heterogeneous book (simr_batch_submit) on the GPU.

Option i of a book uses Philox counter word 3 = i, so its estimate is the one
simr_price / simr_greeks_adjoint give with option_index = i; the two group the
paths into the same 32-path FP32 sums and differ only in the order of the FP64
additions that follow (relative 1e-12).  A sample of the book is also checked
against the FP64 oracle (prices 1e-5 relative + branch-flip allowance).
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def simr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2402_12111_gb300 as simr

    simr.load()
    return simr


@pytest.fixture(scope="module")
def small_book():
    # the book generator's distributions, scaled down in paths and steps for test time
    return workloads.book(n_options=48, seed=3, steps_range=(1, 96), paths_range=(1, 20000))


def test_batch_prices_equal_per_option_calls(simr, small_book):
    p, se, g = simr.batch(small_book, seed=9)
    assert g is None
    for i, o in enumerate(small_book):
        pi, si = simr.price(o["model"], torch.tensor([o["K"]], dtype=torch.float64, device="cuda"), o["is_put"],
                            o["steps"], o["paths"], 9, option_index=i)
        torch.testing.assert_close(p[i:i + 1], pi, rtol=1e-12, atol=1e-12)
        torch.testing.assert_close(se[i:i + 1], si, rtol=1e-9, atol=1e-12)


def test_batch_adjoint_equals_per_option_calls(simr, small_book):
    p, se, g = simr.batch(small_book, seed=4, adjoint=True)
    for i, o in enumerate(small_book):
        pi, _, gi = simr.greeks_adjoint(o["model"], torch.tensor([o["K"]], dtype=torch.float64, device="cuda"),
                                        o["is_put"], o["steps"], o["paths"], 4, ckpt_every=0, option_index=i)
        torch.testing.assert_close(p[i:i + 1], pi, rtol=1e-12, atol=1e-12)
        torch.testing.assert_close(g[i:i + 1], gi, rtol=1e-9, atol=1e-9)


def test_batch_adjoint_long_options_use_shared_segments(simr):
    # a book whose longest option exceeds 1,024 steps runs the shared-memory
    # checkpoint layout instead of one global segment per path: the same results
    book = workloads.book(n_options=6, seed=8, steps_range=(200, 400), paths_range=(300, 3000))
    book[2]["steps"] = 1500
    p, _, g = simr.batch(book, seed=6, adjoint=True)
    for i, o in enumerate(book):
        pi, _, gi = simr.greeks_adjoint(o["model"], torch.tensor([o["K"]], dtype=torch.float64, device="cuda"),
                                        o["is_put"], o["steps"], o["paths"], 6, ckpt_every=0, option_index=i)
        torch.testing.assert_close(p[i:i + 1], pi, rtol=1e-12, atol=1e-12)
        torch.testing.assert_close(g[i:i + 1], gi, rtol=1e-9, atol=1e-9)


def test_every_kernel_shape_gives_the_same_results(simr, small_book):
    # threads per block, paths per thread and unroll change the schedule, never
    # the arithmetic or the grouping of the sums: bit for bit the same
    ref = simr.batch(small_book, seed=12, variant=0)
    for v in range(1, 8):
        got = simr.batch(small_book, seed=12, variant=v)
        torch.testing.assert_close(got[0], ref[0], rtol=0, atol=0)
        torch.testing.assert_close(got[1], ref[1], rtol=0, atol=0)
    refa = simr.batch(small_book[:12], seed=12, adjoint=True, variant=0)
    got = simr.batch(small_book[:12], seed=12, adjoint=True, variant=1)
    for a, b in zip(got, refa):
        torch.testing.assert_close(a, b, rtol=0, atol=0)
    with pytest.raises(simr.SimrError):
        simr.batch(small_book[:4], seed=12, adjoint=True, variant=2)  # adjoint books have two shapes


def test_tuned_shape_is_written_to_the_cache_file(simr, tmp_path, monkeypatch):
    import json
    import subprocess
    import sys

    path = tmp_path / "tune.jsonl"
    monkeypatch.setenv("SIMR_TUNE_CACHE", str(path))
    # a book size class of its own (so this process tunes it now)
    book = workloads.book(n_options=3, seed=21, steps_range=(2, 4), paths_range=(7, 9))
    p0 = simr.batch(book, seed=3)[0]
    lines = [json.loads(ln) for ln in path.read_text().splitlines()]
    assert len(lines) == 1
    e = lines[0]
    assert set(e) >= {"gpu", "key", "chunk", "variant", "tpb", "ppt", "unroll"}
    assert 0 <= e["variant"] < 8 and e["tpb"] in (128, 256) and e["ppt"] in (1, 2) and e["unroll"] in (1, 2)
    assert e["chunk"] % 64 == 0
    # a fresh process reads the file (a malformed line is skipped) and prices the same book
    path.write_text("not json\n" + path.read_text())
    code = ("import sys, torch, workloads, paper_2402_12111_gb300 as simr; "
            "b = workloads.book(n_options=3, seed=21, steps_range=(2, 4), paths_range=(7, 9)); "
            "print(repr(simr.batch(b, seed=3)[0].cpu().tolist()))")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=root,
                         env=dict(os.environ, SIMR_TUNE_CACHE=str(path)), timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert eval(out.stdout.strip().splitlines()[-1]) == p0.cpu().tolist()
    assert len(path.read_text().splitlines()) == 2  # read, nothing re-tuned


def test_batch_graph_replay_and_autotune_agree(simr, small_book):
    ref = simr.batch(small_book, seed=5, autotune=False)[0]
    a = simr.batch(small_book, seed=5, graph=True)[0]   # capture
    b = simr.batch(small_book, seed=5, graph=True)[0]   # replay
    torch.testing.assert_close(a, ref, rtol=1e-12, atol=1e-12)
    torch.testing.assert_close(b, ref, rtol=1e-12, atol=1e-12)
    c = simr.batch(small_book[:7], seed=5, graph=True)[0]  # another book: fresh capture
    torch.testing.assert_close(c, ref[:7], rtol=1e-12, atol=1e-12)


def test_batch_graph_recaptured_after_buffer_growth(simr, small_book):
    # a graph holds the context's device tables; a larger book in between grows
    # (reallocates) them, and the next replay of the first book must not use the
    # freed ones
    ref = simr.batch(small_book, seed=6, autotune=False)[0]
    a = simr.batch(small_book, seed=6, graph=True)[0]
    big = workloads.book(n_options=3000, seed=8, steps_range=(1, 4), paths_range=(1, 64))
    simr.batch(big, seed=6, autotune=False)
    b = simr.batch(small_book, seed=6, graph=True)[0]
    torch.testing.assert_close(a, ref, rtol=1e-12, atol=1e-12)
    torch.testing.assert_close(b, ref, rtol=1e-12, atol=1e-12)


def test_batch_sample_matches_oracle(simr, small_book):
    p, _, _ = simr.batch(small_book, seed=2)
    p = p.cpu().numpy()
    for i in range(0, len(small_book), 6):
        o = small_book[i]
        po, _ = oracle.price(o["model"], [o["K"]], o["is_put"], o["steps"], o["paths"], 2, option_index=i)
        x, _, mg = oracle.terminal(o["model"], o["steps"], 2, 0, o["paths"], option_index=i)
        close = mg < 1e-4
        S = o["model"]["S0"] * np.exp(x[close])
        allow = math.exp(-o["model"]["r"] * o["model"]["T"]) * close.sum() * \
            (o["K"] if o["is_put"] else max(S.max(initial=o["K"]) * 1.5, o["K"])) / o["paths"]
        assert abs(p[i] - po[0]) <= 1e-5 * abs(po[0]) + allow + 1e-12, (i, p[i], po[0])


def test_batch_host_outputs_and_errors(simr, small_book):
    ph, _, _ = simr.batch(small_book[:5], seed=1, out_device="cpu")
    pd, _, _ = simr.batch(small_book[:5], seed=1)
    torch.testing.assert_close(ph, pd.cpu(), rtol=0, atol=0)
    bad = [dict(small_book[0], K=-1.0)]
    with pytest.raises(simr.SimrError):
        simr.batch(bad)


def test_book_at_full_size_matches_oracle_price_and_adjoint(simr):
    # The 1,024-option heterogeneous book at its full sizes (steps log-uniform in
    # [16, 512], paths in [16,384, 2^20]), prices and adjoint Greeks in one
    # submission; options sampled across the book -- the most steps, the most
    # paths, the most path-steps and nine more -- checked directly against the
    # oracle's FP64 price and reverse-mode adjoint of the same counters
    # (option_index = the option's position).  Tolerances: prices 1e-5 relative
    # plus the oracle's flip allowance; each Greek 1e-4 relative plus 1e-4 of the
    # price per unit of its parameter's own size (a floor for sensitivities near
    # zero) plus the oracle-only kink and decision allowances of
    # test_gpu_adjoint (many of the book's models violate the Feller condition).
    from test_gpu_adjoint import oracle_allowances

    book = workloads.book()
    p, _, g = simr.batch(book, seed=1, adjoint=True)
    p, g = p.cpu().numpy(), g.cpu().numpy()
    sizes = np.array([o["steps"] * o["paths"] for o in book])
    rng = np.random.default_rng(17)
    pick = {int(np.argmax([o["steps"] for o in book])), int(np.argmax([o["paths"] for o in book])),
            int(np.argmax(sizes))} | set(int(i) for i in rng.choice(len(book), 9, replace=False))
    cols = ("S0", "v0", "kappa", "theta", "sigma", "rho", "r")
    for i in sorted(pick):
        o = book[i]
        m, K = o["model"], np.array([o["K"]])
        po, go = oracle.adjoint(m, K, o["is_put"], o["steps"], o["paths"], 1, option_index=i)
        x, _, mg = oracle.terminal(m, o["steps"], 1, 0, o["paths"], option_index=i)
        close = mg < 1e-4
        Sx = m["S0"] * np.exp(x[close])
        allow_p = math.exp(-m["r"] * m["T"]) * close.sum() * \
            (o["K"] if o["is_put"] else max(Sx.max(initial=o["K"]) * 1.5, o["K"])) / o["paths"]
        assert abs(p[i] - po[0]) <= 1e-5 * abs(po[0]) + allow_p + 1e-12, (i, p[i], po[0])
        a_kink, a_dec, _, _, _, _ = oracle_allowances(m, K, o["is_put"], o["steps"], o["paths"], 1, option_index=i)
        floor = 1e-4 * abs(po[0]) / np.array([max(abs(m[c]), 0.01) for c in cols])
        tol = 1e-4 * np.abs(go[0]) + floor + a_kink[0] + a_dec[0]
        assert np.all(np.abs(g[i] - go[0]) <= tol), (i, o["steps"], o["paths"], g[i], go[0], tol)

