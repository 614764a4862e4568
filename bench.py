"""Benchmark: Heston path-steps/s for price + bump-and-revalue Greeks on GB300.

A step is one pass of the whole hot path over one batch: simr_greeks_fd on the
32-strike grid workload (252 steps, 2^20 paths, delta/gamma/vega/theta/rho,
relative bump 1e-4) -- Philox draws, inverse normals, QE variance and log-spot
steps for the base and the four re-simulated scenarios, payoffs and the FP64
reduction, one kernel launch.  value = underlying path-steps (paths x time
steps) priced with Greeks per second, summed over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With torchrun (N > 1) every rank prices its own path range [rank P, (rank+1) P)
(weak scaling, no collective in the timed loop); the shards' FP64 sums are
combined once afterwards.  --impl reference times the FP64 CPU oracle on the
host cores on a bounded path sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "Heston path-steps/s (price+Greeks) on 1 GB300; % FP32 peak; adjoint vs FD speedup"
UNIT = "path-steps/s"
FP32_LANES_PER_SM = 128
# Algorithmic FP32 flops per path-step (FMA = 2 flops; special-function
# evaluations -- reciprocal, square root, logarithm -- are counted apart, not
# here), in the method's own operation count:
#   shared per step: the two inverse normals Z_V, Z_X, 22 each                   = 44
#   per simulated scenario: QE variance step 16 (moments, psi, b^2, a, v')
#   + log-spot step 7 (K0 + K1 v + K2 v' + sqrt(K3 v + K4 v') Z_X)               = 23
# Work of this implementation's own choosing is left out: the uniform mapping,
# the Kahan compensation of x, the CRN scenarios' constant deltas, Philox.
FLOPS_SHARED = 44
FLOPS_PER_SCENARIO = 23
# The reverse step of the pathwise adjoint, in the same count (the oracle's
# reverse-mode step, reusing the forward step's quantities): the log-spot step's
# adjoint 14 (d sqrt(w) Z / dw, the adjoints of v_n, v_n+1 and K0..K4), the QE
# map's 24 (abar, bbar, b2bar, tbar, mbar, s2bar), the moments' 13 (through E,
# theta, c1, c2 and v_n) = 51; price + adjoint Greeks = 44 + 23 + 51 = 118.
FLOPS_ADJOINT_REVERSE = 51
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-unit-rates", action="store_true",
                    help="skip the measurement of the FP32 / MUFU / multiply / FP64 unit rates")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint vs bump-and-revalue leg")
    ap.add_argument("--no-book", action="store_true", help="skip the 1,024-option heterogeneous book leg")
    ap.add_argument("--no-lsm", action="store_true", help="skip the Longstaff-Schwartz Bermudan put leg")
    ap.add_argument("--no-headline", action="store_true",
                    help="skip the 8-underlying, 1,024-step, 2^26-path adjoint vs bump-and-revalue leg")
    ap.add_argument("--paths", type=int, default=0, help="override the path count (profiling small cases)")
    ap.add_argument("--time-steps", type=int, default=0, help="override the time-step count of --profile-leg")
    ap.add_argument("--ckpt-every", type=int, default=0,
                    help="checkpoint interval of --profile-leg adjoint (0: the library's choice)")
    ap.add_argument("--profile-leg", default="", choices=["", "fd", "price", "adjoint", "book", "book_price", "lsm",
                                                          "basket"],
                    help="only run one call W + K times on the workload (for profilers); prints no JSON")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def greek_list(w):
    return list(w.greeks)


def simulated_scenarios(greeks) -> int:
    """Base + up/down for each re-simulated Greek (delta, gamma, rho reuse the base path)."""
    return 1 + 2 * sum(g in ("vega", "theta", "kappa", "lrvar", "volvol", "corr") for g in greeks)


def flops_per_path_step(greeks) -> int:
    return FLOPS_SHARED + FLOPS_PER_SCENARIO * simulated_scenarios(greeks)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# The sources the bench step's kernel (heston_paths_kernel) is compiled from.
PATH_KERNEL_SOURCES = ("paper_2402_12111_gb300/csrc/simr_paths.cu", "paper_2402_12111_gb300/csrc/simr_device.cuh",
                       "paper_2402_12111_gb300/csrc/simr_reduce.cuh", "paper_2402_12111_gb300/csrc/simr_internal.h",
                       "include/simr.h")


def _code_only(text: str) -> str:
    """C/C++ source without its comments, blank lines and indentation (string literals kept as they are)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"':
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(ln.strip() for ln in "".join(out).splitlines() if ln.strip())


def kernel_source_sha() -> str:
    """Hash of the code (comments aside) the bench step's kernel is compiled from."""
    h = hashlib.sha256()
    for name in PATH_KERNEL_SOURCES:
        with open(os.path.join(ROOT, name), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


PATH_KERNEL_PROFILE = os.path.join("profiles", "heston_paths_grid32_252x1048576.txt")
ADJOINT_KERNEL_SOURCES = ("paper_2402_12111_gb300/csrc/simr_adjoint.cu",
                          "paper_2402_12111_gb300/csrc/simr_adjoint_path.cuh") + PATH_KERNEL_SOURCES[1:]
ADJOINT_KERNEL_PROFILE = os.path.join("profiles", "heston_adjoint_grid32_252x1048576.txt")


def adjoint_source_sha() -> str:
    """Hash of the code (comments aside) the adjoint kernel is compiled from."""
    h = hashlib.sha256()
    for name in ADJOINT_KERNEL_SOURCES:
        with open(os.path.join(ROOT, name), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def _profile_values(sha: str, profile: str = PATH_KERNEL_PROFILE) -> dict:
    """The key: value lines of a committed ncu summary, if it was taken on the current kernel
    sources (else {})."""
    try:
        lines = open(os.path.join(ROOT, profile)).read().splitlines()
    except OSError:
        return {}
    kv = {}
    for ln in lines:
        if ":" in ln:
            k, v = ln.split(":", 1)
            kv[k.strip()] = v.strip()
    return kv if kv.get("kernel_source_sha") == sha else {}


def profiled_adjoint_k32_traffic(sha: str):
    """DRAM bytes per launch of the adjoint kernel at a checkpoint every 32 steps from the committed
    ncu summary (or None).  Captured at 2^22 paths: the kernel's only DRAM traffic is its partial rows,
    one per block of the persistent grid, which does not grow with the paths."""
    try:
        return float(_profile_values(sha, ADJOINT_KERNEL_PROFILE)["traffic_bytes_per_launch_k32"])
    except (KeyError, ValueError):
        return None


def profiled_traffic(sha: str):
    """DRAM bytes per launch of the path kernel from the committed ncu summary (or None)."""
    try:
        return float(_profile_values(sha)["traffic_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def profiled_pipes(sha: str):
    """The path kernel's ncu pipe utilisation from the committed summary (or None)."""
    kv = _profile_values(sha)
    keys = ("fmaheavy_pipe_cycles_active_pct_of_active", "fmalite_pipe_cycles_active_pct_of_active",
            "xu_pipe_cycles_active_pct_of_active", "issue_active_pct_of_active")
    try:
        out = {k: float(kv[k]) for k in keys}
    except (KeyError, ValueError):
        return None
    out["source"] = PATH_KERNEL_PROFILE
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.out = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.out = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.out:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_run(w, paths_sample: int, with_result: bool = False):
    """One oracle pass (price + the same FD Greeks) on paths [0, paths_sample) of the workload:
    its wall time (and its (price, greeks) with with_result)."""
    import oracle

    bits = {"delta": oracle.G_DELTA, "gamma": oracle.G_GAMMA, "vega": oracle.G_VEGA, "theta": oracle.G_THETA,
            "rho": oracle.G_RHO}
    mask = sum(bits[g] for g in w.greeks)
    t0 = time.perf_counter()
    res = oracle.greeks_fd(w.model, w.strikes, w.is_put, w.steps, paths_sample, w.seed, w.rel_bump, mask)
    dt = time.perf_counter() - t0
    return (dt, res) if with_result else dt


def cpu_baseline(w, paths_sample: int = 1 << 20):
    """The oracle on the host cores; by default the whole workload (2^20 paths, ~12 s on 16 cores).
    Returns the baseline record and, for a whole-workload run, the oracle's (price, greeks)."""
    import oracle

    oracle.build()
    cores = oracle.max_threads()
    paths_sample = min(paths_sample, w.paths)
    dt, res = cpu_oracle_run(w, paths_sample, with_result=True)
    rec = {"value": paths_sample * w.steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{w.name}: paths [0, {paths_sample}) of {w.paths}, all {w.steps} steps, all "
                     f"{len(w.strikes)} strikes and the same Greeks; {dt:.2f} s wall on {cores} threads"}
    return rec, (res if paths_sample == w.paths else None)


def result_errors(gpu, ref):
    """Per column: "rel", the largest |GPU - oracle| / |oracle| over the strikes whose oracle value
    is at least 1e-3 of the column's largest, and "rel_col", the largest |GPU - oracle| over the
    column's largest |oracle|."""
    gpu, ref = np.asarray(gpu, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    scale = np.abs(ref).max()
    keep = np.abs(ref) >= 1e-3 * scale
    err = np.abs(gpu - ref)
    return {"rel": float(np.max(err[keep] / np.abs(ref[keep]))), "rel_col": float(err.max() / scale)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = workloads.grid()
    import oracle

    oracle.build()
    cores = oracle.max_threads()
    sample = 1 << 13
    for _ in range(max(args.warmup, 3)):
        cpu_oracle_run(w, sample)
    times = [cpu_oracle_run(w, sample) for _ in range(args.steps)]
    total = sum(times)
    value = args.steps * sample * w.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "paths": w.paths, "time_steps": w.steps, "strikes": len(w.strikes),
                       "greeks": greek_list(w), "rel_bump": w.rel_bump, "seed": w.seed,
                       "sample_paths_per_step": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"paths [0, {sample}) of {w.paths} per step, all {w.steps} steps, "
                                       f"{len(w.strikes)} strikes, same Greeks"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_profile_leg(args):
    """One kind of call, W + K times, for an external profiler."""
    import torch

    import paper_2402_12111_gb300 as simr

    w = workloads.grid()
    if args.paths:
        w.paths = args.paths
    if args.time_steps:
        w.steps = args.time_steps
    K = torch.as_tensor(w.strikes, dtype=torch.float64, device="cuda")
    legs = {
        "fd": lambda: simr.greeks_fd(w.model, K, w.is_put, w.steps, w.paths, w.seed, greeks=list(w.greeks),
                                     rel_bump=w.rel_bump),
        "price": lambda: simr.price(w.model, K, w.is_put, w.steps, w.paths, w.seed),
        "adjoint": lambda: simr.greeks_adjoint(w.model, K, w.is_put, w.steps, w.paths, w.seed,
                                               ckpt_every=args.ckpt_every),
    }
    if args.profile_leg in ("book", "book_price"):
        opts = workloads.book(n_options=128, paths_range=(16384, args.paths or 1 << 18))
        adj = args.profile_leg == "book"
        fn = lambda: simr.batch(opts, seed=1, adjoint=adj, autotune=False)  # noqa: E731
    elif args.profile_leg == "basket":
        bm, C, wts, kb, bsteps, bpaths = workloads.basket()
        Kb = torch.as_tensor(kb, dtype=torch.float64, device="cuda")
        n = args.paths or bpaths
        fn = lambda: simr.basket_price(bm, C, wts, Kb, False, bsteps, n, 1)  # noqa: E731
    elif args.profile_leg == "lsm":
        lw = workloads.lsm()
        n = args.paths or lw.paths
        fn = lambda: simr.lsm_price(lw.model, float(lw.strikes[0]), True, lw.steps, 1, n, lw.seed)  # noqa: E731
    else:
        fn = legs[args.profile_leg]
    for _ in range(args.warmup + args.steps):
        fn()
    torch.cuda.synchronize()
    return 0


def run_headline(args, simr, dev, stream):
    """The 8-underlying headline workload: price + adjoint Greeks at a checkpoint every 32 steps."""
    import torch

    hw = workloads.headline()
    fd7 = ("delta", "vega", "rho", "kappa", "lrvar", "volvol", "corr")
    ps_head = sum(u.steps * u.paths for u in hw)
    k_cfg = 32
    head = {"metric": "Heston path-steps/s (price + adjoint Greeks, checkpoint every 32 steps) on 1 GB300",
            "unit": UNIT, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "heston_book8_1024x67108864_adjoint_k32", "underlyings": len(hw),
                       "time_steps": hw[0].steps, "paths": hw[0].paths, "strikes": len(hw[0].strikes),
                       "ckpt_every": k_cfg, "sensitivities": ["S0", "v0", "kappa", "theta", "sigma", "rho", "r"],
                       "path_steps": ps_head,
                       "l2": "inputs (model, strikes) negligible; each pass reads and writes far more than L2"},
            "library_ckpt_every": simr.adjoint_interval(len(hw[0].strikes), hw[0].steps, dev.index or 0)}
    Kh = [torch.as_tensor(u.strikes, dtype=torch.float64, device=dev) for u in hw]
    legs = {
        "price": lambda u, k: simr.price(u.model, k, u.is_put, u.steps, u.paths, u.seed),
        "adjoint_k32": lambda u, k: simr.greeks_adjoint(u.model, k, u.is_put, u.steps, u.paths, u.seed,
                                                        ckpt_every=k_cfg),
        # the library's interval (one segment of the whole path in global memory, no forward pass)
        "adjoint_lib": lambda u, k: simr.greeks_adjoint(u.model, k, u.is_put, u.steps, u.paths, u.seed),
        "fd7": lambda u, k: simr.greeks_fd(u.model, k, u.is_put, u.steps, u.paths, u.seed, greeks=fd7,
                                           rel_bump=u.rel_bump),
    }
    clk_k32 = None
    for name, fn in legs.items():
        u0 = hw[0]
        small = workloads.Workload(u0.name, u0.model, u0.strikes, u0.steps, 1 << 16, ckpt_every=u0.ckpt_every)
        fn(small, Kh[0])  # warm-up (context scratch, module load)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev.index or 0) as clk:
            a.record(stream)
            for u, k in zip(hw, Kh):
                fn(u, k)
            b.record(stream)
            torch.cuda.synchronize()
        if name == "adjoint_k32":
            clk_k32 = clk.summary()
        sec = a.elapsed_time(b) * 1e-3
        head[f"{name}_s"] = sec
        head[f"{name}_path_steps_per_s"] = ps_head / sec
    head["value"] = head["adjoint_k32_path_steps_per_s"]
    head["ms_per_step"] = head["adjoint_k32_s"] * 1e3 / len(hw)  # one underlying = one launch
    head["adjoint_k32_cost_vs_price"] = head["adjoint_k32_s"] / head["price_s"]
    head["adjoint_lib_cost_vs_price"] = head["adjoint_lib_s"] / head["price_s"]
    head["adjoint_k32_speedup_vs_fd"] = head["fd7_s"] / head["adjoint_k32_s"]
    head["clocks"] = clk_k32
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clk_k32.get("sm_mhz") or float(measured_peaks().get("sm_max_mhz", 2070.0))
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    flops = FLOPS_SHARED + FLOPS_PER_SCENARIO + FLOPS_ADJOINT_REVERSE
    achieved = flops * ps_head / head["adjoint_k32_s"] / 1e12
    head["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": profiled_adjoint_k32_traffic(adjoint_source_sha()),
                        "traffic_source": ADJOINT_KERNEL_PROFILE,
                        "peak_kind": f"derived: {props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes "
                                     f"x 2 x {sm_mhz:.0f} MHz (the median SM clock sampled during the pass)",
                        "flops_per_path_step": flops,
                        "kernel": "heston_adjoint_kernel (shared-memory segments of 32 steps)"}
    # end to end through the public API with host buffers: strikes in, prices and 7 Greeks out
    if not args.no_e2e:
        K_host = [torch.as_tensor(u.strikes, dtype=torch.float64).pin_memory() for u in hw]
        simr.greeks_adjoint(hw[0].model, K_host[0], hw[0].is_put, hw[0].steps, 1 << 16, hw[0].seed,
                            ckpt_every=k_cfg, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out_b = 0
        for u, k in zip(hw, K_host):
            p_h, se_h, g_h = simr.greeks_adjoint(u.model, k, u.is_put, u.steps, u.paths, u.seed, ckpt_every=k_cfg,
                                                 device=dev)
            out_b += (p_h.numel() + se_h.numel() + g_h.numel()) * 8
        e2e_s = time.perf_counter() - t0
        head["e2e"] = {"value": ps_head / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": sum(k.numel() for k in K_host) * 8 // len(hw),
                       "d2h_bytes_per_step": out_b // len(hw), "steps": len(hw),
                       "note": "one step = one underlying's call with host strike and result buffers"}
    # the FP64 oracle's reverse mode on the host cores, on a path sample of every underlying
    if not args.no_cpu_baseline:
        import oracle

        oracle.build()
        n_s = 1 << 10
        t0 = time.perf_counter()
        for u in hw:
            oracle.adjoint(u.model, u.strikes, u.is_put, u.steps, n_s, u.seed)
        dt = time.perf_counter() - t0
        cores = oracle.max_threads()
        head["cpu_baseline"] = {"value": len(hw) * n_s * hw[0].steps / dt, "unit": UNIT, "cores": cores,
                                "kind": "oracle",
                                "sample": f"paths [0, {n_s}) of each of the {len(hw)} underlyings, all "
                                          f"{hw[0].steps} steps and {len(hw[0].strikes)} strikes, price + the 7 "
                                          f"pathwise sensitivities; {dt:.2f} s wall on {cores} threads"}
    return head


def run_native(args):
    import torch

    import paper_2402_12111_gb300 as simr

    rank, world, local = dist_env()
    if world != args.gpus:
        print(f"warning: --gpus {args.gpus} but WORLD_SIZE {world}", file=sys.stderr)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    w = workloads.grid()
    if args.paths:
        w.paths = args.paths
        w.name = f"{w.name}_paths{args.paths}"
    greeks = greek_list(w)
    mask = simr.greek_mask(greeks)
    K = torch.as_tensor(w.strikes, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    path_begin = rank * w.paths

    def step():
        if world == 1:
            return simr.greeks_fd(w.model, K, w.is_put, w.steps, w.paths, w.seed, greeks=mask, rel_bump=w.rel_bump)
        return simr.path_sums(w.model, K, w.is_put, w.steps, path_begin, w.paths, seed=w.seed, greeks=mask,
                              rel_bump=w.rel_bump)

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        step()
        flush.zero_()
    barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        t_wall = time.perf_counter()
        for i in range(args.steps):
            starts[i].record(stream)
            out = step()
            ends[i].record(stream)
            flush.zero_()
        barrier()
        t_wall = time.perf_counter() - t_wall
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = sum(step_ms) / len(step_ms)
    ms_t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if pg is not None:
        pg.all_reduce(ms_t, op=pg.ReduceOp.MAX)
        sums = out.clone()
        pg.all_reduce(sums)
    ms = float(ms_t.item())
    path_steps = w.paths * w.steps
    value = world * path_steps / (ms * 1e-3)

    # end to end through the public API with host buffers (pinned strikes in, results out)
    e2e = None
    if not args.no_e2e:
        K_host = torch.as_tensor(w.strikes, dtype=torch.float64).pin_memory()
        e2e_steps = max(5, min(args.steps, 20))
        simr.greeks_fd(w.model, K_host, w.is_put, w.steps, w.paths, w.seed, greeks=mask, rel_bump=w.rel_bump,
                       device=dev)
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            p_h, g_h = simr.greeks_fd(w.model, K_host, w.is_put, w.steps, w.paths, w.seed, greeks=mask,
                                      rel_bump=w.rel_bump, device=dev)
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        e2e_t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        if pg is not None:
            pg.all_reduce(e2e_t, op=pg.ReduceOp.MAX)
        e2e = {"value": world * path_steps / float(e2e_t.item()), "unit": UNIT,
               "h2d_bytes_per_step": K_host.numel() * 8, "d2h_bytes_per_step": (p_h.numel() + g_h.numel()) * 8,
               "steps": e2e_steps}

    # adjoint vs bump-and-revalue on the same GPU and workload (the adjoint workload:
    # 7 sensitivities d/d{S0, v0, kappa, theta, sigma, rho, r}, the library's checkpoint interval)
    adj = None
    if not args.no_adjoint:
        fd7 = ("delta", "vega", "rho", "kappa", "lrvar", "volvol", "corr")
        legs = {
            "price_ms": lambda: simr.price(w.model, K, w.is_put, w.steps, w.paths, w.seed),
            "fd7_ms": lambda: simr.greeks_fd(w.model, K, w.is_put, w.steps, w.paths, w.seed, greeks=fd7,
                                             rel_bump=w.rel_bump),
            "adjoint_ms": lambda: simr.greeks_adjoint(w.model, K, w.is_put, w.steps, w.paths, w.seed),
            # the same with a checkpoint every 16 steps (shared-memory segments, forward pass)
            "adjoint_k16_ms": lambda: simr.greeks_adjoint(w.model, K, w.is_put, w.steps, w.paths, w.seed,
                                                          ckpt_every=16),
        }
        adj = {}
        reps = max(3, min(args.steps, 10))
        for name, fn in legs.items():
            for _ in range(3):
                fn()
                flush.zero_()
            times = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                flush.zero_()
                times.append((a, b))
            torch.cuda.synchronize()
            adj[name] = sum(x.elapsed_time(y) for x, y in times) / reps
        # the pricing pass, the adjoint and the 7-Greek bump-and-revalue under QE-M
        # (Andersen's martingale correction)
        simr.set_scheme("qem", dev.index or 0)
        try:
            for name in ("price_ms", "adjoint_ms", "fd7_ms"):
                for _ in range(3):
                    legs[name]()
                    flush.zero_()
                times = []
                for _ in range(reps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    legs[name]()
                    b.record(stream)
                    flush.zero_()
                    times.append((a, b))
                torch.cuda.synchronize()
                adj[name.replace("_ms", "_qem_ms")] = sum(x.elapsed_time(y) for x, y in times) / reps
        finally:
            simr.set_scheme("qe", dev.index or 0)
        adj["qem_cost_vs_qe"] = adj["price_qem_ms"] / adj["price_ms"]
        adj["qem_adjoint_cost_vs_price"] = adj["adjoint_qem_ms"] / adj["price_qem_ms"]
        adj["speedup_vs_fd"] = adj["fd7_ms"] / adj["adjoint_ms"]
        adj["cost_vs_price"] = adj["adjoint_ms"] / adj["price_ms"]
        adj["k16_cost_vs_price"] = adj["adjoint_k16_ms"] / adj["price_ms"]
        adj["ckpt_every"] = simr.adjoint_interval(len(w.strikes), w.steps, dev.index or 0)  # the library's choice
        adj["sensitivities"] = list(fd7)

    # heterogeneous book: 1,024 options (log-uniform steps and paths), one persistent launch
    # per submission, replayed from a captured CUDA graph; prices, then prices + adjoint Greeks
    book = None
    if not args.no_book:
        opts = workloads.book()
        ps_book = sum(o["steps"] * o["paths"] for o in opts)
        book = {"options": len(opts), "path_steps": ps_book}
        for name, adj_flag in (("price", False), ("adjoint", True)):
            simr.batch(opts, seed=1, adjoint=adj_flag, graph=True)  # autotune + capture
            simr.batch(opts, seed=1, adjoint=adj_flag, graph=True)
            torch.cuda.synchronize()
            reps = 3
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                simr.batch(opts, seed=1, adjoint=adj_flag, graph=True)
            b.record(stream)
            torch.cuda.synchronize()
            ms_b = a.elapsed_time(b) / reps
            book[f"{name}_ms"] = ms_b
            book[f"{name}_path_steps_per_s"] = ps_book / (ms_b * 1e-3)

    # the paper's problem sizes (Table 1: A assets analysed x T steps x P paths), each
    # as one batched submission of A independent options: elements (A T P) per second
    paper = None
    if not args.no_book:
        paper = {}
        for size in workloads.PAPER_SIZES:
            opts = workloads.paper_book(size)
            simr.batch(opts, seed=1, graph=True)
            simr.batch(opts, seed=1, graph=True)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 10
            a.record(stream)
            for _ in range(reps):
                simr.batch(opts, seed=1, graph=True)
            b.record(stream)
            torch.cuda.synchronize()
            ms_p = a.elapsed_time(b) / reps
            paper[size] = {"A": workloads.PAPER_SIZES[size][0], "T": workloads.PAPER_SIZES[size][1],
                           "P": workloads.PAPER_SIZES[size][2], "elements": workloads.paper_elements(size),
                           "ms": ms_p, "elements_per_s": workloads.paper_elements(size) / (ms_p * 1e-3)}

    # correlated basket: 8 assets (book-style parameters), 252 steps, 2^20 paths,
    # 32 strikes on the equally weighted basket
    basket = None
    if not args.no_book:
        bm, C, wts, kb, bsteps, bpaths = workloads.basket()
        Kb = torch.as_tensor(kb, dtype=torch.float64, device=dev)
        call = lambda: simr.basket_price(bm, C, wts, Kb, False, bsteps, bpaths, 1)  # noqa: E731
        call()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(5):
            call()
        b.record(stream)
        torch.cuda.synchronize()
        ms_b = a.elapsed_time(b) / 5
        basket = {"assets": 8, "time_steps": 252, "paths": 1 << 20, "strikes": int(Kb.numel()), "ms": ms_b,
                  "asset_path_steps_per_s": 8 * 252 * (1 << 20) / (ms_b * 1e-3)}

    # large-scale headline: 8 underlyings (book-style parameters), 32 strikes each,
    # 1,024 steps, 2^26 paths; price plus adjoint Greeks with a checkpoint every 32
    # steps -- a record of its own (metric, value, roofline, e2e, cpu_baseline) --
    # beside the library's interval, a pricing pass and CRN bump-and-revalue of the
    # same 7 sensitivities, one timed pass each
    head = None
    if not args.no_headline:
        head = run_headline(args, simr, dev, stream)

    # Longstaff-Schwartz Bermudan put (252 steps, exercisable after every step, 2^20
    # paths): the path kernel, then the backward induction (one cooperative sweep
    # launch); the per-date cost is the difference to a one-date valuation (path
    # kernel + the final reduction) over the remaining dates
    lsm_leg = None
    if not args.no_lsm:
        lw = workloads.lsm()
        K_l = float(lw.strikes[0])
        every = lw.extra["exercise_every"]
        n_ex = lw.steps // every

        def lsm_time(ev, reps=5):
            simr.lsm_price(lw.model, K_l, True, lw.steps, ev, lw.paths, lw.seed)
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                simr.lsm_price(lw.model, K_l, True, lw.steps, ev, lw.paths, lw.seed)
                b.record(stream)
                flush.zero_()
                ts.append((a, b))
            torch.cuda.synchronize()
            return sum(x.elapsed_time(y) for x, y in ts) / reps

        ms_all = lsm_time(every)
        ms_one = lsm_time(lw.steps)
        per_date_us = 1e3 * (ms_all - ms_one) / max(n_ex - 1, 1)
        date_bytes = 8 * lw.paths  # per date the sweep reads each path's S and v of that date once
        hbm = float(measured_peaks().get("hbm_gbs", 6800.0))
        gbs = date_bytes / (per_date_us * 1e-6) / 1e9
        lsm_leg = {"workload": lw.name, "exercise_dates": n_ex, "ms": ms_all,
                   "path_steps_per_s": lw.paths * lw.steps / (ms_all * 1e-3),
                   "path_kernel_plus_one_date_ms": ms_one, "per_date_us": per_date_us,
                   "sweep_roofline": {"bound": "latency", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                      "frac": gbs / hbm, "bytes_per_date": date_bytes,
                                      "note": "each date waits on a grid barrier, a cross-block sum and a 6x6 "
                                              "solve; HBM traffic is a small fraction of the date's time"}}

    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return 0

    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    flops_step = flops_per_path_step(greeks)
    achieved_tflops = flops_step * path_steps / (ms * 1e-3) / 1e12  # per GPU, one launch per step
    sha = kernel_source_sha()
    # the units' measured throughput on this GPU (after the timed legs): the derived
    # FP32 peak above is the denominator, the measured packed-FMA rate its check
    rates = None if args.no_unit_rates else simr.unit_rates(dev if isinstance(dev, int) else dev.index or 0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "paths": w.paths, "time_steps": w.steps, "strikes": len(w.strikes),
                   "greeks": greeks, "rel_bump": w.rel_bump, "seed": w.seed,
                   "simulated_scenarios": simulated_scenarios(greeks),
                   "l2": "flushed between timed iterations (256 MiB write, outside the step events)",
                   "parallelism": f"paths sharded over {world} rank(s)"},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved_tflops / fp32_peak_tflops, "traffic": profiled_traffic(sha),
                     "peak_kind": f"derived: {props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 "
                                  f"x {sm_max:.0f} MHz (FMA = 2 flops)",
                     "flops_per_path_step": flops_step,
                     # the same kernel's FP32 (FMA) and MUFU pipe activity as ncu counts it, from the
                     # committed summary of this source (None if the sources changed since)
                     "ncu_pipes": profiled_pipes(sha),
                     "measured_fp32_fma2_tflops": rates["fp32_fma2_tflops"] if rates else None,
                     "frac_of_measured_fma2": achieved_tflops / rates["fp32_fma2_tflops"] if rates else None},
        "fp32_peak_frac": achieved_tflops / fp32_peak_tflops,
        "clocks": clk.summary(),
        "e2e": e2e,
        "gpu_launches": args.steps,
        "adjoint_vs_fd": adj,
        "book": book,
        "paper_sizes": paper,
        "basket": basket,
        "headline": head,
        "lsm": lsm_leg,
        "unit_rates": rates,
        "kernel_source_sha": sha,
        "wall_s_timed_region": t_wall,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"], ref = cpu_baseline(w)
        # the stated error of every result against the FP64 oracle on the same draws:
        # the bench step's price and Greeks (the baseline's oracle run is the same
        # workload), and the 7 adjoint sensitivities of the grid at 2^18 paths
        if ref is not None and world == 1:
            p_g, g_g = (t.cpu().numpy() for t in out)
            errs = {"price": result_errors(p_g, ref[0])}
            for j, n in enumerate(greeks):
                errs[n] = result_errors(g_g[:, j], ref[1][:, j])
            import oracle

            n_adj = 1 << 18
            pa, _, ga = simr.greeks_adjoint(w.model, K, w.is_put, w.steps, n_adj, w.seed, ckpt_every=16)
            pao, gao = oracle.adjoint(w.model, w.strikes, w.is_put, w.steps, n_adj, w.seed)
            aerr = {"price": result_errors(pa.cpu().numpy(), pao)}
            for j, n in enumerate(simr.ADJOINT_COLUMNS):
                aerr["d/d" + n] = result_errors(ga.cpu().numpy()[:, j], gao[:, j])
            line["errors"] = {
                "note": "rel: max over strikes of |GPU - oracle| / |oracle| (strikes with |oracle| >= 1e-3 of "
                        "the column's largest); rel_col: max |GPU - oracle| / max |oracle column|",
                f"{w.name}_fd": errs, f"heston_grid32_252x{n_adj}_adjoint_k16": aerr}
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_leg:
        return run_profile_leg(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
