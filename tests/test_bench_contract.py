"""bench.py's output contract, checked on its CPU arm (no GPU).

`bench.py --impl reference` times the FP64 oracle on the host cores and prints
one JSON line with the same keys as the GPU arm; under torchrun only rank 0
prints, the other ranks exit 0 without work.  The GPU arm's line (the same
keys plus roofline, clocks and gpu_launches) needs a GPU and is produced by the
GPU runs of bench.py.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
COMMON = {"metric": str, "value": float, "unit": str, "n_gpus": int, "steps": int, "warmup": int,
          "ms_per_step": float, "higher_is_better": bool, "scaling": str, "dtype": str, "data": str,
          "config": dict, "cpu_baseline": dict, "e2e": dict}


def _json_lines(out):
    return [json.loads(line) for line in out.splitlines() if line.startswith("{")]


def _check_reference_line(line, n_gpus):
    for key, kind in COMMON.items():
        assert isinstance(line[key], kind), (key, line.get(key))
    assert line["impl"] == "reference"
    assert line["n_gpus"] == n_gpus and line["steps"] == 1 and line["warmup"] >= 3
    assert line["value"] > 0 and line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["dtype"] == "f64" and line["data"] == "synthetic"
    assert line["config"]["workload"] == "heston_grid32_252x1048576"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_prints_one_contract_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = _json_lines(p.stdout)
    assert len(lines) == 1, p.stdout
    _check_reference_line(lines[0], 1)


def test_reference_arm_under_torchrun_prints_once():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4"))
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = _json_lines(p.stdout)
    assert len(lines) == 1, p.stdout
    _check_reference_line(lines[0], 2)


@pytest.mark.parametrize("flag", ["--no-e2e", "--no-book", "--no-lsm", "--no-adjoint", "--no-headline"])
def test_bench_flags_are_accepted(flag):
    # argument parsing only: --help exits before any work
    p = subprocess.run([sys.executable, "bench.py", flag, "--help"], cwd=ROOT, capture_output=True, text=True,
                       timeout=120)
    assert p.returncode == 0 and "--profile-leg" in p.stdout


def _bench():
    sys.path.insert(0, ROOT)
    import bench

    return bench


def test_algorithmic_flops_of_the_bench_step():
    # 44 flops shared per step (two inverse normals) + 23 per simulated scenario (QE
    # variance step 16, log-spot step 7); the bench step simulates base, v0 +- and
    # T +- (delta, gamma and rho revalue the base path); pricing alone is 67
    b = _bench()
    g5 = ["delta", "gamma", "vega", "theta", "rho"]
    assert b.simulated_scenarios(g5) == 5
    assert b.flops_per_path_step(g5) == 159
    assert b.flops_per_path_step([]) == 67
    assert b.simulated_scenarios(["delta", "vega", "rho", "kappa", "lrvar", "volvol", "corr"]) == 11


def test_clock_summary_reads_clocks_and_throttle_reasons():
    b = _bench()
    s = b.ClockSampler(0)
    s.out = ["0, 2070, 2070, 910.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2055, 2070, 1101.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 2040, 2070, 1200.5, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
             "garbage line"]
    out = s.summary()
    assert out["sm_mhz"] == 2055 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    s.out = []
    assert s.summary()["reasons"] == ["unsampled"]


def test_profile_provenance_is_parsed_by_source_hash():
    # roofline.traffic comes from a committed ncu summary only when the summary names
    # the hash of the sources the kernel is compiled from; any other hash gives None
    import bench

    assert len(bench.kernel_source_sha()) == 16 and len(bench.adjoint_source_sha()) == 16
    assert bench.profiled_traffic("0" * 16) is None
    assert bench.profiled_adjoint_k32_traffic("0" * 16) is None
    t = bench.profiled_traffic(bench.kernel_source_sha())
    assert t is None or t > 0


def test_committed_profiles_were_taken_on_the_current_kernel_sources():
    # the bench-step and adjoint summaries under profiles/ name the hashes of the
    # sources they were captured on; a change to those sources (comments aside)
    # needs a new capture, else the bench line's roofline.traffic goes null
    import bench

    assert bench.profiled_traffic(bench.kernel_source_sha()) is not None, "re-capture the bench-step profile"
    assert bench.profiled_adjoint_k32_traffic(bench.adjoint_source_sha()) is not None, "re-capture the adjoint profile"
