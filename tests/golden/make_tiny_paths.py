"""Writes tiny_paths.txt: per-path terminal states of the FP64 oracle on tiny cases.

Run from the repository root: python tests/golden/make_tiny_paths.py
It calls the oracle alone (oracle.terminal: Andersen's QE scheme for Heston on the
Philox4x32-10 counters); the file is a regression fixture of the oracle's paths at
1 and 2 steps, 8 paths, for two models, which the GPU's per-path output must
reproduce within FP32 rounding.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

MODELS = {
    "standard": dict(S0=100.0, r=0.05, T=1.0, v0=0.04, kappa=1.5, theta=0.04, sigma=0.3, rho=-0.7),
    "vol_of_vol_0.9": dict(S0=100.0, r=0.05, T=1.0, v0=0.09, kappa=1.0, theta=0.04, sigma=0.9, rho=-0.3),
}
SEED, PATHS = 7, 8


def main():
    lines = ["# Terminal states of the FP64 oracle (oracle.terminal, Andersen 2008 QE for Heston 1993;",
             "# Philox4x32-10 counters, seed 7, option index 0): model steps path x_T v_T",
             "# written by tests/golden/make_tiny_paths.py"]
    for name, m in MODELS.items():
        for steps in (1, 2):
            x, v, _ = oracle.terminal(m, steps, SEED, 0, PATHS)
            for p in range(PATHS):
                lines.append(f"{name} {steps} {p} {float(x[p])!r} {float(v[p])!r}")
    with open(os.path.join(HERE, "tiny_paths.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
