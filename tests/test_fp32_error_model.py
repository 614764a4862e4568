"""The FP32 error model behind the GPU tolerances, reproduced on the CPU (no GPU).

The kernels run each path step in FP32.  Their tolerances against the FP64
oracle rest on the per-path error of x_T = ln(S_T/S0): it grows roughly like
sqrt(N) with a coefficient of order 1e-8.  This emulates one FP32 path step in
numpy float32 on the oracle's own uniforms.  Each operation is rounded to FP32
as a scalar FP32 instruction would round it, the normals are exact, and x is
Kahan-compensated as in the kernels.  Two algebraically equal forms of the
log-spot update are measured against the FP64 oracle:

* Andersen's form: K0 + K1 v + K2 v' + sqrt(K3 v + K4 v') Z_X, whose
  -rho/sigma and +rho/sigma terms nearly cancel;
* the form the kernels use: with s = v + v', m the conditional mean and
  dl = v' - m,
      r dt - (dt/4) s + Cd (theta - v) + Cdl dl + sqrt(dt (1 - rho^2) / 2) sqrt(s) Z_X,
  where Cdl = (rho/sigma)(1 + kappa dt/2) and
  Cd = (rho/sigma)(1 - E - kappa dt (1 + E)/2) = O((kappa dt)^3).  In the
  quadratic branch dl = a (Z_V (Z_V + 2b) - 1) needs no subtraction of m.

The second form has a third (at 16-64 steps) to an eighth (at 252) of the first
one's error, which is why the kernels use it.
"""
import math

import numpy as np
import pytest
from scipy.special import ndtri

import oracle
import workloads

f32 = np.float32


def _uniforms(seed, paths, steps):
    U = np.empty((steps, 2, paths))
    for n in range(steps):
        for p in range(paths):
            U[n, 0, p], U[n, 1, p] = oracle.step_uniforms(seed, 0, p, n)
    return U


def _fp32_paths(m, steps, U, form):
    """x_T of each path with every operation of the step rounded to FP32."""
    P = U.shape[2]
    dt, k, th, sg, rho = m["T"] / steps, m["kappa"], m["theta"], m["sigma"], m["rho"]
    E, omE = math.exp(-k * dt), -math.expm1(-k * dt)
    Ef, thf = f32(E), f32(th)
    c1, c2 = f32(sg * sg * E * omE / k), f32(th * sg * sg * omE * omE / (2 * k))
    K = oracle.qe_constants(m, steps)
    K0, K1, K2, K3, K4 = (f32(K[n]) for n in ("K0", "K1", "K2", "K3", "K4"))
    rs = rho / sg
    C0, Cv = f32(m["r"] * dt), f32(-0.25 * dt)
    Cd, Cdl = f32(rs * (omE - 0.5 * k * dt * (1 + E))), f32(rs * (1 + 0.5 * k * dt))
    sK3 = f32(math.sqrt(0.5 * dt * (1 - rho * rho)))
    one, two = f32(1), f32(2)
    v = np.full(P, f32(m["v0"]))
    x = np.zeros(P, f32)
    comp = np.zeros(P, f32)
    for n in range(steps):
        uv, ux = U[n, 0], U[n, 1]
        zv, zx, uvf = ndtri(uv).astype(f32), ndtri(ux).astype(f32), uv.astype(f32)
        mm = thf + (v - thf) * Ef
        ss = v * c1 + c2
        with np.errstate(all="ignore"):
            psi = ss / (mm * mm)
            quad = psi <= f32(1.5)
            t = two / psi
            b2 = (t - one) + np.sqrt(t) * np.sqrt(t - one)
            a = mm / (one + b2)
            b = np.sqrt(b2)
            vq = a * (b + zv) * (b + zv)
            dlq = a * (zv * (zv + two * b) - one)
            p = (psi - one) / (psi + one)
            beta = (one - p) / mm
            ve = np.where(uvf <= p, f32(0), np.log((one - p) / (one - uvf)) / beta).astype(f32)
        live = mm > 0
        vn = np.where(live, np.where(quad, vq, ve), f32(0)).astype(f32)
        dl = np.where(live & quad, dlq, vn - mm).astype(f32)
        if form == "andersen":
            inc = K0 + K1 * v + K2 * vn + np.sqrt(K3 * v + K4 * vn) * zx
        else:
            s = v + vn
            inc = C0 + Cv * s + Cd * (thf - v) + Cdl * dl + sK3 * np.sqrt(s) * zx
        y = inc.astype(f32) - comp
        tt = x + y
        comp = (tt - x) - y
        x = tt
        v = vn
    assert x.dtype == f32 and v.dtype == f32  # no operation was promoted to FP64
    return x.astype(np.float64) - comp.astype(np.float64)


@pytest.mark.parametrize("steps", [16, 64, 252])
def test_fp32_path_error_and_the_rewritten_log_spot_step(steps):
    # measured rms / sqrt(N): Andersen's form 1.4e-8, 1.7e-8, 5.9e-8 and the
    # kernels' form 6.5e-9, 5.4e-9, 7.0e-9 at 16, 64 and 252 steps
    m = dict(workloads.BASE_MODEL)
    P = 2048
    U = _uniforms(1, P, steps)
    x64, _, _ = oracle.terminal(m, steps, 1, 0, P)
    rms = {f: float(np.sqrt(np.mean((_fp32_paths(m, steps, U, f) - x64) ** 2))) for f in ("andersen", "kernel")}
    # the kernels' form: FP32 round-off growing like sqrt(N) with a coefficient near 1e-8 ...
    assert 1e-9 * math.sqrt(steps) < rms["kernel"] < 2e-8 * math.sqrt(steps), rms
    # ... and at most half of the error of the form with the cancelling terms
    assert rms["kernel"] < 0.5 * rms["andersen"], rms
