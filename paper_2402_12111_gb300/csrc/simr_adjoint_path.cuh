// simr_adjoint_path.cuh -- per-path pathwise adjoint of the Heston QE path (forward pass
// with checkpoints, reverse sweep), shared by the per-strike adjoint kernel and
// the batched book kernel.  See simr_adjoint.cu for the method.
#pragma once

#include <cstdint>

#include "simr_device.cuh"
#include "simr_internal.h"

#ifndef SIMR_ADJ_PREFETCH
#define SIMR_ADJ_PREFETCH 4  // steps ahead the reverse sweep asks global segment data into L2 (4-32 within 2%)
#endif

namespace simr {
namespace {

// One QE variance step from v given the step's draws (no log-spot update).
__device__ __forceinline__ float qe_only(const ScenConst& c, float v, float xv, float zv) {
  float vn, dl;
  qe_from_moments(fmaf(v, c.E, c.thE), fmaf(v, c.h1, c.h2), xv, zv, vn, dl);
  return vn;
}

struct AdjSums {
  float vbar, Am, Amv, As, Asv, Ad, Adl, Ak3;
  float x, comp;  // x_T accumulated over the reverse sweep (Kahan-compensated)
  // QE-M only: sum (v + m), sum (v' - m) and sum lam's A-adjoint over the corrected
  // steps, and the count of steps that took the plain log-spot step
  float Aqa, AK2, AA, Np;
};

// What a reverse step needs besides the adjoint carried in from the later steps.
// Common to both branches: the log-spot increment inc and the innovation dl,
// q = sqrt(v + v'), Z_X, hzc = Cv + d(sK3 q Z_X)/ds (s = v + v'), hzcd = hzc - Cd
// and tmv = theta - v.  Quadratic branch: the factors of the chain from the
// adjoint of v' to those of m and s^2 (with t = m^2 / (s^2/2) formed exactly as
// the forward step forms it, qe_t, so the two take the same branch):
//   v' = a (b + Z_V)^2, dl = a g, g = Z_V (Z_V + 2b) - 1, a = m / (1 + b^2):
//   abar = vnbar bz^2 + Cdl g,  bbar = 2 a (vnbar bz + Cdl Z_V),
//   b2bar = bbar / (2b) - abar a / (1 + b^2),  mbar = abar / (1 + b^2) + tbar 4m / s^2,
//   tbar = b2bar (1 + (2t - 1) / (2 sqrt(t(t - 1)))),  s2bar = -tbar t / s^2,
// the factors (bz, bz^2, Cdl g, Cdl Z_V, 2a, 1/(2b), a/(1 + b^2), 1/(1 + b^2), the
// bracket F, 4m/s^2, t/s^2) all functions of the step's state and draws.
struct AdjPre {
  float inc, dl, q, zx, hzc, hzcd, tmv, vc;
  float bz, bz2, cg, cz, am2, hrb, amr, ropb2, F, m4r, tr;
  float am, b2, g;  // a, b^2 and g themselves (the QE-M step's correction needs them)
};

// a * b, rounded on its own when RN (no FMA formed by the compiler from it and a
// later sum), else left to the compiler.
template <bool RN>
__device__ __forceinline__ float mul_rn(float a, float b) {
  if constexpr (RN)
    return __fmul_rn(a, b);
  else
    return a * b;
}

// The quadratic branch's factors from m, t = m^2/(s^2/2), rs2h = 1/(s^2/2), Z_V
// (RN: for adjoint_step_qem, every product rounded on its own).
template <bool RN = false>
__device__ __forceinline__ void adj_quad_pre(const ScenConst& c, float m, float t, float rs2h, float zv, AdjPre& P) {
  const float tt = fmaf(t, t, -t);
  const float rroot = rsqrt_approx(tt);
  const float root = mul_rn<RN>(tt, rroot);
  const float b2 = (t - 1.0f) + root;
  const float rb = rsqrt_approx(b2);
  const float b = mul_rn<RN>(b2, rb);
  P.ropb2 = rcp_approx(t + root);  // 1 / (1 + b^2)
  const float am = mul_rn<RN>(m, P.ropb2);
  P.bz = b + zv;
  const float g = fmaf(zv, zv + 2.0f * b, -1.0f);
  P.am = am;
  P.b2 = b2;
  P.g = g;
  P.dl = mul_rn<RN>(am, g);
  P.bz2 = mul_rn<RN>(P.bz, P.bz);
  P.cg = mul_rn<RN>(c.Cdl, g);
  P.cz = mul_rn<RN>(c.Cdl, zv);
  P.am2 = am + am;
  P.hrb = 0.5f * rb;
  P.amr = mul_rn<RN>(am, P.ropb2);
  P.F = fmaf(fmaf(2.0f, t, -1.0f), 0.5f * rroot, 1.0f);
  P.m4r = mul_rn<RN>(m + m, rs2h);      // 4 m / s^2
  P.tr = mul_rn<RN>(t, 0.5f * rs2h);  // t / s^2
}

// The step's log-spot increment (LogPricePathQE), summed into x_T in the
// reverse sweep rather than in the forward pass.
__device__ __forceinline__ float adj_inc(const ScenConst& c, float s, float vc, float dl, float q, float zx) {
  float inc = fmaf(c.Cv, s, c.C0);
  inc = fmaf(-c.Cd, vc, inc);
  inc = fmaf(c.Cdl, dl, inc);
  return fmaf(c.sK3 * q, zx, inc);
}

// The end of a reverse step once mbar and s2bar are known: x_T's increment
// (Kahan-compensated), the adjoint of v_n, and the seven sums.
__device__ __forceinline__ void adj_tail(float E, float c1, const AdjPre& P, float mbar, float s2bar, AdjSums& a) {
  const float y = P.inc - a.comp;
  const float tx = a.x + y;
  a.comp = (tx - a.x) - y;
  a.x = tx;
  a.vbar = fmaf(mbar, E, fmaf(s2bar, c1, P.hzcd));
  a.Am += mbar;
  a.Amv = fmaf(-mbar, P.tmv, a.Amv);  // + mbar (v - theta)
  a.As += s2bar;
  a.Asv = fmaf(s2bar, P.vc, a.Asv);
  a.Ad += P.tmv;
  a.Adl += P.dl;
  a.Ak3 = fmaf(P.q, P.zx, a.Ak3);
}

// The adjoint chain of a quadratic-branch reverse step: from the adjoint of
// v_{n+1} through the QE map's derivatives to mbar and s2bar, then adj_tail.
__device__ __forceinline__ void adj_chain_quad(float E, float c1, const AdjPre& P, AdjSums& a) {
  const float vnbar = a.vbar + P.hzc;  // total adjoint of v_{n+1}
  const float abar = fmaf(vnbar, P.bz2, P.cg);
  const float bbar = P.am2 * fmaf(vnbar, P.bz, P.cz);
  const float b2bar = fmaf(bbar, P.hrb, -(abar * P.amr));
  const float tbar = b2bar * P.F;
  const float mbar = fmaf(tbar, P.m4r, abar * P.ropb2);
  const float s2bar = -(tbar * P.tr);
  adj_tail(E, c1, P, mbar, s2bar, a);
}

// The common part of a reverse step's quantities from vc, vn and Z_X.
__device__ __forceinline__ void adj_common_pre(const ScenConst& c, float theta, float vc, float vn, float zx,
                                               AdjPre& P) {
  const float s = vc + vn;
  const float rq = rsqrt_approx(s);
  const float sq = s * rq;
  const float hq = 0.5f * c.sK3 * zx * rq;
  P.q = s > 0.0f ? sq : 0.0f;
  P.zx = zx;
  P.hzc = (s > 0.0f ? hq : 0.0f) + c.Cv;  // Cv + d(sK3 sqrt(s) Z)/ds
  P.hzcd = P.hzc - c.Cd;
  P.tmv = theta - vc;
  P.vc = vc;
}

// The exponential branch's innovation dl = v' - m of a reverse step (m <= 0:
// v' = 0 and dl = 0), with d = 1 - U_V its stored draw; *atom: v' = 0 by the
// atom (W >= 2 m^2, the forward step's test).
__device__ __forceinline__ float adj_exp_dl(float m, float m2, float s2h, float vn, float d, bool* atom) {
  *atom = true;
  if (!(m > 0.0f)) return 0.0f;
  const float ms = m2 + (s2h + s2h);
  *atom = d * ms >= 2.0f * m2;
  return *atom ? -m : vn - m;
}

// The adjoint chain of an exponential-branch reverse step, then adj_tail (P.dl
// and P.inc already set by adj_exp_dl and adj_inc).
__device__ __forceinline__ void adj_chain_exp(float E, float c1, float Cdl, float m, float m2, float s2h, float d,
                                              bool atom, const AdjPre& P, AdjSums& a) {
  const float vnbar = a.vbar + P.hzc;  // total adjoint of v_{n+1}
  const float dlbar = Cdl;
  float mbar = 0.0f, s2bar = 0.0f;
  if (atom) {  // v' = 0 (the atom, or a zero mean): dl = -m
    mbar = -dlbar;
  } else {  // m > 0
    const float s2 = s2h + s2h;
    const float ms = m2 + s2;
    const float W = d * ms;
    const float rm = rcp_approx(m), rms = rcp_approx(ms);
    const float L = 0.69314718055994531f * lg2_approx(2.0f * m2 * rcp_approx(W));
    const float A = 0.5f * ms * rm;
    const float dA_dm = 0.5f * (m2 - s2) * rm * rm;
    const float dL_dm = 2.0f * rm - 2.0f * m * rms;
    const float dv_dm = fmaf(dA_dm, L, A * dL_dm);
    const float dv_ds = fmaf(0.5f * rm, L, -A * rms);
    mbar = fmaf(vnbar, dv_dm, dlbar * (dv_dm - 1.0f));
    s2bar = (vnbar + dlbar) * dv_ds;
  }
  adj_tail(E, c1, P, mbar, s2bar, a);
}

// Reverse step n: state vc -> vn (both known), the step's stored draw d (Z_V in
// the quadratic branch, 1 - U_V in the exponential one; the branch follows from
// vc) and Z_X; vbar holds the adjoint of v_{n+1} on entry and of v_n on exit.
// Each square root and its reciprocal come from one rsqrt.
__device__ __forceinline__ void adjoint_step(const ScenConst& c, float theta, float c1, float vc, float vn, float d,
                                             float zx, AdjSums& a) {
  const float m = fmaf(vc, c.E, c.thE);
  const float s2h = fmaf(vc, c.h1, c.h2);
  const float m2 = m * m;
  const float rs2h = rcp_approx(s2h);
  const float t = __fmul_rn(m2, rs2h);  // qe_t
  AdjPre P;
  adj_common_pre(c, theta, vc, vn, zx, P);
  if (t > kQuadT) {  // the forward step's branch test
    adj_quad_pre(c, m, t, rs2h, d, P);
    P.inc = adj_inc(c, vc + vn, vc, P.dl, P.q, zx);
    adj_chain_quad(c.E, c1, P, a);
    return;
  }
  bool atom;
  P.dl = adj_exp_dl(m, m2, s2h, vn, d, &atom);
  P.inc = adj_inc(c, vc + vn, vc, P.dl, P.q, zx);
  adj_chain_exp(c.E, c1, c.Cdl, m, m2, s2h, d, atom, P, a);
}

// adjoint_step2 for a warp whose every lane takes the quadratic branch in both
// steps (the same operations as its general form, without the exponential
// branch's code and registers).
__device__ __forceinline__ void adjoint_step2_quad(const ScenConst& c, float theta, float c1, float2 vc, float2 vn,
                                                   float2 d, float2 zx, float2 m, float2 m2, float2 rs2h, float2 t,
                                                   AdjSums& a) {
  const float2 s = p_add(vc, vn);
  const float2 rq = make_float2(rsqrt_approx(s.x), rsqrt_approx(s.y));
  const float2 sq = p_mul(s, rq);
  const float2 hq = p_mul(p_mul(p_bc(0.5f * c.sK3), zx), rq);
  const float2 q = make_float2(s.x > 0.0f ? sq.x : 0.0f, s.y > 0.0f ? sq.y : 0.0f);
  const float2 hzc = p_add(make_float2(s.x > 0.0f ? hq.x : 0.0f, s.y > 0.0f ? hq.y : 0.0f), p_bc(c.Cv));
  const float2 hzcd = p_sub(hzc, p_bc(c.Cd));
  const float2 tmv = p_sub(p_bc(theta), vc);
  const float2 tt = p_fma(t, t, p_mul(t, p_bc(-1.0f)));
  const float2 rroot = make_float2(rsqrt_approx(tt.x), rsqrt_approx(tt.y));
  const float2 root = p_mul(tt, rroot);
  const float2 b2 = p_add(p_sub(t, p_bc(1.0f)), root);
  const float2 rb = make_float2(rsqrt_approx(b2.x), rsqrt_approx(b2.y));
  const float2 b = p_mul(b2, rb);
  const float2 ropb2 = p_rcp(p_add(t, root));
  const float2 am = p_mul(m, ropb2);
  const float2 bz = p_add(b, d);
  const float2 g = p_fma(d, p_add(d, p_mul(p_bc(2.0f), b)), p_bc(-1.0f));
  const float2 dl = p_mul(am, g);
  float2 inc = p_fma(p_bc(c.Cv), s, p_bc(c.C0));
  inc = p_fma(p_bc(-c.Cd), vc, inc);
  inc = p_fma(p_bc(c.Cdl), dl, inc);
  inc = p_fma(p_mul(p_bc(c.sK3), q), zx, inc);
  const float2 bz2 = p_mul(bz, bz);
  const float2 cg = p_mul(p_bc(c.Cdl), g);
  const float2 cz = p_mul(p_bc(c.Cdl), d);
  const float2 am2 = p_add(am, am);
  const float2 hrb = p_mul(p_bc(0.5f), rb);
  const float2 amr = p_mul(am, ropb2);
  const float2 F = p_fma(p_fma(p_bc(2.0f), t, p_bc(-1.0f)), p_mul(p_bc(0.5f), rroot), p_bc(1.0f));
  const float2 m4r = p_mul(p_add(m, m), rs2h);
  const float2 tr = p_mul(t, p_mul(p_bc(0.5f), rs2h));
  const AdjPre Px{inc.x, dl.x, q.x,  zx.x,  hzc.x, hzcd.x,  tmv.x, vc.x, bz.x,
                  bz2.x, cg.x, cz.x, am2.x, hrb.x, amr.x, ropb2.x, F.x,   m4r.x, tr.x};
  const AdjPre Py{inc.y, dl.y, q.y,  zx.y,  hzc.y, hzcd.y,  tmv.y, vc.y, bz.y,
                  bz2.y, cg.y, cz.y, am2.y, hrb.y, amr.y, ropb2.y, F.y,   m4r.y, tr.y};
  adj_chain_quad(c.E, c1, Px, a);
  adj_chain_quad(c.E, c1, Py, a);
}

// Two consecutive reverse steps, n (lane x) then n - 1 (lane y): their
// quantities that do not depend on the carried adjoint (adj_common_pre,
// adj_quad_pre -- used only by a lane in the quadratic branch -- and the
// log-spot increment, with each lane's innovation from its own branch) in packed
// FP32, then the two adjoint chains in order, each by its lane's branch.  Lane
// for lane adjoint_step's operations, so the same sums bit for bit however the
// steps are paired; lanes of a warp in different branches diverge only in the
// chains.
__device__ __forceinline__ void adjoint_step2(const ScenConst& c, float theta, float c1, float2 vc, float2 vn,
                                              float2 d, float2 zx, AdjSums& a) {
  const float2 m = p_fma(vc, p_bc(c.E), p_bc(c.thE));
  const float2 s2h = p_fma(vc, p_bc(c.h1), p_bc(c.h2));
  const float2 m2 = p_mul(m, m);
  const float2 rs2h = p_rcp(s2h);
  const float2 t = p_mul(m2, rs2h);  // qe_t, lane for lane
  const bool qx = t.x > kQuadT, qy = t.y > kQuadT;
  if (__all_sync(0xffffffffu, qx && qy)) {  // the whole warp in the quadratic branch
    adjoint_step2_quad(c, theta, c1, vc, vn, d, zx, m, m2, rs2h, t, a);
    return;
  }
  // adj_common_pre, paired
  const float2 s = p_add(vc, vn);
  const float2 rq = make_float2(rsqrt_approx(s.x), rsqrt_approx(s.y));
  const float2 sq = p_mul(s, rq);
  const float2 hq = p_mul(p_mul(p_bc(0.5f * c.sK3), zx), rq);
  const float2 q = make_float2(s.x > 0.0f ? sq.x : 0.0f, s.y > 0.0f ? sq.y : 0.0f);
  const float2 hzc = p_add(make_float2(s.x > 0.0f ? hq.x : 0.0f, s.y > 0.0f ? hq.y : 0.0f), p_bc(c.Cv));
  const float2 hzcd = p_sub(hzc, p_bc(c.Cd));
  const float2 tmv = p_sub(p_bc(theta), vc);
  // adj_quad_pre, paired (its values are used by quadratic-branch lanes only)
  const float2 tt = p_fma(t, t, p_mul(t, p_bc(-1.0f)));
  const float2 rroot = make_float2(rsqrt_approx(tt.x), rsqrt_approx(tt.y));
  const float2 root = p_mul(tt, rroot);
  const float2 b2 = p_add(p_sub(t, p_bc(1.0f)), root);
  const float2 rb = make_float2(rsqrt_approx(b2.x), rsqrt_approx(b2.y));
  const float2 b = p_mul(b2, rb);
  const float2 ropb2 = p_rcp(p_add(t, root));
  const float2 am = p_mul(m, ropb2);
  const float2 bz = p_add(b, d);
  const float2 g = p_fma(d, p_add(d, p_mul(p_bc(2.0f), b)), p_bc(-1.0f));
  float2 dl = p_mul(am, g);
  const float2 bz2 = p_mul(bz, bz);
  const float2 cg = p_mul(p_bc(c.Cdl), g);
  const float2 cz = p_mul(p_bc(c.Cdl), d);
  const float2 am2 = p_add(am, am);
  const float2 hrb = p_mul(p_bc(0.5f), rb);
  const float2 amr = p_mul(am, ropb2);
  const float2 F = p_fma(p_fma(p_bc(2.0f), t, p_bc(-1.0f)), p_mul(p_bc(0.5f), rroot), p_bc(1.0f));
  const float2 m4r = p_mul(p_add(m, m), rs2h);
  const float2 tr = p_mul(t, p_mul(p_bc(0.5f), rs2h));
  // each lane's innovation from its own branch
  bool ax = false, ay = false;
  if (!qx) dl.x = adj_exp_dl(m.x, m2.x, s2h.x, vn.x, d.x, &ax);
  if (!qy) dl.y = adj_exp_dl(m.y, m2.y, s2h.y, vn.y, d.y, &ay);
  // adj_inc, paired
  float2 inc = p_fma(p_bc(c.Cv), s, p_bc(c.C0));
  inc = p_fma(p_bc(-c.Cd), vc, inc);
  inc = p_fma(p_bc(c.Cdl), dl, inc);
  inc = p_fma(p_mul(p_bc(c.sK3), q), zx, inc);
  const AdjPre Px{inc.x, dl.x, q.x,  zx.x,  hzc.x, hzcd.x,  tmv.x, vc.x, bz.x,
                  bz2.x, cg.x, cz.x, am2.x, hrb.x, amr.x, ropb2.x, F.x,   m4r.x, tr.x};
  const AdjPre Py{inc.y, dl.y, q.y,  zx.y,  hzc.y, hzcd.y,  tmv.y, vc.y, bz.y,
                  bz2.y, cg.y, cz.y, am2.y, hrb.y, amr.y, ropb2.y, F.y,   m4r.y, tr.y};
  if (qx)
    adj_chain_quad(c.E, c1, Px, a);
  else
    adj_chain_exp(c.E, c1, c.Cdl, m.x, m2.x, s2h.x, d.x, ax, Px, a);
  if (qy)
    adj_chain_quad(c.E, c1, Py, a);
  else
    adj_chain_exp(c.E, c1, c.Cdl, m.y, m2.y, s2h.y, d.y, ay, Py, a);
}

// Reverse step n under QE-M (Andersen's martingale correction, QemConst q): where
// the correction exists the step's increment is
//   r dt - qa (v + m) - lam + K2 (v' - m) + sK3 sqrt(v + v') Z_X,
// lam = ln M - A m formed as the forward step forms it (qem_from_moments), and
// the plain increment elsewhere.  lam's adjoint (bar lam = -1):
//   quadratic: lam = u^2 b^2 / (2 (1 - u)) + g(u)/2, u = 2 A a, g(u) = -u - ln(1 - u):
//     dlam/du = b^2 u (2 - u) / (2 (1 - u)^2) + u / (2 (1 - u)), dlam/db^2 = u^2 / (2 (1 - u)),
//     into a (du/da = 2A), b^2 and A (du/dA = 2a);
//   exponential: lam = ln(1 + q w / (1 - w)) - q w, q = 2 m^2 / (m^2 + s^2), w = A (m^2 + s^2) / (2 m):
//     dlam/dq = w / (1 - w + q w) - w, dlam/dw = q / ((1 - w)(1 - w + q w)) - q,
//     into m, s^2 and A;
//   a zero mean (v = theta = 0): v' = 0 and M = 1 with no derivative, so lam = -A m
//     and the increment r dt - qa v does not depend on m.
// The sums Aqa, AK2, AA carry the dependence on qa, K2 and A; Np counts the plain
// steps (their C0 = r dt + Cd theta).  One step at a time (no packed pairs).
__device__ __forceinline__ void adjoint_step_qem(const ScenConst& c, const QemConst& q, float theta, float c1,
                                                 float vc, float vn, float d, float zx, AdjSums& a) {
  // every product is rounded on its own (__fmul_rn) or fused explicitly (fmaf), so
  // the compiler forms no FMA of its own: the same values in every kernel
  const float m = fmaf(vc, c.E, c.thE);
  const float s2h = fmaf(vc, c.h1, c.h2);
  const float m2 = __fmul_rn(m, m);
  const float rs2h = rcp_approx(s2h);
  const float t = __fmul_rn(m2, rs2h);  // qe_t
  const float s = vc + vn;
  const float rq = rsqrt_approx(s);
  const float qs = s > 0.0f ? __fmul_rn(s, rq) : 0.0f;
  const float hz = s > 0.0f ? __fmul_rn(__fmul_rn(0.5f * c.sK3, zx), rq) : 0.0f;  // d(sK3 sqrt(s) Z)/ds
  float mbar = 0.0f, s2bar = 0.0f, Abar = 0.0f, dl, lam = 0.0f;
  bool ok = true;
  if (t > kQuadT) {
    AdjPre P;
    adj_quad_pre<true>(c, m, t, rs2h, d, P);
    dl = P.dl;
    const float am = P.am, bb2 = P.b2;
    const float Aa = __fmul_rn(q.A, am);
    const float u = 2.0f * Aa;
    ok = u < 1.0f;
    float lu = 0.0f, lb2 = 0.0f;
    if (ok) {
      const float r1u = rcp_approx(1.0f - u);
      const float ur = __fmul_rn(u, r1u);
      lam = fmaf(0.5f, neg_log1m_tail(u), __fmul_rn(__fmul_rn(__fmul_rn(2.0f * Aa, Aa), bb2), r1u));
      lu = fmaf(__fmul_rn(__fmul_rn(bb2, ur), 2.0f - u), 0.5f * r1u, 0.5f * ur);
      lb2 = __fmul_rn(0.5f * u, ur);
    }
    const float vnbar = a.vbar + hz + (ok ? 0.0f : c.Cv);  // adjoint of v_{n+1}
    const float dlbar = ok ? q.K2 : c.Cdl;
    float abar = fmaf(vnbar, P.bz2, __fmul_rn(dlbar, P.g));
    if (ok) {
      const float lu2 = 2.0f * lu;
      abar = fmaf(-lu2, q.A, abar);
      Abar = __fmul_rn(-lu2, am);
    }
    const float bbar = __fmul_rn(P.am2, fmaf(vnbar, P.bz, __fmul_rn(dlbar, d)));
    const float b2bar = fmaf(bbar, P.hrb, -__fmul_rn(abar, P.amr)) - (ok ? lb2 : 0.0f);
    const float tbar = __fmul_rn(b2bar, P.F);
    mbar = fmaf(tbar, P.m4r, __fmul_rn(abar, P.ropb2));
    s2bar = -__fmul_rn(tbar, P.tr);
  } else {
    bool atom;
    dl = adj_exp_dl(m, m2, s2h, vn, d, &atom);
    float qq = 0.0f, w = 0.0f, ms = 0.0f;
    if (m > 0.0f) {
      ms = m2 + (s2h + s2h);
      qq = __fmul_rn(2.0f * m2, rcp_approx(ms));             // 1 - p
      w = __fmul_rn(__fmul_rn(0.5f * q.A, ms), rcp_approx(m));  // A / beta
      ok = w < 1.0f;
      if (ok) {
        const float qw = __fmul_rn(qq, w);
        lam = log1pf(__fmul_rn(qw, rcp_approx(1.0f - w))) - qw;
      }
    }
    const float vnbar = a.vbar + hz + (ok ? 0.0f : c.Cv);
    const float dlbar = ok ? q.K2 : c.Cdl;
    // a zero mean: v' = 0 (dl = -m) and M = 1 with no derivative (lam = -A m), so
    // -K2 + A = qa, and with the -qa below m drops out exactly
    if (!(m > 0.0f)) mbar = q.qa;
    if (m > 0.0f) {
      if (atom) mbar = -dlbar;  // v' = 0 by the atom: dl = -m
      const float rm = rcp_approx(m), rms = rcp_approx(ms);
      const float s2 = s2h + s2h;
      if (!atom) {
        const float W = __fmul_rn(d, ms);
        const float L = 0.69314718055994531f * lg2_approx(__fmul_rn(2.0f * m2, rcp_approx(W)));
        const float Av = __fmul_rn(0.5f * ms, rm);
        const float dA_dm = __fmul_rn(__fmul_rn(0.5f * (m2 - s2), rm), rm);
        const float dL_dm = 2.0f * rm - __fmul_rn(2.0f * m, rms);
        const float dv_dm = fmaf(dA_dm, L, __fmul_rn(Av, dL_dm));
        const float dv_ds = fmaf(0.5f * rm, L, -__fmul_rn(Av, rms));
        mbar = fmaf(vnbar, dv_dm, __fmul_rn(dlbar, dv_dm - 1.0f));
        s2bar = __fmul_rn(vnbar + dlbar, dv_ds);
      }
      if (ok) {
        const float den = (1.0f - w) + __fmul_rn(qq, w);
        const float lq = __fmul_rn(w, rcp_approx(den)) - w;
        const float lw = __fmul_rn(qq, rcp_approx(__fmul_rn(1.0f - w, den))) - qq;
        const float rms2 = __fmul_rn(rms, rms), rm2 = __fmul_rn(rm, rm);
        const float dq_dm = __fmul_rn(__fmul_rn(4.0f * m, s2), rms2), dq_ds = __fmul_rn(-2.0f * m2, rms2);
        const float dw_dm = __fmul_rn(q.A, 0.5f - __fmul_rn(0.5f * s2, rm2)), dw_ds = __fmul_rn(0.5f * q.A, rm);
        mbar -= fmaf(lq, dq_dm, __fmul_rn(lw, dw_dm));
        s2bar -= fmaf(lq, dq_ds, __fmul_rn(lw, dw_ds));
        Abar = __fmul_rn(__fmul_rn(-0.5f * lw, ms), rm);
      }
    }
  }
  // the increment, x_T (Kahan), the adjoint of v_n, the sums
  float inc;
  if (ok) {
    inc = fmaf(-q.qa, vc + m, q.rdt) - lam;
    inc = fmaf(q.K2, dl, inc);
    mbar -= q.qa;
  } else {
    inc = fmaf(c.Cv, s, c.C0);
    inc = fmaf(-c.Cd, vc, inc);
    inc = fmaf(c.Cdl, dl, inc);
  }
  inc = fmaf(__fmul_rn(c.sK3, qs), zx, inc);
  const float y = inc - a.comp;
  const float tx = a.x + y;
  a.comp = (tx - a.x) - y;
  a.x = tx;
  a.vbar = fmaf(mbar, c.E, fmaf(s2bar, c1, ok ? hz - q.qa : (c.Cv - c.Cd) + hz));
  a.Am += mbar;
  a.Amv = fmaf(mbar, vc - theta, a.Amv);
  a.As += s2bar;
  a.Asv = fmaf(s2bar, vc, a.Asv);
  a.Ak3 = fmaf(qs, zx, a.Ak3);
  if (ok) {
    a.Aqa += vc + m;
    a.AK2 += dl;
    a.AA += Abar;
  } else {
    a.Ad += theta - vc;
    a.Adl += dl;
    a.Np += 1.0f;
  }
}

// The draw the reverse step of state v needs: Z_V in the quadratic branch,
// 1 - U_V otherwise (same branch test as the forward step).
__device__ __forceinline__ float branch_draw(const ScenConst& c, float v, float xv, float zv) {
  const float m = fmaf(v, c.E, c.thE);
  const float s2h = fmaf(v, c.h1, c.h2);
  return qe_t(m * m, s2h) > kQuadT ? zv : one_minus_u(xv);
}

// The stored data of one step (recompute pass): (state, branch draw) as one
// pair and Z_X, from the step's centred variance uniform and its two normals.
__device__ __forceinline__ void keep_step(const ScenConst& c, float xv_v, float zv, float zx, float2* bvd, float* bz,
                                          float& v) {
  *bvd = make_float2(v, branch_draw(c, v, xv_v, zv));
  *bz = zx;
  v = qe_only(c, v, xv_v, zv);
}

// A thread's column of a segment buffer of `stride` columns (8-byte aligned):
// `rows` (state, draw) float2 pairs at pairs[i * stride], then `rows` Z_X floats
// at zx[i * stride].  SegShared: the block's buffer in shared memory, column
// threadIdx.x of blockDim.x; SegGlobal: a grid-wide buffer in global memory,
// column `col` (the thread's index in the grid) of `stride`.
struct SegShared {
  static constexpr bool kGlobal = false;
  float* base;
  int rows;
  __device__ __forceinline__ int stride() const { return (int)blockDim.x; }
  __device__ __forceinline__ float2* pairs() const { return reinterpret_cast<float2*>(base) + threadIdx.x; }
  __device__ __forceinline__ float* zx() const { return base + 2 * rows * (int)blockDim.x + threadIdx.x; }
};

struct SegGlobal {
  static constexpr bool kGlobal = true;
  float* base;
  long long col, rows, cols;
  __device__ __forceinline__ long long stride() const { return cols; }
  __device__ __forceinline__ float2* pairs() const { return reinterpret_cast<float2*>(base) + col; }
  __device__ __forceinline__ float* zx() const { return base + 2 * rows * cols + col; }
};

// The FP64 map of the sweep's sums onto d x_T / d(v0, kappa, theta, sigma, rho).
// Under QE-M the plain steps' C0 contributes Cd theta per plain step (Np of them)
// instead of every step's, and qa, K2 and A add their sums.
template <bool QEM = false>
__device__ __forceinline__ void adjoint_map(const AdjConst& A, const AdjSums& a, float (&g)[5]) {
  const double Amv = a.Amv, Asv = a.Asv, As = a.As, Ad = a.Ad, Adl = a.Adl, Am = a.Am, Ak3 = a.Ak3;
  g[0] = a.vbar;
  double gk = A.dE_dk * Amv + A.dc1_dk * Asv + A.dc2_dk * As + A.dCd_dk * Ad + A.dCdl_dk * Adl;
  double gt = A.omE * Am + A.dc2_dth * As + (QEM ? A.Cd * (double)a.Np : A.N_Cd);
  double gs = A.two_over_sigma * (A.c1 * Asv + A.c2 * As) - A.Cd_over_sigma * Ad - A.Cdl_over_sigma * Adl;
  double gr = A.D_over_sigma * Ad + A.B_over_sigma * Adl + A.dsK3_drho * Ak3;
  if (QEM) {
    const double Aqa = a.Aqa, AK2 = a.AK2, AA = a.AA;
    gk += A.dK2_dk * AK2 + A.dA_dk * AA;
    gs += A.dK2_ds * AK2 + A.dA_ds * AA;
    gr += -A.dqa_drho * Aqa + A.dK2_dr * AK2 + A.dA_dr * AA;
  }
  g[1] = (float)gk;
  g[2] = (float)gt;
  g[3] = (float)gs;
  g[4] = (float)gr;
}

// Reverse sweep of one path, segment by segment, last first: each segment's
// states are recomputed from its checkpoint (the last checkpoint is v_last, the
// forward pass's final state; earlier ones ck[slot * cstride], each loaded a
// segment ahead of its use) and kept with the step's branch draw and Z_X in this
// thread's segment column S (at least k rows) -- then the steps are
// differentiated backwards.  x_T (with its Kahan remainder) is summed on the
// way; g = d x_T / d(v0, kappa, theta, sigma, rho).
template <typename Seg, bool PAIRED, bool QEM = false>
__device__ __forceinline__ void path_sweep(const ScenConst& c, const AdjConst& A, uint32_t N, uint32_t option,
                                           const uint32_t (&rk)[10][2], const PhiloxLane& pl,
                                           const float* ck, int cstride, float v_last, const Seg& S,
                                           float& x_out, float& comp_out, float (&g)[5], const QemConst& qm) {
  using I = decltype(S.stride());
  const float theta = A.theta;
  const float c1 = c.h1 + c.h1;  // s^2 = v c1 + c2
  const uint32_t k = (uint32_t)A.ckpt_every;
  const int n_seg = A.n_seg;
  AdjSums as = AdjSums{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  float2* s01 = S.pairs();
  float* s2 = S.zx();
  const I bd = S.stride();
  float ck_next = v_last;
  for (int sgi = n_seg - 1; sgi >= 0; --sgi) {
    const uint32_t n0 = (uint32_t)sgi * k, n1 = min(n0 + k, N);
    float vv = ck_next;
    if (sgi > 0) ck_next = ck[(sgi - 1) * cstride];
    // recompute v_n0 .. v_n1 and keep the draws: rows 2 (p - n0/2) and the next of
    // this thread's column, by pointers stepped two rows per pair (n0 is even)
    float2* wp = s01;
    float* wz = s2;
    for (uint32_t p = n0 / 2; 2 * p < n1; ++p, wp += 2 * bd, wz += 2 * bd) {
      const uint4 w = philox_draw(pl, philox_ctr(p, option, rk), rk);
      const float2 xv = centered_uniform2(w.x, w.z);
      const float2 zv = norminv_centered2(xv);  // the pair's normals two at a time
      const float2 zx = norminv_centered2(centered_uniform2(w.y, w.w));
      keep_step(c, xv.x, zv.x, zx.x, wp, wz, vv);
      if (2 * p + 1 < n1) keep_step(c, xv.y, zv.y, zx.y, wp + bd, wz + bd, vv);
    }
    float vnext = vv;  // v_{n1}
    // the reverse steps read row i by pointers rp, rz stepped down from the top row
    int i = (int)(n1 - n0) - 1;
    const float2* rp = s01 + (I)i * bd;
    const float* rz = s2 + (I)i * bd;
    if constexpr (QEM) {
      for (; i >= 0; --i, rp -= bd, rz -= bd) {
        const float2 vd = rp[0];
        adjoint_step_qem(c, qm, theta, c1, vd.x, vnext, vd.y, rz[0], as);
        vnext = vd.x;
      }
    } else if constexpr (PAIRED) {
      if constexpr (Seg::kGlobal) {
        // global memory: the steps in pairs (n, n - 1) from the top, each pair's
        // data loaded one pair ahead into registers and asked into L2
        // kPrefetchSteps steps ahead
        constexpr int kPrefetchSteps = SIMR_ADJ_PREFETCH;
        const I o2 = 2 * bd, o3 = 3 * bd, f2 = (2 + kPrefetchSteps) * bd, f3 = (3 + kPrefetchSteps) * bd;
        float2 pa = rp[0], pb = make_float2(0.0f, 0.0f);
        float za = rz[0], zb = 0.0f;
        if (i >= 1) {
          pb = rp[-bd];
          zb = rz[-bd];
        }
        for (; i >= 1; i -= 2, rp -= o2, rz -= o2) {
          const float2 ca = pa, cb = pb;
          const float cza = za, czb = zb;
          if (i - 2 - kPrefetchSteps >= 0) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(rp - f2));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(rz - f2));
          }
          if (i - 3 - kPrefetchSteps >= 0) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(rp - f3));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(rz - f3));
          }
          if (i >= 2) {
            pa = rp[-o2];
            za = rz[-o2];
          }
          if (i >= 3) {
            pb = rp[-o3];
            zb = rz[-o3];
          }
          adjoint_step2(c, theta, c1, make_float2(ca.x, cb.x), make_float2(vnext, ca.x), make_float2(ca.y, cb.y),
                        make_float2(cza, czb), as);
          vnext = cb.x;
        }
        if (i == 0) {  // an odd count: the last step alone (loaded as pa)
          adjoint_step(c, theta, c1, pa.x, vnext, pa.y, za, as);
          vnext = pa.x;
        }
      } else {
        for (; i >= 1; i -= 2, rp -= 2 * bd, rz -= 2 * bd) {
          const float2 ca = rp[0], cb = rp[-bd];
          adjoint_step2(c, theta, c1, make_float2(ca.x, cb.x), make_float2(vnext, ca.x), make_float2(ca.y, cb.y),
                        make_float2(rz[0], rz[-bd]), as);
          vnext = cb.x;
        }
        if (i == 0) {
          const float2 vd = s01[0];
          adjoint_step(c, theta, c1, vd.x, vnext, vd.y, s2[0], as);
          vnext = vd.x;
        }
      }
    } else {
      if constexpr (Seg::kGlobal) {
        // global memory: each step's data loaded one step ahead into registers,
        // and asked into L2 kPrefetchSteps steps ahead
        constexpr int kPrefetchSteps = SIMR_ADJ_PREFETCH;
        const I f = (I)kPrefetchSteps * bd;
        float2 vd_n = rp[0];
        float zx_n = rz[0];
        for (; i >= 0; --i, rp -= bd, rz -= bd) {
          const float2 vd = vd_n;
          const float zx = zx_n;
          if (i >= kPrefetchSteps) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(rp - f));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(rz - f));
          }
          if (i > 0) {
            vd_n = rp[-bd];
            zx_n = rz[-bd];
          }
          adjoint_step(c, theta, c1, vd.x, vnext, vd.y, zx, as);
          vnext = vd.x;
        }
      } else {
        for (; i >= 0; --i, rp -= bd, rz -= bd) {
          const float2 vd = rp[0];
          adjoint_step(c, theta, c1, vd.x, vnext, vd.y, rz[0], as);
          vnext = vd.x;
        }
      }
    }
  }
  x_out = as.x;
  comp_out = as.comp;
  adjoint_map<QEM>(A, as, g);
}

// Forward pass with checkpoints, then the reverse sweeps, for PPT paths: the
// forward pass runs the variance recursion only, and only up to the last
// checkpoint (x_T is not needed before the sweep ends; the last segment is
// recomputed from its checkpoint anyway), the PPT paths together -- two paths
// paired (qe_from_moments2, lane for lane the scalar step); the reverse sweeps
// then run one path at a time through the same shared segment buffer.
// Checkpoint (slot, path j) of this thread at ck[(slot * PPT + j) * ck_stride]
// (n_seg - 1 slots; shared or global memory); S is this thread's segment column
// (shared or global memory, at least k rows).
template <int PPT, typename Seg, bool PAIRED = true, bool QEM = false>
__device__ __forceinline__ void path_adjoint_ppt(const ScenConst& c, const AdjConst& A, uint32_t N, uint32_t option,
                                                 const uint32_t (&rk)[10][2], const uint64_t (&path)[PPT], float* ck,
                                                 int ck_stride, const Seg& S, float (&x_out)[PPT],
                                                 float (&comp_out)[PPT], float (&g)[PPT][5],
                                                 const QemConst& qm = QemConst{}) {
  static_assert(PPT == 1 || PPT == 2, "one or two paths per thread");
  const uint32_t k = (uint32_t)A.ckpt_every;
  const int n_seg = A.n_seg;
  PhiloxLane pl[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) pl[j] = philox_lane(path[j], rk);
  // forward pass: the variance recursion up to the last checkpoint, (n_seg - 1) k
  // < N; k is even, so every pair of steps below it is whole
  float v[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) v[j] = c.v0;
  for (int sg = 0; sg < n_seg - 1; ++sg) {
#pragma unroll
    for (int j = 0; j < PPT; ++j) ck[(sg * PPT + j) * ck_stride] = v[j];
    const uint32_t p0 = (uint32_t)sg * (k / 2);
    for (uint32_t p = p0; p < p0 + k / 2; ++p) {
      uint4 w[PPT];
#pragma unroll
      for (int j = 0; j < PPT; ++j) w[j] = philox_draw(pl[j], philox_ctr(p, option, rk), rk);
      if constexpr (PPT == 2) {
        const float2 xa = centered_uniform2(w[0].x, w[1].x), xb = centered_uniform2(w[0].z, w[1].z);
        const float2 za = norminv_centered2(xa);
        const float2 zb = norminv_centered2(xb);
        float2 vv = make_float2(v[0], v[1]), vn, dl;
        qe_from_moments2(p_fma(vv, p_bc(c.E), p_bc(c.thE)), p_fma(vv, p_bc(c.h1), p_bc(c.h2)), xa, za, vn, dl);
        vv = vn;
        qe_from_moments2(p_fma(vv, p_bc(c.E), p_bc(c.thE)), p_fma(vv, p_bc(c.h1), p_bc(c.h2)), xb, zb, vn, dl);
        v[0] = vn.x;
        v[1] = vn.y;
      } else {  // the pair's two variance normals together
        const float2 xv = centered_uniform2(w[0].x, w[0].z);
        const float2 zv = norminv_centered2(xv);
        v[0] = qe_only(c, v[0], xv.x, zv.x);
        v[0] = qe_only(c, v[0], xv.y, zv.y);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < PPT; ++j)
    path_sweep<Seg, PAIRED, QEM>(c, A, N, option, rk, pl[j], ck + j * ck_stride, PPT * ck_stride, v[j], S,
                                 x_out[j], comp_out[j], g[j], qm);
}

// Floats per thread of path_adjoint_ppt: checkpoints and the segment buffer.
__host__ __device__ inline size_t adjoint_ckpt_floats(const AdjConst& A, int ppt) { return (size_t)A.n_seg * ppt; }
__host__ __device__ inline size_t adjoint_seg_floats(const AdjConst& A, int /*ppt: the sweeps share one buffer*/) {
  return (size_t)3 * A.ckpt_every;
}

// Terms per strike: 0 f, 1 f^2, 2 S0, 3 v0, 4 kappa, 5 theta, 6 sigma, 7 rho,
// 8 r: the signed in-the-money indicator.  d/dr of e^{-rT} E[f] with dx_T/dr = T
// is e^{-rT} T E[w - f], and w - f = K 1{S_T > K} for a call, -K 1{S_T < K} for
// a put: the column is e^{-rT} T K E[indicator], with no cancellation of
// E[w T] against T P (which loses the column when S_T >> K).
constexpr int kAdjAcc = 9;

__device__ __forceinline__ float adj_term(int a, bool put, float S, float K, const float (&g)[5], float invS0,
                                          float /*T: applied in the normalisation*/) {
  const float f = put ? fmaxf(K - S, 0.0f) : fmaxf(S - K, 0.0f);
  if (a == 0) return f;
  if (a == 1) return f * f;
  if (a == 8) return put ? (S < K ? -1.0f : 0.0f) : (S > K ? 1.0f : 0.0f);
  const float w = put ? (S < K ? -S : 0.0f) : (S > K ? S : 0.0f);
  if (a == 2) return w * invS0;
  return w * g[a - 3];
}

}  // namespace
}  // namespace simr
