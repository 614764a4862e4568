// simr_device.cuh -- device primitives of the fused Heston QE path kernels (sm_103a).
//
// One thread carries one path's state (v, x = ln S/S0) in registers through all
// time steps: the paper's per-path cached state of the asset/timestep/path loop
// nest (Sec. 5.1, Listing 2) becomes register state, with the timestep loop
// inside the thread.  Random inputs are drawn in-kernel (no V/Z arrays in
// HBM, unlike the host-streamed inputs of the paper's Table 1).
#pragma once

#include <cstdint>

namespace simr {

constexpr int kMaxScen = 13;  // base + 6 re-simulated Greeks x (up, down)

// Per-scenario FP32 constants of the QE variance step and the log-spot step
// (Andersen 2008 with gamma1 = gamma2 = 1/2, risk-neutral drift r), computed on
// the host in FP64 and rounded once:
//   m     = theta + (v - theta) E        = fma(v, E, thE)
//   s^2/2 = v h1 + h2                    (h1 = c1/2, h2 = c2/2 of s^2 = v c1 + c2:
//           the step needs t = 2 m^2 / s^2 = m^2 / (s^2/2), so it carries half the
//           conditional variance; the halving is exact)
//   x' = x + K0 + K1 v + K2 v' + sqrt(K3 v + K4 v') Z_X, rewritten without
//   the large cancelling rho/sigma terms as
//   x' = x + C0 + Cv (v + v') - Cd v + Cdl (v' - m) + sK3 sqrt(v + v') Z_X
// with Cd = (rho/sigma)((1-E) - kappa dt (1+E)/2), C0 = r dt + Cd theta,
// Cv = -dt/4, Cdl = (rho/sigma)(1 + kappa dt/2), sK3 = sqrt(dt (1 - rho^2)/2):
// the same polynomial in (v, v'), since v' - v = (theta - v)(1 - E) + (v' - m).
//
// A bumped scenario (bump-and-revalue) stores DELTAS to the base scenario's
// constants instead (dE = E_s - E_0 etc., exact differences taken in FP64 and
// added to the base's FP32 constants): a 1e-4
// bump moves E or Cdl by only a few FP32 ulps, so bumped constants rounded on
// their own would bias the finite difference.  Each delta is added inside an
// FMA whose product varies from path to path (so its rounding is unbiased),
// and every scenario adds the base constants in the same order, so the
// systematic part of their rounding is common to all scenarios and cancels in
// the difference.  The initial variance is not a delta: each scenario starts
// from its own FP32 v0, and the host divides by the realised FP32 bump.
struct ScenConst {
  float E, thE, h1, h2;
  float C0, Cv, Cd, Cdl;
  float sK3;
  float ratio;  // base: 1; bumped: (discount of this scenario / base discount) - 1
  float v0;     // initial variance of this scenario (FP32 value)
  float pad;
};

// The step constants of two lanes, packed (lane x, lane y): the operands of the
// paired steps, read from the launch parameters as they are (the same values
// in both lanes for two paths or the v0 bumps; a bumped pair's own deltas).
struct ScenConst2 {
  float2 E, thE, h1, h2, C0, Cv, mCd, Cdl, sK3;  // mCd = -Cd
};

__host__ __device__ inline ScenConst2 pack_const(const ScenConst& a, const ScenConst& b) {
  ScenConst2 p;
  p.E = make_float2(a.E, b.E);
  p.thE = make_float2(a.thE, b.thE);
  p.h1 = make_float2(a.h1, b.h1);
  p.h2 = make_float2(a.h2, b.h2);
  p.C0 = make_float2(a.C0, b.C0);
  p.Cv = make_float2(a.Cv, b.Cv);
  p.mCd = make_float2(-a.Cd, -b.Cd);
  p.Cdl = make_float2(a.Cdl, b.Cdl);
  p.sK3 = make_float2(a.sK3, b.sK3);
  return p;
}

// First-step constants of a scenario (all paths share v0, so every step-0
// quantity except the draws is a per-scenario constant).  Computed on the host
// in FP64: base scenario full values, bumped scenarios their exact differences
// to the base's -- except q (decision threshold) and v0, which are full values.
//   quadratic: v1 = a (b + Z_V)^2, v1 - m0 = a (Z_V (Z_V + 2b) - 1)
//   exponential: v1 = 0 if 1 - U_V >= q, else C (L - ln(1 - U_V)), C = m0/q, L = ln q
//   increment: x1 = K0p + Cv v1 + Cdl (v1 - m0) + sK3 sqrt(v0 + v1) Z_X, K0p = C0 + (Cv - Cd) v0
struct FirstConst {
  float a, b, q, C, L, m0, K0p;
  int branch;  // 0 quadratic, 1 exponential, 2 zero mean
};

// ---------------------------------------------------------------- PTX ----
// The special-function unit's approximations (MUFU), or with SIMR_IEEE=1 (a
// build for error studies) the correctly rounded division, square root and
// reciprocal square root and the library's log2f in their place.
#ifndef SIMR_IEEE
#define SIMR_IEEE 0
#endif
__device__ __forceinline__ float rcp_approx(float x) {
#if SIMR_IEEE
  return __frcp_rn(x);
#else
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#endif
}
__device__ __forceinline__ float sqrt_approx(float x) {
#if SIMR_IEEE
  return __fsqrt_rn(x);
#else
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#endif
}
__device__ __forceinline__ float rsqrt_approx(float x) {
#if SIMR_IEEE
  return __frsqrt_rn(x);
#else
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#endif
}
__device__ __forceinline__ float lg2_approx(float x) {
#if SIMR_IEEE
  return log2f(x);
#else
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
#endif
}

// ------------------------------------------------- packed FP32 (f32x2) ----
// sm_100-family paired FP32 instructions: one instruction computes two lanes,
// each rounded exactly as the scalar __fmaf_rn / __fmul_rn / __fadd_rn /
// __fsub_rn (bitwise, checked on the device).  The path kernels are bound by
// instruction issue, not by the FMA pipe, so pairing two scenarios (or two
// paths) that run the same arithmetic halves the issue slots of that part.
// Functions with a "2" suffix below repeat their scalar namesake's operation
// sequence lane for lane, so a lane's result is the scalar function's, bit for bit.
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 p_add(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 p_bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 p_rcp(float2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }
__device__ __forceinline__ float2 p_sqrt(float2 a) { return make_float2(sqrt_approx(a.x), sqrt_approx(a.y)); }
__device__ __forceinline__ float2 p_lg2(float2 a) { return make_float2(lg2_approx(a.x), lg2_approx(a.y)); }

// ------------------------------------------------------------- Philox ----
// Philox4x32-10 (Salmon et al., SC'11) of the counter (p, plo, phi, option):
// ten rounds (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
// lo(M0 c0)) under the round keys rk[i] = key + i * (0x9E3779B9, 0xBB67AE85),
// precomputed on the host (the key is uniform over the launch).
// The first two rounds are split by what their words depend on.  Round 0
// multiplies phi (path) and p (step pair); round 1 multiplies round 0's
// path-only word s0 and its step-only word s2.  So round 1's output is
//   (a(p) ^ s1, b(p), h0 ^ c(p), l0)
// with (s1, h0, l0) a function of the path alone (PhiloxLane, formed once per
// path) and (a, b, c) of the step pair and option alone (PhiloxCtr, formed once
// per step pair and shared by every path that draws it); rounds 2..9 run per
// path: 16 of the 20 32x32 -> 64-bit products a path needs per draw.
constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;

struct PhiloxLane {
  uint32_t s1, h0, l0;  // lo(M1 phi); hi and lo of M0 s0, s0 = hi(M1 phi) ^ plo ^ rk[0][0]
};
struct PhiloxCtr {
  uint32_t a, b, c;  // hi(M1 s2) ^ rk[1][0]; lo(M1 s2); lo(M0 p) ^ rk[1][1], s2 = hi(M0 p) ^ option ^ rk[0][1]
};

__device__ __forceinline__ PhiloxLane philox_lane(uint32_t plo, uint32_t phi, const uint32_t (&rk)[10][2]) {
  const uint32_t s0 = __umulhi(kPhiloxM1, phi) ^ plo ^ rk[0][0];
  PhiloxLane l;
  l.s1 = kPhiloxM1 * phi;
  l.h0 = __umulhi(kPhiloxM0, s0);
  l.l0 = kPhiloxM0 * s0;
  return l;
}
__device__ __forceinline__ PhiloxLane philox_lane(uint64_t path, const uint32_t (&rk)[10][2]) {
  return philox_lane((uint32_t)path, (uint32_t)(path >> 32), rk);
}

__device__ __forceinline__ PhiloxCtr philox_ctr(uint32_t p, uint32_t option, const uint32_t (&rk)[10][2]) {
  const uint32_t s2 = __umulhi(kPhiloxM0, p) ^ option ^ rk[0][1];
  PhiloxCtr u;
  u.a = __umulhi(kPhiloxM1, s2) ^ rk[1][0];
  u.b = kPhiloxM1 * s2;
  u.c = (kPhiloxM0 * p) ^ rk[1][1];
  return u;
}

// Rounds 2..9 from the two halves of round 1's output.
__device__ __forceinline__ uint4 philox_draw(const PhiloxLane& l, const PhiloxCtr& u, const uint32_t (&rk)[10][2]) {
  uint32_t c0 = u.a ^ l.s1, c1 = u.b, c2 = l.h0 ^ u.c, c3 = l.l0;
#pragma unroll
  for (int i = 2; i < 10; ++i) {
    const uint32_t lo0 = kPhiloxM0 * c0, hi0 = __umulhi(kPhiloxM0, c0);
    const uint32_t lo1 = kPhiloxM1 * c2, hi1 = __umulhi(kPhiloxM1, c2);
    const uint32_t n0 = hi1 ^ c1 ^ rk[i][0];
    const uint32_t n2 = hi0 ^ c3 ^ rk[i][1];
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// The whole generator for one counter.
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               const uint32_t (&rk)[10][2]) {
  return philox_draw(philox_lane(c1, c2, rk), philox_ctr(c0, c3, rk), rk);
}

// x = 2u - 1 for u = ((w >> 9) + 1/2) 2^-23, exact in FP32:
// f = 1 + (w >> 9) 2^-23 from the bits, f - 1.5 is exact, and
// 2 (f - 1.5) + 2^-23 = (2k + 1 - 2^23) 2^-23 needs at most 23 significant bits.
__device__ __forceinline__ float centered_uniform(uint32_t w) {
  const float f = __uint_as_float(0x3f800000u | (w >> 9));
  return fmaf(2.0f, f - 1.5f, 0x1p-23f);
}
// Two of them in packed FP32 (the same operations, lane for lane).
__device__ __forceinline__ float2 centered_uniform2(uint32_t wa, uint32_t wb);
// 1 - U_V from x = 2 U_V - 1 (exact): the exponential branch's uniform.
__device__ __forceinline__ float one_minus_u(float x) { return 0.5f * (1.0f - x); }

// Z = Phi^-1(u) = sqrt(2) erfinv(x), x = 2u - 1, by M. Giles' single-precision
// erfinv approximation ("Approximating the erfinv function", GPU Computing Gems
// Jade Edition, 2011): w = -ln(1 - x^2); a degree-8 polynomial in w - 2.5 for
// w < 5, else in sqrt(w) - 3, times x.  The coefficients below are Giles'
// multiplied by sqrt(2) (in double, rounded once), so no final scaling is needed.
// 1 - x^2 is formed by one FMA (exact product, one rounding) -- as x^2 - 1 with
// the sign dropped at the logarithm, which rounds to the same magnitude -- and
// w - 2.5 = -ln2 lg2(1 - x^2) - 2.5 by one more.
#define SIMR_S2(c) ((float)((c) * 1.4142135623730951))
// the tail branch (w >= 5, |x| > 0.9966: about 0.3% of the draws)
__device__ __forceinline__ float norminv_tail(float w) {
  w = __fsub_rn(sqrt_approx(w), 3.0f);
  float p = SIMR_S2(-0.000200214257);
  p = __fmaf_rn(p, w, SIMR_S2(0.000100950558));
  p = __fmaf_rn(p, w, SIMR_S2(0.00134934322));
  p = __fmaf_rn(p, w, SIMR_S2(-0.00367342844));
  p = __fmaf_rn(p, w, SIMR_S2(0.00573950773));
  p = __fmaf_rn(p, w, SIMR_S2(-0.0076224613));
  p = __fmaf_rn(p, w, SIMR_S2(0.00943887047));
  p = __fmaf_rn(p, w, SIMR_S2(1.00167406));
  p = __fmaf_rn(p, w, SIMR_S2(2.83297682));
  return p;
}
// w - 2.5 from lg2(1 - x^2)
__device__ __forceinline__ float norminv_wc(float x) {
  return __fmaf_rn(lg2_approx(fabsf(__fmaf_rn(x, x, -1.0f))), -0.69314718055994531f, -2.5f);
}
__device__ __forceinline__ float norminv_central(float wc) {
  float p = SIMR_S2(2.81022636e-08);
  p = __fmaf_rn(p, wc, SIMR_S2(3.43273939e-07));
  p = __fmaf_rn(p, wc, SIMR_S2(-3.5233877e-06));
  p = __fmaf_rn(p, wc, SIMR_S2(-4.39150654e-06));
  p = __fmaf_rn(p, wc, SIMR_S2(0.00021858087));
  p = __fmaf_rn(p, wc, SIMR_S2(-0.00125372503));
  p = __fmaf_rn(p, wc, SIMR_S2(-0.00417768164));
  p = __fmaf_rn(p, wc, SIMR_S2(0.246640727));
  p = __fmaf_rn(p, wc, SIMR_S2(1.50140941));
  return p;
}
__device__ __forceinline__ float norminv_centered(float x) {
  const float wc = norminv_wc(x);
  const float p = wc < 2.5f ? norminv_central(wc) : norminv_tail(__fadd_rn(wc, 2.5f));
  return __fmul_rn(p, x);
}
// Two inverse normals at once (the central polynomial paired, the rare tail per lane).
__device__ __forceinline__ float2 norminv_centered2(float2 x) {
  const float2 t = p_fma(x, x, p_bc(-1.0f));
  const float2 L = make_float2(lg2_approx(fabsf(t.x)), lg2_approx(fabsf(t.y)));
  const float2 wc = p_fma(L, p_bc(-0.69314718055994531f), p_bc(-2.5f));
  float2 p = p_bc(SIMR_S2(2.81022636e-08));
  p = p_fma(p, wc, p_bc(SIMR_S2(3.43273939e-07)));
  p = p_fma(p, wc, p_bc(SIMR_S2(-3.5233877e-06)));
  p = p_fma(p, wc, p_bc(SIMR_S2(-4.39150654e-06)));
  p = p_fma(p, wc, p_bc(SIMR_S2(0.00021858087)));
  p = p_fma(p, wc, p_bc(SIMR_S2(-0.00125372503)));
  p = p_fma(p, wc, p_bc(SIMR_S2(-0.00417768164)));
  p = p_fma(p, wc, p_bc(SIMR_S2(0.246640727)));
  p = p_fma(p, wc, p_bc(SIMR_S2(1.50140941)));
  if (!(wc.x < 2.5f && wc.y < 2.5f)) {  // one test on the common path
    if (!(wc.x < 2.5f)) p.x = norminv_tail(__fadd_rn(wc.x, 2.5f));
    if (!(wc.y < 2.5f)) p.y = norminv_tail(__fadd_rn(wc.y, 2.5f));
  }
  return p_mul(p, x);
}
#undef SIMR_S2

__device__ __forceinline__ float2 centered_uniform2(uint32_t wa, uint32_t wb) {
  const float2 f = make_float2(__uint_as_float(0x3f800000u | (wa >> 9)), __uint_as_float(0x3f800000u | (wb >> 9)));
  return p_fma(p_bc(2.0f), p_sub(f, p_bc(1.5f)), p_bc(0x1p-23f));
}

// ------------------------------------------------------------ QE step ----
// VariancePathQE (paper Sec. 4) with Andersen's QE rule, psi_c = 1.5, given
// m = E[v'|v] and s2h = Var[v'|v] / 2:
//   psi = s^2/m^2 <= 1.5 : v' = a (b + Z_V)^2, b^2 = t - 1 + sqrt(t (t - 1)),
//                          t = 2/psi = m^2 / s2h, a = m / (1 + b^2)
//   psi > 1.5            : p = (psi-1)/(psi+1); v' = 0 if U_V <= p,
//                          else ((1-p)/m)^-1 ln((1-p)/(1-U_V))
// The branch test is t > 4/3 in FP32, strictly: t is needed by the quadratic
// branch anyway, and m = 0 (theta = 0 and v = 0, so s2h = 0 as well: t = NaN)
// falls through to the exponential branch's m > 0 test (v' = 0) with no test of
// its own in the common path; a decision at FP32 distance from the threshold,
// where the FP64 reading psi <= psi_c can go either way anyway, may differ from
// it.  t - 1 is exact for t in [1, 2^24], so t (t - 1) rounds as t^2 - t.
// U_V <= p is tested as (1 - U_V)(m^2 + s^2) >= 2 m^2.  Besides v' the step
// returns dl = v' - m (the innovation the log-spot step needs) without
// cancellation in the quadratic branch: a (b + Z)^2 - m = a (Z (Z + 2b) - 1)
// since m = a (1 + b^2).  xv = 2 U_V - 1 (1 - U_V is formed only where the
// exponential branch needs it), zv = Phi^-1(U_V).
constexpr float kQuadT = 1.33333333333333333f;  // t above it: the quadratic branch (psi < 1.5)

__device__ __forceinline__ float qe_t(float m2, float s2h) { return __fmul_rn(m2, rcp_approx(s2h)); }

// the exponential branch (and the zero-mean case) of qe_from_moments
__device__ __forceinline__ void qe_exp_branch(float m, float s2h, float m2, float xv, float& v_next, float& dl) {
  if (m > 0.0f) {
    const float ms = __fadd_rn(m2, __fadd_rn(s2h, s2h));
    const float W = __fmul_rn(one_minus_u(xv), ms);
    if (W >= __fmul_rn(2.0f, m2)) {
      v_next = 0.0f;
    } else {
      const float L = __fmul_rn(0.69314718055994531f, lg2_approx(__fmul_rn(__fmul_rn(2.0f, m2), rcp_approx(W))));
      v_next = __fmul_rn(__fmul_rn(__fmul_rn(0.5f, ms), rcp_approx(m)), L);
    }
    dl = __fsub_rn(v_next, m);
  } else {
    v_next = 0.0f;
    dl = 0.0f;
  }
}

// the quadratic branch from t = m^2 / s2h
__device__ __forceinline__ void qe_quad_branch(float m, float t, float zv, float& v_next, float& dl, float* b2_out = nullptr,
                                               float* a_out = nullptr) {
  const float tm1 = __fsub_rn(t, 1.0f);
  const float root = sqrt_approx(__fmul_rn(t, tm1));
  const float b2 = __fadd_rn(tm1, root);
  const float b = sqrt_approx(b2);
  const float a = __fmul_rn(m, rcp_approx(__fadd_rn(t, root)));
  const float bz = __fadd_rn(b, zv);
  v_next = __fmul_rn(__fmul_rn(a, bz), bz);
  dl = __fmul_rn(a, __fmaf_rn(zv, __fadd_rn(bz, b), -1.0f));
  if (b2_out) *b2_out = b2;
  if (a_out) *a_out = a;
}

__device__ __forceinline__ void qe_from_moments(float m, float s2h, float xv, float zv, float& v_next, float& dl) {
  const float m2 = __fmul_rn(m, m);
  const float t = qe_t(m2, s2h);
  if (t > kQuadT)
    qe_quad_branch(m, t, zv, v_next, dl);
  else
    qe_exp_branch(m, s2h, m2, xv, v_next, dl);
}

// Two QE variance steps: the quadratic branch paired for both lanes, then any
// lane outside it redone by the scalar exponential branch.
__device__ __forceinline__ void qe_from_moments2(float2 m, float2 s2h, float2 xv, float2 zv, float2& v_next,
                                                 float2& dl) {
  const float2 m2 = p_mul(m, m);
  const float2 t = p_mul(m2, p_rcp(s2h));
  const float2 tm1 = p_sub(t, p_bc(1.0f));
  const float2 root = p_sqrt(p_mul(t, tm1));
  const float2 b2 = p_add(tm1, root);
  const float2 b = p_sqrt(b2);
  const float2 a = p_mul(m, p_rcp(p_add(t, root)));
  const float2 bz = p_add(b, zv);
  v_next = p_mul(p_mul(a, bz), bz);
  dl = p_mul(a, p_fma(zv, p_add(bz, b), p_bc(-1.0f)));
  const bool qx = t.x > kQuadT, qy = t.y > kQuadT;
  if (!(qx && qy)) {  // one test on the common path
    if (!qx) qe_exp_branch(m.x, s2h.x, m2.x, xv.x, v_next.x, dl.x);
    if (!qy) qe_exp_branch(m.y, s2h.y, m2.y, xv.y, v_next.y, dl.y);
  }
}

// One step of the base scenario: QE variance step, then LogPricePathQE (paper
// Sec. 5), Kahan-compensated in x.  CRN: with bumped scenarios alongside, the
// moments are formed in the bumped scenarios' rounding order (product, then
// the additive constant) so the two share their systematic rounding.
template <bool CRN>
__device__ __forceinline__ void step_base(const ScenConst& c, float xv, float zv, float zx, float& v, float& x,
                                          float& comp) {
  float vn, dl;
  // CRN: round(round(v E) + thE), exactly the bumped scenarios' sequence with zero
  // deltas (__fmul_rn / __fadd_rn are never contracted into an FMA)
  const float m = CRN ? __fadd_rn(__fmul_rn(v, c.E), c.thE) : __fmaf_rn(v, c.E, c.thE);
  const float s2h = CRN ? __fadd_rn(__fmul_rn(v, c.h1), c.h2) : __fmaf_rn(v, c.h1, c.h2);
  qe_from_moments(m, s2h, xv, zv, vn, dl);
  const float s = __fadd_rn(v, vn);
  float inc = __fmaf_rn(c.Cv, s, c.C0);
  inc = __fmaf_rn(-c.Cd, v, inc);
  inc = __fmaf_rn(c.Cdl, dl, inc);
  inc = __fmaf_rn(__fmul_rn(c.sK3, sqrt_approx(s)), zx, inc);
  const float y = __fsub_rn(inc, comp);
  const float t = __fadd_rn(x, y);
  comp = __fsub_rn(__fsub_rn(t, x), y);
  x = t;
  v = vn;
}

// step_base for two lanes sharing the constants (two paths, or two scenarios
// that differ only in v0).
template <bool CRN>
__device__ __forceinline__ void step_base2(const ScenConst2& c, float2 xv, float2 zv, float2 zx, float2& v,
                                           float2& x, float2& comp) {
  float2 vn, dl;
  const float2 m = CRN ? p_add(p_mul(v, c.E), c.thE) : p_fma(v, c.E, c.thE);
  const float2 s2h = CRN ? p_add(p_mul(v, c.h1), c.h2) : p_fma(v, c.h1, c.h2);
  qe_from_moments2(m, s2h, xv, zv, vn, dl);
  const float2 s = p_add(v, vn);
  float2 inc = p_fma(c.Cv, s, c.C0);
  inc = p_fma(c.mCd, v, inc);
  inc = p_fma(c.Cdl, dl, inc);
  inc = p_fma(p_mul(c.sK3, p_sqrt(s)), zx, inc);
  const float2 y = p_sub(inc, comp);
  const float2 t = p_add(x, y);
  comp = p_sub(p_sub(t, x), y);
  x = t;
  v = vn;
}

template <bool CRN>
__device__ __forceinline__ void step_base2(const ScenConst& c, float2 xv, float2 zv, float2 zx, float2& v,
                                           float2& x, float2& comp) {
  step_base2<CRN>(pack_const(c, c), xv, zv, zx, v, x, comp);
}

// QE-M (Andersen 2008, martingale correction): the constant K0 - r dt of the
// log-spot step becomes K0* = -ln M - (K1 + K3/2) v with M = E[exp(A v') | v],
// A = K2 + K4/2, so that the discounted spot is an exact martingale of the
// scheme.  Written around the same m and dl as the plain step,
//   x' - x = r dt - qa (v + m) - lam + K2 (v' - m) + sK3 sqrt(v + v') Z_X,
// qa = K3/2 = K4/2 = dt (1 - rho^2)/4 and lam = ln M - A m >= 0, which has no
// large cancelling terms (the rho/sigma parts of K1, K2 cancel exactly).
struct QemConst {
  float rdt, qa, K2, A;  // r dt, dt (1 - rho^2)/4, K2, K2 + K4/2
};
struct QemConst2 {  // two scenarios' QemConst (their deltas), lane by lane
  float2 rdt, qa, K2, A;
};

// g(u) = -u - ln(1 - u) = sum_{k >= 2} u^k / k, u < 1: the series to u^8 for
// |u| < 1/8 (remainder below 6e-8 relative), else the logarithm.
__device__ __forceinline__ float neg_log1m_tail(float u) {
  if (fabsf(u) < 0.125f) {
    float t = __fmaf_rn(u, 0.125f, 0.14285714285714285f);
    t = __fmaf_rn(u, t, 0.16666666666666666f);
    t = __fmaf_rn(u, t, 0.2f);
    t = __fmaf_rn(u, t, 0.25f);
    t = __fmaf_rn(u, t, 0.33333333333333333f);
    t = __fmaf_rn(u, t, 0.5f);
    return __fmul_rn(__fmul_rn(u, u), t);
  }
  return -u - log1pf(-u);
}

// The QE variance step of qe_from_moments (the same expressions, so the same
// v_next and dl) together with lam = ln M - A m of the QE-M correction; false
// where M does not exist (quadratic branch: 2 A a >= 1; exponential branch:
// A >= beta).  Quadratic: lam = 2 (A a)^2 b^2 / (1 - 2 A a) + g(2 A a)/2;
// exponential: lam = ln(1 + (1 - p) w / (1 - w)) - (1 - p) w with w = A / beta,
// 1 - p = 2 m^2 / (m^2 + s^2), beta = 2 m / (m^2 + s^2).
__device__ __forceinline__ bool qem_from_moments(float m, float s2h, float xv, float zv, float A, float& v_next,
                                                 float& dl, float& lam) {
  const float m2 = __fmul_rn(m, m);
  const float t = qe_t(m2, s2h);
  lam = 0.0f;
  if (t > kQuadT) {
    float b2, a;
    qe_quad_branch(m, t, zv, v_next, dl, &b2, &a);
    const float Aa = __fmul_rn(A, a);
    const float u = __fmul_rn(2.0f, Aa);
    if (!(u < 1.0f)) return false;
    lam = __fmaf_rn(0.5f, neg_log1m_tail(u),
                    __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(2.0f, Aa), Aa), b2), rcp_approx(__fsub_rn(1.0f, u))));
    return true;
  }
  if (m > 0.0f) {
    qe_exp_branch(m, s2h, m2, xv, v_next, dl);
    const float ms = m2 + (s2h + s2h);
    const float onep = 2.0f * m2 * rcp_approx(ms);  // 1 - p
    const float w = 0.5f * A * ms * rcp_approx(m);  // A / beta
    if (!(w < 1.0f)) return false;
    lam = log1pf(onep * w * rcp_approx(1.0f - w)) - onep * w;
    return true;
  }
  v_next = 0.0f;
  dl = 0.0f;
  return true;  // m = 0: v' = 0, M = 1
}

// One QE-M step of the base scenario (variance step identical to step_base's);
// where the correction does not exist the plain QE increment is taken.
__device__ __forceinline__ void step_qem(const ScenConst& c, const QemConst& q, float xv, float zv, float zx,
                                         float& v, float& x, float& comp) {
  float vn, dl, lam;
  const float m = __fmaf_rn(v, c.E, c.thE);
  const float s2h = __fmaf_rn(v, c.h1, c.h2);
  const bool ok = qem_from_moments(m, s2h, xv, zv, q.A, vn, dl, lam);
  const float s = __fadd_rn(v, vn);
  float inc;
  if (ok) {
    inc = __fsub_rn(__fmaf_rn(-q.qa, __fadd_rn(v, m), q.rdt), lam);
    inc = __fmaf_rn(q.K2, dl, inc);
  } else {
    inc = __fmaf_rn(c.Cv, s, c.C0);
    inc = __fmaf_rn(-c.Cd, v, inc);
    inc = __fmaf_rn(c.Cdl, dl, inc);
  }
  inc = __fmaf_rn(__fmul_rn(c.sK3, sqrt_approx(s)), zx, inc);
  const float y = __fsub_rn(inc, comp);
  const float t = __fadd_rn(x, y);
  comp = __fsub_rn(__fsub_rn(t, x), y);
  x = t;
  v = vn;
}

// The QE-M variance step of two lanes with their own A (qem_from_moments lane
// for lane): the quadratic branch and the series part of lam paired when both
// lanes take them, every other case per lane by the scalar function.
__device__ __forceinline__ void qem_from_moments2(float2 m, float2 s2h, float2 xv, float2 zv, float2 A, float2& vn,
                                                  float2& dl, float2& lam, bool& okx, bool& oky) {
  const float2 m2 = p_mul(m, m);
  const float2 t = p_mul(m2, p_rcp(s2h));
  if (t.x > kQuadT && t.y > kQuadT) {
    const float2 tm1 = p_sub(t, p_bc(1.0f));
    const float2 root = p_sqrt(p_mul(t, tm1));
    const float2 b2 = p_add(tm1, root);
    const float2 b = p_sqrt(b2);
    const float2 a = p_mul(m, p_rcp(p_add(t, root)));
    const float2 bz = p_add(b, zv);
    vn = p_mul(p_mul(a, bz), bz);
    dl = p_mul(a, p_fma(zv, p_add(bz, b), p_bc(-1.0f)));
    const float2 Aa = p_mul(A, a);
    const float2 u = p_mul(p_bc(2.0f), Aa);
    okx = u.x < 1.0f;
    oky = u.y < 1.0f;
    // g(u) by its series (neg_log1m_tail), the logarithm per lane outside |u| < 1/8
    float2 g = p_fma(u, p_bc(0.125f), p_bc(0.14285714285714285f));
    g = p_fma(u, g, p_bc(0.16666666666666666f));
    g = p_fma(u, g, p_bc(0.2f));
    g = p_fma(u, g, p_bc(0.25f));
    g = p_fma(u, g, p_bc(0.33333333333333333f));
    g = p_fma(u, g, p_bc(0.5f));
    g = p_mul(p_mul(u, u), g);
    if (!(fabsf(u.x) < 0.125f && fabsf(u.y) < 0.125f)) {
      if (!(fabsf(u.x) < 0.125f)) g.x = neg_log1m_tail(u.x);
      if (!(fabsf(u.y) < 0.125f)) g.y = neg_log1m_tail(u.y);
    }
    lam = p_fma(p_bc(0.5f), g, p_mul(p_mul(p_mul(p_mul(p_bc(2.0f), Aa), Aa), b2), p_rcp(p_sub(p_bc(1.0f), u))));
    if (!okx) lam.x = 0.0f;
    if (!oky) lam.y = 0.0f;
  } else {
    okx = qem_from_moments(m.x, s2h.x, xv.x, zv.x, A.x, vn.x, dl.x, lam.x);
    oky = qem_from_moments(m.y, s2h.y, xv.y, zv.y, A.y, vn.y, dl.y, lam.y);
  }
}

// Two QE-M steps (two paths on the same constants) in packed FP32, lane for
// lane step_qem.
__device__ __forceinline__ void step_qem2(const ScenConst& c, const QemConst& q, float2 xv, float2 zv, float2 zx,
                                          float2& v, float2& x, float2& comp) {
  const float2 m = p_fma(v, p_bc(c.E), p_bc(c.thE));
  const float2 s2h = p_fma(v, p_bc(c.h1), p_bc(c.h2));
  float2 vn, dl, lam;
  bool okx, oky;
  qem_from_moments2(m, s2h, xv, zv, p_bc(q.A), vn, dl, lam, okx, oky);
  const float2 s = p_add(v, vn);
  float2 inc;
  if (okx && oky) {
    inc = p_sub(p_fma(p_bc(-q.qa), p_add(v, m), p_bc(q.rdt)), lam);
    inc = p_fma(p_bc(q.K2), dl, inc);
  } else {
    const float vv[2] = {v.x, v.y}, mm[2] = {m.x, m.y}, ss[2] = {s.x, s.y}, dd[2] = {dl.x, dl.y},
                ll[2] = {lam.x, lam.y};
    const bool ok[2] = {okx, oky};
    float r[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (ok[j]) {
        r[j] = __fmaf_rn(q.K2, dd[j], __fsub_rn(__fmaf_rn(-q.qa, __fadd_rn(vv[j], mm[j]), q.rdt), ll[j]));
      } else {
        float t = __fmaf_rn(c.Cv, ss[j], c.C0);
        t = __fmaf_rn(-c.Cd, vv[j], t);
        r[j] = __fmaf_rn(c.Cdl, dd[j], t);
      }
    }
    inc = make_float2(r[0], r[1]);
  }
  inc = p_fma(p_mul(p_bc(c.sK3), p_sqrt(s)), zx, inc);
  const float2 y = p_sub(inc, comp);
  const float2 t2 = p_add(x, y);
  comp = p_sub(p_sub(t2, x), y);
  x = t2;
  v = vn;
}

// One step of the base scenario under scheme QEM (false: QE) with the CRN
// rounding order of step_base<CRN> for the plain scheme.
template <bool CRN, bool QEM>
__device__ __forceinline__ void step_scheme(const ScenConst& c, const QemConst& q, float xv, float zv, float zx,
                                            float& v, float& x, float& comp) {
  if constexpr (QEM)
    step_qem(c, q, xv, zv, zx, v, x, comp);
  else
    step_base<CRN>(c, xv, zv, zx, v, x, comp);
}

#ifndef SIMR_KAHAN_BUMPED
#define SIMR_KAHAN_BUMPED 1  // Kahan-compensate x in bumped scenarios too
#endif

// One step of a bumped scenario: base constants b plus deltas d.
__device__ __forceinline__ void step_bumped(const ScenConst& b, const ScenConst& d, float xv, float zv, float zx,
                                            float& v, float& x, float& comp) {
  const float m = __fadd_rn(__fmaf_rn(v, b.E, __fmaf_rn(v, d.E, d.thE)), b.thE);
  const float s2h = __fadd_rn(__fmaf_rn(v, b.h1, __fmaf_rn(v, d.h1, d.h2)), b.h2);
  float vn, dl;
  qe_from_moments(m, s2h, xv, zv, vn, dl);
  const float s = __fadd_rn(v, vn);
  const float q = sqrt_approx(s);
  float inc = __fmaf_rn(b.Cv, s, b.C0);
  inc = __fmaf_rn(-b.Cd, v, inc);
  inc = __fmaf_rn(b.Cdl, dl, inc);
  inc = __fmaf_rn(__fmul_rn(b.sK3, q), zx, inc);
  float sm = __fmaf_rn(d.Cv, s, d.C0);
  sm = __fmaf_rn(-d.Cd, v, sm);
  sm = __fmaf_rn(d.Cdl, dl, sm);
  sm = __fmaf_rn(__fmul_rn(d.sK3, q), zx, sm);
  inc = __fadd_rn(inc, sm);
#if SIMR_KAHAN_BUMPED
  const float y = __fsub_rn(inc, comp);
  const float t = __fadd_rn(x, y);
  comp = __fsub_rn(__fsub_rn(t, x), y);
  x = t;
#else
  x = __fadd_rn(x, inc);
#endif
  v = vn;
}

// One QE-M step of a scenario in a common-random-number launch: base constants
// b, q plus deltas d, qd (zero for the base scenario itself).  The variance step
// is step_bumped's; the correction lam comes from the scenario's own moments
// and A; the deltas of r dt, qa, K2 and sK3 enter as a separate sum, so the bump
// is not lost to the base terms' rounding.  Where M does not exist the plain
// bumped increment is taken.
__device__ __forceinline__ void step_qem_bumped(const ScenConst& b, const ScenConst& d, const QemConst& q,
                                                const QemConst& qd, float xv, float zv, float zx, float& v,
                                                float& x, float& comp) {
  const float m = __fadd_rn(__fmaf_rn(v, b.E, __fmaf_rn(v, d.E, d.thE)), b.thE);
  const float s2h = __fadd_rn(__fmaf_rn(v, b.h1, __fmaf_rn(v, d.h1, d.h2)), b.h2);
  float vn, dl, lam;
  const bool ok = qem_from_moments(m, s2h, xv, zv, __fadd_rn(q.A, qd.A), vn, dl, lam);
  const float s = __fadd_rn(v, vn);
  const float r = sqrt_approx(s);
  float inc, sm;
  if (ok) {
    const float vm = __fadd_rn(v, m);
    inc = __fmaf_rn(-q.qa, vm, q.rdt);
    inc = __fmaf_rn(q.K2, dl, inc);
    inc = __fmaf_rn(__fmul_rn(b.sK3, r), zx, inc);
    sm = __fmaf_rn(-qd.qa, vm, qd.rdt);
    sm = __fmaf_rn(qd.K2, dl, sm);
    sm = __fmaf_rn(__fmul_rn(d.sK3, r), zx, sm);
    sm = __fsub_rn(sm, lam);
  } else {
    inc = __fmaf_rn(b.Cv, s, b.C0);
    inc = __fmaf_rn(-b.Cd, v, inc);
    inc = __fmaf_rn(b.Cdl, dl, inc);
    inc = __fmaf_rn(__fmul_rn(b.sK3, r), zx, inc);
    sm = __fmaf_rn(d.Cv, s, d.C0);
    sm = __fmaf_rn(-d.Cd, v, sm);
    sm = __fmaf_rn(d.Cdl, dl, sm);
    sm = __fmaf_rn(__fmul_rn(d.sK3, r), zx, sm);
  }
  inc = __fadd_rn(inc, sm);
  const float y = __fsub_rn(inc, comp);
  const float t = __fadd_rn(x, y);
  comp = __fsub_rn(__fsub_rn(t, x), y);
  x = t;
  v = vn;
}

// step_qem_bumped for two scenarios (lane for lane its operations): base
// constants b, q (both lanes), deltas d, qd (lane x the first scenario's, lane y
// the second's).
__device__ __forceinline__ void step_qem_bumped2(const ScenConst2& b, const ScenConst2& d, const QemConst& q,
                                                 const QemConst2& qd, float2 xv, float2 zv, float2 zx, float2& v,
                                                 float2& x, float2& comp) {
  const float2 m = p_add(p_fma(v, b.E, p_fma(v, d.E, d.thE)), b.thE);
  const float2 s2h = p_add(p_fma(v, b.h1, p_fma(v, d.h1, d.h2)), b.h2);
  float2 vn, dl, lam;
  bool okx, oky;
  qem_from_moments2(m, s2h, xv, zv, p_add(p_bc(q.A), qd.A), vn, dl, lam, okx, oky);
  const float2 s = p_add(v, vn);
  const float2 r = p_sqrt(s);
  float2 inc, sm;
  if (okx && oky) {
    const float2 vm = p_add(v, m);
    inc = p_fma(p_bc(-q.qa), vm, p_bc(q.rdt));
    inc = p_fma(p_bc(q.K2), dl, inc);
    inc = p_fma(p_mul(b.sK3, r), zx, inc);
    sm = p_fma(p_mul(p_bc(-1.0f), qd.qa), vm, qd.rdt);
    sm = p_fma(qd.K2, dl, sm);
    sm = p_fma(p_mul(d.sK3, r), zx, sm);
    sm = p_sub(sm, lam);
  } else {  // per lane, step_qem_bumped's increment of that lane's branch
    const float vv[2] = {v.x, v.y}, mm[2] = {m.x, m.y}, ss[2] = {s.x, s.y}, dd[2] = {dl.x, dl.y},
                ll[2] = {lam.x, lam.y}, rr[2] = {r.x, r.y};
    const float bsk[2] = {b.sK3.x, b.sK3.y}, dsk[2] = {d.sK3.x, d.sK3.y};
    const float bC0[2] = {b.C0.x, b.C0.y}, bCv[2] = {b.Cv.x, b.Cv.y}, bmCd[2] = {b.mCd.x, b.mCd.y},
                bCdl[2] = {b.Cdl.x, b.Cdl.y};
    const float dC0[2] = {d.C0.x, d.C0.y}, dCv[2] = {d.Cv.x, d.Cv.y}, dmCd[2] = {d.mCd.x, d.mCd.y},
                dCdl[2] = {d.Cdl.x, d.Cdl.y};
    const float qrdt[2] = {qd.rdt.x, qd.rdt.y}, qqa[2] = {qd.qa.x, qd.qa.y}, qK2[2] = {qd.K2.x, qd.K2.y};
    const float zz[2] = {zx.x, zx.y};
    const bool ok[2] = {okx, oky};
    float ri[2], rs[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float a, c;
      if (ok[j]) {
        const float vm = __fadd_rn(vv[j], mm[j]);
        a = __fmaf_rn(-q.qa, vm, q.rdt);
        a = __fmaf_rn(q.K2, dd[j], a);
        a = __fmaf_rn(__fmul_rn(bsk[j], rr[j]), zz[j], a);
        c = __fmaf_rn(-qqa[j], vm, qrdt[j]);
        c = __fmaf_rn(qK2[j], dd[j], c);
        c = __fmaf_rn(__fmul_rn(dsk[j], rr[j]), zz[j], c);
        c = __fsub_rn(c, ll[j]);
      } else {
        a = __fmaf_rn(bCv[j], ss[j], bC0[j]);
        a = __fmaf_rn(bmCd[j], vv[j], a);
        a = __fmaf_rn(bCdl[j], dd[j], a);
        a = __fmaf_rn(__fmul_rn(bsk[j], rr[j]), zz[j], a);
        c = __fmaf_rn(dCv[j], ss[j], dC0[j]);
        c = __fmaf_rn(dmCd[j], vv[j], c);
        c = __fmaf_rn(dCdl[j], dd[j], c);
        c = __fmaf_rn(__fmul_rn(dsk[j], rr[j]), zz[j], c);
      }
      ri[j] = a;
      rs[j] = c;
    }
    inc = make_float2(ri[0], ri[1]);
    sm = make_float2(rs[0], rs[1]);
  }
  inc = p_add(inc, sm);
  const float2 y = p_sub(inc, comp);
  const float2 t = p_add(x, y);
  comp = p_sub(p_sub(t, x), y);
  x = t;
  v = vn;
}

// step_bumped for two scenarios: base constants b (both lanes), deltas d (lane
// x the first scenario's, lane y the second's).
__device__ __forceinline__ void step_bumped2(const ScenConst2& b, const ScenConst2& d, float2 xv, float2 zv,
                                             float2 zx, float2& v, float2& x, float2& comp) {
  const float2 m = p_add(p_fma(v, b.E, p_fma(v, d.E, d.thE)), b.thE);
  const float2 s2h = p_add(p_fma(v, b.h1, p_fma(v, d.h1, d.h2)), b.h2);
  float2 vn, dl;
  qe_from_moments2(m, s2h, xv, zv, vn, dl);
  const float2 s = p_add(v, vn);
  const float2 q = p_sqrt(s);
  float2 inc = p_fma(b.Cv, s, b.C0);
  inc = p_fma(b.mCd, v, inc);
  inc = p_fma(b.Cdl, dl, inc);
  inc = p_fma(p_mul(b.sK3, q), zx, inc);
  float2 sm = p_fma(d.Cv, s, d.C0);
  sm = p_fma(d.mCd, v, sm);
  sm = p_fma(d.Cdl, dl, sm);
  sm = p_fma(p_mul(d.sK3, q), zx, sm);
  inc = p_add(inc, sm);
#if SIMR_KAHAN_BUMPED
  const float2 y = p_sub(inc, comp);
  const float2 t = p_add(x, y);
  comp = p_sub(p_sub(t, x), y);
  x = t;
#else
  x = p_add(x, inc);
#endif
  v = vn;
}

// a + b rounded, plus the exact rounding error (Knuth's TwoSum; plain adds only).
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  const float s = a + b;
  const float bb = s - a;
  err = (a - (s - bb)) + (b - bb);
  return s;
}

// Step 0 of a scenario in a common-random-number launch: base first-step
// constants fb plus deltas fd (zero for the base scenario itself), base step
// constants b plus deltas d.  Each delta enters through the exact rounding
// error of a sum with a path-dependent operand, so no quantisation of the
// bump is shared by all paths.
__device__ __forceinline__ void step0_crn(const FirstConst& fb, const FirstConst& fd, const ScenConst& b,
                                          const ScenConst& d, float v0, float omu, float zv, float zx, float& v,
                                          float& x, float& comp) {
  float v1 = 0.0f, dl = 0.0f;
  if (fb.branch == 0) {
    float e;
    const float hi = two_sum(fb.b, zv, e);
    const float bz = hi + (e + fd.b);
    const float bz2 = bz * bz;
    v1 = fmaf(fb.a, bz2, fd.a * bz2);
    float g = fmaf(zv, zv + 2.0f * fb.b, -1.0f);
    g = fmaf(2.0f * fd.b, zv, g);
    dl = fmaf(fb.a, g, fd.a * g);
  } else if (fb.branch == 1) {
    if (omu < fd.q) {  // fd.q: this scenario's own threshold
      const float lnomu = 0.69314718055994531f * lg2_approx(omu);
      float e;
      const float hi = two_sum(fb.L, -lnomu, e);
      const float w = hi + (e + fd.L);
      v1 = fmaf(fb.C, w, fd.C * w);
    }
    float e;
    const float hi = two_sum(v1, -fb.m0, e);
    dl = hi + (e - fd.m0);
  }
  const float q = sqrt_approx(v0 + v1);
  float inc = fmaf(b.Cv, v1, fb.K0p);
  inc = fmaf(b.Cdl, dl, inc);
  inc = fmaf(b.sK3 * q, zx, inc);
  float sm = fmaf(d.Cv, v1, fd.K0p);
  sm = fmaf(d.Cdl, dl, sm);
  sm = fmaf(d.sK3 * q, zx, sm);
  x = inc + sm;
  comp = 0.0f;
  v = v1;
}

// One path of one scenario over all steps: x_T with its Kahan remainder (U:
// the step-pair loop unrolled U times).
template <bool QEM = false, int U = 1>
__device__ __forceinline__ void simulate_one(const ScenConst& c, uint32_t steps, uint32_t option,
                                             const uint32_t (&rk)[10][2], uint64_t path, float& x, float& comp,
                                             const QemConst& q = QemConst{}) {
  const PhiloxLane pl = philox_lane(path, rk);
  float v = c.v0;
  x = 0.0f;
  comp = 0.0f;
#pragma unroll U
  for (uint32_t p = 0; 2 * p < steps; ++p) {
    const uint4 w = philox_draw(pl, philox_ctr(p, option, rk), rk);
    {
      const float xv = centered_uniform(w.x);
      step_scheme<false, QEM>(c, q, xv, norminv_centered(xv), norminv_centered(centered_uniform(w.y)), v, x, comp);
    }
    if (2 * p + 1 < steps) {
      const float xv = centered_uniform(w.z);
      step_scheme<false, QEM>(c, q, xv, norminv_centered(xv), norminv_centered(centered_uniform(w.w)), v, x, comp);
    }
  }
}

// Two paths of one scenario in lockstep: simulate_one's arithmetic, paired lane
// for lane (QE, or QE-M through step_qem2), so each path's x_T and remainder
// equal simulate_one's (U: the step-pair loop unrolled U times).
template <int U = 1, bool QEM = false>
__device__ __forceinline__ void simulate_two(const ScenConst& c, uint32_t steps, uint32_t option,
                                             const uint32_t (&rk)[10][2], uint64_t path0, uint64_t path1,
                                             float2& x, float2& comp, const QemConst& q = QemConst{}) {
  const PhiloxLane pl0 = philox_lane(path0, rk), pl1 = philox_lane(path1, rk);
  float2 v = make_float2(c.v0, c.v0);
  x = make_float2(0.0f, 0.0f);
  comp = make_float2(0.0f, 0.0f);
#pragma unroll U
  for (uint32_t p = 0; 2 * p < steps; ++p) {
    const PhiloxCtr u = philox_ctr(p, option, rk);
    const uint4 w0 = philox_draw(pl0, u, rk);
    const uint4 w1 = philox_draw(pl1, u, rk);
    {
      const float2 xv = centered_uniform2(w0.x, w1.x);
      const float2 zv = norminv_centered2(xv);
      const float2 zx = norminv_centered2(centered_uniform2(w0.y, w1.y));
      if constexpr (QEM)
        step_qem2(c, q, xv, zv, zx, v, x, comp);
      else
        step_base2<false>(c, xv, zv, zx, v, x, comp);
    }
    if (2 * p + 1 < steps) {
      const float2 xv = centered_uniform2(w0.z, w1.z);
      const float2 zv = norminv_centered2(xv);
      const float2 zx = norminv_centered2(centered_uniform2(w0.w, w1.w));
      if constexpr (QEM)
        step_qem2(c, q, xv, zv, zx, v, x, comp);
      else
        step_base2<false>(c, xv, zv, zx, v, x, comp);
    }
  }
}

// AssetPathExponential (paper Sec. 5): S_T = S0 e^{x} with the Kahan remainder
// (true sum = x - comp) applied as S (1 - comp).  expf is the accurate one.
__device__ __forceinline__ float terminal_spot(float S0, float x, float comp) {
  const float e = S0 * expf(x);
  return fmaf(-comp, e, e);
}

}  // namespace simr
