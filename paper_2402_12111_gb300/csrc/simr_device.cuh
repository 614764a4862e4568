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
//   m   = theta + (v - theta) E          = fma(v, E, thE)
//   s^2 = v c1 + c2
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
  float E, thE, c1, c2;
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
  float2 E, thE, c1, c2, C0, Cv, mCd, Cdl, sK3;  // mCd = -Cd
};

__host__ __device__ inline ScenConst2 pack_const(const ScenConst& a, const ScenConst& b) {
  ScenConst2 p;
  p.E = make_float2(a.E, b.E);
  p.thE = make_float2(a.thE, b.thE);
  p.c1 = make_float2(a.c1, b.c1);
  p.c2 = make_float2(a.c2, b.c2);
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
// Philox4x32-10 (Salmon et al., SC'11).  rk[i] = key + i * (0x9E3779B9, 0xBB67AE85)
// is precomputed on the host (the key is uniform over the launch), so each round
// is two 32x32->64 multiplies and two three-input XORs with a constant operand.
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               const uint32_t (&rk)[10][2]) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ rk[i][0];
    const uint32_t n2 = hi0 ^ c3 ^ rk[i][1];
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// x = 2u - 1 for u = ((w >> 9) + 1/2) 2^-23, exact in FP32:
// f = 1 + (w >> 9) 2^-23 from the bits, f - 1.5 is exact, and
// 2 (f - 1.5) + 2^-23 = (2k + 1 - 2^23) 2^-23 needs at most 23 significant bits.
__device__ __forceinline__ float centered_uniform(uint32_t w) {
  const float f = __uint_as_float(0x3f800000u | (w >> 9));
  return fmaf(2.0f, f - 1.5f, 0x1p-23f);
}

// Z = Phi^-1(u) = sqrt(2) erfinv(x), x = 2u - 1, by M. Giles' single-precision
// erfinv approximation ("Approximating the erfinv function", GPU Computing Gems
// Jade Edition, 2011): w = -ln(1 - x^2); a degree-8 polynomial in w - 2.5 for
// w < 5, else in sqrt(w) - 3, times x.  The coefficients below are Giles'
// multiplied by sqrt(2) (in double, rounded once), so no final scaling is needed.
// 1 - x^2 is formed by one FMA (exact product, one rounding).
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
__device__ __forceinline__ float norminv_centered(float x) {
  const float w = __fmul_rn(-0.69314718055994531f, lg2_approx(__fmaf_rn(-x, x, 1.0f)));
  float p;
  if (w < 5.0f) {
    const float wc = __fsub_rn(w, 2.5f);
    p = SIMR_S2(2.81022636e-08);
    p = __fmaf_rn(p, wc, SIMR_S2(3.43273939e-07));
    p = __fmaf_rn(p, wc, SIMR_S2(-3.5233877e-06));
    p = __fmaf_rn(p, wc, SIMR_S2(-4.39150654e-06));
    p = __fmaf_rn(p, wc, SIMR_S2(0.00021858087));
    p = __fmaf_rn(p, wc, SIMR_S2(-0.00125372503));
    p = __fmaf_rn(p, wc, SIMR_S2(-0.00417768164));
    p = __fmaf_rn(p, wc, SIMR_S2(0.246640727));
    p = __fmaf_rn(p, wc, SIMR_S2(1.50140941));
  } else {
    p = norminv_tail(w);
  }
  return __fmul_rn(p, x);
}
// Two inverse normals at once (the central polynomial paired, the rare tail per lane).
__device__ __forceinline__ float2 norminv_centered2(float2 x) {
  const float2 w = p_mul(p_bc(-0.69314718055994531f), p_lg2(p_fma(p_mul(x, p_bc(-1.0f)), x, p_bc(1.0f))));
  const float2 wc = p_sub(w, p_bc(2.5f));
  float2 p = p_bc(SIMR_S2(2.81022636e-08));
  p = p_fma(p, wc, p_bc(SIMR_S2(3.43273939e-07)));
  p = p_fma(p, wc, p_bc(SIMR_S2(-3.5233877e-06)));
  p = p_fma(p, wc, p_bc(SIMR_S2(-4.39150654e-06)));
  p = p_fma(p, wc, p_bc(SIMR_S2(0.00021858087)));
  p = p_fma(p, wc, p_bc(SIMR_S2(-0.00125372503)));
  p = p_fma(p, wc, p_bc(SIMR_S2(-0.00417768164)));
  p = p_fma(p, wc, p_bc(SIMR_S2(0.246640727)));
  p = p_fma(p, wc, p_bc(SIMR_S2(1.50140941)));
  if (!(w.x < 5.0f && w.y < 5.0f)) {  // one test on the common path
    if (!(w.x < 5.0f)) p.x = norminv_tail(w.x);
    if (!(w.y < 5.0f)) p.y = norminv_tail(w.y);
  }
  return p_mul(p, x);
}
#undef SIMR_S2

// ------------------------------------------------------------ QE step ----
// VariancePathQE (paper Sec. 4) with Andersen's QE rule, psi_c = 1.5, given
// m = E[v'|v] and s2 = Var[v'|v]:
//   psi = s^2/m^2 <= 1.5 : v' = a (b + Z_V)^2, b^2 = t - 1 + sqrt(t (t - 1)),
//                          t = 2/psi, a = m / (1 + b^2)
//   psi > 1.5            : p = (psi-1)/(psi+1); v' = 0 if U_V <= p,
//                          else ((1-p)/m)^-1 ln((1-p)/(1-U_V))
// The branch test needs no division: s^2 < 1.5 m^2 in FP32, strictly, so that
// m = 0 (theta = 0 and v = 0: then s^2 = 0 as well) falls through to the
// exponential branch's m > 0 test (v' = 0) with no test of its own in the
// common path; an exact FP32 tie -- at FP32 distance from the threshold, where
// the FP64 reading psi <= psi_c can go either way anyway -- takes the
// exponential branch.  U_V <= p is tested as
// (1 - U_V)(m^2 + s^2) >= 2 m^2.  Besides v' it returns dl = v' - m (the
// innovation the log-spot step needs) without cancellation in the quadratic
// branch: a (b + Z)^2 - m = a (Z (Z + 2b) - 1) since m = a (1 + b^2).
// omu = 1 - U_V (exact), zv = Phi^-1(U_V).
// the exponential branch (and the zero-mean case) of qe_from_moments
__device__ __forceinline__ void qe_exp_branch(float m, float s2, float m2, float omu, float& v_next, float& dl) {
  if (m > 0.0f) {
    const float ms = __fadd_rn(m2, s2);
    const float W = __fmul_rn(omu, ms);
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

__device__ __forceinline__ void qe_from_moments(float m, float s2, float omu, float zv, float& v_next,
                                                float& dl) {
  const float m2 = __fmul_rn(m, m);
  if (s2 < __fmul_rn(1.5f, m2)) {
    const float t = __fmul_rn(__fmul_rn(2.0f, m2), rcp_approx(s2));
    const float root = sqrt_approx(__fmaf_rn(t, t, -t));
    const float b2 = __fadd_rn(__fsub_rn(t, 1.0f), root);
    const float b = sqrt_approx(b2);
    const float a = __fmul_rn(m, rcp_approx(__fadd_rn(t, root)));
    const float bz = __fadd_rn(b, zv);
    v_next = __fmul_rn(__fmul_rn(a, bz), bz);
    dl = __fmul_rn(a, __fmaf_rn(zv, __fadd_rn(zv, __fmul_rn(2.0f, b)), -1.0f));
  } else {
    qe_exp_branch(m, s2, m2, omu, v_next, dl);
  }
}

// Two QE variance steps: the quadratic branch paired for both lanes, then any
// lane outside it redone by the scalar exponential branch.
__device__ __forceinline__ void qe_from_moments2(float2 m, float2 s2, float2 omu, float2 zv, float2& v_next,
                                                 float2& dl) {
  const float2 m2 = p_mul(m, m);
  const float2 lim = p_mul(p_bc(1.5f), m2);
  const float2 t = p_mul(p_mul(p_bc(2.0f), m2), p_rcp(s2));
  const float2 root = p_sqrt(p_fma(t, t, p_mul(t, p_bc(-1.0f))));
  const float2 b2 = p_add(p_sub(t, p_bc(1.0f)), root);
  const float2 b = p_sqrt(b2);
  const float2 a = p_mul(m, p_rcp(p_add(t, root)));
  const float2 bz = p_add(b, zv);
  v_next = p_mul(p_mul(a, bz), bz);
  dl = p_mul(a, p_fma(zv, p_add(zv, p_mul(p_bc(2.0f), b)), p_bc(-1.0f)));
  const bool qx = s2.x < lim.x, qy = s2.y < lim.y;
  if (!(qx && qy)) {  // one test on the common path
    if (!qx) qe_exp_branch(m.x, s2.x, m2.x, omu.x, v_next.x, dl.x);
    if (!qy) qe_exp_branch(m.y, s2.y, m2.y, omu.y, v_next.y, dl.y);
  }
}

// One step of the base scenario: QE variance step, then LogPricePathQE (paper
// Sec. 5), Kahan-compensated in x.  CRN: with bumped scenarios alongside, the
// moments are formed in the bumped scenarios' rounding order (product, then
// the additive constant) so the two share their systematic rounding.
template <bool CRN>
__device__ __forceinline__ void step_base(const ScenConst& c, float omu, float zv, float zx, float& v, float& x,
                                          float& comp) {
  float vn, dl;
  // CRN: round(round(v E) + thE), exactly the bumped scenarios' sequence with zero
  // deltas (__fmul_rn / __fadd_rn are never contracted into an FMA)
  const float m = CRN ? __fadd_rn(__fmul_rn(v, c.E), c.thE) : __fmaf_rn(v, c.E, c.thE);
  const float s2 = CRN ? __fadd_rn(__fmul_rn(v, c.c1), c.c2) : __fmaf_rn(v, c.c1, c.c2);
  qe_from_moments(m, s2, omu, zv, vn, dl);
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
__device__ __forceinline__ void step_base2(const ScenConst2& c, float2 omu, float2 zv, float2 zx, float2& v,
                                           float2& x, float2& comp) {
  float2 vn, dl;
  const float2 m = CRN ? p_add(p_mul(v, c.E), c.thE) : p_fma(v, c.E, c.thE);
  const float2 s2 = CRN ? p_add(p_mul(v, c.c1), c.c2) : p_fma(v, c.c1, c.c2);
  qe_from_moments2(m, s2, omu, zv, vn, dl);
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
__device__ __forceinline__ void step_base2(const ScenConst& c, float2 omu, float2 zv, float2 zx, float2& v,
                                           float2& x, float2& comp) {
  step_base2<CRN>(pack_const(c, c), omu, zv, zx, v, x, comp);
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
__device__ __forceinline__ bool qem_from_moments(float m, float s2, float omu, float zv, float A, float& v_next,
                                                 float& dl, float& lam) {
  const float m2 = __fmul_rn(m, m);
  lam = 0.0f;
  if (s2 < __fmul_rn(1.5f, m2)) {
    const float t = __fmul_rn(__fmul_rn(2.0f, m2), rcp_approx(s2));
    const float root = sqrt_approx(__fmaf_rn(t, t, -t));
    const float b2 = __fadd_rn(__fsub_rn(t, 1.0f), root);
    const float b = sqrt_approx(b2);
    const float a = __fmul_rn(m, rcp_approx(__fadd_rn(t, root)));
    const float bz = __fadd_rn(b, zv);
    v_next = __fmul_rn(__fmul_rn(a, bz), bz);
    dl = __fmul_rn(a, __fmaf_rn(zv, __fadd_rn(zv, __fmul_rn(2.0f, b)), -1.0f));
    const float Aa = __fmul_rn(A, a);
    const float u = __fmul_rn(2.0f, Aa);
    if (!(u < 1.0f)) return false;
    lam = __fmaf_rn(0.5f, neg_log1m_tail(u),
                    __fmul_rn(__fmul_rn(__fmul_rn(__fmul_rn(2.0f, Aa), Aa), b2), rcp_approx(__fsub_rn(1.0f, u))));
    return true;
  }
  if (m > 0.0f) {
    const float ms = m2 + s2;
    const float W = omu * ms;
    if (W >= 2.0f * m2) {
      v_next = 0.0f;
    } else {
      const float L = 0.69314718055994531f * lg2_approx(2.0f * m2 * rcp_approx(W));
      v_next = 0.5f * ms * rcp_approx(m) * L;
    }
    dl = v_next - m;
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
__device__ __forceinline__ void step_qem(const ScenConst& c, const QemConst& q, float omu, float zv, float zx,
                                         float& v, float& x, float& comp) {
  float vn, dl, lam;
  const float m = __fmaf_rn(v, c.E, c.thE);
  const float s2 = __fmaf_rn(v, c.c1, c.c2);
  const bool ok = qem_from_moments(m, s2, omu, zv, q.A, vn, dl, lam);
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

// Two QE-M steps (two paths on the same constants) in packed FP32, lane for
// lane step_qem: the quadratic branch and the series part of lam paired when
// both lanes take them, every other case per lane by the scalar functions.
__device__ __forceinline__ void step_qem2(const ScenConst& c, const QemConst& q, float2 omu, float2 zv, float2 zx,
                                          float2& v, float2& x, float2& comp) {
  const float2 m = p_fma(v, p_bc(c.E), p_bc(c.thE));
  const float2 s2 = p_fma(v, p_bc(c.c1), p_bc(c.c2));
  const float2 m2 = p_mul(m, m);
  const float2 lim = p_mul(p_bc(1.5f), m2);
  float2 vn, dl, lam;
  bool okx, oky;
  if (s2.x < lim.x && s2.y < lim.y) {
    const float2 t = p_mul(p_mul(p_bc(2.0f), m2), p_rcp(s2));
    const float2 root = p_sqrt(p_fma(t, t, p_mul(t, p_bc(-1.0f))));
    const float2 b2 = p_add(p_sub(t, p_bc(1.0f)), root);
    const float2 b = p_sqrt(b2);
    const float2 a = p_mul(m, p_rcp(p_add(t, root)));
    const float2 bz = p_add(b, zv);
    vn = p_mul(p_mul(a, bz), bz);
    dl = p_mul(a, p_fma(zv, p_add(zv, p_mul(p_bc(2.0f), b)), p_bc(-1.0f)));
    const float2 Aa = p_mul(p_bc(q.A), a);
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
    okx = qem_from_moments(m.x, s2.x, omu.x, zv.x, q.A, vn.x, dl.x, lam.x);
    oky = qem_from_moments(m.y, s2.y, omu.y, zv.y, q.A, vn.y, dl.y, lam.y);
  }
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
  const float2 t = p_add(x, y);
  comp = p_sub(p_sub(t, x), y);
  x = t;
  v = vn;
}

// One step of the base scenario under scheme QEM (false: QE) with the CRN
// rounding order of step_base<CRN> for the plain scheme.
template <bool CRN, bool QEM>
__device__ __forceinline__ void step_scheme(const ScenConst& c, const QemConst& q, float omu, float zv, float zx,
                                            float& v, float& x, float& comp) {
  if constexpr (QEM)
    step_qem(c, q, omu, zv, zx, v, x, comp);
  else
    step_base<CRN>(c, omu, zv, zx, v, x, comp);
}

#ifndef SIMR_KAHAN_BUMPED
#define SIMR_KAHAN_BUMPED 1  // Kahan-compensate x in bumped scenarios too
#endif

// One step of a bumped scenario: base constants b plus deltas d.
__device__ __forceinline__ void step_bumped(const ScenConst& b, const ScenConst& d, float omu, float zv, float zx,
                                            float& v, float& x, float& comp) {
  const float m = __fadd_rn(__fmaf_rn(v, b.E, __fmaf_rn(v, d.E, d.thE)), b.thE);
  const float s2 = __fadd_rn(__fmaf_rn(v, b.c1, __fmaf_rn(v, d.c1, d.c2)), b.c2);
  float vn, dl;
  qe_from_moments(m, s2, omu, zv, vn, dl);
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

// step_bumped for two scenarios: base constants b (both lanes), deltas d (lane
// x the first scenario's, lane y the second's).
__device__ __forceinline__ void step_bumped2(const ScenConst2& b, const ScenConst2& d, float2 omu, float2 zv,
                                             float2 zx, float2& v, float2& x, float2& comp) {
  const float2 m = p_add(p_fma(v, b.E, p_fma(v, d.E, d.thE)), b.thE);
  const float2 s2 = p_add(p_fma(v, b.c1, p_fma(v, d.c1, d.c2)), b.c2);
  float2 vn, dl;
  qe_from_moments2(m, s2, omu, zv, vn, dl);
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
  const uint32_t plo = (uint32_t)path, phi = (uint32_t)(path >> 32);
  float v = c.v0;
  x = 0.0f;
  comp = 0.0f;
#pragma unroll U
  for (uint32_t p = 0; 2 * p < steps; ++p) {
    const uint4 w = philox4x32_10(p, plo, phi, option, rk);
    {
      const float xv = centered_uniform(w.x);
      step_scheme<false, QEM>(c, q, 0.5f * (1.0f - xv), norminv_centered(xv),
                              norminv_centered(centered_uniform(w.y)), v, x, comp);
    }
    if (2 * p + 1 < steps) {
      const float xv = centered_uniform(w.z);
      step_scheme<false, QEM>(c, q, 0.5f * (1.0f - xv), norminv_centered(xv),
                              norminv_centered(centered_uniform(w.w)), v, x, comp);
    }
  }
}

// Two paths of one scenario in lockstep (plain QE): simulate_one's arithmetic,
// paired lane for lane, so each path's x_T and remainder equal simulate_one's
// (U: the step-pair loop unrolled U times).
template <int U = 1>
__device__ __forceinline__ void simulate_two(const ScenConst& c, uint32_t steps, uint32_t option,
                                             const uint32_t (&rk)[10][2], uint64_t path0, uint64_t path1,
                                             float2& x, float2& comp) {
  const uint32_t plo0 = (uint32_t)path0, phi0 = (uint32_t)(path0 >> 32);
  const uint32_t plo1 = (uint32_t)path1, phi1 = (uint32_t)(path1 >> 32);
  float2 v = make_float2(c.v0, c.v0);
  x = make_float2(0.0f, 0.0f);
  comp = make_float2(0.0f, 0.0f);
#pragma unroll U
  for (uint32_t p = 0; 2 * p < steps; ++p) {
    const uint4 w0 = philox4x32_10(p, plo0, phi0, option, rk);
    const uint4 w1 = philox4x32_10(p, plo1, phi1, option, rk);
    {
      const float xa = centered_uniform(w0.x), xb = centered_uniform(w1.x);
      const float2 zv = norminv_centered2(make_float2(xa, xb));
      const float2 zx = norminv_centered2(make_float2(centered_uniform(w0.y), centered_uniform(w1.y)));
      step_base2<false>(c, make_float2(0.5f * (1.0f - xa), 0.5f * (1.0f - xb)), zv, zx, v, x, comp);
    }
    if (2 * p + 1 < steps) {
      const float xa = centered_uniform(w0.z), xb = centered_uniform(w1.z);
      const float2 zv = norminv_centered2(make_float2(xa, xb));
      const float2 zx = norminv_centered2(make_float2(centered_uniform(w0.w), centered_uniform(w1.w)));
      step_base2<false>(c, make_float2(0.5f * (1.0f - xa), 0.5f * (1.0f - xb)), zv, zx, v, x, comp);
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
