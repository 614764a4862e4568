// simr_adjoint_path.cuh -- per-path pathwise adjoint of the Heston QE path (forward pass
// with checkpoints, reverse sweep), shared by the per-strike adjoint kernel and
// the batched book kernel.  See simr_adjoint.cu for the method.
#pragma once

#include <cstdint>

#include "simr_device.cuh"
#include "simr_internal.h"

namespace simr {
namespace {

// One QE variance step from v given the step's draws (no log-spot update).
__device__ __forceinline__ float qe_only(const ScenConst& c, float v, float omu, float zv) {
  float vn, dl;
  qe_from_moments(fmaf(v, c.E, c.thE), fmaf(v, c.c1, c.c2), omu, zv, vn, dl);
  return vn;
}

struct AdjSums {
  float vbar, Am, Amv, As, Asv, Ad, Adl, Ak3;
  float x, comp;  // x_T accumulated over the reverse sweep (Kahan-compensated)
};

// Reverse step n: state vc -> vn (both known), the step's stored draw d (Z_V in
// the quadratic branch, 1 - U_V in the exponential one; the branch follows from
// vc) and Z_X; vbar holds the adjoint of v_{n+1} on entry and of v_n on exit.
// Each square root and its reciprocal come from one rsqrt.
__device__ __forceinline__ void adjoint_step(const ScenConst& c, float theta, float vc, float vn, float d, float zx,
                                             AdjSums& a) {
  const float m = fmaf(vc, c.E, c.thE);
  const float s2 = fmaf(vc, c.c1, c.c2);
  const float m2 = m * m;
  const float s = vc + vn;
  const float rq = rsqrt_approx(s);
  const float q = s > 0.0f ? s * rq : 0.0f;
  const float hz = s > 0.0f ? 0.5f * c.sK3 * zx * rq : 0.0f;  // d(sK3 sqrt(s) Z)/ds
  const float vnbar = a.vbar + c.Cv + hz;  // total adjoint of v_{n+1}
  const float dlbar = c.Cdl;
  float mbar = 0.0f, s2bar = 0.0f, dl = 0.0f;
  if (s2 <= 1.5f * m2 && m2 > 0.0f) {
    const float zv = d;
    const float rs2 = rcp_approx(s2);
    const float t = 2.0f * m2 * rs2;
    const float tt = fmaf(t, t, -t);
    const float rroot = rsqrt_approx(tt);
    const float root = tt * rroot;
    const float b2 = (t - 1.0f) + root;
    const float rb = rsqrt_approx(b2);
    const float b = b2 * rb;
    const float ropb2 = rcp_approx(t + root);  // 1 / (1 + b^2)
    const float am = m * ropb2;
    const float bz = b + zv;
    const float g = fmaf(zv, zv + 2.0f * b, -1.0f);
    dl = am * g;
    const float abar = fmaf(vnbar, bz * bz, dlbar * g);
    const float bbar = 2.0f * am * fmaf(vnbar, bz, dlbar * zv);
    const float b2bar = fmaf(0.5f * bbar, rb, -abar * am * ropb2);
    mbar = abar * ropb2;
    const float tbar = b2bar * fmaf(2.0f * t - 1.0f, 0.5f * rroot, 1.0f);
    mbar = fmaf(tbar * 4.0f * m, rs2, mbar);
    s2bar = -tbar * t * rs2;
  } else if (m > 0.0f) {
    const float omu = d;
    const float ms = m2 + s2;
    const float W = omu * ms;
    if (W >= 2.0f * m2) {
      dl = -m;
      mbar = -dlbar;
    } else {
      const float rm = rcp_approx(m), rms = rcp_approx(ms);
      const float L = 0.69314718055994531f * lg2_approx(2.0f * m2 * rcp_approx(W));
      const float A = 0.5f * ms * rm;
      const float dA_dm = 0.5f * (m2 - s2) * rm * rm;
      const float dL_dm = 2.0f * rm - 2.0f * m * rms;
      const float dv_dm = fmaf(dA_dm, L, A * dL_dm);
      const float dv_ds = fmaf(0.5f * rm, L, -A * rms);
      dl = vn - m;
      mbar = fmaf(vnbar, dv_dm, dlbar * (dv_dm - 1.0f));
      s2bar = (vnbar + dlbar) * dv_ds;
    }
  }
  // the step's log-spot increment (LogPricePathQE), summed into x_T here rather
  // than in the forward pass
  float inc = fmaf(c.Cv, s, c.C0);
  inc = fmaf(-c.Cd, vc, inc);
  inc = fmaf(c.Cdl, dl, inc);
  inc = fmaf(c.sK3 * q, zx, inc);
  const float y = inc - a.comp;
  const float tx = a.x + y;
  a.comp = (tx - a.x) - y;
  a.x = tx;
  a.vbar = (c.Cv - c.Cd + hz) + fmaf(mbar, c.E, s2bar * c.c1);
  a.Am += mbar;
  a.Amv = fmaf(mbar, vc - theta, a.Amv);
  a.As += s2bar;
  a.Asv = fmaf(s2bar, vc, a.Asv);
  a.Ad += theta - vc;
  a.Adl += dl;
  a.Ak3 = fmaf(q, zx, a.Ak3);
}

// The draw the reverse step of state v needs: Z_V in the quadratic branch,
// 1 - U_V otherwise (same branch test as the forward step).
__device__ __forceinline__ float branch_draw(const ScenConst& c, float v, float omu, float zv) {
  const float m = fmaf(v, c.E, c.thE);
  const float s2 = fmaf(v, c.c1, c.c2);
  return (s2 <= 1.5f * (m * m) && m * m > 0.0f) ? zv : omu;
}

// The stored data of one step (recompute pass): state, branch draw, Z_X, from
// the step's centred variance uniform and its two normals.
__device__ __forceinline__ void keep_step(const ScenConst& c, float xv_v, float zv, float zx, float* bv, float* bd_,
                                          float* bz, float& v) {
  const float omu = 0.5f * (1.0f - xv_v);
  *bv = v;
  *bd_ = branch_draw(c, v, omu, zv);
  *bz = zx;
  v = qe_only(c, v, omu, zv);
}

// The FP64 map of the sweep's sums onto d x_T / d(v0, kappa, theta, sigma, rho).
__device__ __forceinline__ void adjoint_map(const AdjConst& A, const AdjSums& a, float (&g)[5]) {
  const double Amv = a.Amv, Asv = a.Asv, As = a.As, Ad = a.Ad, Adl = a.Adl, Am = a.Am, Ak3 = a.Ak3;
  g[0] = a.vbar;
  g[1] = (float)(A.dE_dk * Amv + A.dc1_dk * Asv + A.dc2_dk * As + A.dCd_dk * Ad + A.dCdl_dk * Adl);
  g[2] = (float)(A.omE * Am + A.dc2_dth * As + A.N_Cd);
  g[3] = (float)(A.two_over_sigma * (A.c1 * Asv + A.c2 * As) - A.Cd_over_sigma * Ad - A.Cdl_over_sigma * Adl);
  g[4] = (float)(A.D_over_sigma * Ad + A.B_over_sigma * Adl + A.dsK3_drho * Ak3);
}

// Forward pass with checkpoints, then the reverse sweep, for PPT paths in
// lockstep (independent dependency chains for the scheduler to interleave):
// x_T (with its Kahan remainder) and g = d x_T / d(v0, kappa, theta, sigma, rho)
// per path.  The forward pass runs the variance recursion only, and only up to
// the last checkpoint (x_T is not needed before the sweep ends; the last
// segment is recomputed from its checkpoint anyway); the reverse sweep adds up
// the log-spot increments as it goes.  Checkpoint (slot, path j) of this thread
// at ck[(slot * PPT + j) * ck_stride] (n_seg - 1 slots; shared or global memory);
// the segment's states, branch draws and Z_X in this thread's column of a
// shared buffer of bd columns: seg[((q * k + i) * PPT + j) * bd], q = 0..2.
// The recompute pass of a segment keeps them there, so the reverse sweep
// regenerates nothing.
template <int PPT>
__device__ __forceinline__ void path_adjoint_ppt(const ScenConst& c, const AdjConst& A, uint32_t N, uint32_t option,
                                                 const uint32_t (&rk)[10][2], const uint64_t (&path)[PPT], float* ck,
                                                 int ck_stride, float* seg, int bd, float (&x_out)[PPT],
                                                 float (&comp_out)[PPT], float (&g)[PPT][5]) {
  const float theta = A.theta;
  const uint32_t k = (uint32_t)A.ckpt_every;
  const int n_seg = A.n_seg;
  const int stride = PPT * bd;  // between consecutive steps of one thread's segment column
  uint32_t plo[PPT], phi[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    plo[j] = (uint32_t)path[j];
    phi[j] = (uint32_t)(path[j] >> 32);
  }
#define SIMR_CK(slot, j) ck[((int)(slot) * PPT + (j)) * ck_stride]

  // forward pass: the variance recursion up to the last checkpoint, (n_seg - 1) k
  // < N; k is even, so every pair of steps below it is whole
  float v[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) v[j] = c.v0;
  for (int sg = 0; sg < n_seg - 1; ++sg) {
#pragma unroll
    for (int j = 0; j < PPT; ++j) SIMR_CK(sg, j) = v[j];
    const uint32_t p0 = (uint32_t)sg * (k / 2);
    for (uint32_t p = p0; p < p0 + k / 2; ++p) {
      uint4 w[PPT];
#pragma unroll
      for (int j = 0; j < PPT; ++j) w[j] = philox4x32_10(p, plo[j], phi[j], option, rk);
#pragma unroll
      for (int j = 0; j < PPT; ++j) {  // the pair's two variance normals together
        const float xa = centered_uniform(w[j].x), xb = centered_uniform(w[j].z);
        const float2 zv = norminv_centered2(make_float2(xa, xb));
        v[j] = qe_only(c, v[j], 0.5f * (1.0f - xa), zv.x);
        v[j] = qe_only(c, v[j], 0.5f * (1.0f - xb), zv.y);
      }
    }
  }

  AdjSums as[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) as[j] = AdjSums{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};

  {
    float* s0 = seg;                   // states
    float* s1 = s0 + (int)k * stride;  // branch draws
    float* s2 = s1 + (int)k * stride;  // Z_X
#define SIMR_SG(q, i, j) s##q[(int)(i) * stride + (j) * bd]
    // the last checkpoint is the forward pass's final state; each earlier one is
    // loaded a segment ahead of its use
    float ck_next[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) ck_next[j] = v[j];
    for (int sgi = n_seg - 1; sgi >= 0; --sgi) {
      const uint32_t n0 = (uint32_t)sgi * k, n1 = min(n0 + k, N);
      float vv[PPT];
#pragma unroll
      for (int j = 0; j < PPT; ++j) vv[j] = ck_next[j];
      if (sgi > 0) {
#pragma unroll
        for (int j = 0; j < PPT; ++j) ck_next[j] = SIMR_CK(sgi - 1, j);
      }
      for (uint32_t p = n0 / 2; 2 * p < n1; ++p) {  // recompute v_n0 .. v_n1 and keep the draws
        const uint32_t i = 2 * p - n0;
        uint4 w[PPT];
#pragma unroll
        for (int j = 0; j < PPT; ++j) w[j] = philox4x32_10(p, plo[j], phi[j], option, rk);
#pragma unroll
        for (int j = 0; j < PPT; ++j) {  // the pair's normals two at a time
          const float xa = centered_uniform(w[j].x), xb = centered_uniform(w[j].z);
          const float2 zv = norminv_centered2(make_float2(xa, xb));
          const float2 zx = norminv_centered2(make_float2(centered_uniform(w[j].y), centered_uniform(w[j].w)));
          keep_step(c, xa, zv.x, zx.x, &SIMR_SG(0, i, j), &SIMR_SG(1, i, j), &SIMR_SG(2, i, j), vv[j]);
          if (2 * p + 1 < n1)
            keep_step(c, xb, zv.y, zx.y, &SIMR_SG(0, i + 1, j), &SIMR_SG(1, i + 1, j), &SIMR_SG(2, i + 1, j), vv[j]);
        }
      }
      float vnext[PPT];
#pragma unroll
      for (int j = 0; j < PPT; ++j) vnext[j] = vv[j];  // v_{n1}
      for (int i = (int)(n1 - n0) - 1; i >= 0; --i) {
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
          const float vc = SIMR_SG(0, i, j);
          adjoint_step(c, theta, vc, vnext[j], SIMR_SG(1, i, j), SIMR_SG(2, i, j), as[j]);
          vnext[j] = vc;
        }
      }
    }
#undef SIMR_SG
  }
#undef SIMR_CK
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    x_out[j] = as[j].x;
    comp_out[j] = as[j].comp;
    adjoint_map(A, as[j], g[j]);
  }
}

// Floats per thread of path_adjoint_ppt: checkpoints and the segment buffer.
__host__ __device__ inline size_t adjoint_ckpt_floats(const AdjConst& A, int ppt) { return (size_t)A.n_seg * ppt; }
__host__ __device__ inline size_t adjoint_seg_floats(const AdjConst& A, int ppt) {
  return (size_t)3 * A.ckpt_every * ppt;
}

// Terms per strike: 0 f, 1 f^2, 2 S0, 3 v0, 4 kappa, 5 theta, 6 sigma, 7 rho, 8 r (before -T P).
constexpr int kAdjAcc = 9;

__device__ __forceinline__ float adj_term(int a, bool put, float S, float K, const float (&g)[5], float invS0,
                                          float T) {
  const float f = put ? fmaxf(K - S, 0.0f) : fmaxf(S - K, 0.0f);
  if (a == 0) return f;
  if (a == 1) return f * f;
  const float w = put ? (S < K ? -S : 0.0f) : (S > K ? S : 0.0f);
  if (a == 2) return w * invS0;
  if (a == 8) return w * T;
  return w * g[a - 3];
}

}  // namespace
}  // namespace simr
