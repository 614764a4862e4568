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
__device__ __forceinline__ float qe_only(const ScenConst& c, float v, float omu, float zv) {
  float vn, dl;
  qe_from_moments(fmaf(v, c.E, c.thE), fmaf(v, c.c1, c.c2), omu, zv, vn, dl);
  return vn;
}

struct AdjSums {
  float vbar, Am, Amv, As, Asv, Ad, Adl, Ak3;
  float x, comp;  // x_T accumulated over the reverse sweep (Kahan-compensated)
};

// The reverse step's quantities of the quadratic branch that do not depend on
// the adjoint carried in from the later steps (functions of v_n, m, s^2, Z_V).
struct AdjQuad {
  float rs2, t, rroot, rb, ropb2, am, bz, g;
};

__device__ __forceinline__ AdjQuad adj_quad(float m, float m2, float s2, float zv) {
  AdjQuad Q;
  Q.rs2 = rcp_approx(s2);
  Q.t = 2.0f * m2 * Q.rs2;
  const float tt = fmaf(Q.t, Q.t, -Q.t);
  Q.rroot = rsqrt_approx(tt);
  const float root = tt * Q.rroot;
  const float b2 = (Q.t - 1.0f) + root;
  Q.rb = rsqrt_approx(b2);
  const float b = b2 * Q.rb;
  Q.ropb2 = rcp_approx(Q.t + root);  // 1 / (1 + b^2)
  Q.am = m * Q.ropb2;
  Q.bz = b + zv;
  Q.g = fmaf(zv, zv + 2.0f * b, -1.0f);
  return Q;
}

// The end of a reverse step once mbar and s2bar are known: x_T's increment
// (Kahan-compensated), the adjoint of v_n, and the seven sums.
__device__ __forceinline__ void adj_tail(const ScenConst& c, float theta, float vc, float q, float zx, float hz,
                                         float dl, float inc, float mbar, float s2bar, AdjSums& a) {
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

// The adjoint chain of a quadratic-branch reverse step: from the adjoint of
// v_{n+1} through the QE map's derivatives to mbar and s2bar, then adj_tail.
__device__ __forceinline__ void adj_chain_quad(const ScenConst& c, float theta, float vc, float m, float zv, float q,
                                               float zx, float hz, float dl, float inc, const AdjQuad& Q,
                                               AdjSums& a) {
  const float vnbar = a.vbar + c.Cv + hz;  // total adjoint of v_{n+1}
  const float dlbar = c.Cdl;
  const float abar = fmaf(vnbar, Q.bz * Q.bz, dlbar * Q.g);
  const float bbar = 2.0f * Q.am * fmaf(vnbar, Q.bz, dlbar * zv);
  const float b2bar = fmaf(0.5f * bbar, Q.rb, -abar * Q.am * Q.ropb2);
  float mbar = abar * Q.ropb2;
  const float tbar = b2bar * fmaf(2.0f * Q.t - 1.0f, 0.5f * Q.rroot, 1.0f);
  mbar = fmaf(tbar * 4.0f * m, Q.rs2, mbar);
  const float s2bar = -tbar * Q.t * Q.rs2;
  adj_tail(c, theta, vc, q, zx, hz, dl, inc, mbar, s2bar, a);
}

// The step's log-spot increment (LogPricePathQE), summed into x_T in the
// reverse sweep rather than in the forward pass.
__device__ __forceinline__ float adj_inc(const ScenConst& c, float s, float vc, float dl, float q, float zx) {
  float inc = fmaf(c.Cv, s, c.C0);
  inc = fmaf(-c.Cd, vc, inc);
  inc = fmaf(c.Cdl, dl, inc);
  return fmaf(c.sK3 * q, zx, inc);
}

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
  if (s2 < 1.5f * m2) {  // the forward step's branch test
    const AdjQuad Q = adj_quad(m, m2, s2, d);
    const float dl = Q.am * Q.g;
    adj_chain_quad(c, theta, vc, m, d, q, zx, hz, dl, adj_inc(c, s, vc, dl, q, zx), Q, a);
    return;
  }
  const float vnbar = a.vbar + c.Cv + hz;  // total adjoint of v_{n+1}
  const float dlbar = c.Cdl;
  float mbar = 0.0f, s2bar = 0.0f, dl = 0.0f;
  if (m > 0.0f) {
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
  adj_tail(c, theta, vc, q, zx, hz, dl, adj_inc(c, s, vc, dl, q, zx), mbar, s2bar, a);
}

// Two consecutive reverse steps, n (lane x) then n - 1 (lane y): when both
// take the quadratic branch, their quantities that do not depend on the
// carried adjoint -- moments, square roots, the branch's terms, the log-spot
// increment -- in packed FP32, then the two adjoint chains in order; else two
// adjoint_step calls.  Lane for lane adjoint_step's operations, so the same
// sums bit for bit however the steps are paired.
__device__ __forceinline__ void adjoint_step2(const ScenConst& c, float theta, float2 vc, float2 vn, float2 d,
                                              float2 zx, AdjSums& a) {
  const float2 m = p_fma(vc, p_bc(c.E), p_bc(c.thE));
  const float2 s2 = p_fma(vc, p_bc(c.c1), p_bc(c.c2));
  const float2 m2 = p_mul(m, m);
  const float2 lim = p_mul(p_bc(1.5f), m2);
  if (!(s2.x < lim.x && s2.y < lim.y)) {
    adjoint_step(c, theta, vc.x, vn.x, d.x, zx.x, a);
    adjoint_step(c, theta, vc.y, vn.y, d.y, zx.y, a);
    return;
  }
  const float2 s = p_add(vc, vn);
  const float2 rq = make_float2(rsqrt_approx(s.x), rsqrt_approx(s.y));
  const float2 sq = p_mul(s, rq);
  const float2 hq = p_mul(p_mul(p_bc(0.5f * c.sK3), zx), rq);
  const float2 q = make_float2(s.x > 0.0f ? sq.x : 0.0f, s.y > 0.0f ? sq.y : 0.0f);
  const float2 hz = make_float2(s.x > 0.0f ? hq.x : 0.0f, s.y > 0.0f ? hq.y : 0.0f);
  // adj_quad, paired
  const float2 rs2 = p_rcp(s2);
  const float2 t = p_mul(p_mul(p_bc(2.0f), m2), rs2);
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
  // adj_inc, paired
  float2 inc = p_fma(p_bc(c.Cv), s, p_bc(c.C0));
  inc = p_fma(p_bc(-c.Cd), vc, inc);
  inc = p_fma(p_bc(c.Cdl), dl, inc);
  inc = p_fma(p_mul(p_bc(c.sK3), q), zx, inc);
  const AdjQuad Qx{rs2.x, t.x, rroot.x, rb.x, ropb2.x, am.x, bz.x, g.x};
  const AdjQuad Qy{rs2.y, t.y, rroot.y, rb.y, ropb2.y, am.y, bz.y, g.y};
  adj_chain_quad(c, theta, vc.x, m.x, d.x, q.x, zx.x, hz.x, dl.x, inc.x, Qx, a);
  adj_chain_quad(c, theta, vc.y, m.y, d.y, q.y, zx.y, hz.y, dl.y, inc.y, Qy, a);
}

// The draw the reverse step of state v needs: Z_V in the quadratic branch,
// 1 - U_V otherwise (same branch test as the forward step).
__device__ __forceinline__ float branch_draw(const ScenConst& c, float v, float omu, float zv) {
  const float m = fmaf(v, c.E, c.thE);
  const float s2 = fmaf(v, c.c1, c.c2);
  return s2 < 1.5f * (m * m) ? zv : omu;
}

// The stored data of one step (recompute pass): (state, branch draw) as one
// pair and Z_X, from the step's centred variance uniform and its two normals.
__device__ __forceinline__ void keep_step(const ScenConst& c, float xv_v, float zv, float zx, float2* bvd, float* bz,
                                          float& v) {
  const float omu = 0.5f * (1.0f - xv_v);
  *bvd = make_float2(v, branch_draw(c, v, omu, zv));
  *bz = zx;
  v = qe_only(c, v, omu, zv);
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
__device__ __forceinline__ void adjoint_map(const AdjConst& A, const AdjSums& a, float (&g)[5]) {
  const double Amv = a.Amv, Asv = a.Asv, As = a.As, Ad = a.Ad, Adl = a.Adl, Am = a.Am, Ak3 = a.Ak3;
  g[0] = a.vbar;
  g[1] = (float)(A.dE_dk * Amv + A.dc1_dk * Asv + A.dc2_dk * As + A.dCd_dk * Ad + A.dCdl_dk * Adl);
  g[2] = (float)(A.omE * Am + A.dc2_dth * As + A.N_Cd);
  g[3] = (float)(A.two_over_sigma * (A.c1 * Asv + A.c2 * As) - A.Cd_over_sigma * Ad - A.Cdl_over_sigma * Adl);
  g[4] = (float)(A.D_over_sigma * Ad + A.B_over_sigma * Adl + A.dsK3_drho * Ak3);
}

// Reverse sweep of one path, segment by segment, last first: each segment's
// states are recomputed from its checkpoint (the last checkpoint is v_last, the
// forward pass's final state; earlier ones ck[slot * cstride], each loaded a
// segment ahead of its use) and kept with the step's branch draw and Z_X in this
// thread's segment column S (at least k rows) -- then the steps are
// differentiated backwards.  x_T (with its Kahan remainder) is summed on the
// way; g = d x_T / d(v0, kappa, theta, sigma, rho).
template <typename Seg, bool PAIRED>
__device__ __forceinline__ void path_sweep(const ScenConst& c, const AdjConst& A, uint32_t N, uint32_t option,
                                           const uint32_t (&rk)[10][2], uint32_t plo, uint32_t phi,
                                           const float* ck, int cstride, float v_last, const Seg& S,
                                           float& x_out, float& comp_out, float (&g)[5]) {
  using I = decltype(S.stride());
  const float theta = A.theta;
  const uint32_t k = (uint32_t)A.ckpt_every;
  const int n_seg = A.n_seg;
  AdjSums as = AdjSums{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  float2* s01 = S.pairs();
  float* s2 = S.zx();
  const I bd = S.stride();
  float ck_next = v_last;
  for (int sgi = n_seg - 1; sgi >= 0; --sgi) {
    const uint32_t n0 = (uint32_t)sgi * k, n1 = min(n0 + k, N);
    float vv = ck_next;
    if (sgi > 0) ck_next = ck[(sgi - 1) * cstride];
    for (uint32_t p = n0 / 2; 2 * p < n1; ++p) {  // recompute v_n0 .. v_n1 and keep the draws
      const I i = (I)(2 * p - n0) * bd;
      const uint4 w = philox4x32_10(p, plo, phi, option, rk);
      const float xa = centered_uniform(w.x), xb = centered_uniform(w.z);
      const float2 zv = norminv_centered2(make_float2(xa, xb));  // the pair's normals two at a time
      const float2 zx = norminv_centered2(make_float2(centered_uniform(w.y), centered_uniform(w.w)));
      keep_step(c, xa, zv.x, zx.x, s01 + i, s2 + i, vv);
      if (2 * p + 1 < n1) keep_step(c, xb, zv.y, zx.y, s01 + i + bd, s2 + i + bd, vv);
    }
    float vnext = vv;  // v_{n1}
    if constexpr (PAIRED) {
      if constexpr (Seg::kGlobal) {
        // global memory: the steps in pairs (n, n - 1) from the top, each pair's
        // data loaded one pair ahead into registers and asked into L2
        // kPrefetchSteps steps ahead
        constexpr int kPrefetchSteps = SIMR_ADJ_PREFETCH;
        int i = (int)(n1 - n0) - 1;
        float2 pa = s01[(I)i * bd], pb = make_float2(0.0f, 0.0f);
        float za = s2[(I)i * bd], zb = 0.0f;
        if (i >= 1) {
          pb = s01[(I)(i - 1) * bd];
          zb = s2[(I)(i - 1) * bd];
        }
        for (; i >= 1; i -= 2) {
          const float2 ca = pa, cb = pb;
          const float cza = za, czb = zb;
          if (i - 2 - kPrefetchSteps >= 0) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s01 + (I)(i - 2 - kPrefetchSteps) * bd));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s2 + (I)(i - 2 - kPrefetchSteps) * bd));
          }
          if (i - 3 - kPrefetchSteps >= 0) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s01 + (I)(i - 3 - kPrefetchSteps) * bd));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s2 + (I)(i - 3 - kPrefetchSteps) * bd));
          }
          if (i >= 2) {
            pa = s01[(I)(i - 2) * bd];
            za = s2[(I)(i - 2) * bd];
          }
          if (i >= 3) {
            pb = s01[(I)(i - 3) * bd];
            zb = s2[(I)(i - 3) * bd];
          }
          adjoint_step2(c, theta, make_float2(ca.x, cb.x), make_float2(vnext, ca.x), make_float2(ca.y, cb.y),
                        make_float2(cza, czb), as);
          vnext = cb.x;
        }
        if (i == 0) {  // an odd count: the last step alone (loaded as pa)
          adjoint_step(c, theta, pa.x, vnext, pa.y, za, as);
          vnext = pa.x;
        }
      } else {
        int i = (int)(n1 - n0) - 1;
        for (; i >= 1; i -= 2) {
          const float2 ca = s01[(I)i * bd], cb = s01[(I)(i - 1) * bd];
          adjoint_step2(c, theta, make_float2(ca.x, cb.x), make_float2(vnext, ca.x), make_float2(ca.y, cb.y),
                        make_float2(s2[(I)i * bd], s2[(I)(i - 1) * bd]), as);
          vnext = cb.x;
        }
        if (i == 0) {
          const float2 vd = s01[0];
          adjoint_step(c, theta, vd.x, vnext, vd.y, s2[0], as);
          vnext = vd.x;
        }
      }
    } else {
      if constexpr (Seg::kGlobal) {
        // global memory: each step's data loaded one step ahead into registers,
        // and asked into L2 kPrefetchSteps steps ahead
        constexpr int kPrefetchSteps = SIMR_ADJ_PREFETCH;
        int i = (int)(n1 - n0) - 1;
        float2 vd_n = s01[(I)i * bd];
        float zx_n = s2[(I)i * bd];
        for (; i >= 0; --i) {
          const float2 vd = vd_n;
          const float zx = zx_n;
          if (i >= kPrefetchSteps) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s01 + (I)(i - kPrefetchSteps) * bd));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(s2 + (I)(i - kPrefetchSteps) * bd));
          }
          if (i > 0) {
            vd_n = s01[(I)(i - 1) * bd];
            zx_n = s2[(I)(i - 1) * bd];
          }
          adjoint_step(c, theta, vd.x, vnext, vd.y, zx, as);
          vnext = vd.x;
        }
      } else {
        for (int i = (int)(n1 - n0) - 1; i >= 0; --i) {
          const float2 vd = s01[(I)i * bd];
          adjoint_step(c, theta, vd.x, vnext, vd.y, s2[(I)i * bd], as);
          vnext = vd.x;
        }
      }
    }
  }
  x_out = as.x;
  comp_out = as.comp;
  adjoint_map(A, as, g);
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
template <int PPT, typename Seg, bool PAIRED = true>
__device__ __forceinline__ void path_adjoint_ppt(const ScenConst& c, const AdjConst& A, uint32_t N, uint32_t option,
                                                 const uint32_t (&rk)[10][2], const uint64_t (&path)[PPT], float* ck,
                                                 int ck_stride, const Seg& S, float (&x_out)[PPT],
                                                 float (&comp_out)[PPT], float (&g)[PPT][5]) {
  static_assert(PPT == 1 || PPT == 2, "one or two paths per thread");
  const uint32_t k = (uint32_t)A.ckpt_every;
  const int n_seg = A.n_seg;
  uint32_t plo[PPT], phi[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    plo[j] = (uint32_t)path[j];
    phi[j] = (uint32_t)(path[j] >> 32);
  }
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
      for (int j = 0; j < PPT; ++j) w[j] = philox4x32_10(p, plo[j], phi[j], option, rk);
      if constexpr (PPT == 2) {
        const float xa0 = centered_uniform(w[0].x), xa1 = centered_uniform(w[1].x);
        const float xb0 = centered_uniform(w[0].z), xb1 = centered_uniform(w[1].z);
        const float2 za = norminv_centered2(make_float2(xa0, xa1));
        const float2 zb = norminv_centered2(make_float2(xb0, xb1));
        float2 vv = make_float2(v[0], v[1]), vn, dl;
        qe_from_moments2(p_fma(vv, p_bc(c.E), p_bc(c.thE)), p_fma(vv, p_bc(c.c1), p_bc(c.c2)),
                         make_float2(0.5f * (1.0f - xa0), 0.5f * (1.0f - xa1)), za, vn, dl);
        vv = vn;
        qe_from_moments2(p_fma(vv, p_bc(c.E), p_bc(c.thE)), p_fma(vv, p_bc(c.c1), p_bc(c.c2)),
                         make_float2(0.5f * (1.0f - xb0), 0.5f * (1.0f - xb1)), zb, vn, dl);
        v[0] = vn.x;
        v[1] = vn.y;
      } else {  // the pair's two variance normals together
        const float xa = centered_uniform(w[0].x), xb = centered_uniform(w[0].z);
        const float2 zv = norminv_centered2(make_float2(xa, xb));
        v[0] = qe_only(c, v[0], 0.5f * (1.0f - xa), zv.x);
        v[0] = qe_only(c, v[0], 0.5f * (1.0f - xb), zv.y);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < PPT; ++j)
    path_sweep<Seg, PAIRED>(c, A, N, option, rk, plo[j], phi[j], ck + j * ck_stride, PPT * ck_stride, v[j], S,
                            x_out[j], comp_out[j], g[j]);
}

// Floats per thread of path_adjoint_ppt: checkpoints and the segment buffer.
__host__ __device__ inline size_t adjoint_ckpt_floats(const AdjConst& A, int ppt) { return (size_t)A.n_seg * ppt; }
__host__ __device__ inline size_t adjoint_seg_floats(const AdjConst& A, int /*ppt: the sweeps share one buffer*/) {
  return (size_t)3 * A.ckpt_every;
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
