// simr_lsm.cu -- Longstaff-Schwartz (least-squares Monte Carlo) price of a Bermudan
// option on the Heston QE paths, sm_103a.
//
// The paper's dataflow ends in writeLongstaffSchwartzPath and
// longstaffSchwartzPathReduction (Sec. 5, Fig. 1): the per-path states are
// written out and reduced across paths with dependencies between the paths
// (Sec. 6).  The method is Longstaff and Schwartz (2001): backwards over the
// exercise dates, regress the discounted cash flows that the in-the-money
// paths realise under the decisions already taken on basis functions of the
// state, and exercise where the payoff exceeds the fitted continuation value.
//
// (1) A persistent path kernel (VariancePathQE / LogPricePathQE /
//     AssetPathExponential, two paths per thread, Philox in the kernel) writes
//     S and v at every exercise date into [date][path] arrays, and the
//     maturity payoff as each path's initial cash flow.
// (2) One kernel per date j, last date first: apply date j's exercise rule
//     (coefficients solved by the previous launch) and accumulate the
//     regression sums of date j - 1 over its in-the-money paths -- the 15
//     monomials xs^a ys^b, a + b <= 4, that make up the Gram matrix of the basis
//     (1, xs, xs^2, ys, xs ys, ys^2), and the 6 products of the basis with the
//     discounted cash flow -- FP32 per thread and across the warp, FP64 from the
//     warp on; the last block sums the block rows in block order and solves the
//     normal equations (lsm_solve_warp: FP32 Cholesky, refined against an FP64
//     residual).  The launch of date 0 applies its rule and reduces the
//     discounted cash flows to the price.
// (2') In place of (2), when the GPU can keep one 1024-thread block per SM
//     resident for up to 7 paths per thread: the whole backward induction as
//     one cooperative launch (lsm_sweep_kernel) -- per date a block row, one
//     grid barrier, and in every block the same cross-block sum and solve; each
//     date's states come into shared memory by TMA bulk copies issued a date
//     ahead.
//
// The coordinates xs = (S - F_j)/sd_j and ys = (v - E v_j)/sd(v_j) are x and y
// of the basis (1, x, x^2, y, xy, y^2), x = S/K - 1, y = v/w - 1, shifted and
// scaled by the model's forward and spreads at date j: the same space of
// quadratics, so the same least-squares fit, but a Gram matrix of order-one
// entries.  In x and y directly the early dates' Gram matrices have condition
// numbers near 1e6 (the spot has barely spread), which FP32 sums cannot
// resolve.  The coefficients are reported in x and y (converted in FP64).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "simr_device.cuh"
#include "simr_internal.h"
#include "simr_reduce.cuh"

namespace simr {
namespace {

constexpr int kLsmTpb = 256;
constexpr int kLsmWarps = kLsmTpb / kWarp;
constexpr int kNMono = 15;  // x^a y^b, a + b <= 4
constexpr int kNB = 6;      // basis functions
constexpr int kNReg = kNMono + kNB;
constexpr int kLsmPpt = 2;

// Double-float sums: hi + lo carries about 48 significant bits, with FP32
// arithmetic only (GB300's FP64 rate makes each FP64 warp instruction cost tens
// of cycles, and the cross-block sums sit on every date's critical path).
// Knuth's TwoSum of the high parts, then the low parts, renormalised.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  const float lo = __fadd_rn(__fadd_rn(err, a.lo), b.lo);
  const float hi = __fadd_rn(s, lo);
  return DF{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

__device__ __forceinline__ float lsm_payoff(bool put, float S, float K) {
  return put ? fmaxf(K - S, 0.0f) : fmaxf(S - K, 0.0f);
}

// One step of the thread's two paths from their (variance, log-spot) words,
// paired in packed FP32 (simulate_two's arithmetic, or step_qem2 for QE-M).
template <bool QEM>
__device__ __forceinline__ void step_two(const LsmLaunch& L, uint32_t wv0, uint32_t wx0, uint32_t wv1, uint32_t wx1,
                                         float (&v)[kLsmPpt], float (&x)[kLsmPpt], float (&comp)[kLsmPpt]) {
  static_assert(kLsmPpt == 2, "two paths per thread");
  const float2 xv = centered_uniform2(wv0, wv1);
  const float2 zv = norminv_centered2(xv);
  const float2 zx = norminv_centered2(centered_uniform2(wx0, wx1));
  float2 vv = make_float2(v[0], v[1]), xx = make_float2(x[0], x[1]), cc = make_float2(comp[0], comp[1]);
  if constexpr (QEM)
    step_qem2(L.sc, L.qm, xv, zv, zx, vv, xx, cc);
  else
    step_base2<false>(L.sc, xv, zv, zx, vv, xx, cc);
  v[0] = vv.x;
  v[1] = vv.y;
  x[0] = xx.x;
  x[1] = xx.y;
  comp[0] = cc.x;
  comp[1] = cc.y;
}

// Path kernel: states at the exercise dates, maturity cash flow.
template <bool QEM>
__global__ void __launch_bounds__(kLsmTpb) lsm_paths_kernel(const __grid_constant__ LsmLaunch L,
                                                            float* __restrict__ S_out, float* __restrict__ V_out,
                                                            float* __restrict__ cash, int32_t* __restrict__ stop) {
  const int lane = threadIdx.x & 31;
  const uint64_t per = (uint64_t)kWarp * kLsmPpt;
  const uint64_t batches = (L.paths + per - 1) / per;
  const uint64_t n_warps = (uint64_t)gridDim.x * kLsmWarps;
  const bool put = L.is_put != 0;
  for (uint64_t bt = (uint64_t)blockIdx.x * kLsmWarps + (threadIdx.x >> 5); bt < batches; bt += n_warps) {
    uint64_t idx[kLsmPpt];
    PhiloxLane pl[kLsmPpt];
    float v[kLsmPpt], x[kLsmPpt], comp[kLsmPpt];
#pragma unroll
    for (int j = 0; j < kLsmPpt; ++j) {
      idx[j] = bt * per + (uint64_t)j * kWarp + lane;
      pl[j] = philox_lane(idx[j], L.rk);
      v[j] = L.sc.v0;
      x[j] = 0.0f;
      comp[j] = 0.0f;
    }
    int cnt = 0;
    size_t row = 0;  // offset of the next date's row
    auto record = [&]() {
#pragma unroll
      for (int j = 0; j < kLsmPpt; ++j) {
        if (idx[j] < L.paths) {
          S_out[row + idx[j]] = terminal_spot(L.S0, x[j], comp[j]);
          V_out[row + idx[j]] = v[j];
        }
      }
      row += L.pitch;
    };
    for (uint32_t p = 0; 2 * p < L.steps; ++p) {
      uint4 w[kLsmPpt];
      const PhiloxCtr u = philox_ctr(p, L.option_index, L.rk);
#pragma unroll
      for (int j = 0; j < kLsmPpt; ++j) w[j] = philox_draw(pl[j], u, L.rk);
      step_two<QEM>(L, w[0].x, w[0].y, w[1].x, w[1].y, v, x, comp);
      if (++cnt == L.every) {
        cnt = 0;
        record();
      }
      if (2 * p + 1 < L.steps) {
        step_two<QEM>(L, w[0].z, w[0].w, w[1].z, w[1].w, v, x, comp);
        if (++cnt == L.every) {
          cnt = 0;
          record();
        }
      }
    }
    // the last date is the maturity: its payoff starts each path's cash flow
#pragma unroll
    for (int j = 0; j < kLsmPpt; ++j) {
      if (idx[j] < L.paths) {
        const float h = lsm_payoff(put, terminal_spot(L.S0, x[j], comp[j]), L.K);
        cash[idx[j]] = h;
        stop[idx[j]] = h > 0.0f ? L.n_ex - 1 : -1;
      }
    }
  }
}

// Coefficients in x, y from those in xs = kx (x - cx), ys = ky (y - cy).
__device__ void lsm_unscale(const double* bt, double kx, double cx, double ky, double cy, double* beta) {
  const double kx2 = kx * kx, ky2 = ky * ky, kxy = kx * ky;
  beta[0] = bt[0] - bt[1] * kx * cx + bt[2] * kx2 * cx * cx - bt[3] * ky * cy + bt[4] * kxy * cx * cy +
            bt[5] * ky2 * cy * cy;
  beta[1] = bt[1] * kx - 2.0 * bt[2] * kx2 * cx - bt[4] * kxy * cy;
  beta[2] = bt[2] * kx2;
  beta[3] = bt[3] * ky - bt[4] * kxy * cx - 2.0 * bt[5] * ky2 * cy;
  beta[4] = bt[4] * kxy;
  beta[5] = bt[5] * ky2;
}

// Gram matrix entry (i, k) of the basis (1, x, x^2, y, xy, y^2) as an index into
// the 15 monomial sums 1, x, y, x^2, xy, y^2, x^3, x^2y, xy^2, y^3, x^4, x^3y,
// x^2y^2, xy^3, y^4: the monomial of exponent e_i + e_k.
__constant__ int c_gram_index[kNB * kNB] = {0, 1, 3, 2,  4,  5,  1, 3,  6,  4,  7,  8,  3,  6,  10, 7,  11, 12,
                                            2, 4, 7, 5,  8,  9,  4, 7,  11, 8,  12, 13, 5,  8,  12, 9,  13, 14};

// 6x6 normal equations G beta = b from the 15 monomial sums and the 6 products
// b (tot[15..20]), solved by one warp (lane r < 6 holds row r of G and of the
// Cholesky factor L; every lane ends with all of beta).  In the standardised
// coordinates G has order-one entries, so the factorisation runs in FP32:
// Cholesky in basis order, basis function k left out (coefficient 0) when its
// pivot is not above 1e-5 G[k][k] -- the threshold at which FP32's own rounding
// of the order-one Gram entries (~1e-7 each) can no longer tell a pivot from
// zero; pivots of non-degenerate fits are near 0.05 or above; then one step of
// iterative refinement with
// the residual b - G x formed in FP64 (row r in lane r), which brings the
// solution to about FP64 accuracy for condition numbers far below 1e7.
__device__ void lsm_solve_warp(const double* tot, double* beta, int lane) {
  const int row = lane < kNB ? lane : 0;
  double g[kNB];
  float gf[kNB], l[kNB], rd[kNB];
  unsigned keep = 0;
#pragma unroll
  for (int k = 0; k < kNB; ++k) {
    g[k] = tot[c_gram_index[row * kNB + k]];
    gf[k] = (float)g[k];
    l[k] = 0.0f;
  }
#pragma unroll
  for (int k = 0; k < kNB; ++k) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < k; ++i) s = fmaf(l[i], l[i], s);  // left-out columns hold 0
    const float d = __shfl_sync(kFull, gf[k] - s, k);
    const float gkk = __shfl_sync(kFull, gf[k], k);
    rd[k] = 0.0f;
    if (!(gkk > 0.0f && d > 1e-5f * gkk)) continue;
    keep |= 1u << k;
    const float lkk = __fsqrt_rn(d);
    rd[k] = __frcp_rn(lkk);
    float t = 0.0f;
#pragma unroll
    for (int i = 0; i < k; ++i) t = fmaf(l[i], __shfl_sync(kFull, l[i], k), t);
    if (lane > k) l[k] = (gf[k] - t) * rd[k];
    if (lane == k) l[k] = lkk;
  }
  // L L^T x = r for r held by every lane; L[k][i] is lane k's l[i]
  auto solve = [&](const float (&r)[kNB], float (&x)[kNB]) {
    float z[kNB];
#pragma unroll
    for (int k = 0; k < kNB; ++k) {
      float t = 0.0f;
#pragma unroll
      for (int i = 0; i < k; ++i) t = fmaf(l[i], z[i], t);
      const float zk = ((keep >> k) & 1u) ? (r[k] - t) * rd[k] : 0.0f;
      z[k] = __shfl_sync(kFull, zk, k);
    }
#pragma unroll
    for (int k = kNB - 1; k >= 0; --k) {
      float t = 0.0f;
#pragma unroll
      for (int i = k + 1; i < kNB; ++i) t = fmaf(__shfl_sync(kFull, l[k], i), x[i], t);
      x[k] = ((keep >> k) & 1u) ? (z[k] - t) * rd[k] : 0.0f;
    }
  };
  float rf[kNB], xf[kNB], dx[kNB];
#pragma unroll
  for (int k = 0; k < kNB; ++k) rf[k] = (float)tot[kNMono + k];
  solve(rf, xf);
  double res = tot[kNMono + row];
#pragma unroll
  for (int k = 0; k < kNB; ++k) res = fma(-g[k], (double)xf[k], res);
#pragma unroll
  for (int k = 0; k < kNB; ++k) rf[k] = (float)__shfl_sync(kFull, res, k);
  solve(rf, dx);
#pragma unroll
  for (int k = 0; k < kNB; ++k) beta[k] = ((keep >> k) & 1u) ? (double)xf[k] + (double)dx[k] : 0.0;
}

// Fitted continuation value in the standardised coordinates (x, y).
__device__ __forceinline__ float lsm_continuation(const float (&b)[kNB], float x, float y) {
  float C = fmaf(b[2], x, b[1]);
  C = fmaf(C, x, b[0]);
  return fmaf(fmaf(b[5], y, fmaf(b[4], x, b[3])), y, C);
}

// One in-the-money path's terms of the regression sums: the 15 monomials
// 1, x, y, x^2, xy, y^2, x^3, x^2y, xy^2, y^3, x^4, x^3y, x^2y^2, xy^3, y^4 and
// the target Y times the basis (1, x, x^2, y, xy, y^2).
__device__ __forceinline__ void lsm_accumulate(float (&acc)[kNReg], float x, float y, float Y) {
  const float x2 = x * x, y2 = y * y, xy = x * y;
  acc[0] += 1.0f;
  acc[1] += x;
  acc[2] += y;
  acc[3] += x2;
  acc[4] += xy;
  acc[5] += y2;
  acc[6] = fmaf(x2, x, acc[6]);
  acc[7] = fmaf(x2, y, acc[7]);
  acc[8] = fmaf(x, y2, acc[8]);
  acc[9] = fmaf(y2, y, acc[9]);
  acc[10] = fmaf(x2, x2, acc[10]);
  acc[11] = fmaf(x2, xy, acc[11]);
  acc[12] = fmaf(x2, y2, acc[12]);
  acc[13] = fmaf(xy, y2, acc[13]);
  acc[14] = fmaf(y2, y2, acc[14]);
  acc[15] += Y;
  acc[16] = fmaf(Y, x, acc[16]);
  acc[17] = fmaf(Y, x2, acc[17]);
  acc[18] = fmaf(Y, y, acc[18]);
  acc[19] = fmaf(Y, xy, acc[19]);
  acc[20] = fmaf(Y, y2, acc[20]);
}

// Date kernel: exercise rule of date j (UPDATE), then the regression sums of
// date j - 1 (REGRESS) or, after date 0, the price (neither flag set: no update).
template <bool UPDATE, bool REGRESS>
__global__ void __launch_bounds__(kLsmTpb) lsm_date_kernel(const __grid_constant__ LsmLaunch L, const LsmBuffers B,
                                                           int j) {
  __shared__ float s_rows[kLsmWarps][kNReg];
  __shared__ DF s_part[kLsmTpb];
  __shared__ double s_tot[kNReg];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // date j's coefficients (scaled basis), read by every thread (one address per warp)
  float bj[kNB];
  bool has = false;
  if (UPDATE) {
    const double* bt = B.beta_t + (size_t)j * kNB;
    has = !isnan(__ldcg(bt));
#pragma unroll
    for (int k = 0; k < kNB; ++k) bj[k] = has ? (float)__ldcg(bt + k) : 0.0f;
  }
  const float* __restrict__ dpow = B.dpow;

  constexpr int NV = REGRESS ? kNReg : 2;
  float acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0f;
  const bool put = L.is_put != 0;
  const bool upd = UPDATE && has;
  const uint64_t P = L.paths;
  const float K = L.K;
  const int jr = j - 1;
  const float4 tj = B.xform[j];                   // update date
  const float4 tr = B.xform[REGRESS ? jr : j];    // regression date
  const float* Sj = B.S + (size_t)j * L.pitch;
  const float* Vj = B.V + (size_t)j * L.pitch;
  const float* Sr = B.S + (size_t)(REGRESS ? jr : 0) * L.pitch;
  const float* Vr = B.V + (size_t)(REGRESS ? jr : 0) * L.pitch;
  // two paths per iteration, all their loads issued before either is used
  const uint64_t gt = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < P; i0 += 2 * gt) {
    const uint64_t ii[2] = {i0, i0 + gt < P ? i0 + gt : i0};
    const bool act[2] = {true, i0 + gt < P};
    float c[2], Su[2], Vu[2], Sg[2], Vg[2];
    int sp[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      c[k] = B.cash[ii[k]];
      sp[k] = B.stop[ii[k]];
      Su[k] = upd ? Sj[ii[k]] : 0.0f;
      Vu[k] = upd ? Vj[ii[k]] : 0.0f;
      Sg[k] = REGRESS ? Sr[ii[k]] : 0.0f;
      Vg[k] = REGRESS ? Vr[ii[k]] : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (!act[k]) continue;
      const uint64_t i = ii[k];
      float cc = c[k];
      int s = sp[k];
      if (upd) {
        const float h = lsm_payoff(put, Su[k], K);
        if (h > 0.0f) {
          const float C = lsm_continuation(bj, fmaf(Su[k], tj.x, tj.y), fmaf(Vu[k], tj.z, tj.w));
          if (h > C) {
            cc = h;
            s = j;
            B.cash[i] = cc;
            B.stop[i] = s;
          }
        }
      }
      if (REGRESS) {
        const float h = lsm_payoff(put, Sg[k], K);
        if (h > 0.0f) {
          const float x = fmaf(Sg[k], tr.x, tr.y), y = fmaf(Vg[k], tr.z, tr.w);
          const float Y = s >= 0 ? cc * __ldg(dpow + (s - jr)) : 0.0f;
          if constexpr (REGRESS) lsm_accumulate(acc, x, y, Y);
        }
      } else {
        const float d = s >= 0 ? cc * __ldg(dpow + s) : 0.0f;  // discounted to t_0
        acc[0] += d;
        acc[1] = fmaf(d, d, acc[1]);
      }
    }
  }

  // FP32 over the warp, double-float over warps and blocks (block rows of (hi, lo)
  // pairs in block order), FP64 for the 21 totals
  if (REGRESS) {
    float vals[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) vals[k] = k < NV ? acc[k] : 0.0f;
    butterfly32(vals, lane);
    if (lane < NV) s_rows[warp][lane] = vals[0];
  } else {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const float t = warp_sum(acc[k]);
      if (lane == 0) s_rows[warp][k] = t;
    }
  }
  __syncthreads();
  float2* rows = reinterpret_cast<float2*>(B.partials);  // [grid][kNReg]
  if (threadIdx.x < NV) {
    DF t{0.0f, 0.0f};
    for (int w = 0; w < kLsmWarps; ++w) t = df_add(t, DF{s_rows[w][threadIdx.x], 0.0f});
    rows[(size_t)blockIdx.x * kNReg + threadIdx.x] = make_float2(t.hi, t.lo);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(B.ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // thread (part, q) sums quantity q of the rows of blocks part, part + n_parts,
  // ... (independent loads, unrolled); then the parts' sums in part order
  constexpr int n_parts = kLsmTpb / NV;
  if (threadIdx.x < n_parts * NV) {
    const int q = threadIdx.x % NV, part = threadIdx.x / NV;
    DF t{0.0f, 0.0f};
#pragma unroll 8
    for (unsigned b = part; b < gridDim.x; b += n_parts) {
      const float2 r = __ldcg(rows + (size_t)b * kNReg + q);
      t = df_add(t, DF{r.x, r.y});
    }
    s_part[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    DF t{0.0f, 0.0f};
    for (int part = 0; part < n_parts; ++part) t = df_add(t, s_part[part * NV + threadIdx.x]);
    s_tot[threadIdx.x] = (double)t.hi + (double)t.lo;
  }
  __syncthreads();
  if (REGRESS && warp == 0) {
    double* beta = B.beta + (size_t)jr * kNB;
    double* bt = B.beta_t + (size_t)jr * kNB;
    if (s_tot[0] < (double)L.min_itm) {
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      if (lane < kNB) beta[lane] = bt[lane] = nan;
    } else {
      double bs[kNB];
      lsm_solve_warp(s_tot, bs, lane);
      if (lane == 0) {
        // xs = a S + b with S = K (1 + x): xs = aK (x - cx), cx = -(aK + b)/(aK); likewise ys
        const double kx = (double)tr.x * L.Kd, cx = -(kx + (double)tr.y) / kx;
        const double ky = (double)tr.z * L.wd, cy = -(ky + (double)tr.w) / ky;
        double bo[kNB];
        lsm_unscale(bs, kx, cx, ky, cy, bo);
#pragma unroll
        for (int k = 0; k < kNB; ++k) {
          bt[k] = bs[k];
          beta[k] = bo[k];
        }
      }
    }
  }
  if (threadIdx.x == 0) {
    if (!REGRESS) {
      const double n = (double)P;
      const double mean = s_tot[0] / n;
      B.price[0] = L.disc0 * mean;
      if (B.stderr_) {
        const double var = n > 1.0 ? (s_tot[1] / n - mean * mean) / (n - 1.0) : 0.0;
        B.stderr_[0] = L.disc0 * sqrt(var > 0.0 ? var : 0.0);
      }
    }
    *B.ticket = 0u;
  }
}

// The same normal equations from double-float totals, with FP32 arithmetic only
// (the sweep's critical path): the FP32 Cholesky of lsm_solve_warp on the high
// parts, then one refinement step whose residual b - G x is formed in
// double-float (each product G x split exactly by an FMA).  The solution is the
// pair (x, dx); x + dx in FP32 is what the exercise rule uses.
__device__ void lsm_solve_df(const DF* tot, float* x_out, float* dx_out, int lane) {
  const int row = lane < kNB ? lane : 0;
  DF g[kNB];
  float l[kNB], rd[kNB];
  unsigned keep = 0;
#pragma unroll
  for (int k = 0; k < kNB; ++k) {
    g[k] = tot[c_gram_index[row * kNB + k]];
    l[k] = 0.0f;
  }
#pragma unroll
  for (int k = 0; k < kNB; ++k) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < k; ++i) s = fmaf(l[i], l[i], s);
    const float d = __shfl_sync(kFull, g[k].hi - s, k);
    const float gkk = __shfl_sync(kFull, g[k].hi, k);
    rd[k] = 0.0f;
    if (!(gkk > 0.0f && d > 1e-5f * gkk)) continue;
    keep |= 1u << k;
    const float lkk = __fsqrt_rn(d);
    rd[k] = __frcp_rn(lkk);
    float t = 0.0f;
#pragma unroll
    for (int i = 0; i < k; ++i) t = fmaf(l[i], __shfl_sync(kFull, l[i], k), t);
    if (lane > k) l[k] = (g[k].hi - t) * rd[k];
    if (lane == k) l[k] = lkk;
  }
  auto solve = [&](const float (&r)[kNB], float (&x)[kNB]) {
    float z[kNB];
#pragma unroll
    for (int k = 0; k < kNB; ++k) {
      float t = 0.0f;
#pragma unroll
      for (int i = 0; i < k; ++i) t = fmaf(l[i], z[i], t);
      const float zk = ((keep >> k) & 1u) ? (r[k] - t) * rd[k] : 0.0f;
      z[k] = __shfl_sync(kFull, zk, k);
    }
#pragma unroll
    for (int k = kNB - 1; k >= 0; --k) {
      float t = 0.0f;
#pragma unroll
      for (int i = k + 1; i < kNB; ++i) t = fmaf(__shfl_sync(kFull, l[k], i), x[i], t);
      x[k] = ((keep >> k) & 1u) ? (z[k] - t) * rd[k] : 0.0f;
    }
  };
  float rf[kNB], x[kNB], dx[kNB];
#pragma unroll
  for (int k = 0; k < kNB; ++k) rf[k] = tot[kNMono + k].hi;
  solve(rf, x);
  DF res = tot[kNMono + row];
#pragma unroll
  for (int k = 0; k < kNB; ++k) {
    const float p = g[k].hi * x[k];
    const float pe = fmaf(g[k].hi, x[k], -p);  // exact remainder of the product
    res = df_add(res, DF{-p, -fmaf(g[k].lo, x[k], pe)});
  }
  const float r = res.hi + res.lo;
#pragma unroll
  for (int k = 0; k < kNB; ++k) rf[k] = __shfl_sync(kFull, r, k);
  solve(rf, dx);
#pragma unroll
  for (int k = 0; k < kNB; ++k) {
    x_out[k] = x[k];
    dx_out[k] = dx[k];
  }
}

// ---------------------------------------------------------------------------
// Persistent sweep: the whole backward induction in one cooperative launch (all
// blocks resident, one per SM).  Each date: apply the date's rule to the
// thread's paths (states kept in shared memory from the previous date's
// regression), load the states of the date before, accumulate its regression
// sums, write the block's row, one grid barrier, then EVERY block sums all
// rows (one warp per quantity, in a fixed order) and solves the same normal
// equations (identical arithmetic, so identical coefficients everywhere and no
// second barrier).  Rows alternate between two buffers: a block writes a buffer
// again only after the next barrier, which every block reaches after reading it.
constexpr int kSweepTpb = 1024;
constexpr int kSweepWarps = kSweepTpb / kWarp;
static_assert(kNReg <= kSweepWarps, "one warp per regression quantity in the cross-block sum");
// Every wait of the sweep (grid barrier, bulk copy) gives up after kWaitLimitNs
// of the GPU's global timer -- 25,000 times a date's whole time -- or, as a
// backstop, after kSpinLimit polls.
constexpr unsigned long long kWaitLimitNs = 250000000ull;
constexpr unsigned kSpinLimit = 1u << 26;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Whether a wait that began at t0 and has polled `it` times should give up
// (the timer read every 256 polls).
__device__ __forceinline__ bool wait_expired(unsigned it, unsigned long long t0) {
  return it > kSpinLimit || ((it & 255u) == 0u && global_ns() - t0 > kWaitLimitNs);
}

// Bulk copies global -> shared memory by the TMA engine (cp.async.bulk, no
// tensor map: contiguous 16-byte-aligned ranges), each completing its bytes on
// an mbarrier in shared memory.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

// The one arrival of a phase, announcing the bytes its copies will complete.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(float* dst, const float* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// Waits for the phase of the given parity to complete (non-blocking polls,
// backing off like the grid barrier); false once the wait has expired.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if (wait_expired(it, t0)) return false;
    if (it > 2048) __nanosleep(32);
  }
}

struct LsmSweep {
  unsigned int* count;  // arrivals at all barriers so far (zeroed before the launch)
  int* status;          // bit 1: a barrier wait timed out (results invalid)
  float2* rows;         // [2][kNReg][grid]: two buffers, quantity-major
};

// Grid-wide barrier number `nb` (0, 1, ...) of the cooperative sweep: every block
// adds one arrival to a counter that is never reset during the launch and waits
// until it reaches (nb + 1) blocks (+ `extra`, 0 but under fault injection) --
// the last block to arrive has nothing more to do, so the barrier costs one
// atomic and the polls.  Bounded: a wait that expires sets status bit 1 and
// returns false, and every later barrier returns false at once, so all blocks
// leave within one time-out.  `idle()` runs in every thread once the block has
// arrived, while thread 0 waits.
template <class Idle>
__device__ bool lsm_grid_sync(const LsmSweep& Y, unsigned nb, unsigned extra, int* s_flag, Idle&& idle) {
  __threadfence();
  __syncthreads();
  idle();
  if (threadIdx.x == 0) {
    int ok = (*(volatile int*)Y.status & 2) == 0;
    if (ok) {
      const unsigned target = (nb + 1u) * gridDim.x + extra;
      atomicAdd(Y.count, 1u);
      const unsigned long long t0 = global_ns();
      unsigned it = 0;
      while (*(volatile unsigned*)Y.count < target) {
        if (wait_expired(++it, t0)) {
          atomicOr(Y.status, 2);
          ok = 0;
          break;
        }
        if (it > 2048) __nanosleep(32);
      }
      __threadfence();
    }
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// Block's FP32 warp sums (s_w[warp][q], q < nv) -> one double-float row: four
// threads per quantity sum 8 warps each, then one sums the four in order.  The
// rows are stored quantity-major, [q][block], so that a warp reads one
// quantity of 32 blocks as one contiguous line.
__device__ __forceinline__ void sweep_block_row(const float (*s_w)[kNReg], int nv, DF* s_quad, float2* rows) {
  if (threadIdx.x < 4 * nv) {
    const int q = threadIdx.x % nv, g = threadIdx.x / nv;
    DF t{0.0f, 0.0f};
#pragma unroll
    for (int w = 8 * g; w < 8 * g + 8; ++w) t = df_add(t, DF{s_w[w][q], 0.0f});
    s_quad[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    DF t{0.0f, 0.0f};
#pragma unroll
    for (int g = 0; g < 4; ++g) t = df_add(t, s_quad[g * nv + threadIdx.x]);
    rows[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = make_float2(t.hi, t.lo);
  }
}

// Sum of all blocks' rows into s_tot (double-float): warp q sums quantity q,
// lane l taking blocks l, l + 32, ... in order (its loads issued together), then
// a butterfly over the lanes; lane 0's total is the same in every block (the same
// operations on the same rows).
__device__ __forceinline__ void sweep_total(const float2* rows, int nv, DF* s_tot) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q < nv) {
    constexpr int kAhead = 8;  // loads in flight per lane
    DF t{0.0f, 0.0f};
    for (unsigned b0 = 0; b0 < gridDim.x; b0 += kAhead * kWarp) {
      float2 r[kAhead];
#pragma unroll
      for (int k = 0; k < kAhead; ++k) {
        const unsigned b = b0 + k * kWarp + lane;
        r[k] = b < gridDim.x ? __ldcg(rows + (size_t)q * gridDim.x + b) : make_float2(0.0f, 0.0f);
      }
#pragma unroll
      for (int k = 0; k < kAhead; ++k)
        if (b0 + k * kWarp + lane < gridDim.x) t = df_add(t, DF{r[k].x, r[k].y});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      t = df_add(t, DF{__shfl_xor_sync(kFull, t.hi, o), __shfl_xor_sync(kFull, t.lo, o)});
    if (lane == 0) s_tot[q] = t;
  }
  __syncthreads();
}

// Each date's states come into shared memory by bulk copies issued a date ahead,
// into two buffers used in turn (every block's range of a date starts on 16
// bytes: the rows' pitch is a multiple of 4 floats).
template <int M>
__global__ void __launch_bounds__(kSweepTpb, 1) lsm_sweep_kernel(const __grid_constant__ LsmLaunch L,
                                                                 const LsmBuffers B, const LsmSweep Y) {
  // dynamic shared memory, [M][thread] each: the states of a date (S, then v; two
  // such buffers, date j in buffer j & 1) -- the regression of date j reads them,
  // the rule of date j reads them again -- then the thread's paths' cash flows
  // and exercise dates for the whole sweep (each thread its own slots), then the
  // discount table (n_ex floats)
  extern __shared__ __align__(16) float s_keep[];
  float* s_c = s_keep + 4 * M * kSweepTpb;
  int* s_st = reinterpret_cast<int*>(s_c + M * kSweepTpb);
  float* s_dpow = s_c + 2 * M * kSweepTpb;
  auto states = [&](int j) { return s_keep + (j & 1) * 2 * M * kSweepTpb; };
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ float s_w[kSweepWarps][kNReg];
  __shared__ DF s_quad[4 * kNReg];
  __shared__ DF s_tot[kNReg];
  __shared__ float s_beta[kNB];
  __shared__ int s_has, s_flag;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t P = L.paths;
  float2* beta_t = reinterpret_cast<float2*>(B.beta_t);  // [n_ex][6] (x, dx) pairs
  const uint64_t gt = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t g0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool put = L.is_put != 0;
  const float K = L.K;
  for (int k = threadIdx.x; k < L.n_ex; k += kSweepTpb) s_dpow[k] = B.dpow[k];
  // this thread's paths g0 + m gt
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const uint64_t i = g0 + (uint64_t)m * gt;
    s_c[m * kSweepTpb + threadIdx.x] = i < P ? B.cash[i] : 0.0f;
    s_st[m * kSweepTpb + threadIdx.x] = i < P ? B.stop[i] : -1;
  }
  // the block's share of date j: for each m the paths m gt + blockIdx.x 1024 +
  // [0, 1024), cut at P rounded up to 4 floats (within the row's pitch; slots of
  // paths >= P are never used); the block's last thread issues the copies
  // (thread 0 runs the grid barrier meanwhile)
  // per buffer b (bit b, the same in every thread): the parity of its next phase,
  // and whether a copy into it is in flight
  uint32_t parity = 0u, pending = 0u;
  auto issue = [&](int j) {
    if (threadIdx.x == kSweepTpb - 1) {
      float* dst = states(j);
      const float* Sg = B.S + (size_t)j * L.pitch;
      const float* Vg = B.V + (size_t)j * L.pitch;
      auto floats = [&](uint64_t a) -> uint32_t {  // the copy's length at path a (a multiple of 4)
        const uint64_t n = a < P ? (P - a < kSweepTpb ? P - a : kSweepTpb) : 0;
        return (uint32_t)((n + 3) & ~3ull);
      };
      uint32_t total = 0;
#pragma unroll
      for (int m = 0; m < M; ++m) total += 8u * floats((uint64_t)m * gt + (uint64_t)blockIdx.x * kSweepTpb);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier reads of the buffer before the copies
      mbar_arrive_expect(&s_bar[j & 1], total);
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const uint64_t a = (uint64_t)m * gt + (uint64_t)blockIdx.x * kSweepTpb;
        if (a < P) {
          const uint32_t bytes = 4u * floats(a);
          bulk_copy_g2s(dst + m * kSweepTpb, Sg + a, bytes, &s_bar[j & 1]);
          bulk_copy_g2s(dst + (M + m) * kSweepTpb, Vg + a, bytes, &s_bar[j & 1]);
        }
      }
    }
    pending |= 1u << (j & 1);
  };
  // before an early return: the copies still in flight land first (bounded)
  auto drain = [&]() {
    for (int b = 0; b < 2; ++b)
      if ((pending >> b) & 1u) (void)mbar_wait(&s_bar[b], (parity >> b) & 1u);
  };
  if (threadIdx.x == 0) {
    s_has = 0;
    mbar_init(&s_bar[0]);
    mbar_init(&s_bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();  // (the barriers' initialisation before the last thread's first copies)
  if (L.n_ex >= 2) issue(L.n_ex - 2);
  float4 tj = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // date d's basis scaling (loaded a date ahead)
  for (int d = L.n_ex - 1; d >= 0; --d) {
    const bool regress = d >= 1;
    const int nv = regress ? kNReg : 2;
    const float4 tr = regress ? __ldg(B.xform + (d - 1)) : tj;  // date d - 1's, requested early
    // date d's rule (no coefficients at the maturity)
    if (s_has) {  // (a rule exists only below the last date: date d's states are in shared memory)
      float bj[kNB];
#pragma unroll
      for (int k = 0; k < kNB; ++k) bj[k] = s_beta[k];
      const float* sd = states(d);
      float Su[M], Vu[M];
#pragma unroll
      for (int m = 0; m < M; ++m) {
        Su[m] = sd[m * kSweepTpb + threadIdx.x];
        Vu[m] = sd[(M + m) * kSweepTpb + threadIdx.x];
      }
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const float h = lsm_payoff(put, Su[m], K);
        if (g0 + (uint64_t)m * gt < P && h > 0.0f &&
            h > lsm_continuation(bj, fmaf(Su[m], tj.x, tj.y), fmaf(Vu[m], tj.z, tj.w))) {
          s_c[m * kSweepTpb + threadIdx.x] = h;
          s_st[m * kSweepTpb + threadIdx.x] = d;
        }
      }
    }
    float acc[kNReg];
#pragma unroll
    for (int k = 0; k < kNReg; ++k) acc[k] = 0.0f;
    if (regress) {
      float Sn[M], Vn[M];
      {  // date d - 1's copies, issued a date ago
        const int b = (d - 1) & 1;
        const bool late = !mbar_wait(&s_bar[b], (parity >> b) & 1u);
        if (__syncthreads_or(late)) {  // the whole block leaves
          if (threadIdx.x == 0) atomicOr(Y.status, 2);
          drain();
          return;
        }
        parity ^= 1u << b;
        pending &= ~(1u << b);
        const float* sr = states(d - 1);
#pragma unroll
        for (int m = 0; m < M; ++m) {
          Sn[m] = sr[m * kSweepTpb + threadIdx.x];
          Vn[m] = sr[(M + m) * kSweepTpb + threadIdx.x];
        }
      }
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const float h = lsm_payoff(put, Sn[m], K);
        if (g0 + (uint64_t)m * gt < P && h > 0.0f) {
          const int st = s_st[m * kSweepTpb + threadIdx.x];
          const float Yv = st >= 0 ? s_c[m * kSweepTpb + threadIdx.x] * s_dpow[st - (d - 1)] : 0.0f;
          lsm_accumulate(acc, fmaf(Sn[m], tr.x, tr.y), fmaf(Vn[m], tr.z, tr.w), Yv);
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int st = s_st[m * kSweepTpb + threadIdx.x];
        const float dv = st >= 0 ? s_c[m * kSweepTpb + threadIdx.x] * s_dpow[st] : 0.0f;  // discounted to t_0
        acc[0] += dv;
        acc[1] = fmaf(dv, dv, acc[1]);
      }
    }
    // FP32 over the warp, double-float over warps and blocks
    {
      float vals[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) vals[k] = k < kNReg ? acc[k] : 0.0f;
      butterfly32(vals, lane);
      if (lane < kNReg) s_w[warp][lane] = vals[0];
    }
    __syncthreads();
    float2* rows = Y.rows + (size_t)(d & 1) * gridDim.x * kNReg;
    sweep_block_row(s_w, nv, s_quad, rows);
    // once every thread is past date d's rule, its buffer takes date d - 2
    const unsigned extra = d == L.n_ex - 1 ? (unsigned)L.barrier_extra : 0u;
    if (!lsm_grid_sync(Y, (unsigned)(L.n_ex - 1 - d), extra, &s_flag, [&] {
          if (d >= 2) issue(d - 2);
        })) {
      drain();
      return;
    }
    sweep_total(rows, nv, s_tot);
    if (regress) {
      // every block: the same solve; block 0 records the coefficients
      if (warp == 0) {
        const bool ok = s_tot[0].hi >= (float)L.min_itm;  // an exact count
        float x[kNB], dx[kNB];
        if (ok) lsm_solve_df(s_tot, x, dx, lane);
        if (lane == 0) {
          s_has = ok ? 1 : 0;
#pragma unroll
          for (int k = 0; k < kNB; ++k) s_beta[k] = ok ? x[k] + dx[k] : 0.0f;
          if (blockIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < kNB; ++k)
              beta_t[(size_t)(d - 1) * kNB + k] = ok ? make_float2(x[k], dx[k]) : make_float2(__int_as_float(0x7fc00000), 0.0f);
          }
        }
      }
      __syncthreads();
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
      const double n = (double)P;
      const double mean = ((double)s_tot[0].hi + (double)s_tot[0].lo) / n;
      B.price[0] = L.disc0 * mean;
      if (B.stderr_) {
        const double var = n > 1.0 ? (((double)s_tot[1].hi + (double)s_tot[1].lo) / n - mean * mean) / (n - 1.0) : 0.0;
        B.stderr_[0] = L.disc0 * sqrt(var > 0.0 ? var : 0.0);
      }
    }
    tj = tr;  // date d - 1's rule comes next
  }
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const uint64_t i = g0 + (uint64_t)m * gt;
    if (i < P) B.stop[i] = s_st[m * kSweepTpb + threadIdx.x];
  }
  // the coefficients in x, y: one date per block (block 0's rows are visible
  // after the last barrier)
  if (threadIdx.x == 0) {
    for (int j = blockIdx.x; j < L.n_ex - 1; j += gridDim.x) {
      const float2* bt = beta_t + (size_t)j * kNB;
      double* bo = B.beta + (size_t)j * kNB;
      if (isnan(__ldcg(bt).x)) continue;  // stays NaN
      double bs[kNB];
#pragma unroll
      for (int k = 0; k < kNB; ++k) {
        const float2 v = __ldcg(bt + k);
        bs[k] = (double)v.x + (double)v.y;
      }
      const float4 tr = B.xform[j];
      const double kx = (double)tr.x * L.Kd, cx = -(kx + (double)tr.y) / kx;
      const double ky = (double)tr.z * L.wd, cy = -(ky + (double)tr.w) / ky;
      lsm_unscale(bs, kx, cx, ky, cy, bo);
    }
  }
}

template <bool U, bool R>
cudaError_t launch_date(const LsmLaunch& L, const LsmBuffers& B, int j, unsigned grid, cudaStream_t st) {
  lsm_date_kernel<U, R><<<grid, kLsmTpb, 0, st>>>(L, B, j);
  return cudaGetLastError();
}

constexpr int kLsmMaxBlocksPerSm = 8;

}  // namespace

size_t lsm_partial_doubles(int num_sms) { return (size_t)num_sms * kLsmMaxBlocksPerSm * kNReg; }

namespace {

template <int M>
cudaError_t try_sweep_m(const LsmLaunch& L, const LsmBuffers& B, const LsmSweep& Y, int num_sms, cudaStream_t st,
                        bool* used) {
  // S and v (two buffers), cash flow, exercise date; the discount table
  const size_t smem = ((size_t)6 * M * kSweepTpb + (size_t)L.n_ex) * sizeof(float);
  auto kern = lsm_sweep_kernel<M>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSweepTpb, smem);
  if (e != cudaSuccess || per_sm < 1) return e;
  const uint64_t resident = (uint64_t)num_sms * per_sm;
  const uint64_t per_block = (uint64_t)M * kSweepTpb;
  const uint64_t need = (L.paths + per_block - 1) / per_block;
  if (need > resident || need > (uint64_t)num_sms * kLsmMaxBlocksPerSm / 2) return cudaSuccess;  // M too small
  const unsigned grid = (unsigned)need;
  e = cudaMemsetAsync(Y.count, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  LsmLaunch Lc = L;
  LsmBuffers Bc = B;
  LsmSweep Yc = Y;
  void* args[] = {&Lc, &Bc, &Yc};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kSweepTpb), args, smem, st);
  if (e == cudaSuccess) *used = true;
  return e;
}

// The backward induction as one cooperative launch when the device supports it
// and the paths fit M <= 7 per thread of the resident blocks; *used reports it.
cudaError_t try_sweep(const LsmLaunch& L, const LsmBuffers& B, const LsmSweep& Y, int num_sms, cudaStream_t st,
                      bool* used) {
  *used = false;
  const char* env = std::getenv("SIMR_LSM_SWEEP");
  if (env && env[0] == '0') return cudaSuccess;
  int dev = 0, coop = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e != cudaSuccess || !coop) return e;
  e = try_sweep_m<1>(L, B, Y, num_sms, st, used);
  if (e == cudaSuccess && !*used) e = try_sweep_m<2>(L, B, Y, num_sms, st, used);
  if (e == cudaSuccess && !*used) e = try_sweep_m<4>(L, B, Y, num_sms, st, used);
  if (e == cudaSuccess && !*used) e = try_sweep_m<7>(L, B, Y, num_sms, st, used);
  return e;
}

}  // namespace

cudaError_t launch_lsm(const LsmLaunch& L, const LsmBuffers& B, int num_sms, cudaStream_t stream) {
  int per_sm = 0;
  auto pk = L.scheme == 1 ? lsm_paths_kernel<true> : lsm_paths_kernel<false>;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pk, kLsmTpb, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t batches = (L.paths + (uint64_t)kWarp * kLsmPpt - 1) / ((uint64_t)kWarp * kLsmPpt);
  uint64_t grid = (uint64_t)num_sms * per_sm;
  const uint64_t need = (batches + kLsmWarps - 1) / kLsmWarps;
  if (grid > need) grid = need;
  pk<<<(unsigned)grid, kLsmTpb, 0, stream>>>(L, B.S, B.V, B.cash, B.stop);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  bool swept = false;
  const LsmSweep Y{B.ticket + 4, B.status, reinterpret_cast<float2*>(B.partials)};
  e = try_sweep(L, B, Y, num_sms, stream, &swept);
  if (e != cudaSuccess || swept) return e;

  // date kernels: resident blocks on all SMs (at most kLsmMaxBlocksPerSm), at most one path per thread more
  int per_sm2 = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, lsm_date_kernel<true, true>, kLsmTpb, 0);
  if (e != cudaSuccess) return e;
  if (per_sm2 < 1) return cudaErrorInvalidConfiguration;
  if (per_sm2 > kLsmMaxBlocksPerSm) per_sm2 = kLsmMaxBlocksPerSm;
  uint64_t g2 = (uint64_t)num_sms * per_sm2;
  const uint64_t need2 = (L.paths + kLsmTpb - 1) / kLsmTpb;
  if (g2 > need2) g2 = need2;
  const unsigned g = (unsigned)g2;
  if (L.n_ex == 1) return launch_date<false, false>(L, B, 0, g, stream);
  e = launch_date<false, true>(L, B, L.n_ex - 1, g, stream);
  for (int j = L.n_ex - 2; j >= 1 && e == cudaSuccess; --j) e = launch_date<true, true>(L, B, j, g, stream);
  if (e != cudaSuccess) return e;
  return launch_date<true, false>(L, B, 0, g, stream);
}

}  // namespace simr
