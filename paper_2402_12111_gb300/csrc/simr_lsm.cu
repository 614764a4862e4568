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
//     normal equations by Cholesky in FP64, leaving out a basis function whose
//     pivot is not above 1e-12 of its diagonal entry.  The launch of date 0
//     applies its rule and reduces the discounted cash flows to the price.
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

// Path kernel: states at the exercise dates, maturity cash flow.
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
    uint32_t plo[kLsmPpt], phi[kLsmPpt];
    float v[kLsmPpt], x[kLsmPpt], comp[kLsmPpt];
#pragma unroll
    for (int j = 0; j < kLsmPpt; ++j) {
      idx[j] = bt * per + (uint64_t)j * kWarp + lane;
      plo[j] = (uint32_t)idx[j];
      phi[j] = (uint32_t)(idx[j] >> 32);
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
      row += L.paths;
    };
    for (uint32_t p = 0; 2 * p < L.steps; ++p) {
      uint4 w[kLsmPpt];
#pragma unroll
      for (int j = 0; j < kLsmPpt; ++j) w[j] = philox4x32_10(p, plo[j], phi[j], L.option_index, L.rk);
#pragma unroll
      for (int j = 0; j < kLsmPpt; ++j) {
        const float xv = centered_uniform(w[j].x);
        step_base<false>(L.sc, 0.5f * (1.0f - xv), norminv_centered(xv), norminv_centered(centered_uniform(w[j].y)),
                         v[j], x[j], comp[j]);
      }
      if (++cnt == L.every) {
        cnt = 0;
        record();
      }
      if (2 * p + 1 < L.steps) {
#pragma unroll
        for (int j = 0; j < kLsmPpt; ++j) {
          const float xv = centered_uniform(w[j].z);
          step_base<false>(L.sc, 0.5f * (1.0f - xv), norminv_centered(xv),
                           norminv_centered(centered_uniform(w[j].w)), v[j], x[j], comp[j]);
        }
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
// Cholesky factor L; every lane ends with all of beta).  Cholesky in basis
// order, basis function k left out (coefficient 0) when its pivot d is not
// above 1e-12 G[k][k]; each dot product runs in ascending index order.
__device__ void lsm_solve_warp(const double* tot, double* beta, int lane) {
  double g[kNB], l[kNB], rd[kNB], z[kNB];
  unsigned keep = 0;
  const int row = lane < kNB ? lane : 0;
#pragma unroll
  for (int k = 0; k < kNB; ++k) {
    g[k] = tot[c_gram_index[row * kNB + k]];
    l[k] = 0.0;
  }
#pragma unroll
  for (int k = 0; k < kNB; ++k) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < k; ++i) s += l[i] * l[i];  // left-out columns hold 0
    const double d = __shfl_sync(kFull, g[k] - s, k);
    const double gkk = __shfl_sync(kFull, g[k], k);
    rd[k] = 0.0;
    if (!(gkk > 0.0 && d > 1e-12 * gkk)) continue;
    keep |= 1u << k;
    const double lkk = sqrt(d);
    rd[k] = 1.0 / lkk;
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < k; ++i) t += l[i] * __shfl_sync(kFull, l[i], k);
    if (lane > k) l[k] = (g[k] - t) * rd[k];
    if (lane == k) l[k] = lkk;
  }
#pragma unroll
  for (int k = 0; k < kNB; ++k) {  // L z = b
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < k; ++i) t += l[i] * z[i];
    const double zk = ((keep >> k) & 1u) ? (tot[kNMono + k] - t) * rd[k] : 0.0;
    z[k] = __shfl_sync(kFull, zk, k);
  }
#pragma unroll
  for (int k = kNB - 1; k >= 0; --k) {  // L^T beta = z; L[i][k] is lane i's l[k]
    double t = 0.0;
#pragma unroll
    for (int i = k + 1; i < kNB; ++i) t += __shfl_sync(kFull, l[k], i) * beta[i];
    beta[k] = ((keep >> k) & 1u) ? (z[k] - t) * rd[k] : 0.0;
  }
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
  const float* Sj = B.S + (size_t)j * P;
  const float* Vj = B.V + (size_t)j * P;
  const float* Sr = B.S + (size_t)(REGRESS ? jr : 0) * P;
  const float* Vr = B.V + (size_t)(REGRESS ? jr : 0) * P;
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
          const float x = fmaf(Su[k], tj.x, tj.y), y = fmaf(Vu[k], tj.z, tj.w);
          float C = fmaf(bj[2], x, bj[1]);
          C = fmaf(C, x, bj[0]);
          C = fmaf(fmaf(bj[5], y, fmaf(bj[4], x, bj[3])), y, C);
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

template <bool U, bool R>
cudaError_t launch_date(const LsmLaunch& L, const LsmBuffers& B, int j, unsigned grid, cudaStream_t st) {
  lsm_date_kernel<U, R><<<grid, kLsmTpb, 0, st>>>(L, B, j);
  return cudaGetLastError();
}

constexpr int kLsmMaxBlocksPerSm = 8;

}  // namespace

size_t lsm_partial_doubles(int num_sms) { return (size_t)num_sms * kLsmMaxBlocksPerSm * kNReg; }

cudaError_t launch_lsm(const LsmLaunch& L, const LsmBuffers& B, int num_sms, cudaStream_t stream) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lsm_paths_kernel, kLsmTpb, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t batches = (L.paths + (uint64_t)kWarp * kLsmPpt - 1) / ((uint64_t)kWarp * kLsmPpt);
  uint64_t grid = (uint64_t)num_sms * per_sm;
  const uint64_t need = (batches + kLsmWarps - 1) / kLsmWarps;
  if (grid > need) grid = need;
  lsm_paths_kernel<<<(unsigned)grid, kLsmTpb, 0, stream>>>(L, B.S, B.V, B.cash, B.stop);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;

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
