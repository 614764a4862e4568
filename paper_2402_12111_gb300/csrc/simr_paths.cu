// simr_paths.cu -- fused Heston QE path kernels for sm_103a: pricing, bump-and-revalue
// Greeks with common random numbers, terminal states.
//
// Per path (one lane) and per time step, entirely in registers:
//   Philox4x32-10 (one call per two steps) -> two 23-bit uniforms per step ->
//   inverse normals -> QE variance step (paper Sec. 4, VariancePathQE) ->
//   log-spot step (Sec. 5, LogPricePathQE), for every simulated scenario, all
//   sharing the same draws (common random numbers).
// Per path at maturity: S_T = S0 e^{x_T} (AssetPathExponential) and the payoff
// terms of each strike.  Reduction over paths (Sec. 6): a transposed warp
// butterfly in FP32 sums 32 paths per strike in 31 shuffle-add steps for 32
// strikes at once, then one FP64 add per lane into per-warp shared-memory
// accumulators; per block the warps are summed in FP64 in fixed order into a
// partial row in global scratch, and the last block to finish (atomic ticket)
// sums the rows in block order and normalises.  No path data touches HBM.
#include <cuda_runtime.h>

#include <cstdint>

#include "simr_device.cuh"
#include "simr_internal.h"
#include "simr_reduce.cuh"

// Tuning knobs (compile-time): resident 256-thread blocks per SM the 5-scenario
// kernel is register-budgeted for.
#ifndef SIMR_FD5_BLOCKS_PER_SM
#define SIMR_FD5_BLOCKS_PER_SM 3
#endif
// paths per thread of the pricing (one scenario) and bump-and-revalue kernels
#ifndef SIMR_PRICE_PPT
#define SIMR_PRICE_PPT 2
#endif
#ifndef SIMR_FD_PPT
#define SIMR_FD_PPT 1
#endif

namespace simr {
namespace {

// Per-path term of accumulator `a` for one strike (call or put), given the
// terminal spots of all scenarios.  a = 0: payoff f; 1: f^2; then per Greek bit.
template <int NS>
__device__ __forceinline__ float acc_term(const PathLaunch& L, int greek_bit, int a,
                                          const StrikeConst& k, const float (&S)[NS]) {
  const float s = S[0];
  const bool put = L.is_put != 0;
  const float f = put ? fmaxf(k.K - s, 0.0f) : fmaxf(s - k.K, 0.0f);
  if (a == 0) return f;
  if (a == 1) return f * f;
  const float h = L.h_s;
  switch (greek_bit) {
    case 0: {  // delta: f(S(1+h)) - f(S(1-h)) = min(max(S(1+h)-K, 0), 2hS) for a call
      const float w = 2.0f * h * s;
      return put ? -fminf(fmaxf(fmaf(h, s, k.K - s), 0.0f), w) : fminf(fmaxf(fmaf(h, s, s - k.K), 0.0f), w);
    }
    case 1:  // gamma: f(S(1+h)) - 2 f(S) + f(S(1-h)) = max(0, hS - |K - S|)
      return fmaxf(fmaf(h, s, -fabsf(k.K - s)), 0.0f);
    case 4:  // rho: e^{-hT} f(S e^{hT}) - e^{hT} f(S e^{-hT}) = f(S; K e^{-hT}) - f(S; K e^{hT})
      return put ? -fminf(fmaxf(k.Km + k.Wr - s, 0.0f), k.Wr) : fminf(fmaxf(s - k.Km, 0.0f), k.Wr);
    default:
      break;
  }
  return 0.0f;
}

// ratio_up f_up - ratio_dn f_dn with ratio = 1 + delta (delta exact in FP32).
template <int NS>
__device__ __forceinline__ float resim_term(const PathLaunch& L, int up, int dn, const StrikeConst& k,
                                            const float (&S)[NS]) {
  float su = 0.0f, sd = 0.0f;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (s == up) su = S[s];
    if (s == dn) sd = S[s];
  }
  const bool put = L.is_put != 0;
  const float fu = put ? fmaxf(k.K - su, 0.0f) : fmaxf(su - k.K, 0.0f);
  const float fd = put ? fmaxf(k.K - sd, 0.0f) : fmaxf(sd - k.K, 0.0f);
  const float ru = up ? L.sc[up].ratio : 0.0f, rd = dn ? L.sc[dn].ratio : 0.0f;
  return fmaf(ru, fu, fmaf(-rd, fd, fu - fd));
}

// One time step for all NS scenarios from the two words (w_v, w_x) of the step.
// NS scenarios in registers; DYN: only the first L.n_scen of them are live.
// Scenarios 1 .. NV differ from the base only in v0 (all constant deltas zero):
// they take the base step, which is the bumped step's arithmetic with zero deltas.
// The two inverse normals run paired, and so do the scenarios after the base,
// two at a time (s, s + 1): the paired functions repeat the scalar ones lane for
// lane, so every scenario's value is the scalar step's, bit for bit.  Constants
// equal in both lanes are broadcast from the scalar ones; a bumped pair's deltas,
// which differ by lane, come pre-packed from the launch parameters (measured:
// 3.4% faster than pre-packing the broadcast constants too, 6% faster than
// packing the deltas in the kernel).
template <int NS, int NV, bool DYN, bool QEM = false>
__device__ __forceinline__ void step_all(const PathLaunch& L, uint32_t w_v, uint32_t w_x, float (&v)[NS],
                                         float (&x)[NS], float (&c)[NS]) {
  const float2 xu = centered_uniform2(w_v, w_x);  // (2 U_V - 1, 2 U_X - 1)
  const float2 z = norminv_centered2(xu);
  const float xv = xu.x, zv = z.x, zx = z.y;
  static_assert(NS % 2 == 1, "the base scenario plus up/down pairs");
  if constexpr (QEM && NS > 1) {  // QE-M with bumped scenarios: the base, then the pairs (DYN: one at a time)
    const ScenConst zero{};
    const QemConst zq{};
    step_qem_bumped(L.sc[0], zero, L.qm, zq, xv, zv, zx, v[0], x[0], c[0]);
#pragma unroll
    for (int s = 1; s < NS; ++s) {
      if constexpr (DYN) {
        if (s >= L.n_scen) break;
        step_qem_bumped(L.sc[0], L.sc[s], L.qm, L.qmd[s], xv, zv, zx, v[s], x[s], c[s]);
      } else if (s % 2 == 1) {
        float2 vv = make_float2(v[s], v[s + 1]), xx = make_float2(x[s], x[s + 1]),
               cc = make_float2(c[s], c[s + 1]);
        step_qem_bumped2(pack_const(L.sc[0], L.sc[0]), L.pair2[(s - 1) / 2], L.qm, L.qmd2[(s - 1) / 2], p_bc(xv),
                         p_bc(zv), p_bc(zx), vv, xx, cc);
        v[s] = vv.x;
        v[s + 1] = vv.y;
        x[s] = xx.x;
        x[s + 1] = xx.y;
        c[s] = cc.x;
        c[s + 1] = cc.y;
      }
    }
    return;
  }
  step_scheme<(NS > 1), QEM>(L.sc[0], L.qm, xv, zv, zx, v[0], x[0], c[0]);
#pragma unroll
  for (int s = 1; s + 1 < NS; s += 2) {
    if (DYN && s >= L.n_scen) break;
    float2 vv = make_float2(v[s], v[s + 1]), xx = make_float2(x[s], x[s + 1]), cc = make_float2(c[s], c[s + 1]);
    if (s + 1 <= NV)
      step_base2<true>(L.sc[0], p_bc(xv), p_bc(zv), p_bc(zx), vv, xx, cc);
    else
      step_bumped2(pack_const(L.sc[0], L.sc[0]), L.pair2[(s - 1) / 2], p_bc(xv), p_bc(zv), p_bc(zx), vv, xx, cc);
    v[s] = vv.x;
    v[s + 1] = vv.y;
    x[s] = xx.x;
    x[s + 1] = xx.y;
    c[s] = cc.x;
    c[s + 1] = cc.y;
  }
}

// One time step of PPT paths.  Pricing with two paths per thread runs the two
// paths' steps paired (their inverse normals too; QE or QE-M); otherwise
// step_all per path.
template <int NS, int NV, bool DYN, int PPT, bool QEM>
__device__ __forceinline__ void step_paths(const PathLaunch& L, const uint32_t (&wv)[PPT], const uint32_t (&wx)[PPT],
                                           float (&v)[PPT][NS], float (&x)[PPT][NS], float (&c)[PPT][NS]) {
  if constexpr (NS == 1 && PPT == 2) {
    const float2 xv = centered_uniform2(wv[0], wv[1]);
    const float2 zv = norminv_centered2(xv);
    const float2 zx = norminv_centered2(centered_uniform2(wx[0], wx[1]));
    float2 vv = make_float2(v[0][0], v[1][0]), xx = make_float2(x[0][0], x[1][0]), cc = make_float2(c[0][0], c[1][0]);
    if constexpr (QEM)
      step_qem2(L.sc[0], L.qm, xv, zv, zx, vv, xx, cc);
    else
      step_base2<false>(L.sc[0], xv, zv, zx, vv, xx, cc);
    v[0][0] = vv.x;
    v[1][0] = vv.y;
    x[0][0] = xx.x;
    x[1][0] = xx.y;
    c[0][0] = cc.x;
    c[1][0] = cc.y;
  } else {
#pragma unroll
    for (int j = 0; j < PPT; ++j) step_all<NS, NV, DYN, QEM>(L, wv[j], wx[j], v[j], x[j], c[j]);
  }
}

// Step 0 of every scenario of a common-random-number launch (see step0_crn).
// Under QE-M the first-step constant K0p is r dt - qa (v0 + m0) - lam(v0) (set
// on the host in FP64, where M exists at every scenario's v0), v' has no term of
// its own and dl the coefficient K2.
template <int NS, bool DYN, bool QEM = false>
__device__ __forceinline__ void step0_all(const PathLaunch& L, uint32_t w_v, uint32_t w_x, float (&v)[NS],
                                          float (&x)[NS], float (&c)[NS]) {
  const float xv = centered_uniform(w_v);
  const float omu = one_minus_u(xv);
  const float zv = norminv_centered(xv);
  const float zx = norminv_centered(centered_uniform(w_x));
  const ScenConst zero{};
  FirstConst fz = L.f0[0];
  fz.a = fz.b = fz.C = fz.L = fz.m0 = fz.K0p = 0.0f;  // base: zero deltas, its own threshold
  ScenConst b0 = L.sc[0];
  if (QEM) {
    b0.Cv = 0.0f;
    b0.Cdl = L.qm.K2;
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (DYN && s >= L.n_scen) break;
    ScenConst d0 = s == 0 ? zero : L.sc[s];
    if (QEM) {
      d0.Cv = 0.0f;
      d0.Cdl = s == 0 ? 0.0f : L.qmd[s].K2;
    }
    step0_crn(L.f0[0], s == 0 ? fz : L.f0[s], b0, d0, L.sc[s].v0, omu, zv, zx, v[s], x[s], c[s]);
  }
}

// PPT paths per thread, simulated step by step in lockstep: independent
// dependency chains the scheduler can interleave (instruction-level
// parallelism at the same occupancy).
template <int NS, int NV, bool DYN, int PPT, bool QEM = false>
__device__ __forceinline__ void simulate_ppt(const PathLaunch& L, const uint64_t (&path)[PPT], float (&v)[PPT][NS],
                                             float (&x)[PPT][NS], float (&c)[PPT][NS]) {
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      v[j][s] = (DYN && s >= L.n_scen) ? 0.0f : L.sc[s].v0;
      x[j][s] = 0.0f;
      c[j][s] = 0.0f;
    }
  }
  PhiloxLane pl[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) pl[j] = philox_lane(path[j], L.rk);
  const uint32_t pairs = L.steps >> 1;
  uint32_t i0 = 0;
  if (NS > 1 && L.first_split) {
    uint4 w[PPT];
    const PhiloxCtr u = philox_ctr(0u, L.option_index, L.rk);
#pragma unroll
    for (int j = 0; j < PPT; ++j) w[j] = philox_draw(pl[j], u, L.rk);
#pragma unroll
    for (int j = 0; j < PPT; ++j) step0_all<NS, DYN, QEM>(L, w[j].x, w[j].y, v[j], x[j], c[j]);
    if (L.steps > 1) {
      uint32_t wv[PPT], wx[PPT];
#pragma unroll
      for (int j = 0; j < PPT; ++j) wv[j] = w[j].z, wx[j] = w[j].w;
      step_paths<NS, NV, DYN, PPT, QEM>(L, wv, wx, v, x, c);
    }
    i0 = 1;
  }
  for (uint32_t i = i0; i < pairs; ++i) {
    uint4 w[PPT];
    uint32_t wv[PPT], wx[PPT];
    const PhiloxCtr u = philox_ctr(i, L.option_index, L.rk);
#pragma unroll
    for (int j = 0; j < PPT; ++j) w[j] = philox_draw(pl[j], u, L.rk);
#pragma unroll
    for (int j = 0; j < PPT; ++j) wv[j] = w[j].x, wx[j] = w[j].y;
    step_paths<NS, NV, DYN, PPT, QEM>(L, wv, wx, v, x, c);
#pragma unroll
    for (int j = 0; j < PPT; ++j) wv[j] = w[j].z, wx[j] = w[j].w;
    step_paths<NS, NV, DYN, PPT, QEM>(L, wv, wx, v, x, c);
  }
  if ((L.steps & 1u) && pairs >= i0) {  // odd last step (step 0 itself when steps == 1 without the split)
    uint32_t wv[PPT], wx[PPT];
    const PhiloxCtr u = philox_ctr(pairs, L.option_index, L.rk);
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const uint4 w = philox_draw(pl[j], u, L.rk);
      wv[j] = w.x;
      wx[j] = w.y;
    }
    step_paths<NS, NV, DYN, PPT, QEM>(L, wv, wx, v, x, c);
  }
}

// Results of strike k from its n_acc sums (sum_a = s[a * stride]): the price
// e^{-rT} sum f / n, its standard error, and each Greek e^{-rT} sum / (n denom);
// or, in raw mode, the sums themselves.  FP64.
// A strike flagged `bad` (not finite and > 0) gets NaN results.
__device__ __forceinline__ void write_results(const PathLaunch& L, int k, const double* s, int stride,
                                              const PathOutputs& out, bool bad) {
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  if (L.raw_sums) {
    for (int a = 0; a < L.n_acc; ++a) out.sums[(size_t)k * L.n_acc + a] = bad ? nan : s[(size_t)a * stride];
    return;
  }
  if (bad) {
    out.price[k] = nan;
    if (out.stderr_) out.stderr_[k] = nan;
    if (out.greeks)
      for (int g = 0; g < L.n_acc - 2; ++g) out.greeks[(size_t)k * (L.n_acc - 2) + g] = nan;
    return;
  }
  const double n = L.paths_total, inv_n = 1.0 / n;
  const double mean = s[0] * inv_n;
  out.price[k] = L.disc * mean;
  if (out.stderr_) {
    const double var = n > 1.0 ? (s[stride] * inv_n - mean * mean) / (n - 1.0) : 0.0;
    out.stderr_[k] = L.disc * sqrt(var > 0.0 ? var : 0.0);
  }
  if (out.greeks) {
    const int ng = L.n_acc - 2;
    for (int g = 0; g < ng; ++g)
      out.greeks[(size_t)k * ng + g] = L.disc * s[(size_t)(2 + g) * stride] * inv_n / L.denom[g];
  }
}

// Fused price / Greeks kernel.  TILE = 1 (single strike) or 32 (strike tiles).
// Dynamic shared memory: accumulators [warps][n_acc][nk_pad] (FP64), then the
// strike constants [nk_pad] (StrikeConst), then a flag word.
template <int NS, int NV, int TILE, bool DYN, int PPT, bool QEM>
__global__ void __launch_bounds__(256, (NS * PPT <= 3 ? 4 : NS * PPT <= 5 ? SIMR_FD5_BLOCKS_PER_SM : 2)) heston_paths_kernel(const __grid_constant__ PathLaunch L,
                                                           const double* __restrict__ strikes,
                                                           PathOutputs out, double* __restrict__ partials,
                                                           unsigned int* __restrict__ ticket) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warps = blockDim.x / kWarp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = L.n_acc * L.nk_pad;
  double* acc = reinterpret_cast<double*>(smem_raw);
  StrikeConst* ks = reinterpret_cast<StrikeConst*>(acc + (size_t)warps * row);
  int* s_last = reinterpret_cast<int*>(ks + L.nk_pad);

  for (int i = threadIdx.x; i < warps * row; i += blockDim.x) acc[i] = 0.0;
  for (int j = threadIdx.x; j < L.nk_pad; j += blockDim.x) {
    StrikeConst k{0.0f, 0.0f, 0.0f, 0.0f};
    if (j < L.n_strikes) {
      const double K = strikes[j];
      if (!(K > 0.0) || !isfinite(K)) atomicOr(out.status, 1);  // reported by simr_sync
      k.K = (float)K;
      k.Km = (float)(K * L.rho_em);
      k.Wr = (float)(K * L.rho_w);
    }
    ks[j] = k;
  }
  __syncthreads();

  double* my_acc = acc + (size_t)warp * row;
  const uint64_t per_batch = (uint64_t)kWarp * PPT;
  const uint64_t batches = (L.path_count + per_batch - 1) / per_batch;
  const uint64_t total_warps = (uint64_t)gridDim.x * warps;
  for (uint64_t b = (uint64_t)blockIdx.x * warps + warp; b < batches; b += total_warps) {
    uint64_t pth[PPT];
    bool act[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const uint64_t local = b * per_batch + (uint64_t)j * kWarp + lane;
      act[j] = local < L.path_count;
      pth[j] = L.path_begin + local;
    }
    float v[PPT][NS], x[PPT][NS], c[PPT][NS];
    simulate_ppt<NS, NV, DYN, PPT, QEM>(L, pth, v, x, c);
    float S[PPT][NS];
#pragma unroll
    for (int j = 0; j < PPT; ++j)
#pragma unroll
      for (int s = 0; s < NS; ++s) S[j][s] = terminal_spot(L.S0, x[j][s], c[j][s]);

    // accumulator list: 0 f, 1 f^2, then set Greek bits in order
    int a = 0, r = 0;
    for (int bit = -2; bit < kMaxGreeks; ++bit) {
      if (bit >= 0 && !((L.greek_mask >> bit) & 1u)) continue;
      const bool resim = bit == 2 || bit == 3 || bit >= 5;
      const int up = resim ? L.resim_up[r] : 0, dn = resim ? L.resim_dn[r] : 0;
      if (TILE == 1) {
        float t = 0.0f;
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
          const float tj = resim ? resim_term<NS>(L, up, dn, ks[0], S[j]) : acc_term<NS>(L, bit, a, ks[0], S[j]);
          t += act[j] ? tj : 0.0f;
        }
        t = warp_sum(t);
        if (lane == 0) my_acc[a] += (double)t;
      } else {
        for (int t0 = 0; t0 < L.nk_pad; t0 += 32) {
          float vals[32];
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const StrikeConst k = ks[t0 + jj];
            float t = 0.0f;
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
              const float tj = resim ? resim_term<NS>(L, up, dn, k, S[j]) : acc_term<NS>(L, bit, a, k, S[j]);
              t += act[j] ? tj : 0.0f;
            }
            vals[jj] = t;
          }
          butterfly32(vals, lane);
          my_acc[(size_t)a * L.nk_pad + t0 + lane] += (double)vals[0];
        }
      }
      if (resim) ++r;
      ++a;
    }
  }
  __syncthreads();

  // block partial: sum the warps in order
  double* my_row = partials + (size_t)blockIdx.x * row;
  for (int i = threadIdx.x; i < row; i += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < warps; ++w) s += acc[(size_t)w * row + i];
    my_row[i] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!*s_last) return;
  __threadfence();

  // last block: sum the partial rows in block order, then normalise per strike
  for (int i = threadIdx.x; i < row; i += blockDim.x) {
    double s = 0.0;
    for (unsigned bidx = 0; bidx < gridDim.x; ++bidx) s += __ldcg(partials + (size_t)bidx * row + i);
    acc[i] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < L.n_strikes; k += blockDim.x) {
    const double K = strikes[k];
    write_results(L, k, acc + k, L.nk_pad, out, !(K > 0.0) || !isfinite(K));
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// Normalise sums of a sharded run: sums[k][n_acc] -> outputs.
__global__ void finalize_sums_kernel(const __grid_constant__ PathLaunch L, const double* __restrict__ sums,
                                     PathOutputs out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < L.n_strikes) write_results(L, k, sums + (size_t)k * L.n_acc, 1, out, false);
}

template <bool QEM>
__global__ void __launch_bounds__(256) heston_terminal_kernel(const __grid_constant__ PathLaunch L,
                                                              float* __restrict__ x_T, float* __restrict__ v_T) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.path_count) return;
  float v[1][1], x[1][1], c[1][1];
  const uint64_t pth[1] = {L.path_begin + i};
  simulate_ppt<1, 0, false, 1, QEM>(L, pth, v, x, c);
  x_T[i] = x[0][0] - c[0][0];
  if (v_T) v_T[i] = v[0][0];
}

template <int NS, int NV, int TILE, bool DYN, bool QEM = false,
          int PPT = (NS == 1 ? SIMR_PRICE_PPT : SIMR_FD_PPT)>
cudaError_t launch_t(const PathLaunch& L, const double* strikes, const PathOutputs& out, const Scratch& s,
                     int num_sms, cudaStream_t stream, int* grid_used) {
  const int tpb = 256, warps = tpb / kWarp;
  const size_t row = (size_t)L.n_acc * L.nk_pad;
  const size_t smem = warps * row * sizeof(double) + L.nk_pad * sizeof(StrikeConst) + 16;
  auto kern = heston_paths_kernel<NS, NV, TILE, DYN, PPT, QEM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tpb, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t batches = (L.path_count + (uint64_t)kWarp * PPT - 1) / ((uint64_t)kWarp * PPT);
  uint64_t grid = (uint64_t)num_sms * per_sm;
  const uint64_t need = (batches + warps - 1) / warps;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  if ((size_t)grid * row > s.partial_doubles) return cudaErrorMemoryAllocation;
  *grid_used = (int)grid;
  kern<<<(unsigned)grid, tpb, smem, stream>>>(L, strikes, out, s.partials, s.ticket);
  return cudaGetLastError();
}

}  // namespace

size_t paths_scratch_doubles(const PathLaunch& L, int num_sms) {
  // at most 8 resident blocks of 256 threads per SM
  return (size_t)num_sms * 8 * (size_t)L.n_acc * L.nk_pad;
}

cudaError_t launch_paths(const PathLaunch& L, const double* strikes, const PathOutputs& out, const Scratch& s,
                         int num_sms, cudaStream_t stream, int* grid_used) {
  const bool one = L.nk_pad == 1;
  const bool v2 = L.n_v0_scen == 2;  // scenarios 1, 2 are the v0 bumps (constant deltas zero)
#define SIMR_LAUNCH(NS_, NV_, DYN_)                                                                \
  (one ? launch_t<NS_, NV_, 1, DYN_>(L, strikes, out, s, num_sms, stream, grid_used)               \
       : launch_t<NS_, NV_, 32, DYN_>(L, strikes, out, s, num_sms, stream, grid_used))
  if (L.scheme == 1) {  // QE-M: the base scenario alone, 5 or 11 scenarios in pairs, any other count dynamic
#define SIMR_LAUNCH_QEM(NS_, DYN_)                                                                     \
  (one ? launch_t<NS_, 0, 1, DYN_, true>(L, strikes, out, s, num_sms, stream, grid_used)               \
       : launch_t<NS_, 0, 32, DYN_, true>(L, strikes, out, s, num_sms, stream, grid_used))
    switch (L.n_scen) {
      case 1:
        return SIMR_LAUNCH_QEM(1, false);
      case 5:
        return SIMR_LAUNCH_QEM(5, false);
      case 11:
        return SIMR_LAUNCH_QEM(11, false);
      default:
        if (L.n_scen < 1 || L.n_scen > kMaxScen) return cudaErrorInvalidValue;
        return SIMR_LAUNCH_QEM(kMaxScen, true);
    }
#undef SIMR_LAUNCH_QEM
  }
  switch (L.n_scen) {
    case 1:
      return SIMR_LAUNCH(1, 0, false);
    case 3:
      return v2 ? SIMR_LAUNCH(3, 2, false) : SIMR_LAUNCH(3, 0, false);
    case 5:
      return v2 ? SIMR_LAUNCH(5, 2, false) : SIMR_LAUNCH(5, 0, false);
    case 11:  // all five re-simulated model-parameter Greeks
      return v2 ? SIMR_LAUNCH(11, 2, false) : SIMR_LAUNCH(11, 0, false);
    default:
      if (L.n_scen < 1 || L.n_scen > kMaxScen) return cudaErrorInvalidValue;
      return v2 ? SIMR_LAUNCH(kMaxScen, 2, true) : SIMR_LAUNCH(kMaxScen, 0, true);
  }
#undef SIMR_LAUNCH
}

cudaError_t launch_finalize(const PathLaunch& L, const double* sums, const PathOutputs& out, cudaStream_t stream) {
  const int tpb = 128;
  finalize_sums_kernel<<<(L.n_strikes + tpb - 1) / tpb, tpb, 0, stream>>>(L, sums, out);
  return cudaGetLastError();
}

cudaError_t launch_terminal(const PathLaunch& L, float* x_T, float* v_T, cudaStream_t stream) {
  const int tpb = 256;
  const uint64_t grid = (L.path_count + tpb - 1) / tpb;
  if (L.scheme == 1)
    heston_terminal_kernel<true><<<(unsigned)grid, tpb, 0, stream>>>(L, x_T, v_T);
  else
    heston_terminal_kernel<false><<<(unsigned)grid, tpb, 0, stream>>>(L, x_T, v_T);
  return cudaGetLastError();
}

}  // namespace simr
