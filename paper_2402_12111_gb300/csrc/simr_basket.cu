// simr_basket.cu -- basket options on correlated Heston assets, sm_103a.
//
// The paper's A assets (Sec. 5, Table 1) each run the VariancePathQE /
// LogPricePathQE / AssetPathExponential stages; here A <= 16 assets of one
// basket are simulated together, one path per thread: asset k uses its own
// model and the Philox counters of option index k (so with no correlation it is
// exactly simr_price's path of option k), except that its log-spot normal is
// z_k = sum_{j <= k} Lc[k][j] eps_j, eps_j the Phi^-1(U_X) of asset j, Lc the
// lower Cholesky factor of the correlation of the spot drivers; the variance
// drivers stay independent.  Payoff on B_T = sum_k w_k S_T,k per strike, and
// the reduction over paths of the price kernel (FP32 over a warp, FP64 on).
// Assets run in pairs, (k, k + 1) in the two halves of packed FP32 (.f32x2)
// operations that round lane for lane as the scalar step; an odd count's last
// asset runs alone in scalar FP32.
#include <cuda_runtime.h>

#include <cstdint>

#include "simr_device.cuh"
#include "simr_internal.h"
#include "simr_reduce.cuh"

namespace simr {
namespace {

constexpr int kBasketTpb = 256;

// step_base<false> of two assets at once in packed FP32, lane for lane the
// scalar step's operations and rounding.
__device__ __forceinline__ void step_pair(const ScenConst2& c, float2 xv, float2 zv, float2 zx, float2& v, float2& x,
                                          float2& comp) {
  float2 vn, dl;
  qe_from_moments2(p_fma(v, c.E, c.thE), p_fma(v, c.h1, c.h2), xv, zv, vn, dl);
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

// step_qem of two assets at once (their own constants and A lane by lane), lane
// for lane the scalar step's operations and rounding.  An asset's log-spot
// normal z_k is standard normal and independent of its own variance path, so
// its martingale correction is the single-asset one.
__device__ __forceinline__ void step_pair_qem(const ScenConst2& c, const QemConst2& q, float2 xv, float2 zv,
                                              float2 zx, float2& v, float2& x, float2& comp) {
  const float2 m = p_fma(v, c.E, c.thE);
  const float2 s2h = p_fma(v, c.h1, c.h2);
  float2 vn, dl, lam;
  bool okx, oky;
  qem_from_moments2(m, s2h, xv, zv, q.A, vn, dl, lam, okx, oky);
  const float2 s = p_add(v, vn);
  float2 inc;
  if (okx && oky) {
    inc = p_sub(p_fma(p_mul(p_bc(-1.0f), q.qa), p_add(v, m), q.rdt), lam);
    inc = p_fma(q.K2, dl, inc);
  } else {
    const float vv[2] = {v.x, v.y}, mm[2] = {m.x, m.y}, ss[2] = {s.x, s.y}, dd[2] = {dl.x, dl.y},
                ll[2] = {lam.x, lam.y};
    const float qa[2] = {q.qa.x, q.qa.y}, rdt[2] = {q.rdt.x, q.rdt.y}, K2[2] = {q.K2.x, q.K2.y};
    const float C0[2] = {c.C0.x, c.C0.y}, Cv[2] = {c.Cv.x, c.Cv.y}, mCd[2] = {c.mCd.x, c.mCd.y},
                Cdl[2] = {c.Cdl.x, c.Cdl.y};
    const bool ok[2] = {okx, oky};
    float r[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (ok[j]) {
        r[j] = __fmaf_rn(K2[j], dd[j], __fsub_rn(__fmaf_rn(-qa[j], __fadd_rn(vv[j], mm[j]), rdt[j]), ll[j]));
      } else {
        float t = __fmaf_rn(Cv[j], ss[j], C0[j]);
        t = __fmaf_rn(mCd[j], vv[j], t);
        r[j] = __fmaf_rn(Cdl[j], dd[j], t);
      }
    }
    inc = make_float2(r[0], r[1]);
  }
  inc = p_fma(p_mul(c.sK3, p_sqrt(s)), zx, inc);
  const float2 y = p_sub(inc, comp);
  const float2 t2 = p_add(x, y);
  comp = p_sub(p_sub(t2, x), y);
  x = t2;
  v = vn;
}

// One step of the asset pair (k, k + 1) from their variance uniforms (centred)
// and spot uniforms' normals eps[0 .. k + 1]: z = Lc eps over the rows k, k + 1,
// summed in column order as for one asset at a time.
template <int NA, bool QEM>
__device__ __forceinline__ void basket_pair_step(const BasketLaunch& L, const ScenConst2& c, int k, float2 xv,
                                                 const float (&eps)[NA], float2& v, float2& x, float2& comp) {
  const float* ra = L.Lc + k * (k + 1) / 2;
  const float* rb = ra + k + 1;  // row k + 1
  float2 z = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    if (j > k) break;
    z = p_fma(make_float2(ra[j], rb[j]), p_bc(eps[j]), z);
  }
  z.y = __fmaf_rn(rb[k + 1], eps[k + 1], z.y);
  const float2 zv = norminv_centered2(xv);
  if constexpr (QEM)
    step_pair_qem(c, L.qk[k / 2], xv, zv, z, v, x, comp);
  else
    step_pair(c, xv, zv, z, v, x, comp);
}

// One step of the lone last asset k of an odd count (k only known at run
// time, its state in plain registers) from its variance uniform (centred), the
// pairs' eps[0 .. k - 1] and its own e, as one lane of basket_pair_step.
template <int NA, bool QEM>
__device__ __forceinline__ void basket_lone_step(const BasketLaunch& L, int k, float xv, const float (&eps)[NA],
                                                 float e, float& v, float& x, float& comp) {
  const float* ra = L.Lc + k * (k + 1) / 2;
  float z = 0.0f;
#pragma unroll
  for (int j = 0; j < NA; ++j)
    if (j < k) z = __fmaf_rn(ra[j], eps[j], z);
  z = __fmaf_rn(ra[k], e, z);
  step_scheme<false, QEM>(L.sc[k], L.qm[k], xv, norminv_centered(xv), z, v, x, comp);
}

template <int NA, int TILE, bool QEM>
__global__ void __launch_bounds__(kBasketTpb) heston_basket_kernel(const __grid_constant__ BasketLaunch L,
                                                                   const double* __restrict__ strikes,
                                                                   BasketOutputs out, double* __restrict__ partials,
                                                                   unsigned int* __restrict__ ticket) {
  static_assert(NA % 2 == 0, "assets are stepped in pairs");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warps = blockDim.x / kWarp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row = 2 * L.nk_pad;
  double* acc = reinterpret_cast<double*>(smem_raw);
  float* ks = reinterpret_cast<float*>(acc + (size_t)warps * row);
  int* s_last = reinterpret_cast<int*>(ks + L.nk_pad);
  for (int i = threadIdx.x; i < warps * row; i += blockDim.x) acc[i] = 0.0;
  for (int j = threadIdx.x; j < L.nk_pad; j += blockDim.x) {
    float K = 0.0f;
    if (j < L.n_strikes) {
      const double Kd = strikes[j];
      if (!(Kd >= 0.0) || !isfinite(Kd)) atomicOr(out.status, 1);
      K = (float)Kd;
    }
    ks[j] = K;
  }
  __syncthreads();

  const bool put = L.is_put != 0;
  const int na = L.n_assets;
  const int kl = na - 1;  // the lone last asset when na is odd
  double* my_acc = acc + (size_t)warp * row;
  const uint64_t batches = (L.paths + kWarp - 1) / kWarp;
  const uint64_t total_warps = (uint64_t)gridDim.x * warps;
  for (uint64_t bt = (uint64_t)blockIdx.x * warps + warp; bt < batches; bt += total_warps) {
    const uint64_t path = bt * kWarp + lane;
    const bool active = path < L.paths;
    const PhiloxLane pl = philox_lane(path, L.rk);  // shared by the assets' counters
    float2 v[NA / 2], x[NA / 2], comp[NA / 2];  // the pairs
    float eps[NA];
    uint32_t wz[NA], ww[NA];  // the odd step's words of each asset
    float vl = L.sc[kl].v0, xl = 0.0f, cl = 0.0f;  // the lone asset (odd counts)
    uint32_t wzl = 0u, wwl = 0u;
#pragma unroll
    for (int q = 0; q < NA / 2; ++q) {
      v[q] = make_float2(L.sc[2 * q].v0, L.sc[2 * q + 1].v0);
      x[q] = make_float2(0.0f, 0.0f);
      comp[q] = make_float2(0.0f, 0.0f);
    }
    for (uint32_t p = 0; 2 * p < L.steps; ++p) {
      // even step 2p: draw each pair's words, correlate, step in pair order (an
      // odd count's last asset alone)
#pragma unroll
      for (int q = 0; q < NA / 2; ++q) {
        const int k = 2 * q;
        if (k + 1 >= na) break;
        const uint4 wa = philox_draw(pl, philox_ctr(p, (uint32_t)k, L.rk), L.rk);
        const uint4 wb = philox_draw(pl, philox_ctr(p, (uint32_t)(k + 1), L.rk), L.rk);
        wz[k] = wa.z;
        ww[k] = wa.w;
        wz[k + 1] = wb.z;
        ww[k + 1] = wb.w;
        const float2 e = norminv_centered2(centered_uniform2(wa.y, wb.y));
        eps[k] = e.x;
        eps[k + 1] = e.y;
        basket_pair_step<NA, QEM>(L, L.pk[q], k, centered_uniform2(wa.x, wb.x), eps, v[q], x[q], comp[q]);
      }
      if (na & 1) {
        const uint4 w = philox_draw(pl, philox_ctr(p, (uint32_t)kl, L.rk), L.rk);
        wzl = w.z;
        wwl = w.w;
        basket_lone_step<NA, QEM>(L, kl, centered_uniform(w.x), eps, norminv_centered(centered_uniform(w.y)), vl, xl, cl);
      }
      if (2 * p + 1 < L.steps) {
#pragma unroll
        for (int q = 0; q < NA / 2; ++q) {
          const int k = 2 * q;
          if (k + 1 >= na) break;
          const float2 e = norminv_centered2(centered_uniform2(ww[k], ww[k + 1]));
          eps[k] = e.x;
          eps[k + 1] = e.y;
          basket_pair_step<NA, QEM>(L, L.pk[q], k, centered_uniform2(wz[k], wz[k + 1]), eps, v[q], x[q], comp[q]);
        }
        if (na & 1)
          basket_lone_step<NA, QEM>(L, kl, centered_uniform(wzl), eps, norminv_centered(centered_uniform(wwl)), vl, xl,
                               cl);
      }
    }
    float B = 0.0f;  // sum_k w_k S0_k e^{x_k}
#pragma unroll
    for (int q = 0; q < NA / 2; ++q) {
      if (2 * q + 1 >= na) break;
      B += terminal_spot(L.S0w[2 * q], x[q].x, comp[q].x);
      B += terminal_spot(L.S0w[2 * q + 1], x[q].y, comp[q].y);
    }
    if (na & 1) B += terminal_spot(L.S0w[kl], xl, cl);

    if (TILE == 1) {
      const float f = active ? (put ? fmaxf(ks[0] - B, 0.0f) : fmaxf(B - ks[0], 0.0f)) : 0.0f;
      const float t0 = warp_sum(f), t1 = warp_sum(f * f);
      if (lane == 0) {
        my_acc[0] += (double)t0;
        my_acc[1] += (double)t1;
      }
    } else {
      for (int t0 = 0; t0 < L.nk_pad; t0 += 32) {
        float vf[32], vq[32];
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const float K = ks[t0 + jj];
          const float f = active ? (put ? fmaxf(K - B, 0.0f) : fmaxf(B - K, 0.0f)) : 0.0f;
          vf[jj] = f;
          vq[jj] = f * f;
        }
        butterfly32(vf, lane);
        butterfly32(vq, lane);
        my_acc[t0 + lane] += (double)vf[0];
        my_acc[L.nk_pad + t0 + lane] += (double)vq[0];
      }
    }
  }
  __syncthreads();

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
  for (int i = threadIdx.x; i < row; i += blockDim.x) {
    double s = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(partials + (size_t)b * row + i);
    acc[i] = s;
  }
  __syncthreads();
  const double inv_n = 1.0 / L.paths_total;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  for (int k = threadIdx.x; k < L.n_strikes; k += blockDim.x) {
    const double K = strikes[k];
    const bool bad = !(K >= 0.0) || !isfinite(K);
    const double mean = acc[k] * inv_n;
    out.price[k] = bad ? nan : L.disc * mean;
    if (out.stderr_) {
      const double n = L.paths_total;
      const double var = n > 1.0 ? (acc[L.nk_pad + k] * inv_n - mean * mean) / (n - 1.0) : 0.0;
      out.stderr_[k] = bad ? nan : L.disc * sqrt(var > 0.0 ? var : 0.0);
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

template <int NA, int TILE, bool QEM>
cudaError_t launch_basket_t(const BasketLaunch& L, const double* strikes, const BasketOutputs& out,
                            double* partials, size_t partial_doubles, unsigned int* ticket, int num_sms,
                            cudaStream_t stream) {
  const int warps = kBasketTpb / kWarp;
  const size_t row = 2 * (size_t)L.nk_pad;
  const size_t smem = warps * row * sizeof(double) + L.nk_pad * sizeof(float) + 16;
  auto kern = heston_basket_kernel<NA, TILE, QEM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBasketTpb, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t batches = (L.paths + kWarp - 1) / kWarp;
  uint64_t grid = (uint64_t)num_sms * per_sm;
  const uint64_t need = (batches + warps - 1) / warps;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  if ((size_t)grid * row > partial_doubles) return cudaErrorMemoryAllocation;
  kern<<<(unsigned)grid, kBasketTpb, smem, stream>>>(L, strikes, out, partials, ticket);
  return cudaGetLastError();
}

template <int NA>
cudaError_t launch_basket_na(const BasketLaunch& L, const double* strikes, const BasketOutputs& out,
                             double* partials, size_t partial_doubles, unsigned int* ticket, int num_sms,
                             cudaStream_t stream) {
  if (L.scheme == 1)
    return L.nk_pad == 1
               ? launch_basket_t<NA, 1, true>(L, strikes, out, partials, partial_doubles, ticket, num_sms, stream)
               : launch_basket_t<NA, 32, true>(L, strikes, out, partials, partial_doubles, ticket, num_sms, stream);
  return L.nk_pad == 1
             ? launch_basket_t<NA, 1, false>(L, strikes, out, partials, partial_doubles, ticket, num_sms, stream)
             : launch_basket_t<NA, 32, false>(L, strikes, out, partials, partial_doubles, ticket, num_sms, stream);
}

}  // namespace

size_t basket_partial_doubles(const BasketLaunch& L, int num_sms) {
  return (size_t)num_sms * 8 * 2 * (size_t)L.nk_pad;  // at most 8 resident blocks per SM
}

cudaError_t launch_basket(const BasketLaunch& L, const double* strikes, const BasketOutputs& out, double* partials,
                          size_t partial_doubles, unsigned int* ticket, int num_sms, cudaStream_t stream) {
  if (L.n_assets <= 2) return launch_basket_na<2>(L, strikes, out, partials, partial_doubles, ticket, num_sms, stream);
  if (L.n_assets <= 4) return launch_basket_na<4>(L, strikes, out, partials, partial_doubles, ticket, num_sms, stream);
  if (L.n_assets <= 8) return launch_basket_na<8>(L, strikes, out, partials, partial_doubles, ticket, num_sms, stream);
  return launch_basket_na<kMaxAssets>(L, strikes, out, partials, partial_doubles, ticket, num_sms, stream);
}

}  // namespace simr
