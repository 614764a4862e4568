// simr_adjoint.cu -- pathwise adjoint (reverse-mode) Greeks of the Heston QE path, sm_103a.
//
// Per path (one lane): a forward pass (Philox draws, QE variance step, log-spot
// step -- the paper's VariancePathQE and LogPricePathQE, Sec. 4-5) that keeps
// the variance every `k` steps in shared memory, then a reverse sweep over the
// segments, last to first: each segment's states are recomputed from its
// checkpoint (the draws are counter-based, so the segment's draws are
// regenerated and kept in shared memory with the states) and the steps are
// differentiated backwards, with the branch taken in the forward pass held
// fixed (pathwise derivative).  Since x' = x + (terms), the
// adjoint of x is 1 throughout; the sweep carries the adjoint of v and seven
// sums that the parameters enter through:
//   Am = sum mbar, Amv = sum mbar (v - theta), As = sum s2bar, Asv = sum s2bar v,
//   Ad = sum (theta - v), Adl = sum (v' - m), Ak3 = sum sqrt(v + v') Z_X,
// mapped once per path onto d x_T / d(v0, kappa, theta, sigma, rho) with
// FP64-derived constants.  Price sensitivities per strike (reduction over paths,
// Sec. 6): dP/dq = e^{-rT} mean[f'(S_T) S_T dx_T/dq], plus S_T/S0 for S0 and
// T - T P for r.  Same FP32-butterfly / FP64 reduction as the pricing kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "simr_device.cuh"
#include "simr_internal.h"
#include "simr_reduce.cuh"

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

// Forward pass with checkpoints, then the reverse sweep, for one path: x_T (with
// its Kahan remainder) and g = d x_T / d(v0, kappa, theta, sigma, rho).
// ckpt: [n_seg][bd] and seg: [3][k][bd] shared-memory slices of this block; the
// recompute pass of a segment keeps the segment's states and draws there, so
// the reverse sweep regenerates nothing.
__device__ __forceinline__ void path_adjoint(const PathLaunch& L, const AdjConst& A, uint64_t path, float* ckpt,
                                             float* seg, int bd, int tid, float& x_out, float& comp_out,
                                             float (&g)[5]) {
  const ScenConst& c = L.sc[0];
  const float theta = A.theta;
  const uint32_t N = L.steps, k = (uint32_t)A.ckpt_every;
  const uint32_t plo = (uint32_t)path, phi = (uint32_t)(path >> 32);
  float* seg_v = seg;
  float* seg_d = seg + (size_t)k * bd;
  float* seg_zx = seg + (size_t)2 * k * bd;

  // forward pass with checkpoints (k is even, so checkpoints fall on even steps)
  float v = c.v0, x = 0.0f, comp = 0.0f;
  for (uint32_t p = 0; 2 * p < N; ++p) {
    const uint4 w = philox4x32_10(p, plo, phi, L.option_index, L.rk);
    const uint32_t n = 2 * p;
    if (n % k == 0) ckpt[(n / k) * bd + tid] = v;
    {
      const float xv = centered_uniform(w.x);
      step_base<false>(c, 0.5f * (1.0f - xv), norminv_centered(xv), norminv_centered(centered_uniform(w.y)), v, x,
                       comp);
    }
    if (n + 1 < N) {
      const float xv = centered_uniform(w.z);
      step_base<false>(c, 0.5f * (1.0f - xv), norminv_centered(xv), norminv_centered(centered_uniform(w.w)), v, x,
                       comp);
    }
  }
  x_out = x;
  comp_out = comp;

  // reverse sweep, segment by segment
  AdjSums as{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  for (int j = A.n_seg - 1; j >= 0; --j) {
    const uint32_t n0 = (uint32_t)j * k, n1 = min(n0 + k, N);
    float vv = ckpt[j * bd + tid];
    for (uint32_t p = n0 / 2; 2 * p < n1; ++p) {  // recompute v_n0 .. v_n1 and keep the draws
      const uint4 w = philox4x32_10(p, plo, phi, L.option_index, L.rk);
      const uint32_t i = 2 * p - n0;
      {
        const float xv = centered_uniform(w.x);
        const float omu = 0.5f * (1.0f - xv), zv = norminv_centered(xv);
        seg_v[i * bd + tid] = vv;
        seg_d[i * bd + tid] = branch_draw(c, vv, omu, zv);
        seg_zx[i * bd + tid] = norminv_centered(centered_uniform(w.y));
        vv = qe_only(c, vv, omu, zv);
      }
      if (2 * p + 1 < n1) {
        const float xv = centered_uniform(w.z);
        const float omu = 0.5f * (1.0f - xv), zv = norminv_centered(xv);
        seg_v[(i + 1) * bd + tid] = vv;
        seg_d[(i + 1) * bd + tid] = branch_draw(c, vv, omu, zv);
        seg_zx[(i + 1) * bd + tid] = norminv_centered(centered_uniform(w.w));
        vv = qe_only(c, vv, omu, zv);
      }
    }
    float vnext = vv;  // v_{n1}
    for (int i = (int)(n1 - n0) - 1; i >= 0; --i) {
      const float vc = seg_v[i * bd + tid];
      adjoint_step(c, theta, vc, vnext, seg_d[i * bd + tid], seg_zx[i * bd + tid], as);
      vnext = vc;
    }
  }
  const double Amv = as.Amv, Asv = as.Asv, As = as.As, Ad = as.Ad, Adl = as.Adl, Am = as.Am, Ak3 = as.Ak3;
  g[0] = as.vbar;
  g[1] = (float)(A.dE_dk * Amv + A.dc1_dk * Asv + A.dc2_dk * As + A.dCd_dk * Ad + A.dCdl_dk * Adl);
  g[2] = (float)(A.omE * Am + A.dc2_dth * As + A.N_Cd);
  g[3] = (float)(A.two_over_sigma * (A.c1 * Asv + A.c2 * As) - A.Cd_over_sigma * Ad - A.Cdl_over_sigma * Adl);
  g[4] = (float)(A.D_over_sigma * Ad + A.B_over_sigma * Adl + A.dsK3_drho * Ak3);
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

template <int TILE>
__global__ void __launch_bounds__(128) heston_adjoint_kernel(const __grid_constant__ PathLaunch L,
                                                             const __grid_constant__ AdjConst A,
                                                             const double* __restrict__ strikes, AdjOutputs out,
                                                             double* __restrict__ partials,
                                                             unsigned int* __restrict__ ticket) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warps = blockDim.x / kWarp;
  const int bd = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
  const int row = kAdjAcc * L.nk_pad;
  double* acc = reinterpret_cast<double*>(smem_raw);
  StrikeConst* ks = reinterpret_cast<StrikeConst*>(acc + (size_t)warps * row);
  int* s_last = reinterpret_cast<int*>(ks + L.nk_pad);
  float* ckpt = reinterpret_cast<float*>(s_last + 4);  // [n_seg][bd]
  float* seg = ckpt + (size_t)A.n_seg * bd;             // [4][k][bd]: v, 1 - U_V, Z_V, Z_X

  for (int i = threadIdx.x; i < warps * row; i += blockDim.x) acc[i] = 0.0;
  for (int j = threadIdx.x; j < L.nk_pad; j += blockDim.x) {
    StrikeConst k{0.0f, 0.0f, 0.0f, 0.0f};
    if (j < L.n_strikes) {
      const double K = strikes[j];
      if (!(K > 0.0) || !isfinite(K)) atomicOr(out.status, 1);
      k.K = (float)K;
    }
    ks[j] = k;
  }
  __syncthreads();

  const bool put = L.is_put != 0;
  double* my_acc = acc + (size_t)warp * row;
  const uint64_t batches = (L.path_count + kWarp - 1) / kWarp;
  const uint64_t total_warps = (uint64_t)gridDim.x * warps;
  for (uint64_t bt = (uint64_t)blockIdx.x * warps + warp; bt < batches; bt += total_warps) {
    const uint64_t local = bt * kWarp + lane;
    const bool active = local < L.path_count;
    float x, comp, g[5];
    path_adjoint(L, A, L.path_begin + local, ckpt, seg, bd, tid, x, comp, g);
    const float S = terminal_spot(L.S0, x, comp);

    // per-strike terms, reduced over the warp's 32 paths
    for (int a = 0; a < kAdjAcc; ++a) {
      if (TILE == 1) {
        float t = adj_term(a, put, S, ks[0].K, g, A.invS0, A.T);
        t = warp_sum(active ? t : 0.0f);
        if (lane == 0) my_acc[a] += (double)t;
      } else {
        for (int t0 = 0; t0 < L.nk_pad; t0 += 32) {
          float vals[32];
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const float t = adj_term(a, put, S, ks[t0 + jj].K, g, A.invS0, A.T);
            vals[jj] = active ? t : 0.0f;
          }
          butterfly32(vals, lane);
          my_acc[(size_t)a * L.nk_pad + t0 + lane] += (double)vals[0];
        }
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
  for (int kk = threadIdx.x; kk < L.n_strikes; kk += blockDim.x) {
    const double K = strikes[kk];
    const bool bad = !(K > 0.0) || !isfinite(K);
    const double mean = acc[kk] * inv_n;
    const double price = L.disc * mean;
    out.price[kk] = bad ? nan : price;
    if (out.stderr_) {
      const double n = L.paths_total;
      const double var = n > 1.0 ? (acc[L.nk_pad + kk] * inv_n - mean * mean) / (n - 1.0) : 0.0;
      out.stderr_[kk] = bad ? nan : L.disc * sqrt(var > 0.0 ? var : 0.0);
    }
    for (int c7 = 0; c7 < 7; ++c7) {
      double gsum = L.disc * acc[(size_t)(2 + c7) * L.nk_pad + kk] * inv_n;
      if (c7 == 6) gsum -= (double)A.T * price;
      out.grad[(size_t)kk * 7 + c7] = bad ? nan : gsum;
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// Per-path output: x_T and g = d x_T / d(v0, kappa, theta, sigma, rho).
__global__ void __launch_bounds__(128) heston_paths_adjoint_kernel(const __grid_constant__ PathLaunch L,
                                                                   const __grid_constant__ AdjConst A,
                                                                   float* __restrict__ x_T, float* __restrict__ grad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int bd = blockDim.x, tid = threadIdx.x;
  float* ckpt = reinterpret_cast<float*>(smem_raw);
  float* seg = ckpt + (size_t)A.n_seg * bd;
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.path_count) return;  // no block-wide synchronisation below
  float x, comp, g[5];
  path_adjoint(L, A, L.path_begin + i, ckpt, seg, bd, tid, x, comp, g);
  x_T[i] = x - comp;
#pragma unroll
  for (int j = 0; j < 5; ++j) grad[i * 5 + j] = g[j];
}

template <int TILE>
cudaError_t launch_adjoint_t(const PathLaunch& L, const AdjConst& A, const double* strikes, const AdjOutputs& out,
                             const Scratch& s, int num_sms, cudaStream_t stream) {
  const int tpb = 128, warps = tpb / kWarp;
  const size_t row = (size_t)kAdjAcc * L.nk_pad;
  const size_t smem = warps * row * sizeof(double) + L.nk_pad * sizeof(StrikeConst) + 16 +
                      (size_t)(A.n_seg + 3 * A.ckpt_every) * tpb * sizeof(float);
  auto kern = heston_adjoint_kernel<TILE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tpb, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t batches = (L.path_count + kWarp - 1) / kWarp;
  uint64_t grid = (uint64_t)num_sms * per_sm;
  const uint64_t need = (batches + warps - 1) / warps;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  if ((size_t)grid * row > s.partial_doubles) return cudaErrorMemoryAllocation;
  kern<<<(unsigned)grid, tpb, smem, stream>>>(L, A, strikes, out, s.partials, s.ticket);
  return cudaGetLastError();
}

}  // namespace

size_t adjoint_scratch_doubles(const PathLaunch& L, int num_sms) {
  return (size_t)num_sms * 16 * kAdjAcc * (size_t)L.nk_pad;  // at most 16 resident blocks of 128 threads per SM
}

size_t adjoint_smem_bytes(const PathLaunch& L, const AdjConst& A) {
  const size_t row = (size_t)kAdjAcc * L.nk_pad;
  return 4 * row * sizeof(double) + L.nk_pad * sizeof(StrikeConst) + 16 +
         (size_t)(A.n_seg + 3 * A.ckpt_every) * 128 * sizeof(float);
}

cudaError_t launch_paths_adjoint(const PathLaunch& L, const AdjConst& A, float* x_T, float* grad, cudaStream_t stream) {
  const int tpb = 128;
  const size_t smem = (size_t)(A.n_seg + 3 * A.ckpt_every) * tpb * sizeof(float);
  cudaError_t e =
      cudaFuncSetAttribute(heston_paths_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const uint64_t grid = (L.path_count + tpb - 1) / tpb;
  heston_paths_adjoint_kernel<<<(unsigned)grid, tpb, smem, stream>>>(L, A, x_T, grad);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const PathLaunch& L, const AdjConst& A, const double* strikes, const AdjOutputs& out,
                           const Scratch& s, int num_sms, cudaStream_t stream) {
  return L.nk_pad == 1 ? launch_adjoint_t<1>(L, A, strikes, out, s, num_sms, stream)
                       : launch_adjoint_t<32>(L, A, strikes, out, s, num_sms, stream);
}

}  // namespace simr
