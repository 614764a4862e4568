// simr_adjoint.cu -- pathwise adjoint (reverse-mode) Greeks of the Heston QE path, sm_103a.
//
// Per path (one lane): a forward pass of the variance recursion (Philox draws,
// QE variance step -- the paper's VariancePathQE, Sec. 4) that keeps the
// variance every `k` steps (a global [slot][resident thread] array), then a
// reverse sweep over the segments, last to first: each segment's states are
// recomputed from its checkpoint (the draws are counter-based, so the
// segment's draws are regenerated) and kept with the step's branch draw and Z_X
// -- in shared memory, or in a global [3 k][resident thread] buffer when the
// segment is longer than shared memory holds -- and the steps are
// differentiated backwards (LogPricePathQE's increments summed on the way),
// with the branch taken in the forward pass held fixed (pathwise derivative).
// With one segment of the whole path there is no forward pass at all: the
// recompute of that segment is the path's only simulation.  Since x' = x + (terms), the
// adjoint of x is 1 throughout; the sweep carries the adjoint of v and seven
// sums that the parameters enter through:
//   Am = sum mbar, Amv = sum mbar (v - theta), As = sum s2bar, Asv = sum s2bar v,
//   Ad = sum (theta - v), Adl = sum (v' - m), Ak3 = sum sqrt(v + v') Z_X,
// mapped once per path onto d x_T / d(v0, kappa, theta, sigma, rho) with
// FP64-derived constants.  Price sensitivities per strike (reduction over paths,
// Sec. 6): dP/dq = e^{-rT} mean[f'(S_T) S_T dx_T/dq], plus S_T/S0 for S0 and
// T - T P for r.  The terms are summed in FP32 over a warp's paths (one strike
// per lane for 32-strike tiles, a warp sum for one strike) and in FP64 on, as
// in the pricing kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "simr_device.cuh"
#include "simr_internal.h"
#include "simr_reduce.cuh"
#include "simr_adjoint_path.cuh"

namespace simr {
namespace {

#ifndef SIMR_ADJ_PPT
#define SIMR_ADJ_PPT 1  // paths per thread of the per-strike adjoint kernel (2 measured slower)
#endif
// Dynamic shared memory of the per-strike kernel: strike constants, the
// last-block flag, then the segment buffers (none when they are in global
// memory, GSEG); the per-warp FP64 accumulator rows come first when they live in
// shared memory throughout (RACC false), or reuse the segment buffers' space
// once the path loop has ended (RACC true: lane l accumulates strike l of the
// one 32-strike tile in registers).
inline size_t adjoint_smem_bytes_t(const PathLaunch& L, const AdjConst& A, int tpb, int ppt, bool racc,
                                   bool gseg = false) {
  const size_t acc_bytes = (size_t)(tpb / kWarp) * kAdjAcc * L.nk_pad * sizeof(double);
  const size_t buf_bytes = gseg ? 0 : adjoint_seg_floats(A, ppt) * tpb * sizeof(float);
  const size_t head = L.nk_pad * sizeof(StrikeConst) + 16;
  return racc ? head + (buf_bytes > acc_bytes ? buf_bytes : acc_bytes) : acc_bytes + head + buf_bytes;
}

// The per-strike terms of a 32-strike tile, lane l owning strike K (the
// tile's strike l): the warp's paths are broadcast one at a time -- terminal
// spot and d x_T / d(v0, kappa, theta, sigma, rho) -- and each lane adds its
// strike's payoff f, f^2, and the in-the-money weight w (S_T for a call above
// its strike, -S_T for a put below) alone and times each derivative; FP32 over
// the warp's paths.  out[0..8]: f, f^2, w, w dx/dv0 .. w dx/drho, the signed
// in-the-money indicator (the S0 column is w / S0, scaled when added to the FP64
// sums; the r column e^{-rT} T K times the indicator's mean, see adj_term).
template <int PPT>
__device__ __forceinline__ void strike_tile_terms(bool put, float K, const float (&S)[PPT], const bool (&act)[PPT],
                                                  const float (&g)[PPT][5], float (&out)[kAdjAcc]) {
#pragma unroll
  for (int a = 0; a < kAdjAcc; ++a) out[a] = 0.0f;
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const unsigned live = __ballot_sync(kFull, act[j]);
#pragma unroll 4
    for (int p = 0; p < kWarp; ++p) {
      const float Sp = __shfl_sync(kFull, S[j], p);
      float gp[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) gp[k] = __shfl_sync(kFull, g[j][k], p);
      if ((live >> p) & 1u) {  // warp-uniform
        const float f = put ? fmaxf(K - Sp, 0.0f) : fmaxf(Sp - K, 0.0f);
        const float w = put ? (Sp < K ? -Sp : 0.0f) : (Sp > K ? Sp : 0.0f);
        out[0] += f;
        out[1] = fmaf(f, f, out[1]);
        out[2] += w;
#pragma unroll
        for (int k = 0; k < 5; ++k) out[3 + k] = fmaf(w, gp[k], out[3 + k]);
        out[8] += put ? (Sp < K ? -1.0f : 0.0f) : (Sp > K ? 1.0f : 0.0f);
      }
    }
  }
}

// Minimum resident blocks per SM asked of the register allocator: 5 for global
// segments (one segment of the whole path: 4-5% faster than its own choice, 7%
// faster than 4), 4 for shared-memory segments (which hold a block's segment
// buffers, 12 k bytes per thread, so that longer segments leave room for 4
// blocks at most: 11% faster at k = 32 and 1% at k = 16 than with 5).
#ifndef SIMR_ADJ_MINB_GSEG
#define SIMR_ADJ_MINB_GSEG 5
#endif
#ifndef SIMR_ADJ_MINB_SMEM
#define SIMR_ADJ_MINB_SMEM 4
#endif

// GSEG: the segment buffers in global memory, [3 k][grid threads] (for a
// segment too long for shared memory, in particular one segment of the whole
// path: no forward pass).
// QEM: the QE-M log-spot step (the launch's scheme 1), differentiated one step
// at a time.
template <int TILE, int PPT, bool RACC, bool GSEG, bool QEM>
__global__ void __launch_bounds__(128, GSEG ? SIMR_ADJ_MINB_GSEG : SIMR_ADJ_MINB_SMEM) heston_adjoint_kernel(const __grid_constant__ PathLaunch L,
                                                             const __grid_constant__ AdjConst A,
                                                             const double* __restrict__ strikes, AdjOutputs out,
                                                             double* __restrict__ partials,
                                                             unsigned int* __restrict__ ticket,
                                                             float* __restrict__ gckpt, float* __restrict__ gseg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warps = blockDim.x / kWarp;
  const int bd = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
  const int row = kAdjAcc * L.nk_pad;
  const size_t acc_bytes = (size_t)warps * row * sizeof(double);
  const size_t ks_off = RACC ? 0 : acc_bytes;
  StrikeConst* ks = reinterpret_cast<StrikeConst*>(smem_raw + ks_off);
  int* s_last = reinterpret_cast<int*>(ks + L.nk_pad);
  float* sbuf = reinterpret_cast<float*>(s_last + 4);  // path_adjoint_ppt's segment buffers
  double* acc = RACC ? reinterpret_cast<double*>(sbuf) : reinterpret_cast<double*>(smem_raw);
  // checkpoints: this thread's column of a [slot][grid threads] global array
  float* ck = gckpt + (int)blockIdx.x * bd + tid;
  const int ck_stride = (int)(gridDim.x * blockDim.x);
  double racc[RACC ? kAdjAcc : 1];
#pragma unroll
  for (int a = 0; a < (RACC ? kAdjAcc : 1); ++a) racc[a] = 0.0;

  if (!RACC)
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
  const uint64_t per_batch = (uint64_t)kWarp * PPT;
  const uint64_t batches = (L.path_count + per_batch - 1) / per_batch;
  const uint64_t total_warps = (uint64_t)gridDim.x * warps;
  for (uint64_t bt = (uint64_t)blockIdx.x * warps + warp; bt < batches; bt += total_warps) {
    uint64_t pth[PPT];
    bool act[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const uint64_t local = bt * per_batch + (uint64_t)j * kWarp + lane;
      act[j] = local < L.path_count;
      pth[j] = L.path_begin + local;
    }
    float x[PPT], comp[PPT], g[PPT][5], S[PPT];
    if constexpr (GSEG)
      path_adjoint_ppt<PPT, SegGlobal, true, QEM>(
          L.sc[0], A, L.steps, L.option_index, L.rk, pth, ck, ck_stride,
          SegGlobal{gseg, (long long)blockIdx.x * bd + tid, A.ckpt_every, (long long)ck_stride}, x, comp, g, L.qm);
    else
      path_adjoint_ppt<PPT, SegShared, true, QEM>(L.sc[0], A, L.steps, L.option_index, L.rk, pth, ck, ck_stride,
                                                  SegShared{sbuf, A.ckpt_every}, x, comp, g, L.qm);
#pragma unroll
    for (int j = 0; j < PPT; ++j) S[j] = terminal_spot(L.S0, x[j], comp[j]);

    // per-strike terms, summed over the warp's paths
    if (RACC) {
      float t[kAdjAcc];
      strike_tile_terms<PPT>(put, ks[lane].K, S, act, g, t);
#pragma unroll
      for (int a = 0; a < kAdjAcc; ++a) racc[a] += (double)t[a];
    } else if (TILE == 1) {
      for (int a = 0; a < kAdjAcc; ++a) {
        float t = 0.0f;
#pragma unroll
        for (int j = 0; j < PPT; ++j) t += act[j] ? adj_term(a, put, S[j], ks[0].K, g[j], A.invS0, A.T) : 0.0f;
        t = warp_sum(t);
        if (lane == 0) my_acc[a] += (double)t;
      }
    } else {
      for (int t0 = 0; t0 < L.nk_pad; t0 += 32) {
        float t[kAdjAcc];
        strike_tile_terms<PPT>(put, ks[t0 + lane].K, S, act, g, t);
        double* row = my_acc + t0 + lane;
        row[0] += (double)t[0];
        row[(size_t)L.nk_pad] += (double)t[1];
        row[(size_t)2 * L.nk_pad] += (double)t[2] * (double)A.invS0;
#pragma unroll
        for (int a = 3; a < kAdjAcc; ++a) row[(size_t)a * L.nk_pad] += (double)t[a];
      }
    }
  }
  __syncthreads();
  if (RACC) {  // the segment buffers are free now: spill the lanes' sums into the rows
    // racc[2] holds the weights w: the S0 column is w / S0
    my_acc[lane] = racc[0];
    my_acc[(size_t)L.nk_pad + lane] = racc[1];
    my_acc[(size_t)2 * L.nk_pad + lane] = racc[2] * (double)A.invS0;
#pragma unroll
    for (int a = 3; a < kAdjAcc; ++a) my_acc[(size_t)a * L.nk_pad + lane] = racc[a];
    __syncthreads();
  }

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
      // e^{-rT} T K E[indicator] with the FP32 T and K the paths use (as the book does)
      if (c7 == 6) gsum *= (double)A.T * (double)(float)K;
      out.grad[(size_t)kk * 7 + c7] = bad ? nan : gsum;
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// Per-path output: x_T and g = d x_T / d(v0, kappa, theta, sigma, rho).
template <bool QEM>
__global__ void __launch_bounds__(128) heston_paths_adjoint_kernel(const __grid_constant__ PathLaunch L,
                                                                   const __grid_constant__ AdjConst A,
                                                                   float* __restrict__ x_T, float* __restrict__ grad) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int bd = blockDim.x, tid = threadIdx.x;
  float* ckpt = reinterpret_cast<float*>(smem_raw);
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.path_count) return;  // no block-wide synchronisation below
  float x[1], comp[1], g[1][5];
  const uint64_t pth[1] = {L.path_begin + i};
  path_adjoint_ppt<1, SegShared, true, QEM>(L.sc[0], A, L.steps, L.option_index, L.rk, pth, ckpt + tid, bd,
                                            SegShared{ckpt + (A.n_seg - 1) * bd, A.ckpt_every}, x, comp, g, L.qm);
  x_T[i] = x[0] - comp[0];
#pragma unroll
  for (int j = 0; j < 5; ++j) grad[i * 5 + j] = g[0][j];
}

// The grid of the per-strike kernel variant (resident blocks, at most what the
// paths need) and its dynamic shared memory.
template <int TILE, bool RACC, bool GSEG, bool QEM>
cudaError_t adjoint_grid_t(const PathLaunch& L, const AdjConst& A, int num_sms, uint64_t* grid, size_t* smem) {
  constexpr int PPT = SIMR_ADJ_PPT;
  const int tpb = 128, warps = tpb / kWarp;
  *smem = adjoint_smem_bytes_t(L, A, tpb, PPT, RACC, GSEG);
  auto kern = heston_adjoint_kernel<TILE, PPT, RACC, GSEG, QEM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tpb, *smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t batches = (L.path_count + (uint64_t)kWarp * PPT - 1) / ((uint64_t)kWarp * PPT);
  uint64_t g = (uint64_t)num_sms * per_sm;
  const uint64_t need = (batches + warps - 1) / warps;
  if (g > need) g = need;
  *grid = g < 1 ? 1 : g;
  return cudaSuccess;
}

template <int TILE, bool RACC, bool GSEG, bool QEM>
cudaError_t launch_adjoint_t(const PathLaunch& L, const AdjConst& A, const double* strikes, const AdjOutputs& out,
                             const Scratch& s, int num_sms, cudaStream_t stream) {
  constexpr int PPT = SIMR_ADJ_PPT;
  const int tpb = 128;
  const size_t row = (size_t)kAdjAcc * L.nk_pad;
  uint64_t grid = 0;
  size_t smem = 0;
  cudaError_t e = adjoint_grid_t<TILE, RACC, GSEG, QEM>(L, A, num_sms, &grid, &smem);
  if (e != cudaSuccess) return e;
  if ((size_t)grid * row > s.partial_doubles) return cudaErrorMemoryAllocation;
  if ((size_t)grid * tpb * adjoint_ckpt_floats(A, PPT) > s.ckpt_floats) return cudaErrorMemoryAllocation;
  if (GSEG && (size_t)grid * tpb * adjoint_seg_floats(A, PPT) > s.gseg_floats) return cudaErrorMemoryAllocation;
  heston_adjoint_kernel<TILE, PPT, RACC, GSEG, QEM>
      <<<(unsigned)grid, tpb, smem, stream>>>(L, A, strikes, out, s.partials, s.ticket, s.ckpt, s.gseg);
  return cudaGetLastError();
}

// Whether the segment buffers go to global memory: when 3 k floats per thread
// do not fit the shared memory of a block.  (Shared-memory segments are kept
// even where they cost resident blocks: at k = 32, 4 blocks per SM with
// shared-memory segments ran 11% faster than 5 with L2-resident global ones.)
bool adjoint_gseg(const PathLaunch& L, const AdjConst& A) {
  return adjoint_smem_bytes_t(L, A, 128, SIMR_ADJ_PPT, L.nk_pad == 32) > kAdjMaxSmem;
}

template <bool QEM>
cudaError_t launch_adjoint_s(const PathLaunch& L, const AdjConst& A, const double* strikes, const AdjOutputs& out,
                             const Scratch& s, int num_sms, cudaStream_t stream) {
  if (adjoint_gseg(L, A)) {
    if (L.nk_pad == 1) return launch_adjoint_t<1, false, true, QEM>(L, A, strikes, out, s, num_sms, stream);
    if (L.nk_pad == 32) return launch_adjoint_t<32, true, true, QEM>(L, A, strikes, out, s, num_sms, stream);
    return launch_adjoint_t<32, false, true, QEM>(L, A, strikes, out, s, num_sms, stream);
  }
  if (L.nk_pad == 1) return launch_adjoint_t<1, false, false, QEM>(L, A, strikes, out, s, num_sms, stream);
  if (L.nk_pad == 32) return launch_adjoint_t<32, true, false, QEM>(L, A, strikes, out, s, num_sms, stream);
  return launch_adjoint_t<32, false, false, QEM>(L, A, strikes, out, s, num_sms, stream);
}

}  // namespace

size_t adjoint_scratch_doubles(const PathLaunch& L, int num_sms) {
  return (size_t)num_sms * 16 * kAdjAcc * (size_t)L.nk_pad;  // at most 16 resident blocks of 128 threads per SM
}

cudaError_t adjoint_max_ckpt_every(const PathLaunch& L, int steps_cap, int* k_max) {
  // the kernel variant launch_adjoint picks for this strike count
  const bool racc = L.nk_pad == 32;
  const void* kern = L.nk_pad == 1 ? (const void*)heston_adjoint_kernel<1, SIMR_ADJ_PPT, false, false, false>
                     : racc      ? (const void*)heston_adjoint_kernel<32, SIMR_ADJ_PPT, true, false, false>
                                 : (const void*)heston_adjoint_kernel<32, SIMR_ADJ_PPT, false, false, false>;
  auto blocks = [&](int k, int* n) -> cudaError_t {
    AdjConst A{};
    A.ckpt_every = k;
    const size_t smem = adjoint_smem_bytes_t(L, A, 128, SIMR_ADJ_PPT, racc);
    *n = 0;
    if (smem > kAdjMaxSmem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, kern, 128, smem);
  };
  int best = 0;
  cudaError_t e = blocks(2, &best);
  if (e != cudaSuccess) return e;
  if (best < 1) return cudaErrorInvalidConfiguration;
  // blocks per SM fall as k grows: the largest even k that keeps `best`
  int lo = 1, hi = (steps_cap + 1) / 2 + 1;  // k = 2 lo keeps it; k = 2 hi is past the cap
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    int n = 0;
    if ((e = blocks(2 * mid, &n)) != cudaSuccess) return e;
    (n >= best ? lo : hi) = mid;
  }
  *k_max = 2 * lo;
  return cudaSuccess;
}

size_t adjoint_smem_bytes(const PathLaunch& L, const AdjConst& A) {
  return adjoint_smem_bytes_t(L, A, 128, SIMR_ADJ_PPT, L.nk_pad == 32, adjoint_gseg(L, A));
}

cudaError_t adjoint_gseg_floats(const PathLaunch& L, const AdjConst& A, int num_sms, size_t* floats) {
  *floats = 0;
  if (!adjoint_gseg(L, A)) return cudaSuccess;
  uint64_t grid = 0;
  size_t smem = 0;
  cudaError_t e = L.nk_pad == 1    ? adjoint_grid_t<1, false, true, false>(L, A, num_sms, &grid, &smem)
                  : L.nk_pad == 32 ? adjoint_grid_t<32, true, true, false>(L, A, num_sms, &grid, &smem)
                                   : adjoint_grid_t<32, false, true, false>(L, A, num_sms, &grid, &smem);
  if (e == cudaSuccess && L.scheme == 1) {  // the QE-M kernel's occupancy may differ: take the larger grid
    uint64_t grid_q = 0;
    e = L.nk_pad == 1    ? adjoint_grid_t<1, false, true, true>(L, A, num_sms, &grid_q, &smem)
        : L.nk_pad == 32 ? adjoint_grid_t<32, true, true, true>(L, A, num_sms, &grid_q, &smem)
                         : adjoint_grid_t<32, false, true, true>(L, A, num_sms, &grid_q, &smem);
    if (grid_q > grid) grid = grid_q;
  }
  if (e == cudaSuccess) *floats = (size_t)grid * 128 * adjoint_seg_floats(A, SIMR_ADJ_PPT);
  return e;
}

size_t adjoint_ckpt_scratch_floats(const AdjConst& A, int num_sms) {
  // at most 16 resident blocks of 128 threads per SM
  return (size_t)num_sms * 16 * 128 * adjoint_ckpt_floats(A, SIMR_ADJ_PPT);
}

cudaError_t launch_paths_adjoint(const PathLaunch& L, const AdjConst& A, float* x_T, float* grad, cudaStream_t stream) {
  const int tpb = 128;
  const size_t smem = (size_t)adjoint_thread_floats(A.n_seg, A.ckpt_every, 1) * tpb * sizeof(float);
  auto kern = L.scheme == 1 ? heston_paths_adjoint_kernel<true> : heston_paths_adjoint_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const uint64_t grid = (L.path_count + tpb - 1) / tpb;
  kern<<<(unsigned)grid, tpb, smem, stream>>>(L, A, x_T, grad);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const PathLaunch& L, const AdjConst& A, const double* strikes, const AdjOutputs& out,
                           const Scratch& s, int num_sms, cudaStream_t stream) {
  if (L.scheme == 1) return launch_adjoint_s<true>(L, A, strikes, out, s, num_sms, stream);
  return launch_adjoint_s<false>(L, A, strikes, out, s, num_sms, stream);
}

}  // namespace simr
