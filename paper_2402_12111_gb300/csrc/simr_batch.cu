// simr_batch.cu -- a heterogeneous book of European options in one persistent launch (sm_103a).
//
// Each option has its own model, maturity, steps and paths.  The host cuts every
// option's path range into items of `chunk` paths, longest options first; the
// persistent kernel's warps take items from an atomic ticket until the queue is
// empty, simulate their paths (the paper's VariancePathQE / LogPricePathQE /
// AssetPathExponential stages, Sec. 4-5, one lane per path, the option index as
// the fourth Philox counter word) and write one FP64 partial row per item; a
// second kernel sums each option's rows in item order (the reduction over paths
// of Sec. 6) and normalises.  Adjoint books run the per-path reverse sweep of
// simr_adjoint_path.cuh instead and add the 7 sensitivities.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "simr_adjoint_path.cuh"
#include "simr_device.cuh"
#include "simr_internal.h"
#include "simr_reduce.cuh"

namespace simr {
namespace {

// GSEG (adjoint books): every option is one segment of its whole path (no
// forward pass), kept in a grid-wide buffer in global memory.  The tunable
// shape: TPB threads per block; PPT paths per thread (price books: 2 stepped
// together in packed FP32, or 1 at a time -- each lane then adds its two paths'
// terms in the same order, so both give the same sums bit for bit); U, the
// unrolling of the step-pair loop.
// Adjoint books ask the register allocator for 640 resident threads per SM (5
// blocks of 128: at most 102 registers), which it would otherwise trade for
// registers it does not need (measured on the 1,024-option book with paired
// reverse steps: 311 ms, against 317 at 768 threads and 393 with no bound).
#ifndef SIMR_BOOK_PAIRED
#define SIMR_BOOK_PAIRED true  // reverse steps in pairs (one at a time: 351 ms against 311 for the book)
#endif
#ifndef SIMR_BOOK_ADJ_THREADS
#define SIMR_BOOK_ADJ_THREADS 640
#endif
// QEM: the options' log-spot steps under QE-M (their QemConst); price books
// then run two paths per thread, unrolled once (two shapes: the block size).
template <bool ADJ, bool GSEG, int TPB, int PPT, int U, bool QEM>
__global__ void __launch_bounds__(TPB, ADJ ? SIMR_BOOK_ADJ_THREADS / TPB : 1) heston_batch_kernel(const __grid_constant__ BatchLaunch B,
                                                           const BatchOption* __restrict__ opts,
                                                           const BatchItem* __restrict__ items,
                                                           unsigned int* __restrict__ counter,
                                                           double* __restrict__ partials) {
  extern __shared__ __align__(16) float smem_f[];
  constexpr int NACC = ADJ ? kAdjAcc : 2;
  const int lane = threadIdx.x & 31, tid = threadIdx.x, bd = blockDim.x;
  while (true) {
    unsigned int it = 0;
    if (lane == 0) it = atomicAdd(counter, 1u);
    it = __shfl_sync(kFull, it, 0);
    if (it >= B.n_items) break;
    const BatchItem I = items[it];
    const BatchOption& O = opts[I.option];
    const ScenConst c = O.sc;
    const float K = O.K, S0 = O.S0;
    const bool put = O.is_put != 0;
    const uint32_t steps = O.steps, oidx = O.option_index;
    double acc[NACC];
#pragma unroll
    for (int a = 0; a < NACC; ++a) acc[a] = 0.0;
    // paths b + lane and b + 32 + lane of each 64-path step (price mode): the
    // grouping of simr_price's two-paths-per-thread kernel, so both form the
    // same FP32 sums of 64 paths
    constexpr uint32_t STEP = ADJ ? 32u : 64u;
    for (uint32_t b = 0; b < I.count; b += STEP) {
      float terms[NACC];
      if (ADJ) {
        const bool active = b + lane < I.count;
        float x[1], comp[1], g[1][5];
        const uint64_t pth[1] = {I.path_begin + b + lane};
        // the block's layout: ckpt_rows checkpoint rows, then the segment
        // arrays of seg_rows rows (the largest over the book), so threads on
        // options with different checkpoint intervals never overlap
        if constexpr (GSEG)  // one segment: no checkpoints are read or written
          path_adjoint_ppt<1, SegGlobal, SIMR_BOOK_PAIRED, QEM>(
              c, O.A, steps, oidx, B.rk, pth, B.gseg, 0,
              SegGlobal{B.gseg, (long long)blockIdx.x * bd + tid, B.seg_rows, (long long)gridDim.x * bd}, x, comp,
              g, O.qm);
        else
          path_adjoint_ppt<1, SegShared, SIMR_BOOK_PAIRED, QEM>(c, O.A, steps, oidx, B.rk, pth, smem_f + tid, bd,
                                                                SegShared{smem_f + B.ckpt_rows * bd, B.seg_rows},
                                                                x, comp, g, O.qm);
        const float S = terminal_spot(S0, x[0], comp[0]);
#pragma unroll
        for (int a = 0; a < NACC; ++a) terms[a] = active ? adj_term(a, put, S, K, g[0], O.invS0, O.T) : 0.0f;
      } else {
        terms[0] = terms[1] = 0.0f;
        float xs[2], cs[2];
        if constexpr (PPT == 2) {
          float2 x2, comp2;
          simulate_two<U, QEM>(c, steps, oidx, B.rk, I.path_begin + b + lane, I.path_begin + b + 32 + lane, x2,
                               comp2, O.qm);
          xs[0] = x2.x;
          xs[1] = x2.y;
          cs[0] = comp2.x;
          cs[1] = comp2.y;
        } else {
#pragma unroll 1
          for (int j = 0; j < 2; ++j)
            simulate_one<QEM, U>(c, steps, oidx, B.rk, I.path_begin + b + 32 * j + lane, xs[j], cs[j], O.qm);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const bool active = b + 32 * j + lane < I.count;
          const float S = terminal_spot(S0, xs[j], cs[j]);
          const float f = put ? fmaxf(K - S, 0.0f) : fmaxf(S - K, 0.0f);
          terms[0] += active ? f : 0.0f;
          terms[1] += active ? f * f : 0.0f;
        }
      }
#pragma unroll
      for (int a = 0; a < NACC; ++a) acc[a] += (double)warp_sum(terms[a]);
    }
    if (lane == 0) {
#pragma unroll
      for (int a = 0; a < NACC; ++a) partials[(size_t)it * NACC + a] = acc[a];
    }
  }
}

// One thread per option: sum its items' rows in item order, normalise.
__global__ void batch_reduce_kernel(const BatchOption* __restrict__ opts, uint32_t n_opts, int nacc,
                                    const double* __restrict__ partials, BatchOutputs out) {
  const uint32_t o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n_opts) return;
  const BatchOption& O = opts[o];
  double s[kAdjAcc];
  for (int a = 0; a < kAdjAcc; ++a) s[a] = 0.0;
  for (uint32_t i = O.item_begin; i < O.item_begin + O.item_count; ++i)
    for (int a = 0; a < nacc; ++a) s[a] += partials[(size_t)i * nacc + a];
  const double n = (double)O.paths, inv_n = 1.0 / n;
  const double mean = s[0] * inv_n;
  const double price = O.disc * mean;
  const uint32_t u = O.option_index;
  out.price[u] = price;
  if (out.stderr_) {
    const double var = n > 1.0 ? (s[1] * inv_n - mean * mean) / (n - 1.0) : 0.0;
    out.stderr_[u] = O.disc * sqrt(var > 0.0 ? var : 0.0);
  }
  if (out.grad && nacc == kAdjAcc) {
    for (int c7 = 0; c7 < 7; ++c7) {
      double g = O.disc * s[2 + c7] * inv_n;
      if (c7 == 6) g *= (double)O.T * (double)O.K;  // e^{-rT} T K E[indicator] (adj_term)
      out.grad[(size_t)u * 7 + c7] = g;
    }
  }
}

using BatchKernel = void (*)(BatchLaunch, const BatchOption*, const BatchItem*, unsigned int*, double*);

// The kernel of a book's mode and shape: price books any of the kBatchVariants
// (threads per block 128 / 256, paths per thread 2 / 1, unroll 1 / 2); adjoint
// books the thread count only.
BatchKernel batch_kernel(bool adjoint, bool gseg, int tpb, int ppt, int unroll, bool qem) {
  const bool t256 = tpb == 256;
  if (qem) {
    if (adjoint) {
      if (gseg)
        return t256 ? heston_batch_kernel<true, true, 256, 1, 1, true> : heston_batch_kernel<true, true, 128, 1, 1, true>;
      return t256 ? heston_batch_kernel<true, false, 256, 1, 1, true> : heston_batch_kernel<true, false, 128, 1, 1, true>;
    }
    return t256 ? heston_batch_kernel<false, false, 256, 2, 1, true> : heston_batch_kernel<false, false, 128, 2, 1, true>;
  }
  if (adjoint) {
    if (gseg) return t256 ? heston_batch_kernel<true, true, 256, 1, 1, false> : heston_batch_kernel<true, true, 128, 1, 1, false>;
    return t256 ? heston_batch_kernel<true, false, 256, 1, 1, false> : heston_batch_kernel<true, false, 128, 1, 1, false>;
  }
  const bool p1 = ppt == 1, u2 = unroll == 2;
  if (t256)
    return p1 ? (u2 ? heston_batch_kernel<false, false, 256, 1, 2, false> : heston_batch_kernel<false, false, 256, 1, 1, false>)
              : (u2 ? heston_batch_kernel<false, false, 256, 2, 2, false> : heston_batch_kernel<false, false, 256, 2, 1, false>);
  return p1 ? (u2 ? heston_batch_kernel<false, false, 128, 1, 2, false> : heston_batch_kernel<false, false, 128, 1, 1, false>)
            : (u2 ? heston_batch_kernel<false, false, 128, 2, 2, false> : heston_batch_kernel<false, false, 128, 2, 1, false>);
}

BatchKernel batch_kernel(const BatchLaunch& B) {
  return batch_kernel(B.adjoint != 0, B.gseg != nullptr, B.tpb, B.ppt, B.unroll, B.qem != 0);
}

size_t batch_smem(const BatchLaunch& B) {
  return B.adjoint && !B.gseg ? (size_t)(B.ckpt_rows + 3 * B.seg_rows) * B.tpb * sizeof(float) : 0;
}

}  // namespace

void batch_variant(int v, bool adjoint, BatchLaunch* B) {
  B->tpb = (v & 1) ? 256 : 128;
  B->ppt = adjoint ? 1 : (((v >> 1) & 1) && !B->qem) ? 1 : 2;
  B->unroll = adjoint ? 1 : (((v >> 2) & 1) && !B->qem) ? 2 : 1;
}

cudaError_t prepare_batch(const BatchLaunch& B) {
  if (!B.adjoint || B.gseg) return cudaSuccess;
  return cudaFuncSetAttribute(batch_kernel(B), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem(B));
}

cudaError_t batch_gseg_threads(int num_sms, size_t* threads) {
  // the largest grid any adjoint variant runs
  *threads = 0;
  for (int q = 0; q < 2; ++q)
    for (int tpb = 128; tpb <= 256; tpb *= 2) {
      int per_sm = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel(true, true, tpb, 1, 1, q),
                                                                    tpb, 0);
      if (e != cudaSuccess) return e;
      *threads = std::max(*threads, (size_t)num_sms * (size_t)per_sm * tpb);
    }
  return cudaSuccess;
}

cudaError_t launch_batch(const BatchLaunch& B, const BatchOption* opts, const BatchItem* items, unsigned int* counter,
                         double* partials, const BatchOutputs& out, int num_sms, cudaStream_t stream) {
  const size_t smem = batch_smem(B);
  int per_sm = 0;
  const BatchKernel kern = batch_kernel(B);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, B.tpb, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const unsigned grid = (unsigned)num_sms * (unsigned)per_sm;
  if (B.adjoint && B.gseg && (size_t)grid * B.tpb * 3 * (size_t)B.seg_rows > B.gseg_floats)
    return cudaErrorMemoryAllocation;
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), stream);
  if (e != cudaSuccess) return e;
  kern<<<grid, B.tpb, smem, stream>>>(B, opts, items, counter, partials);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nacc = B.adjoint ? kAdjAcc : 2;
  batch_reduce_kernel<<<(B.n_opts + 127) / 128, 128, 0, stream>>>(opts, B.n_opts, nacc, partials, out);
  return cudaGetLastError();
}

}  // namespace simr
