// simr_draws.cu -- the path kernels' random inputs, exposed: the raw Philox4x32-10
// words of given counters and their FP32 standard normals, computed by the same
// device functions (philox_lane / philox_ctr / philox_draw, centered_uniform,
// norminv_centered and its paired form) that every path kernel calls.  They let
// a caller check the generator word for word and the normal transform draw by
// draw (the paper streams its random inputs V and Z from the host, Sec. 3 Table 1
// and Sec. 4; here they are drawn inside the kernels).
#include <cuda_runtime.h>

#include <cstdint>

#include "simr_device.cuh"
#include "simr_internal.h"

namespace simr {
namespace {

// One thread per (path, step pair): words[(path - path_begin) * n_pairs + pair - pair_begin].
__global__ void __launch_bounds__(256) philox_words_kernel(const __grid_constant__ DrawLaunch D,
                                                           uint4* __restrict__ words) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D.n_paths * (uint64_t)D.n_pairs) return;
  const uint64_t path = D.path_begin + i / D.n_pairs;
  const uint32_t pair = D.pair_begin + (uint32_t)(i % D.n_pairs);
  words[i] = philox_draw(philox_lane(path, D.rk), philox_ctr(pair, D.option_index, D.rk), D.rk);
}

// z[i] from words[i] one at a time; zp[2j], zp[2j + 1] from words 2j, 2j + 1 as one
// packed pair (a last odd word paired with itself, its second lane dropped).
__global__ void __launch_bounds__(256) normals_kernel(const uint32_t* __restrict__ words, uint64_t n,
                                                      float* __restrict__ z, float* __restrict__ zp) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = norminv_centered(centered_uniform(words[i]));
  if (zp && 2 * i < n) {
    const uint32_t wa = words[2 * i], wb = 2 * i + 1 < n ? words[2 * i + 1] : wa;
    const float2 r = norminv_centered2(centered_uniform2(wa, wb));
    zp[2 * i] = r.x;
    if (2 * i + 1 < n) zp[2 * i + 1] = r.y;
  }
}

}  // namespace

cudaError_t launch_philox_words(const DrawLaunch& D, uint32_t* words, cudaStream_t stream) {
  const uint64_t n = D.n_paths * (uint64_t)D.n_pairs;
  const int tpb = 256;
  philox_words_kernel<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, stream>>>(D, reinterpret_cast<uint4*>(words));
  return cudaGetLastError();
}

cudaError_t launch_normals(const uint32_t* words, uint64_t n, float* z, float* zp, cudaStream_t stream) {
  const int tpb = 256;
  normals_kernel<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, stream>>>(words, n, z, zp);
  return cudaGetLastError();
}

}  // namespace simr
