// simr_reduce.cuh -- warp-level reduction helpers of the path kernels (reduction over
// paths, paper Sec. 6): FP32 sums of 32 paths, FP64 from there on.
#pragma once

#include <cstdint>

namespace simr {
namespace {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// In-place transposed butterfly: on entry vals[j] is this lane's term for strike
// j of the tile; on exit vals[0] of lane l is the sum over the 32 lanes for strike l.
__device__ __forceinline__ void butterfly32(float (&vals)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < o; ++j) {
      const float send = upper ? vals[j] : vals[j + o];
      const float keep = upper ? vals[j + o] : vals[j];
      vals[j] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

struct StrikeConst {
  float K, Km, Wr, pad;  // strike; K e^{-h_r T}; K e^{h_r T} - K e^{-h_r T}
};

}  // namespace
}  // namespace simr
