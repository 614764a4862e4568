// simr_rates.cu -- measured throughput of the execution units the path kernels
// lean on, for the roofline's denominators on the GPU in use (no counterpart in
// the paper): FP32 FMA (scalar and packed .f32x2), the special-function unit's
// reciprocal square root, the 32 x 32 -> 64-bit integer multiply of Philox, and
// FP64 FMA.  Each kernel runs one operation in long dependent chains, eight
// independent chains per thread and 2,048 threads per SM, so that latency is
// hidden and the unit's issue rate is what the clock measures.
#include <cuda_runtime.h>

#include <cstdint>

#include "simr_device.cuh"
#include "simr_internal.h"

namespace simr {
namespace {

constexpr int kRateChains = 8;
constexpr int kRateTpb = 256;
constexpr int kRateBlocksPerSm = 8;

enum RateOp { kFma = 0, kFma2 = 1, kRsqrt = 2, kMulWide = 3, kDfma = 4, kRateOps = 5 };

__device__ __forceinline__ float rsqrt_unit(float x) {
  float y;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t mul_wide_fold(uint32_t a, uint32_t m) {
  uint64_t p;
  asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a), "r"(m));
  return (uint32_t)(p >> 32) ^ (uint32_t)p;
}

// `iters` rounds of kRateChains independent operations per thread; every thread
// writes its chains' combination so that no operation is dead.
template <int OP>
__global__ void __launch_bounds__(kRateTpb) rate_kernel(int iters, float seed, float* __restrict__ out) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  float r = 0.0f;
  if constexpr (OP == kFma) {
    float a[kRateChains];
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) a[c] = seed + 0.01f * (float)(c + 1) + 1e-9f * (float)tid;
    const float b = 0.99993f, d = 7e-5f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kRateChains; ++c) a[c] = __fmaf_rn(a[c], b, d);
    }
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) r += a[c];
  } else if constexpr (OP == kFma2) {
    float2 a[kRateChains];
#pragma unroll
    for (int c = 0; c < kRateChains; ++c)
      a[c] = make_float2(seed + 0.01f * (float)(c + 1), seed - 0.01f * (float)(c + 1) + 1e-9f * (float)tid);
    const float2 b = p_bc(0.99993f), d = p_bc(7e-5f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kRateChains; ++c) a[c] = p_fma(a[c], b, d);
    }
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) r += a[c].x + a[c].y;
  } else if constexpr (OP == kRsqrt) {
    float a[kRateChains];
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) a[c] = seed + 0.5f * (float)(c + 1) + 1e-6f * (float)(tid & 1023u);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kRateChains; ++c) a[c] = rsqrt_unit(a[c]);  // x -> x^(-1/2): stays positive
    }
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) r += a[c];
  } else if constexpr (OP == kMulWide) {
    uint32_t a[kRateChains];
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) a[c] = tid * 2654435761u + (uint32_t)c * 40503u + __float_as_uint(seed);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kRateChains; ++c) a[c] = mul_wide_fold(a[c], 0xD2511F53u);
    }
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) r += (float)(a[c] >> 8);
  } else {
    double a[kRateChains];
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) a[c] = (double)seed + 0.01 * (double)(c + 1) + 1e-12 * (double)tid;
    const double b = 0.99993, d = 7e-5;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kRateChains; ++c) a[c] = __fma_rn(a[c], b, d);
    }
#pragma unroll
    for (int c = 0; c < kRateChains; ++c) r += (float)a[c];
  }
  out[tid] = r;
}

// Operations per thread and round (flops counted as 2 per FMA lane).
constexpr double kUnitsPerOp[kRateOps] = {2.0 * kRateChains, 4.0 * kRateChains, kRateChains, kRateChains,
                                          2.0 * kRateChains};
// Rounds per thread: each kernel runs for a few milliseconds at GB300's rates.
constexpr int kIters[kRateOps] = {200000, 100000, 40000, 40000, 4000};

template <int OP>
cudaError_t time_op(int grid, float* out, cudaStream_t st, cudaEvent_t a, cudaEvent_t b, double* per_s) {
  rate_kernel<OP><<<grid, kRateTpb, 0, st>>>(kIters[OP] / 8, 1.0f, out);  // warm-up
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  if (e == cudaSuccess) {
    rate_kernel<OP><<<grid, kRateTpb, 0, st>>>(kIters[OP], 1.0f, out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (e != cudaSuccess) return e;
  const double units = (double)grid * kRateTpb * (double)kIters[OP] * kUnitsPerOp[OP];
  *per_s = units / ((double)ms * 1e-3);
  return cudaSuccess;
}

}  // namespace

cudaError_t measure_unit_rates(int num_sms, float* scratch, cudaStream_t st, double* rates) {
  const int grid = num_sms * kRateBlocksPerSm;
  cudaEvent_t a = nullptr, b = nullptr, t0 = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventRecord(t0, st);
  double v[kRateOps] = {0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = time_op<kFma>(grid, scratch, st, a, b, &v[kFma]);
  if (e == cudaSuccess) e = time_op<kFma2>(grid, scratch, st, a, b, &v[kFma2]);
  if (e == cudaSuccess) e = time_op<kRsqrt>(grid, scratch, st, a, b, &v[kRsqrt]);
  if (e == cudaSuccess) e = time_op<kMulWide>(grid, scratch, st, a, b, &v[kMulWide]);
  if (e == cudaSuccess) e = time_op<kDfma>(grid, scratch, st, a, b, &v[kDfma]);
  float total = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&total, t0, b);
  if (e == cudaSuccess) {
    for (int i = 0; i < kRateOps; ++i) rates[i] = v[i] * 1e-12;  // tera-units per second
    rates[kRateOps] = total;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (t0) cudaEventDestroy(t0);
  return e;
}

size_t unit_rates_scratch_floats(int num_sms) { return (size_t)num_sms * kRateBlocksPerSm * kRateTpb; }

}  // namespace simr
