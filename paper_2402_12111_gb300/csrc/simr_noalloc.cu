// simr_noalloc.cu -- simr_price_noalloc: the European pricing call of simr_price
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: latency-bound serving loops that must
// never block on the allocator (cudaMalloc can synchronise the device), and
// host applications or plugins that hand out all device memory themselves and
// forbid libraries from taking more.  This entry point takes
// device pointers for its inputs and outputs, needs no context, and keeps its
// reduction scratch (partial sums of each block, the finishing ticket and a
// status word) in one file-scope __device__ array of fixed size, which every
// GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "simr.h"
#include "simr_internal.h"

namespace {

constexpr int kNoAllocMaxStrikes = 32;
constexpr int kNoAllocMaxBlocks = 2048;  // blocks of the persistent grid, any SM count up to 256
constexpr size_t kHeaderBytes = 256;      // ticket word at 0, status word at 64
constexpr size_t kPartialDoubles = (size_t)kNoAllocMaxBlocks * 2 * kNoAllocMaxStrikes;
constexpr int kMaxDevices = 64;

// 1 MiB + 256 B: the scratch of every simr_price_noalloc call on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kHeaderBytes + kPartialDoubles * sizeof(double)];

struct DeviceSlot {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
  int num_sms = 0;
};
DeviceSlot g_slots[kMaxDevices];
std::mutex g_mutex;

// Once per device, with that device current: the device address of the
// scratch array (its host-side name is only a stand-in, not an address a kernel
// may use) and the SM count.
int setup(int device, DeviceSlot** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceSlot& s = g_slots[device];
  if (!s.ready) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return simr::internal_cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return simr::internal_cuda_fail(e, "querying the SM count");
    if ((size_t)sms * 8 > (size_t)kNoAllocMaxBlocks)
      return simr::internal_fail(SIMR_EUNSUPPORTED, "device has more SMs than the static scratch covers");
    s.base = static_cast<unsigned char*>(ptr);
    s.num_sms = sms;
    s.ready = true;
  }
  *out = &s;
  return SIMR_OK;
}

// Device memory of `device` (or managed memory).  Device memory of another GPU
// would pass a plain device-pointer test and then fault in the kernel.
bool on_device(const void* p, int device) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

extern "C" SIMR_API int simr_price_noalloc(const simr_heston* model, const double* strikes, int n_strikes,
                                           int is_put, uint32_t steps, uint64_t paths, uint64_t seed,
                                           uint32_t option_index, double* price, double* stderr_out,
                                           void* stream) {
  int rc = simr::internal_check_price_args(model, strikes, n_strikes, kNoAllocMaxStrikes, steps, paths);
  if (rc) return rc;
  if (!price) return simr::internal_fail(SIMR_EINVAL, "price is NULL");
  if (!simr::internal_is_device_ptr(strikes) || !simr::internal_is_device_ptr(price) ||
      (stderr_out && !simr::internal_is_device_ptr(stderr_out)))
    return simr::internal_fail(SIMR_EINVAL, "simr_price_noalloc takes device pointers only");
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return simr::internal_cuda_fail(e, "cudaGetDevice");
  if (!on_device(strikes, device) || !on_device(price, device) || (stderr_out && !on_device(stderr_out, device)))
    return simr::internal_fail(SIMR_EINVAL, "simr_price_noalloc takes device pointers only, of the current device");
  if (device < 0 || device >= kMaxDevices) return simr::internal_fail(SIMR_EUNSUPPORTED, "device ordinal too large");
  DeviceSlot* slot = nullptr;
  if ((rc = setup(device, &slot))) return rc;

  simr::PathLaunch L;
  if ((rc = simr::internal_build_price_launch(model, n_strikes, is_put, steps, paths, seed, option_index, &L)))
    return rc;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int* ticket = reinterpret_cast<unsigned int*>(slot->base);
  // the ticket and status words must start at zero; the array keeps the last call's contents
  e = cudaMemsetAsync(slot->base, 0, kHeaderBytes, st);
  if (e != cudaSuccess) return simr::internal_cuda_fail(e, "clearing the static scratch header");
  simr::PathOutputs out{};
  out.price = price;
  out.stderr_ = stderr_out;
  out.status = reinterpret_cast<int*>(slot->base + 64);
  simr::Scratch s{reinterpret_cast<double*>(slot->base + kHeaderBytes), ticket, kPartialDoubles};
  int grid = 0;
  e = simr::take_fault(SIMR_FAULT_LAUNCH) ? cudaErrorLaunchOutOfResources
                                          : simr::launch_paths(L, strikes, out, s, slot->num_sms, st, &grid);
  if (e == cudaErrorMemoryAllocation)
    return simr::internal_fail(SIMR_EUNSUPPORTED, "launch needs more partial sums than the static scratch holds");
  if (e != cudaSuccess) return simr::internal_cuda_fail(e, "launching the path kernel");
  return SIMR_OK;
}
