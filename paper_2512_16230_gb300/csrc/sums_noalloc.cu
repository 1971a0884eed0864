// Conservation sums without any device allocation.
//
// Some callers cannot call cudaMalloc when they need the sums: hosts that hand all device memory
// to their own pool allocator (a cudaMalloc behind the pool's back would fragment or exceed what
// it manages), runtimes that run under a fixed device-memory budget, and diagnostics that must
// still work after the device has run out of memory. lbm_model_conserved_sums_noalloc serves
// them: its reduction scratch is the file-scope device array below, compiled into the
// library and resident on every GPU that loads it until the process exits, and its result goes
// to a buffer the caller already owns.
//
// The array holds one partial sum per reduction block (608 blocks x 4 quantities = 19,456
// bytes). Every call overwrites all the slots it reads, so nothing has to be cleared between
// calls, but all calls share the one array: two calls whose kernels overlap on the GPU (on
// different streams, or different models on the same device) race on it and must be ordered by
// the caller.
//
// Host code cannot use the array's name as a device address (in host code it names a host-side
// stand-in), so the first call on each device looks the address up with cudaGetSymbolAddress,
// with that device current, and caches it. That first call may also load the library's device
// code for this file; make it before any stream capture begins. The cached address belongs to
// the device's current context: after cudaDeviceReset the library must be reloaded.
#include <mutex>
#include <string>

#include "lbm_internal.cuh"

namespace {

constexpr int kNoAllocSlots = lbm::kRedBlocks;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoAllocSlots * 4];

std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {};

lbm_status scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return lbm::set_error(LBM_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[device]) {
    void* ptr = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
    if (err != cudaSuccess) return lbm::cuda_error(err, "reduction scratch address");
    g_addr[device] = static_cast<double*>(ptr);
  }
  *out = g_addr[device];
  return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_model_conserved_sums_noalloc(lbm_model* m, double* out_dev) {
  if (!m || !out_dev) return lbm::set_error(LBM_ERR_ARG, "NULL argument");
  if (reinterpret_cast<uintptr_t>(out_dev) % alignof(double) != 0)
    return lbm::set_error(LBM_ERR_ARG, "out_dev must be 8-byte aligned device memory");
  // the result is written by a kernel on the model's GPU: out_dev must be memory of that GPU
  // (a host pointer or a peer GPU's buffer would fault there)
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, out_dev) != cudaSuccess) {
    cudaGetLastError();
    return lbm::set_error(LBM_ERR_ARG, "out_dev is not a device pointer");
  }
  if (!((attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) && attr.device == m->device))
    return lbm::set_error(LBM_ERR_ARG, "out_dev must be device or managed memory of the model's GPU (device " +
                                           std::to_string(m->device) + ")");
  if (lbm::kRedBlocks > kNoAllocSlots)
    return lbm::set_error(LBM_ERR_ARG, "the reduction needs " + std::to_string(lbm::kRedBlocks) +
                                           " scratch slots, the static array holds " + std::to_string(kNoAllocSlots));
  int prev = -1;
  cudaError_t err = cudaGetDevice(&prev);
  if (err != cudaSuccess) return lbm::cuda_error(err, "cudaGetDevice");
  if (prev != m->device) {
    err = cudaSetDevice(m->device);
    if (err != cudaSuccess) return lbm::cuda_error(err, "cudaSetDevice");
  }
  double* scratch = nullptr;
  lbm_status st = scratch_address(m->device, &scratch);
  if (st == LBM_OK) st = lbm::launch_sums_into(m, scratch, kNoAllocSlots, out_dev);
  if (prev != m->device) cudaSetDevice(prev);
  return st;
}
