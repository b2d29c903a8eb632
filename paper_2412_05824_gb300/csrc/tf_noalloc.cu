// turbofft_exec_static_scratch: the two-pass transform with its intermediate
// buffer in a fixed, file-scope device array, so that the call allocates no
// device memory at all.
//
// Who needs it: code that can create its plans up front but must not call
// cudaMalloc (or any allocating routine) when it transforms, for example a
// program whose device memory is owned by another allocator that hands out
// no raw buffers, or one that runs under a device-memory budget fixed when it
// starts.  turbofft_exec would otherwise allocate a two-pass plan's
// intermediate on its first call, and turbofft_set_workspace needs a device
// buffer that such a caller cannot obtain.
//
// The array holds TURBOFFT_STATIC_SCRATCH_BYTES (32 MiB).  It lives in this
// file's module, so every GPU on which that module is loaded keeps the
// 32 MiB until the process exits.  All calls on a device share it: two calls
// whose kernels overlap on the GPU (different streams, no ordering between
// them) race on it.  Nothing in it needs to start at zero: the first pass of a
// two-pass transform writes every element of the intermediate before the
// second pass reads it, so the contents left by the previous call are never
// read.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/turbofft.h"
#include "tf_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[TURBOFFT_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch per device, looked up once per device
// (with that device current) on the first call that needs it.  With lazy
// module loading the lookup is what loads this file's module, so the 32 MiB
// is reserved on the device at that first call.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

turbofft_status scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return TURBOFFT_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[device]) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
      cudaGetLastError();
      return TURBOFFT_CUDA_ERROR;
    }
    if (cur != device && cudaSetDevice(device) != cudaSuccess) {
      cudaGetLastError();
      return TURBOFFT_CUDA_ERROR;
    }
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return TURBOFFT_CUDA_ERROR;
    }
    g_scratch_ptr[device] = ptr;
  }
  *out = g_scratch_ptr[device];
  return TURBOFFT_SUCCESS;
}

}  // namespace

extern "C" const uint64_t turbofft_static_scratch_bytes = TURBOFFT_STATIC_SCRATCH_BYTES;

extern "C" turbofft_status turbofft_exec_static_scratch(turbofft_plan* plan, const void* in, void* out,
                                                        turbofft_stream stream) {
  if (!plan) return TURBOFFT_INVALID_VALUE;
  const size_t need = tf::plan_scratch_bytes(plan);
  if (need > (size_t)TURBOFFT_STATIC_SCRATCH_BYTES) {
    std::string msg = "turbofft_exec_static_scratch: the plan's intermediate needs " + std::to_string(need) +
                      " bytes; the static scratch holds " + std::to_string((size_t)TURBOFFT_STATIC_SCRATCH_BYTES);
    tf::plan_set_error(plan, msg.c_str());
    return TURBOFFT_INVALID_VALUE;
  }
  void* scratch = nullptr;
  if (need > 0) {
    turbofft_status st = scratch_address(tf::plan_device(plan), &scratch);
    if (st != TURBOFFT_SUCCESS) {
      tf::plan_set_error(plan, "turbofft_exec_static_scratch: device address of the static scratch not available");
      return st;
    }
  }
  return tf::exec_given_scratch(plan, in, out, scratch, reinterpret_cast<cudaStream_t>(stream));
}
