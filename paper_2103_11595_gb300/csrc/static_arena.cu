// A fixed device arena for evaluations that must not allocate device memory.
//
// The arena is a file-scope __device__ array, so every GPU that loads libajf's module for this
// file reserves kStaticArenaBytes for it until the process exits. CUDA loads modules lazily by
// default; ajf_create looks the address up for every device context, which loads the module (and
// reserves the array) at set-up rather than inside the first no-allocation call. Host code must
// not use the array's name as a device address: its device address comes from
// cudaGetSymbolAddress with the device current.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"

namespace ajf {

static __device__ __align__(256) unsigned char g_static_arena[kStaticArenaBytes];

namespace {
std::mutex g_mutex;
}  // namespace

// Not cached across calls: after a device reset the array lives at a new address, and every
// context created afterwards must see it.
cudaError_t static_arena_address(int device, void** ptr) {
  if (device < 0) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return e;
  if (cur != device) return cudaErrorInvalidDevice;  // the caller makes `device` current first
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_static_arena);
  if (e != cudaSuccess) return e;
  *ptr = p;
  return cudaSuccess;
}

}  // namespace ajf
