// A fixed device arena for evaluations that must not allocate device memory.
//
// The arena is a file-scope __device__ array, so every GPU that loads libajf reserves
// kStaticArenaBytes for it until the process exits. Host code must not use the array's name as a
// device address: its device address is looked up with cudaGetSymbolAddress once per device (with
// that device current) and cached here.
#include <cuda_runtime.h>

#include <mutex>

#include "kernels.h"

namespace ajf {

static __device__ __align__(256) unsigned char g_static_arena[kStaticArenaBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};
}  // namespace

cudaError_t static_arena_address(int device, void** ptr) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_arena);
    if (e != cudaSuccess) return e;
    g_addr[device] = p;
  }
  *ptr = g_addr[device];
  return cudaSuccess;
}

}  // namespace ajf
