// Persistent step interpreter (sm_103a): one launch runs the default-lowered programs of many
// networks -- Sec. IV-A remarks that the traces, and so the evaluations of different circuits, are
// independent -- as one queue of tasks. Every launch of every program is a phase; a phase's blocks
// (or a tensor-core GEMM's work items) are cut into tasks; the queue lists the tasks phase by
// phase, the programs' phases interleaved (first phases of all programs, then second phases, ...).
//
// One block per SM (320 threads, ~200 KB of shared memory, 512 TMEM columns allocated for the
// block's lifetime) takes tasks in queue order from a global counter. Before a task runs, thread 0
// waits (bounded) until the previous phase of the task's program has completed all its tasks:
// that keeps each program's launch order, while different programs fill the GPU together. Every
// task waits only for tasks earlier in the queue, and all blocks are resident, so the queue
// always drains. After a task, thread 0 publishes its writes (fence, then the phase's completion
// count). A wait that expires sets the launch's error flag; every block then stops taking tasks,
// drains what its GEMM pipeline issued, frees its TMEM and returns.
//
// Tasks run the same device code as the standalone kernels: the CUDA-core bodies of bodies.cuh on
// threads 0..255 (a named barrier; the block's last two warps sit out), and the tensor-core GEMM
// roles of tc_gemm_dev.cuh on all ten warps, whose slot and TMEM rings continue from one GEMM
// task to the next. The GEMM's shared-memory slots double as the scratch of the other bodies.
#include <cuda.h>
#include <cuda_runtime.h>

#include "bodies.cuh"
#include "device.h"
#include "kernels.h"
#include "tc_gemm_dev.cuh"

#include <cstring>

namespace ajf {
namespace {

using namespace tc;

// fixed GEMM pipeline geometry of the interpreter: every GEMM task uses the same ring
constexpr int kQSlots = 6;
constexpr uint32_t kQSlotBytes = (kBM + 128) * kRowBytes;  // room for the widest B tile
constexpr int kQBufs = 2;
constexpr int kQTmemStride = 256;                          // two partials of up to 128 columns
constexpr uint32_t kQTmemCols = kQBufs * kQTmemStride;
constexpr size_t kQScratch = size_t(kQSlots) * kQSlotBytes;  // 192 KiB
constexpr size_t kQArrays = 96 * 1024;                     // body arrays after the offset tables
constexpr size_t kQSmem = kQScratch + kTcControlBytes + 1024 /* alignment */;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Each kind of task is its own (not inlined) function, so that the register allocation of one
// body does not constrain the others.
template <int BN, int KIND>
__device__ __noinline__ bool gemm_task(const QPhase& ph, const QTask& t, const TcShared& sh, TcRing& ring) {
  const TcParams& p = *static_cast<const TcParams*>(ph.gemm);
  if (threadIdx.x == 0) {
    // the tensor maps live in global memory (written before the launch): acquire them for the
    // tensor-map proxy before the producer's first TMA load through them
    for (int i = 0; i < p.terms; ++i) {
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&p.amap[i]) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&p.bmap[i]) : "memory");
    }
  }
  return tc_gemm_items<BN, KIND>(p, static_cast<uint32_t>(t.b0), static_cast<uint32_t>(t.b1), 1u, sh, ring);
}

// One virtual block v of a CUDA-core phase (threads 0..255), one function per kind of body.
__device__ __noinline__ void q_leaves(const QPhase& ph, int v) {
  leaf_body<double>(static_cast<const LeafDev*>(ph.desc), ph.p0, reinterpret_cast<double*>(ph.base), v);
}
__device__ __noinline__ void q_small(const QPhase& ph, int v, uint8_t* smem) {
  small_body<double, double, SyncBody>(static_cast<const StepDev*>(ph.desc), ph.count, ph.nblocks,
                                       reinterpret_cast<double*>(ph.base), v, reinterpret_cast<int64_t*>(smem));
}
__device__ __noinline__ void q_splitk(const QPhase& ph, int v, uint8_t* smem) {
  double* red = reinterpret_cast<double*>(smem + kQArrays);
  splitk_body<double, SyncBody>(static_cast<const StepDev*>(ph.desc), ph.count, reinterpret_cast<double*>(ph.base),
                                reinterpret_cast<double2*>(ph.p0), v, reinterpret_cast<int64_t*>(smem), red,
                                red + kBodyThreads);
}
__device__ __noinline__ void q_splitk_done(const QPhase& ph, int v, uint8_t* smem) {
  double* red = reinterpret_cast<double*>(smem + kQArrays);
  splitk_done_body<double, SyncBody>(static_cast<const StepDev*>(ph.desc), reinterpret_cast<const double2*>(ph.p0),
                                     reinterpret_cast<double*>(ph.base), reinterpret_cast<double2*>(ph.p1), v, red,
                                     red + kBodyThreads);
}
template <bool kF32>
__device__ __noinline__ void q_dot(const QPhase& ph, int v, uint8_t* smem) {
  double* red = reinterpret_cast<double*>(smem + kQArrays);
  dot_body<double, kF32, SyncBody>(static_cast<const StepDev*>(ph.desc), ph.count, reinterpret_cast<double*>(ph.base),
                                   reinterpret_cast<double2*>(ph.p0), v, reinterpret_cast<int64_t*>(smem), red,
                                   red + kBodyThreads);
}
__device__ __noinline__ void q_perm(const QPhase& ph, int v, uint8_t* smem) {
  perm_body<float, SyncBody>(static_cast<const PermDev*>(ph.desc), reinterpret_cast<const double*>(ph.base), ph.base,
                             v % ph.grid_x, ph.grid_x, v / ph.grid_x, reinterpret_cast<int64_t*>(smem),
                             *reinterpret_cast<PermSmem<float>*>(smem + kQArrays));
}
__device__ __noinline__ void q_split_sum(const QPhase& ph, int v) {
  split_sum_body(reinterpret_cast<const float*>(ph.p0), ph.ksplit, ph.n, reinterpret_cast<float*>(ph.p1), v,
                 ph.nblocks);
}
__device__ __noinline__ void q_open(const QPhase& ph, int v, uint8_t* smem) {
  open_body<double, SyncBody>(static_cast<const FinalDev*>(ph.desc), reinterpret_cast<const double*>(ph.base),
                              reinterpret_cast<const double2*>(ph.p0), ph.p1, ph.p2, v, ph.nblocks,
                              reinterpret_cast<int64_t*>(smem), reinterpret_cast<double*>(smem + kQArrays));
}
__device__ __noinline__ void q_final(const QPhase& ph) {
  if (threadIdx.x == 0) {
    final_body(static_cast<const FinalDev*>(ph.desc), reinterpret_cast<const double2*>(ph.p0), ph.p2, ph.p1);
    if (ph.p3) {
      ph.p3[0] = ph.p1[0];
      ph.p3[1] = ph.p1[1];
      ph.p3[2] = ph.p1[2];
    }
  }
}

__device__ __forceinline__ void body_task(const QPhase& ph, int v, uint8_t* smem) {
  switch (ph.kind) {
    case QK_LEAVES: q_leaves(ph, v); break;
    case QK_SMALL: q_small(ph, v, smem); break;
    case QK_SPLITK: q_splitk(ph, v, smem); break;
    case QK_SPLITK_DONE: q_splitk_done(ph, v, smem); break;
    case QK_DOT:
      if (ph.flag) q_dot<true>(ph, v, smem);
      else q_dot<false>(ph, v, smem);
      break;
    case QK_PERM: q_perm(ph, v, smem); break;
    case QK_SPLIT_SUM: q_split_sum(ph, v); break;
    case QK_OPEN: q_open(ph, v, smem); break;
    default: q_final(ph); break;
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_queue(const QPhase* __restrict__ phases,
                                                       const QTask* __restrict__ tasks, int ntasks,
                                                       int* __restrict__ counters, int* __restrict__ status,
                                                       unsigned long long wait_ns,
                                                       unsigned long long* __restrict__ prof) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ int s_task;
  const int tid = threadIdx.x, warp = tid >> 5;
  TcShared sh;
  uint32_t* tmem_slot = tc_layout(smem, smem + kQScratch, sh);
  if (tid == 0) tc_init_barriers(sh, kQSlots, kQBufs);
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kQTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  sh.tmem = *tmem_slot;
  TcRing ring;
  __shared__ unsigned long long s_t0, s_t1;
  for (;;) {
    if (tid == 0) {
      if (prof) s_t0 = globaltimer();
      int t = ntasks;
      if (!*sh.abort_flag && ld_acquire(&counters[kQError]) == 0) t = atomicAdd(&counters[kQNext], 1);
      if (t < ntasks) {
        const int prev = phases[tasks[t].phase].prev;
        if (prev >= 0) {
          const int need = phases[prev].ntasks;
          if (ld_acquire(&counters[kQPhase0 + prev]) < need) {
            const unsigned long long t0 = globaltimer();
            unsigned ns = 32;
            while (ld_acquire(&counters[kQPhase0 + prev]) < need) {
              if (ld_acquire(&counters[kQError]) != 0) {
                t = ntasks;
                break;
              }
              if (globaltimer() - t0 > wait_ns) {
                atomicExch(status, 21);
                atomicExch(&counters[kQError], 1);
                t = ntasks;
                break;
              }
              __nanosleep(ns);
              if (ns < 1024) ns *= 2;
            }
          }
        }
        // the task's inputs were written by other blocks through the generic proxy: make them
        // visible to this thread's TMA loads (async proxy), and order this block's earlier generic
        // shared-memory writes before the TMA writes into the same bytes
        asm volatile("fence.proxy.async.global;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      s_task = t;
      if (prof) s_t1 = globaltimer();
    }
    __syncthreads();
    const int t = s_task;
    if (t >= ntasks) break;
    const QTask task = tasks[t];
    const QPhase& ph = phases[task.phase];
    if (ph.kind == QK_GEMM) {
      if (ph.flag == 2) {
        if (ph.bn == 128) gemm_task<128, 2>(ph, task, sh, ring);
        else if (ph.bn == 64) gemm_task<64, 2>(ph, task, sh, ring);
        else gemm_task<32, 2>(ph, task, sh, ring);
      } else if (ph.flag == 1) {
        if (ph.bn == 128) gemm_task<128, 1>(ph, task, sh, ring);
        else if (ph.bn == 64) gemm_task<64, 1>(ph, task, sh, ring);
        else gemm_task<32, 1>(ph, task, sh, ring);
      } else {
        if (ph.bn == 128) gemm_task<128, 0>(ph, task, sh, ring);
        else if (ph.bn == 64) gemm_task<64, 0>(ph, task, sh, ring);
        else gemm_task<32, 0>(ph, task, sh, ring);
      }
      __syncwarp();
    } else if (warp < kBodyThreads / 32) {
      for (int v = task.b0; v < task.b1; ++v) {
        body_task(ph, v, smem);
        SyncBody::sync();
      }
    }
    __syncthreads();
    if (tid == 0) {
      if (*sh.abort_flag) atomicExch(&counters[kQError], 1);
      __threadfence();
      atomicAdd(&counters[kQPhase0 + task.phase], 1);
      if (prof) {  // per kind of task: busy time, time waiting for the previous phase, tasks
        const unsigned long long t2 = globaltimer();
        atomicAdd(&prof[3 * ph.kind + 0], t2 - s_t1);
        atomicAdd(&prof[3 * ph.kind + 1], s_t1 - s_t0);
        atomicAdd(&prof[3 * ph.kind + 2], 1ull);
      }
    }
  }
  if (*sh.abort_flag) tc_drain_after_abort(kQSlots, kQBufs, wait_ns, status, sh, ring);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncwarp();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sh.tmem), "r"(kQTmemCols) : "memory");
  }
}

}  // namespace

size_t queue_smem_bytes() { return kQSmem; }

cudaError_t queue_gemm_params(const TcPrepared& t, void* out, int* bn, int* bf16, int* nwork) {
  if (!t.ready) return cudaErrorInvalidValue;
  TcParams p;
  std::memcpy(&p, t.params, sizeof(p));
  // the interpreter's fixed pipeline: every GEMM task shares one slot ring and one TMEM ring
  p.slots = kQSlots;
  p.slot_bytes = kQSlotBytes;
  p.bufs = kQBufs;
  p.tmem_stride = kQTmemStride;
  const uint32_t bnbits = (p.idesc >> 17) & 0x3Fu;  // N >> 3 in the instruction descriptor
  *bn = static_cast<int>(bnbits << 3);
  const uint32_t fmt = (p.idesc >> 7) & 0x7u;  // 2 TF32, 1 bf16, 0 fp16 (scaled)
  *bf16 = fmt == 2u ? 0 : (fmt == 1u ? 1 : 2);
  *nwork = static_cast<int>(p.tiles * p.ksplit);
  std::memcpy(out, &p, sizeof(p));
  return cudaSuccess;
}

size_t queue_gemm_params_bytes() { return (sizeof(TcParams) + 1023) / 1024 * 1024; }

cudaError_t launch_queue(const QPhase* d_phases, int nphases, const QTask* d_tasks, int ntasks, int* d_counters,
                         int* d_status, int blocks, cudaStream_t s, unsigned long long wait_ns,
                         unsigned long long* d_prof) {
  if (ntasks == 0) return cudaSuccess;
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(k_queue, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kQSmem));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  e = cudaMemsetAsync(d_counters, 0, sizeof(int) * (kQPhase0 + static_cast<size_t>(nphases)), s);
  if (e != cudaSuccess) return e;
  k_queue<<<blocks, kThreads, kQSmem, s>>>(d_phases, d_tasks, ntasks, d_counters, d_status, wait_ns, d_prof);
  return cudaGetLastError();
}

}  // namespace ajf
