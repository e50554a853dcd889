// Launch wrappers of the device kernels (host-callable).
#pragma once
#include <cuda_runtime.h>

#include "device.h"

namespace ajf {

cudaError_t set_kernel_smem_limits();

// Fixed device arena (static_arena.cu) for evaluations that allocate nothing: its size, and its
// device address on `device`, which must be the current device (cudaErrorInvalidDevice otherwise).
constexpr size_t kStaticArenaBytes = size_t(64) << 20;
cudaError_t static_arena_address(int device, void** ptr);
size_t step_table_bytes(const StepDev& st);
size_t perm_table_bytes(const PermDev& p);

cudaError_t launch_leaves(const LeafDev* d_leaves, int n, const double* d_in, void* arena, cudaStream_t s);
cudaError_t launch_small(const StepDev* d_steps, int nsteps, int total_blocks, size_t smem, void* arena, cudaStream_t s);
cudaError_t launch_splitk(const StepDev* d_steps, int nsteps, int total_blocks, size_t smem, void* arena,
                          double2* partial, double2* scalars, cudaStream_t s);
// op_f64: the operands are FP64 (staged in FP64); otherwise every format is staged in FP32.
cudaError_t launch_perm(const PermDev* d_perms, int nperm, int grid_x, size_t smem, const void* arena, void* base,
                        bool op_f64, cudaStream_t s);
// Tiled FP64 full contraction (k_dot) of steps with a scalar result, then the partial-sum pass.
// The tiled dot's staged form (FP32 operands, FP32 products): the step qualifies on the host side;
// the kernel also checks the operands' bit positions and alignment and otherwise falls back.
bool dot_staged(const StepDev& st, bool f32_products);
size_t dot_smem_bytes(const StepDev& st, bool f32_products);
// f32_products: FP32 products summed in FP32 per tile, tile sums in FP64 (reduced-precision modes).
cudaError_t launch_dot(const StepDev* d_steps, int nsteps, int total_blocks, size_t smem, const void* arena,
                       double2* partial, double2* scalars, bool f32_products, cudaStream_t s);
cudaError_t launch_gemm_simt(const void* A, const void* B, void* C, int64_t M, int64_t N, int64_t K, bool f64,
                             cudaStream_t s);
cudaError_t launch_final(const FinalDev* d_fd, int open_bits_nchunks, int nblocks, const void* arena,
                         const double2* scalars, double* traces, double* partial, double* result, cudaStream_t s);
// Persistent kernel: one thread block per network runs that network's whole program (leaves,
// all steps level by level, the FP64 trace and F) -- n_jobs networks in one launch. `smem`:
// dynamic shared memory per block (the largest work region among the jobs with job.smem = 1).
cudaError_t launch_persistent(const InterpJob* d_jobs, int n_jobs, const InterpOp* d_ops, size_t smem, int threads,
                              cudaStream_t s);
constexpr size_t kPersistentSmemMax = 96 * 1024;

// Tensor-core GEMM (tcgen05, tc_gemm.cu): C[M][N] (FP32, row-major) =
// sum_{i + j < terms} A_i[M][K] . B_j[N][K]^T for the split terms A_t, B_t (byte offsets from
// `base`), FP32 accumulation promoted per K block. kind 0: tf32, 1: bf16, 2: scaled fp16.
// Returns cudaErrorNotSupported when the shape is not tile-aligned.
bool tc_gemm_supported(int64_t M, int64_t N, int64_t K, int kind);
// K splits for an M x N x K GEMM: GEMMs with fewer 128 x BN tiles than SMs divide K over several
// CTAs, each writing an FP32 partial tile to a workspace of ksplit * M * N floats that a
// deterministic pass then sums into C. 1 = no split (no workspace).
int tc_gemm_splits(int64_t M, int64_t N, int64_t K, int kind);
// A tensor-core GEMM launch prepared on the host (tensor maps, tiling, kernel parameters), so that
// enqueueing it later costs one kernel launch (two with a K split) and no host set-up.
struct TcPrepared {
  alignas(64) unsigned char params[1024];  // the kernel's parameter block
  void (*run)(const void* params, unsigned grid, size_t smem, cudaStream_t s) = nullptr;
  unsigned grid = 0;
  size_t smem = 0;
  int ksplit = 1;
  float* ws = nullptr;
  float* C = nullptr;
  int64_t n = 0;  // M * N
  bool ready = false;
};
cudaError_t tc_gemm_prepare(TcPrepared* t, char* base, const int64_t* a_off, const int64_t* b_off, int terms,
                            float* C, int64_t M, int64_t N, int64_t K, int kind, float* ws, int ksplit,
                            int* d_status, unsigned long long wait_ns, int stall_loads);
cudaError_t tc_gemm_run(const TcPrepared& t, cudaStream_t s);
// Bound of every device-side wait in the GEMM and the step interpreter (nanoseconds).
constexpr unsigned long long kTcWaitNs = 2000000000ull;
// Persistent step interpreter (queue.cu): one launch of `blocks` blocks (at most one per SM) runs
// the tasks of the phases (device tables; see device.h). d_counters: kQPhase0 + nphases ints,
// zeroed by the launch. A dependency wait that expires sets *d_status (code 21) and the error
// counter; a GEMM wait sets its own code, as in the standalone kernel.
size_t queue_smem_bytes();
// d_prof (optional, 3 * kQKinds counters, accumulated): per kind of task, its busy nanoseconds,
// the nanoseconds its block waited for the previous phase, and its task count.
constexpr int kQKinds = 10;
cudaError_t launch_queue(const QPhase* d_phases, int nphases, const QTask* d_tasks, int ntasks, int* d_counters,
                         int* d_status, int blocks, cudaStream_t s, unsigned long long wait_ns = kTcWaitNs,
                         unsigned long long* d_prof = nullptr);
// A prepared tensor-core GEMM's parameter block for the interpreter (its fixed pipeline geometry),
// written to `out` (queue_gemm_params_bytes() bytes, 64-byte aligned in device memory when used);
// its tile width, operand kind and work-item count.
size_t queue_gemm_params_bytes();
cudaError_t queue_gemm_params(const TcPrepared& t, void* out, int* bn, int* bf16, int* nwork);
cudaError_t launch_gemm_tc(char* base, const int64_t* a_off, const int64_t* b_off, int terms, float* C, int64_t M,
                           int64_t N, int64_t K, int kind, float* ws, int ksplit, int* d_status, cudaStream_t s);
// Same with an explicit bound on every device-side wait and a test hook: stall_loads = 1 makes the
// producer issue no loads, so the MMA and epilogue waits expire and the kernel reports a status
// code and returns.
cudaError_t launch_gemm_tc_ex(char* base, const int64_t* a_off, const int64_t* b_off, int terms, float* C, int64_t M,
                              int64_t N, int64_t K, int kind, float* ws, int ksplit, int* d_status, cudaStream_t s,
                              unsigned long long wait_ns, int stall_loads);

}  // namespace ajf
