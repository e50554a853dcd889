// A lowered contraction: descriptor arrays, the launch sequence and the arena layout.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "ajf_internal.h"
#include "device.h"

namespace ajf {

enum LaunchKind : int32_t { LK_SMALL = 0, LK_SPLITK = 1, LK_PERM = 2, LK_GEMM_SIMT = 3, LK_GEMM_TC = 4, LK_DOT = 5 };

struct Launch {
  int32_t kind = 0;
  int32_t first = 0, count = 0;  // range in steps (SMALL/SPLITK) or perms (PERM)
  int32_t blocks = 0;            // grid size (SMALL/SPLITK total blocks, PERM grid.x)
  size_t smem = 0;
  // GEMM: C[M][N] = sum_p A_p[M][K] . B_p[N][K]^T (byte offsets into the arena)
  int64_t a_off[6] = {0, 0, 0, 0, 0, 0}, b_off[6] = {0, 0, 0, 0, 0, 0};
  int32_t npass = 0;
  int32_t tc_kind = 0;           // 0 tf32, 1 bf16
  int32_t op_f64 = 1;            // CUDA-core GEMM: FP64 (1) or FP32 (0) operands
  int64_t c_off = 0;             // byte offset of C
  int32_t ksplit = 1;            // tensor-core GEMM: K splits (> 1: FP32 partials in the workspace)
  int64_t ws_off = 0;            // byte offset of the split workspace (ksplit * M * N floats)
  int64_t M = 0, N = 0, K = 0;
  double flops = 0, bytes = 0;   // algorithmic work of the complex step this launch belongs to
};

struct Program {
  int alg = 0;
  int precision = AJF_PREC_F64;
  size_t elem = 8;               // bytes per real element of a complex128 tensor (complex64 ones: 4)
  std::vector<LeafDev> leaves;
  std::vector<StepDev> steps;
  std::vector<PermDev> perms;
  std::vector<Launch> launches;
  FinalDev fin{};
  int final_nchunks = 0;
  int final_blocks = 1;
  int n_scalars = 0;
  int64_t n_traces = 1;          // 2^open_bits
  // arena layout (bytes)
  size_t off_desc = 0, desc_bytes = 0;        // leaves | steps | perms | final
  size_t off_leaves = 0, off_steps = 0, off_perms = 0, off_final = 0;
  size_t off_inputs = 0, input_bytes = 0;     // packed complex128 inputs
  size_t off_result = 0;                      // 4 doubles: S, F, 1-F, status
  size_t off_scalars = 0;                     // double2 per scalar slot
  size_t off_partial = 0, partial_count = 0;  // double2 split-K partials
  size_t off_open_partial = 0;                // double per k_open block
  size_t off_traces = 0;                      // double2 per trace (Alg. I)
  size_t off_status = 0;                      // int32 device status words
  size_t off_work = 0;                        // tensors and GEMM scratch
  size_t work_bytes = 0;                      // size of the work region
  size_t arena_bytes = 0;
  bool persistent = false;                    // lowered for the persistent kernel (CUDA-core steps only)
  // statistics
  double flops = 0, bytes = 0, gemm_flops = 0, gemm_bytes = 0;
  int n_gemm = 0;
  int tensor_cores = 0;          // GEMM launches on tcgen05
};

// Lower `path` over `net` to a device program for `precision`. `inputs_complex` is the number
// of complex128 values in the packed input buffer. `tc_ok`: tensor-core GEMMs may be used.
// `persistent`: every step becomes a CUDA-core gather step (LK_SMALL) or a reduction step
// (LK_SPLITK), so that one thread block of the persistent kernel can run the whole program.
Program lower(const Network& net, const Path& path, int precision, size_t inputs_complex, bool tc_ok,
              bool persistent = false);

// Host-side replay of a lowered program's address arithmetic and buffer lifetimes (no device
// needed): "" if every access stays inside its buffer and region and no launch overwrites a buffer
// still to be read; otherwise the first violation.
std::string check_program(const Program& P);

}  // namespace ajf
