// Device-side step descriptors shared by the lowering (host) and the kernels (device).
//
// Storage: every tensor lives in one device arena in planar complex form -- a real plane of
// 2^r elements followed by an imaginary plane of 2^r elements. Tensors are complex128 (FP64
// planes), except the products of reduced-precision GEMMs, which are complex64 (FP32 planes: the
// GEMM promotes each result to one FP32 register sum, so nothing is lost); an element offset is in
// units of the tensor's own element type from the arena base. Element index = sum_i bit_i * 2^i,
// where bit i is the tensor's i-th label. Scalars produced by full contractions are FP64 (double2
// slots).
#pragma once
#include <cstdint>

namespace ajf {

constexpr int kMaxBits = 48;

// Map from the bits of an index to element offsets of one tensor: offset(idx) =
// sum_i bit_i(idx) << pos[i] (pos < 0: the bit does not address this tensor). Evaluated on the
// device through 8-bit lookup tables built in shared memory.
struct BitMap {
  int32_t nbits;
  int8_t pos[kMaxBits];
};

// One pairwise contraction C[o] = sum_kk A[a + oa(o) + ka(kk)] * B[b + ob(o) + kb(kk)].
struct StepDev {
  int64_t a, b, c;        // element offsets of the real planes in the arena
  int64_t pa, pb, pc;     // plane strides (elements) = tensor sizes
  int64_t poff;           // split-K: offset (in double2) of this step's partial sums
  BitMap oa, ob;          // output-index bits -> A / B offsets
  BitMap ka, kb;          // contracted-index bits -> A / B offsets
  int32_t rc, rk;         // output and contracted bit counts
  int32_t block0;         // first block of this step within its launch
  int32_t scalar_slot;    // >= 0: the result is a scalar written to a double2 slot (FP64)
  int32_t nsplit;         // split-K: blocks per output element
  int32_t ntl;            // tiled dot: bits of a tile (<= 10)
  int8_t tl[16];          // tiled dot: contracted-index bits of a tile, ordered by A position
  int8_t tlb[16];         // tiled dot: the same bits ordered by B position
  int8_t fa, fb;          // A / B is complex64 (FP32 planes); the output C is always complex128
  int8_t pad8[6];
};

// Operand preparation for a GEMM step: gather a complex tensor into a real row-major,
// K-contiguous GEMM operand. Embedded (X side): rows (s, m), cols (t, k) hold
// [[Re, -Im], [Im, Re]] (2M x 2K). Plain (Y side, stored transposed): rows n, cols (t, k) hold
// plane t (N x 2K).
struct PermDev {
  int64_t src, plane;     // source tensor (element offset of the real plane) and plane stride
  int64_t dst[3];         // destination operand arrays (split terms: hi, mid, lo), byte offsets;
                          // OPM_F16X2S: hi, lo and the scale array
  BitMap rows, cols;      // row-index bits / k-index bits -> source offsets
  int32_t rbits, kbits;   // log2 rows (M or N), log2 K
  int32_t embed;          // 1: X side (embedded), 0: Y side
  int32_t rows_fast;      // 1: read with lanes along rows (the source's stride-1 bit is a row bit)
  int32_t mode;           // operand format, see OperandMode
  int32_t src_f32;        // the source is complex64 (FP32 planes), else complex128
};

enum OperandMode : int32_t {
  OPM_F64 = 0,     // double
  OPM_F32 = 1,     // float
  OPM_TF32 = 2,    // float rounded to TF32
  OPM_TF32X2 = 3,  // hi, lo (float, each TF32)
  OPM_BF16X2 = 4,  // hi, lo (bf16)
  OPM_BF16X3 = 5,  // hi, mid, lo (bf16)
  OPM_F16X2S = 6,  // hi, lo (fp16) of x / q, with q a power of two per row and K block (dst[2]: the
                   // FP32 q's, [K block][row])
};

// Leaf construction from the uploaded complex128 inputs.
struct LeafDev {
  int64_t off, plane;     // destination (element offset of the real plane), plane stride
  int64_t src;            // complex offset of the source matrix in the input buffer
  int32_t kind, a, nk, kbits;
  int32_t bits;           // total tensor bits
  uint16_t fix_mask;      // bond slicing: positions of sliced labels in the full leaf index
  uint16_t fix_val;       // their values in this slice (bits under fix_mask)
};

// Final reduction: scalars, open tensor, result.
struct FinalDev {
  int64_t open_off;              // open tensor (working precision); -1 if none
  int64_t open_plane;
  BitMap open_map;               // canonical open-index bits -> offsets in the open tensor
  int32_t open_bits;
  int32_t n_scalars;
  int32_t loops;                 // untouched wires: factor 2 each on every trace
  int32_t n_qubits;
  int32_t alg;
  int32_t nblocks;               // blocks of the open-tensor pass
  int32_t open_f32;              // the open tensor is complex64 (FP32 planes), else complex128
  int32_t pad;
};

// One network of a persistent-kernel launch (one thread block each). Byte offsets are into the
// network's own arena; the program is a sequence of ops, each a range of independent steps.
struct InterpJob {
  char* base;                    // the network's arena (device)
  double* out;                   // optional copy of (S, F, 1 - F); nullptr: none
  int64_t off_leaves, off_steps, off_final, off_inputs, off_scalars, off_traces, off_result;
  int64_t work0;                 // element offset of the work region in the arena
  int32_t n_leaves, op0, n_ops;  // leaves; first op and op count in the op table
  int32_t smem;                  // 1: the work region lives in shared memory for the whole program
};

struct InterpOp {
  int32_t kind;                  // LK_SMALL (0) or LK_SPLITK (1)
  int32_t first, count;          // range of steps (all at one level: independent)
  int32_t pad;
};

}  // namespace ajf

namespace ajf {

// ------------------------------------------------------------------ persistent step interpreter
// One launch (k_queue, queue.cu) runs the default-lowered programs of many networks: every launch
// of every program becomes a phase, every phase a few tasks (ranges of the kernel's blocks, or of
// a tensor-core GEMM's work items), and the tasks form one queue that the launch's persistent
// thread blocks take in order. A task waits until the previous phase of its program is complete,
// which keeps each program's launch order; different programs overlap freely.

enum QKind : int32_t {
  QK_LEAVES = 0,       // leaf_body, one block per leaf
  QK_SMALL = 1,        // small_body
  QK_SPLITK = 2,       // splitk_body
  QK_SPLITK_DONE = 3,  // splitk_done_body, one block per step
  QK_DOT = 4,          // dot_body
  QK_PERM = 5,         // perm_body, blocks = grid_x * (number of perms)
  QK_GEMM = 6,         // tensor-core GEMM work items
  QK_SPLIT_SUM = 7,    // split_sum_body over the K-split workspace
  QK_OPEN = 8,         // open_body
  QK_FINAL = 9,        // final_body (one block)
};

struct QPhase {
  int32_t kind;
  int32_t ntasks;      // tasks of the phase: its completion count
  int32_t prev;        // phase that must be complete first (-1: none)
  int32_t nblocks;     // the kernel's blocks, or the GEMM's work items
  int32_t count;       // steps / perms / leaves of the launch
  int32_t grid_x;      // QK_PERM: blocks per perm
  int32_t flag;        // QK_DOT: FP32 products; QK_GEMM: operand kind (0 TF32, 1 bf16, 2 scaled fp16)
  int32_t bn;          // QK_GEMM: tile width
  int32_t ksplit;      // QK_SPLIT_SUM: splits
  int32_t pad;
  int64_t n;           // QK_SPLIT_SUM: elements of the result
  char* base;          // the program's arena
  const void* desc;    // steps / perms / leaves / final record (device)
  const void* gemm;    // QK_GEMM: the GEMM's parameter block (device, 64-byte aligned)
  // per kind: LEAVES p0 = packed inputs; SPLITK / DOT p0 = split partials; SPLITK_DONE p0 =
  // partials, p1 = scalar slots; SPLIT_SUM p0 = workspace, p1 = result (both FP32, cast to this
  // field's type); OPEN p0 = scalar slots, p1 = traces, p2 = block partials; FINAL p0 = scalar
  // slots, p1 = result, p2 = block partials, p3 = optional copy of (S, F, 1 - F)
  double* p0;
  double* p1;
  double* p2;
  double* p3;
};

struct QTask {
  int32_t phase;
  int32_t b0, b1;      // blocks (work items) [b0, b1) of the phase
  int32_t pad;
};

// Counters of one interpreter launch (int32, zeroed before it): the next task to take, an error
// flag (a bounded wait expired), then one completion count per phase.
constexpr int kQNext = 0, kQError = 1, kQPhase0 = 4;

}  // namespace ajf
