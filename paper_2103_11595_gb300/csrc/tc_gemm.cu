// Tensor-core GEMM on sm_103a: tcgen05.mma with TMEM accumulators, TMA-fed shared-memory stages,
// and promotion of partial sums to round-to-nearest FP32 on the CUDA cores.
//
//   C[M][N] (FP32, row-major) = sum_{i + j < T} A_i[M][K] . B_j[N][K]^T
//
// A_t and B_t (t < T) are the terms of a split operand -- x = x_0 + x_1 (+ x_2) -- stored
// K-contiguous (K-major) in TF32 (FP32 containers) or bf16. T = 1 is a plain one-pass product;
// T = 2 is the three-product split (x_0.y_0 + x_0.y_1 + x_1.y_0); T = 3 the six-product split.
// The complex contraction step arrives here as one real GEMM (the caller embedded the complex
// operand as [[Re,-Im],[Im,Re]]).
//
// Accuracy. The tensor core's FP32 accumulation truncates toward zero: measured on GB300 with
// positive operands, a TMEM accumulation over K drifts by about -(K/8) * 2^-24 relative, far above
// round-to-nearest FP32, and a drift of that kind compounds over the dozens of GEMMs of one
// contraction. In the six-product split the kernel removes the drift by construction instead of
// correcting it:
//  * exact leading product: the operand preparation (k_perm) makes every leading term x_0 an
//    integer multiple of a power of two q fixed per row and 128-byte K block, with |x_0 / q| <= 2^8.
//    Within one K block every product x_0 y_0 is then a multiple of q_x q_y of magnitude at most
//    2^16 q_x q_y, and the block's sum of 64 of them stays below 2^24 q_x q_y: the TMEM accumulation
//    of the leading product loses no bit at all (the middle and low terms carry the remainder
//    x - x_0 to 2^-26 of the block's largest entry);
//  * two partials per K block: the leading product goes into its own fresh TMEM partial P0, the
//    correction products (about 2^-8 of it) into a second fresh partial P1, whose truncation is
//    relative to |P1| and so at most ~2^-31 of the result per instruction;
//  * promotion: eight epilogue warps add P0 + P1 of every K block into FP32 registers with
//    round-to-nearest (unbiased), at most kMaxBlocksPerSplit blocks per register sum; longer
//    contractions are split over K and the FP32 partial tiles summed (compensated) in a fixed order.
// No calibrated correction factor is involved; the promoted FP32 sums are the stored result.
// The two-term splits (TF32 and bf16 three-product modes) keep a floating leading term, whose 11
// or 8 significant bits follow each entry: their P0 truncates like a plain accumulation, one
// promoted K block at a time, and they are bounded modes, not FP32-class ones.
//
// Kernel structure (persistent: at most one CTA per SM walks the 128 x BN output tiles in a
// grouped raster order; 320 threads; the slot and TMEM-buffer rings continue from tile to tile so
// the loads and MMAs of the next tile overlap the store of the current one):
//   warp 0, lane 0 : TMA producer -- for every K block and term, the A tile (128 rows x 128 B) and
//                    the B tile (BN rows x 128 B), 128-byte swizzle, into a ring of slots
//                    (mbarrier expect-tx / complete-tx);
//   warp 1         : allocates TMEM; lane 0 issues tcgen05.mma (M=128, N=BN, 32 B of K each) into
//                    a ring of TMEM buffers (two partials of BN columns each) and tcgen05.commit
//                    to release slots and hand partials to the epilogue;
//   warps 2..9     : epilogue -- two warps per TMEM lane quarter (warp % 4), each owning half of
//                    the BN columns of its rows: tcgen05.ld, FP32 round-to-nearest accumulation in
//                    registers, FP32 store of the tile (rows < M, columns < N) staged through
//                    shared memory so that every warp store writes whole 128-byte row segments.
// Work items are (tile, K split) pairs. GEMMs with fewer tiles than SMs, or with more than
// kMaxBlocksPerSplit K blocks, split K over several work items; each split writes an FP32 partial
// tile to a workspace and k_split_sum adds the splits in a fixed order (deterministic).
// Every wait is bounded by the global timer (2 s); on expiry the kernel records a status code,
// stops issuing work, waits (bounded again) for the TMA loads and MMAs it already issued,
// releases TMEM and returns, so the host sees AJF_E_TIMEOUT instead of a hang.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "bodies.cuh"
#include "kernels.h"
#include "tc_gemm_dev.cuh"

namespace ajf {
namespace {

using namespace tc;

template <int BN, int kKind>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(const __grid_constant__ TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5;
  // TMEM: NB buffers of two partials (P0: leading product, P1: corrections), BN columns each
  const uint32_t ncols =
      static_cast<uint32_t>(2 * p.bufs * BN) < 32u ? 32u : static_cast<uint32_t>(2 * p.bufs * BN);
  TcShared sh;
  uint32_t* tmem_slot = tc_layout(smem, smem + p.slots * p.slot_bytes, sh);
  if (threadIdx.x == 0) tc_init_barriers(sh, p.slots, p.bufs);
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  sh.tmem = *tmem_slot;
  TcRing ring;
  const uint32_t nwork = static_cast<uint32_t>(p.tiles) * static_cast<uint32_t>(p.ksplit);
  tc_gemm_items<BN, kKind>(p, blockIdx.x, nwork, gridDim.x, sh, ring);
  if (*sh.abort_flag) tc_drain_after_abort(p.slots, p.bufs, p.wait_ns, p.status, sh, ring);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  // __syncthreads (bar.sync, the aligned form) must be executed by all threads of a warp
  // together; warps 0 and 1 get here diverged (lane 0 ran the producer / MMA loop, lanes 1-31 came
  // straight through), so they reconverge first. The barrier then orders warp 1's TMEM release
  // after every epilogue warp's last TMEM read and after the abort drains above.
  __syncwarp();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sh.tmem), "r"(ncols) : "memory");
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(f);
  });
  return fn;
}

bool make_map(CUtensorMap* map, void* ptr, int64_t rows, int64_t k, uint32_t box_rows, int kind) {
  EncodeFn fn = encode_fn();
  if (!fn) return false;
  const size_t es = kind != 0 ? 2 : 4;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(k), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(k * es)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kRowBytes / es), box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : (kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
  return fn(map, dt, 2, ptr, dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// SM count of the current device (queried once per device).
int sm_count() {
  static int counts[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (counts[dev] == 0) cudaDeviceGetAttribute(&counts[dev], cudaDevAttrMultiProcessorCount, dev);
  return counts[dev];
}

template <int BN, int KIND>
void run_tile(const void* params, unsigned grid, size_t smem, cudaStream_t s) {
  k_gemm_tc<BN, KIND><<<grid, kThreads, smem, s>>>(*static_cast<const TcParams*>(params));
}

// Fill the tile geometry of `p` and the launch shape of `t` (host only; nothing is enqueued).
template <int BN, int KIND>
cudaError_t prepare_tile(TcParams& p, TcPrepared* t, int64_t M, int64_t N) {
  p.slot_bytes = static_cast<uint32_t>((kBM + BN) * kRowBytes);
  p.slots = static_cast<int32_t>(kSmemBudget / p.slot_bytes);
  if (p.slots > kMaxSlots) p.slots = kMaxSlots;
  if (p.slots < p.terms) return cudaErrorInvalidValue;
  p.bufs = 256 / BN > kMaxBufs ? kMaxBufs : 256 / BN;  // each buffer: 2 partials x BN TMEM columns
  p.tmem_stride = 2 * BN;
  const size_t smem = size_t(p.slots) * p.slot_bytes + kTcControlBytes + 1024 /* alignment */;
  const int64_t mt = (M + kBM - 1) / kBM, nt = (N + BN - 1) / BN;
  const int64_t tiles = mt * nt;
  if (mt > 0x7FFFFFFF || nt > 0x7FFFFFFF) return cudaErrorInvalidValue;
  p.ntn = static_cast<int32_t>(nt);
  p.mtn = static_cast<int32_t>(mt);
  p.group = static_cast<int32_t>(mt < 8 ? mt : 8);
  p.tiles = tiles;
  // persistent grid: at most one CTA per SM (the kernel holds 1 CTA/SM), each walking tiles with a stride
  const int sms = sm_count();
  if (sms <= 0) return cudaErrorInvalidDevice;
  // work items are (tile, K split) pairs: a GEMM with few tiles but many K splits still spreads
  // over every SM
  const int64_t work = tiles * static_cast<int64_t>(p.ksplit);
  // as few CTAs as keep the number of rounds (work items per CTA) at its minimum: the last round
  // is no longer partly empty, and the SMs left over run other streams' kernels meanwhile
  const int64_t rounds = (work + sms - 1) / sms;
  const int64_t grid = (work + rounds - 1) / rounds;
  // A/B type: TF32 = 2 (kind::tf32), BF16 = 1, F16 = 0 (kind::f16); D = F32; both K-major
  const uint32_t fmt = KIND == 0 ? 2u : (KIND == 1 ? 1u : 0u);
  p.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(BN >> 3) << 17) |
            (static_cast<uint32_t>(kBM >> 4) << 24);
  // the shared-memory opt-in is a per-function attribute: set once per device (the size is the
  // same for every launch of one instantiation)
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(k_gemm_tc<BN, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  t->grid = static_cast<unsigned>(grid);
  t->smem = smem;
  t->run = &run_tile<BN, KIND>;
  return cudaSuccess;
}

}  // namespace

// Shapes are powers of two (binary-index tensors). Tiles may overhang the matrices: TMA fills the
// rows of a box beyond M or N, and the K columns beyond the last full 128-byte row, with zeros, and
// the epilogue stores only rows < M and columns < N. Row strides must be multiples of 16 bytes.
bool tc_gemm_supported(int64_t M, int64_t N, int64_t K, int kind) {
  const int64_t es = kind != 0 ? 2 : 4;
  const bool pow2 = (M & (M - 1)) == 0 && (N & (N - 1)) == 0 && (K & (K - 1)) == 0;
  return pow2 && M >= 32 && N >= 16 && K * es >= 32 && M * N <= (int64_t(1) << 40) && K * es <= (int64_t(1) << 38);
}

int tc_gemm_splits(int64_t M, int64_t N, int64_t K, int kind) {
  const int64_t es = kind != 0 ? 2 : 4;
  const int64_t bn = N >= 128 ? 128 : (N >= 64 ? 64 : 32);
  const int64_t tiles = ((M + kBM - 1) / kBM) * ((N + bn - 1) / bn);
  const int64_t kblocks = (K * es + kRowBytes - 1) / kRowBytes;
  // accuracy: at most kMaxBlocksPerSplit K blocks per split
  int64_t ks = (kblocks + kMaxBlocksPerSplit - 1) / kMaxBlocksPerSplit;
  // parallelism: with fewer tiles than SMs, about two work items per SM, at least 8 K blocks each
  if (tiles < kPlanSMs) {
    int64_t kp = (2 * kPlanSMs + tiles - 1) / tiles;
    if (kp > kblocks / 8) kp = kblocks / 8;
    if (kp > ks) ks = kp;
  }
  // workspace of ksplit * M * N FP32 values: at most 2^30 of them (beyond that, fewer and longer splits)
  while (ks > 1 && ks * M * N * 8 > (int64_t(8) << 30)) --ks;
  if (ks <= 1) return 1;
  const int64_t per = (kblocks + ks - 1) / ks;
  return static_cast<int>((kblocks + per - 1) / per);
}

namespace {

// C[i] = sum over splits s (in order) of W[s][i] (compensated FP32 sum)
__global__ void __launch_bounds__(kBodyThreads) k_split_sum(const float* __restrict__ W, int ksplit, int64_t n,
                                                            float* __restrict__ C) {
  split_sum_body(W, ksplit, n, C, static_cast<int>(blockIdx.x), static_cast<int>(gridDim.x));
}

}  // namespace

cudaError_t tc_gemm_prepare(TcPrepared* t, char* base, const int64_t* a_off, const int64_t* b_off, int terms,
                            float* C, int64_t M, int64_t N, int64_t K, int kind, float* ws, int ksplit,
                            int* d_status, unsigned long long wait_ns, int stall_loads) {
  static_assert(sizeof(TcParams) <= sizeof(t->params), "kernel parameters exceed the prepared-launch buffer");
  t->ready = false;
  if (!tc_gemm_supported(M, N, K, kind) || terms < 1 || terms > kMaxTerms) return cudaErrorNotSupported;
  if (ksplit < 1 || (ksplit > 1 && !ws)) return cudaErrorInvalidValue;
  if (kind < 0 || kind > 2 || (kind == 2 && terms != 2)) return cudaErrorInvalidValue;
  // BN = 256 would need 128 FP32 accumulators per epilogue thread and spill at 320 threads.
  const int bn = N >= 128 ? 128 : (N >= 64 ? 64 : 32);
  TcParams p;
  std::memset(&p, 0, sizeof(p));
  for (int i = 0; i < terms; ++i) {
    if (!make_map(&p.amap[i], base + a_off[i], M, K, kBM, kind)) return cudaErrorInvalidValue;
    if (!make_map(&p.bmap[i], base + b_off[i], N, K, static_cast<uint32_t>(bn), kind)) return cudaErrorInvalidValue;
  }
  if (kind == 2) {  // the scale arrays ride in the third offset: [K block][M] and [K block][N] floats
    p.sa = reinterpret_cast<const float*>(base + a_off[2]);
    p.sb = reinterpret_cast<const float*>(base + b_off[2]);
  }
  p.C = C;
  p.ws = ws;
  p.status = d_status;
  p.M = M;
  p.N = N;
  p.terms = terms;
  p.wait_ns = wait_ns;
  p.stall_loads = stall_loads;
  const int64_t row_elems = kRowBytes / (kind != 0 ? 2 : 4);
  p.kblocks = static_cast<int32_t>((K + row_elems - 1) / row_elems);
  p.kb_split = (p.kblocks + ksplit - 1) / ksplit;
  p.ksplit = (p.kblocks + p.kb_split - 1) / p.kb_split;
  if (p.ksplit != ksplit) return cudaErrorInvalidValue;  // the workspace was sized for `ksplit` splits
  cudaError_t e;
  if (kind == 2) {
    if (bn == 128) e = prepare_tile<128, 2>(p, t, M, N);
    else if (bn == 64) e = prepare_tile<64, 2>(p, t, M, N);
    else e = prepare_tile<32, 2>(p, t, M, N);
  } else if (kind == 1) {
    if (bn == 128) e = prepare_tile<128, 1>(p, t, M, N);
    else if (bn == 64) e = prepare_tile<64, 1>(p, t, M, N);
    else e = prepare_tile<32, 1>(p, t, M, N);
  } else {
    if (bn == 128) e = prepare_tile<128, 0>(p, t, M, N);
    else if (bn == 64) e = prepare_tile<64, 0>(p, t, M, N);
    else e = prepare_tile<32, 0>(p, t, M, N);
  }
  if (e != cudaSuccess) return e;
  std::memcpy(t->params, &p, sizeof(p));
  t->ksplit = ksplit;
  t->ws = ws;
  t->C = C;
  t->n = M * N;
  t->ready = true;
  return cudaSuccess;
}

cudaError_t tc_gemm_run(const TcPrepared& t, cudaStream_t s) {
  if (!t.ready) return cudaErrorInvalidValue;
  t.run(t.params, t.grid, t.smem, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || t.ksplit == 1) return e;
  const int64_t blocks = (t.n + 255) / 256 < 4096 ? (t.n + 255) / 256 : 4096;
  k_split_sum<<<static_cast<unsigned>(blocks), kBodyThreads, 0, s>>>(t.ws, t.ksplit, t.n, t.C);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(char* base, const int64_t* a_off, const int64_t* b_off, int terms, float* C, int64_t M,
                           int64_t N, int64_t K, int kind, float* ws, int ksplit, int* d_status, cudaStream_t s) {
  return launch_gemm_tc_ex(base, a_off, b_off, terms, C, M, N, K, kind, ws, ksplit, d_status, s, kWaitNs, 0);
}

cudaError_t launch_gemm_tc_ex(char* base, const int64_t* a_off, const int64_t* b_off, int terms, float* C, int64_t M,
                              int64_t N, int64_t K, int kind, float* ws, int ksplit, int* d_status, cudaStream_t s,
                              unsigned long long wait_ns, int stall_loads) {
  TcPrepared t;
  cudaError_t e = tc_gemm_prepare(&t, base, a_off, b_off, terms, C, M, N, K, kind, ws, ksplit, d_status, wait_ns,
                                  stall_loads);
  if (e != cudaSuccess) return e;
  return tc_gemm_run(t, s);
}

}  // namespace ajf
