// Tensor-core GEMM on sm_103a: tcgen05.mma with TMEM accumulators, TMA-fed shared-memory stages,
// and promotion of partial sums to round-to-nearest FP32 on the CUDA cores.
//
//   C[M][N] (FP64, row-major) = sum_{i + j < T} A_i[M][K] . B_j[N][K]^T
//
// A_t and B_t (t < T) are the terms of a split operand -- x = x_0 + x_1 (+ x_2) -- stored
// K-contiguous (K-major) in TF32 (FP32 containers, pre-rounded) or bf16. T = 1 is a plain
// one-pass product; T = 2 is the three-product split (hi.hi + hi.lo + lo.hi); T = 3 the
// six-product split. The complex contraction step arrives here as one real GEMM (the caller
// embedded the complex operand as [[Re,-Im],[Im,Re]]).
//
// Why promotion: the tensor core's FP32 accumulation truncates. Measured on GB300 with positive
// operands, the mean relative error of a TMEM accumulation over K is about -(K/8) * 2^-24 (one
// half-ulp per MMA instruction, always toward zero), a bias far above what round-to-nearest FP32
// gives. Here every 128-byte K block is accumulated into fresh TMEM partials, two slices of two
// leading-term instructions each; the small correction products of the block are issued first
// into slice 0 (while its magnitude is still small), and the epilogue warps add both slices into
// FP32 registers with round-to-nearest. Partials are double buffered (2 blocks x 2 slices x BN
// columns = 512 TMEM columns at BN = 128), so draining one block overlaps the MMAs of the next.
//
// Kernel structure (one CTA per 128 x BN output tile, 320 threads):
//   warp 0, lane 0 : TMA producer -- per K block, the T terms of the A tile (128 rows x 128 B) and
//                    of the B tile (BN rows x 128 B), 128-byte swizzle, loaded once each into one
//                    shared-memory slot of a ring (mbarrier expect-tx / complete-tx);
//   warp 1         : allocates TMEM; lane 0 issues tcgen05.mma (M=128, N=BN, 32 B of K each) and
//                    tcgen05.commit to release slots and hand partials to the epilogue;
//   warps 2..9     : epilogue -- two warps per TMEM lane quarter (warp % 4), each owning half of
//                    the BN columns: tcgen05.ld, FP32 round-to-nearest accumulation in registers,
//                    FP64 store of C.
// Every wait is bounded by the global timer (2 s); on expiry the kernel records a status code,
// stops issuing work, releases TMEM and returns, so the host sees AJF_E_TIMEOUT instead of a hang.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "kernels.h"

namespace ajf {
namespace {

constexpr int kBM = 128;             // rows per tile (UMMA M)
constexpr int kRowBytes = 128;       // bytes of K per tile row (one 128-byte swizzle span)
constexpr int kMaxSlots = 6;
constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;
constexpr int kMaxTerms = 3;
constexpr uint32_t kSmemBudget = 192 * 1024;
constexpr unsigned long long kWaitNs = 2000000000ull;

struct TcParams {
  CUtensorMap amap[kMaxTerms];
  CUtensorMap bmap[kMaxTerms];
  double* C;
  int* status;
  int64_t N;
  int32_t terms, kblocks, ntn, slots;
  uint32_t idesc;
  uint32_t slot_bytes;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false (and status set) if the phase did not complete within kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t n = 1;; ++n) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((n & 255) == 0 && globaltimer() - t0 > kWaitNs) {
      atomicExch(status, code);
      return false;
    }
  }
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFF);        // start address
  d |= static_cast<uint64_t>(1) << 16;                      // leading byte offset (unused for SW128 K-major)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;              // stride byte offset: 8 rows x 128 B
  d |= static_cast<uint64_t>(1) << 46;                      // descriptor version for tcgen05
  d |= static_cast<uint64_t>(2) << 61;                      // 128-byte swizzle
  return d;
}

template <bool kBF16>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (kBF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <int BN, bool kBF16>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_tc(const __grid_constant__ TcParams p) {
  static_assert(BN == 32 || BN == 64 || BN == 128, "tile width");
  constexpr uint32_t ncols = 4 * BN;  // 2 buffers x 2 slices
  constexpr int HALF = BN / 2;        // columns per epilogue warp
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t a_bytes = kBM * kRowBytes, b_bytes = BN * kRowBytes;
  const int S = p.slots, T = p.terms;
  uint8_t* bars = smem + S * p.slot_bytes;
  const uint32_t full0 = smem_u32(bars);
  const uint32_t empty0 = full0 + 8 * kMaxSlots;
  const uint32_t accf0 = empty0 + 8 * kMaxSlots;  // partial buffer b ready (MMA -> epilogue)
  const uint32_t acce0 = accf0 + 16;              // partial buffer b drained (epilogue -> MMA)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 16 * kMaxSlots + 32);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 16 * kMaxSlots + 36);
  const int64_t m0 = static_cast<int64_t>(blockIdx.x / p.ntn) * kBM;
  const int64_t n0 = static_cast<int64_t>(blockIdx.x % p.ntn) * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, kEpiWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int kblocks = p.kblocks;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: one slot per K block holds every term of A and B
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb % S;
      const uint32_t ph = static_cast<uint32_t>(kb / S) & 1u;
      if (*abort_flag || !mbar_wait(empty0 + 8 * s, ph ^ 1u, p.status, 11)) {
        *abort_flag = 1;
        break;
      }
      const uint32_t base = smem_u32(smem + s * p.slot_bytes);
      const int32_t kx = kb * (kRowBytes / (kBF16 ? 2 : 4));
      mbar_expect_tx(full0 + 8 * s, static_cast<uint32_t>(T) * (a_bytes + b_bytes));
      for (int t = 0; t < T; ++t) {
        const uint32_t sa = base + t * (a_bytes + b_bytes);
        tma_load_2d(sa, &p.amap[t], kx, static_cast<int32_t>(m0), full0 + 8 * s);
        tma_load_2d(sa + a_bytes, &p.bmap[t], kx, static_cast<int32_t>(n0), full0 + 8 * s);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    bool ok = true;
    for (int kb = 0; kb < kblocks; ++kb) {
      const int b = kb & 1;
      const int s = kb % S;
      if (*abort_flag || !mbar_wait(acce0 + 8 * b, (static_cast<uint32_t>(kb >> 1) & 1u) ^ 1u, p.status, 14) ||
          !mbar_wait(full0 + 8 * s, static_cast<uint32_t>(kb / S) & 1u, p.status, 12)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(smem + s * p.slot_bytes);
      const uint32_t slice0 = tmem + static_cast<uint32_t>((2 * b) * BN);
      const uint32_t slice1 = slice0 + BN;
      uint32_t acc0 = 0;
      // correction products (i + j >= 1), smallest first, into slice 0
      for (int sum = T - 1; sum >= 1; --sum)
        for (int i = 0; i <= sum; ++i) {
          const int j = sum - i;
          const uint32_t sa = base + i * (a_bytes + b_bytes);
          const uint32_t sb = base + j * (a_bytes + b_bytes) + a_bytes;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            mma<kBF16>(slice0, smem_desc(sa + 32 * kk), smem_desc(sb + 32 * kk), p.idesc, acc0);
            acc0 = 1;
          }
        }
      // leading product: instructions 0-1 into slice 0, 2-3 into slice 1
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t da = smem_desc(base + 32 * kk), db = smem_desc(base + a_bytes + 32 * kk);
        if (kk < 2) {
          mma<kBF16>(slice0, da, db, p.idesc, acc0);
          acc0 = 1;
        } else {
          mma<kBF16>(slice1, da, db, p.idesc, kk == 3 ? 1u : 0u);
        }
      }
      mma_commit(empty0 + 8 * s);
      mma_commit(accf0 + 8 * b);
    }
    if (!ok) *abort_flag = 1;
  } else if (warp >= 2) {
    // ---- epilogue: promote partials into round-to-nearest FP32 registers, store FP64
    const int q = warp & 3, h = (warp - 2) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(32 * q) << 16;
    float acc[HALF];
#pragma unroll
    for (int j = 0; j < HALF; ++j) acc[j] = 0.0f;
    bool ok = true;
    for (int kb = 0; kb < kblocks; ++kb) {
      const int b = kb & 1;
      int w = 1;
      if (lane == 0) w = mbar_wait(accf0 + 8 * b, static_cast<uint32_t>(kb >> 1) & 1u, p.status, 13) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, w, 0) != 0;
      if (!ok || *abort_flag) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) {
        const uint32_t col = static_cast<uint32_t>((2 * b + sl) * BN + h * HALF);
        uint32_t r[HALF];
#pragma unroll
        for (int c0 = 0; c0 < HALF; c0 += 16)
          tmem_ld16(tmem + lane_base + col + c0, *reinterpret_cast<uint32_t(*)[16]>(&r[c0]));
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < HALF; ++j) acc[j] += __uint_as_float(r[j]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * b);
    }
    if (ok && !*abort_flag) {
      const int64_t row = m0 + 32 * q + lane;
      double2* dst = reinterpret_cast<double2*>(p.C + row * p.N + n0 + h * HALF);
#pragma unroll
      for (int j = 0; j < HALF / 2; ++j)
        dst[j] = make_double2(static_cast<double>(acc[2 * j]), static_cast<double>(acc[2 * j + 1]));
    } else {
      *abort_flag = 1;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
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

bool make_map(CUtensorMap* map, void* ptr, int64_t rows, int64_t k, uint32_t box_rows, bool bf16) {
  EncodeFn fn = encode_fn();
  if (!fn) return false;
  const size_t es = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(k), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(k * es)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kRowBytes / es), box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ptr, dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, bool BF16>
cudaError_t launch_tile(TcParams p, int64_t M, int64_t N, cudaStream_t s) {
  p.slot_bytes = static_cast<uint32_t>(p.terms) * (kBM + BN) * kRowBytes;
  p.slots = static_cast<int32_t>(kSmemBudget / p.slot_bytes);
  if (p.slots > kMaxSlots) p.slots = kMaxSlots;
  if (p.slots < 1) return cudaErrorInvalidValue;
  const size_t smem = size_t(p.slots) * p.slot_bytes + 1024 /* barriers */ + 1024 /* alignment */;
  const int64_t tiles = (M / kBM) * (N / BN);
  if (tiles > 0x7FFFFFFF) return cudaErrorInvalidValue;
  p.ntn = static_cast<int32_t>(N / BN);
  const uint32_t fmt = BF16 ? 1u : 2u;  // A/B type: TF32 = 2, BF16 = 1; D = F32; both K-major
  p.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(BN >> 3) << 17) |
            (static_cast<uint32_t>(kBM >> 4) << 24);
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<BN, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_gemm_tc<BN, BF16><<<static_cast<unsigned>(tiles), kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

bool tc_gemm_supported(int64_t M, int64_t N, int64_t K, int kind) {
  const int64_t bk = kind == 1 ? 64 : 32;  // elements per 128-byte row
  return M >= kBM && (M % kBM) == 0 && N >= 32 && (N & (N - 1)) == 0 && K >= bk && (K % bk) == 0 &&
         M * N <= (int64_t(1) << 40);
}

cudaError_t launch_gemm_tc(char* base, const int64_t* a_off, const int64_t* b_off, int terms, double* C, int64_t M,
                           int64_t N, int64_t K, int kind, int* d_status, cudaStream_t s) {
  if (!tc_gemm_supported(M, N, K, kind) || terms < 1 || terms > kMaxTerms) return cudaErrorNotSupported;
  const bool bf16 = kind == 1;
  const int bn = N >= 128 ? 128 : static_cast<int>(N);
  TcParams p;
  std::memset(&p, 0, sizeof(p));
  for (int t = 0; t < terms; ++t) {
    if (!make_map(&p.amap[t], base + a_off[t], M, K, kBM, bf16)) return cudaErrorInvalidValue;
    if (!make_map(&p.bmap[t], base + b_off[t], N, K, static_cast<uint32_t>(bn), bf16)) return cudaErrorInvalidValue;
  }
  p.C = C;
  p.status = d_status;
  p.N = N;
  p.terms = terms;
  p.kblocks = static_cast<int32_t>(K / (kRowBytes / (bf16 ? 2 : 4)));
  if (bf16) {
    if (bn == 128) return launch_tile<128, true>(p, M, N, s);
    if (bn == 64) return launch_tile<64, true>(p, M, N, s);
    return launch_tile<32, true>(p, M, N, s);
  }
  if (bn == 128) return launch_tile<128, false>(p, M, N, s);
  if (bn == 64) return launch_tile<64, false>(p, M, N, s);
  return launch_tile<32, false>(p, M, N, s);
}

}  // namespace ajf
