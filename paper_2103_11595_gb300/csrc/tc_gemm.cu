// Tensor-core GEMM on sm_103a: tcgen05.mma with TMEM accumulators, TMA-fed shared-memory stages,
// and promotion of partial sums to round-to-nearest FP32 on the CUDA cores.
//
//   C[M][N] (FP64, row-major) = sum_{i + j < T} A_i[M][K] . B_j[N][K]^T
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
//    contractions are split over K and the FP64 partial tiles summed in a fixed order.
// No calibrated correction factor is involved; the result is stored as FP32 -> FP64 exactly.
// The two-term splits (TF32 and bf16 three-product modes) keep a floating leading term, whose 11
// or 8 significant bits follow each entry: their P0 truncates like a plain accumulation, one
// promoted K block at a time, and they are bounded modes, not FP32-class ones.
//
// Kernel structure (persistent: one CTA per SM walks the 128 x BN output tiles in a grouped
// raster order; 320 threads; the slot and TMEM-buffer rings continue from tile to tile so the
// loads and MMAs of the next tile overlap the FP64 store of the current one):
//   warp 0, lane 0 : TMA producer -- for every K block and term, the A tile (128 rows x 128 B) and
//                    the B tile (BN rows x 128 B), 128-byte swizzle, into a ring of slots
//                    (mbarrier expect-tx / complete-tx);
//   warp 1         : allocates TMEM; lane 0 issues tcgen05.mma (M=128, N=BN, 32 B of K each) into
//                    a ring of TMEM buffers (two partials of BN columns each) and tcgen05.commit
//                    to release slots and hand partials to the epilogue;
//   warps 2..9     : epilogue -- two warps per TMEM lane quarter (warp % 4), each owning half of
//                    the BN columns of its rows: tcgen05.ld, FP32 round-to-nearest accumulation in
//                    registers, FP64 store of the tile (rows < M, columns < N).
// Work items are (tile, K split) pairs. GEMMs with fewer tiles than SMs, or with more than
// kMaxBlocksPerSplit K blocks, split K over several work items; each split writes an FP64 partial
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

#include "fp_bits.h"
#include "kernels.h"

namespace ajf {
namespace {

constexpr int kBM = 128;             // rows per tile (UMMA M)
constexpr int kRowBytes = 128;       // bytes of K per tile row (one 128-byte swizzle span)
constexpr int kMaxSlots = 8;
constexpr int kMaxBufs = 4;
constexpr int kThreads = 320;
constexpr int kEpiWarps = 8;
constexpr int kEpiWarp0 = 2;       // epilogue warps 2..9: warp w reads TMEM lanes 32 * (w % 4) .. + 31
// The FP32 register accumulation of promoted partials spans at most this many K blocks: longer
// contractions are split over K (FP64 partial tiles summed afterwards), so the small late
// partials of a long FP32 running sum are not lost.
constexpr int kMaxBlocksPerSplit = 64;
// SM count the K-split heuristic plans for (GB300); the split count only changes how work is
// divided, never the result beyond rounding.
constexpr int64_t kPlanSMs = 152;
constexpr int kMaxTerms = 3;
constexpr uint32_t kSmemBudget = 192 * 1024;
constexpr unsigned long long kWaitNs = kTcWaitNs;

struct TcParams {
  CUtensorMap amap[kMaxTerms];
  CUtensorMap bmap[kMaxTerms];
  double* C;
  int* status;
  int64_t M, N;
  int32_t terms, kblocks, ntn, slots, bufs;
  int32_t mtn;                       // tiles along M
  int32_t group;                     // M tiles per raster group (L2 reuse of B tiles)
  int32_t ksplit, kb_split;          // K splits and K blocks per split
  int64_t tiles;
  double* ws;                        // split partials [ksplit][M][N] (ksplit > 1)
  uint32_t idesc;
  uint32_t slot_bytes;
  unsigned long long wait_ns;        // bound of every wait
  int32_t stall_loads;               // test hook: the producer issues no loads, so every wait expires
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

// Bounded wait: false (and status set) if the phase did not complete within limit_ns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns, int* status,
                                          int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t n = 1;; ++n) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((n & 255) == 0 && globaltimer() - t0 > limit_ns) {
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
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
  constexpr int COLS = BN / 2;                       // columns per epilogue thread (one TMEM lane = one row)
  constexpr int CH = COLS < 16 ? COLS : 16;          // columns per drain chunk
  constexpr uint32_t a_bytes = kBM * kRowBytes, b_bytes = BN * kRowBytes;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = p.slots, T = p.terms, NB = p.bufs;
  // TMEM: NB buffers of two partials (P0: leading product, P1: corrections), BN columns each
  const uint32_t ncols = static_cast<uint32_t>(2 * NB * BN) < 32u ? 32u : static_cast<uint32_t>(2 * NB * BN);
  uint8_t* bars = smem + S * p.slot_bytes;
  const uint32_t full0 = smem_u32(bars);
  const uint32_t empty0 = full0 + 8 * kMaxSlots;
  const uint32_t accf0 = empty0 + 8 * kMaxSlots;  // partial buffer b ready (MMA -> epilogue)
  const uint32_t acce0 = accf0 + 8 * kMaxBufs;    // partial buffer b drained (epilogue -> MMA)
  const uint32_t drain0 = acce0 + 8 * kMaxBufs;   // MMAs issued before an abort have completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 16 * kMaxSlots + 16 * kMaxBufs + 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 16 * kMaxSlots + 16 * kMaxBufs + 12);
  // persistent tile loop: tile = blockIdx.x, blockIdx.x + gridDim.x, ...; every role walks the
  // same tiles, and its ring positions (slots, TMEM buffers) continue across tiles
  // grouped raster: `group` M tiles sweep the N tiles together, so concurrently running CTAs
  // share each B tile through L2 instead of streaming all of B once per M tile. Work item wi is
  // tile wi % tiles of K split wi / tiles (tile and work counts fit 32 bits).
  const uint32_t tiles = static_cast<uint32_t>(p.tiles);
  const uint32_t nwork = tiles * static_cast<uint32_t>(p.ksplit);
  auto work_item = [&](uint32_t wi, int32_t& m0, int32_t& n0, int& kb0, int& kb1) {
    const uint32_t tile = wi % tiles, ks = wi / tiles;
    const uint32_t per_group = static_cast<uint32_t>(p.group) * static_cast<uint32_t>(p.ntn);
    const uint32_t g = tile / per_group, r = tile % per_group;
    const uint32_t first_m = g * static_cast<uint32_t>(p.group);
    const uint32_t left = static_cast<uint32_t>(p.mtn) - first_m;
    const uint32_t gm = left < static_cast<uint32_t>(p.group) ? left : static_cast<uint32_t>(p.group);
    m0 = static_cast<int32_t>((first_m + r % gm) * kBM);
    n0 = static_cast<int32_t>((r / gm) * BN);
    kb0 = static_cast<int>(ks) * p.kb_split;
    kb1 = kb0 + p.kb_split < p.kblocks ? kb0 + p.kb_split : p.kblocks;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < NB; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, kEpiWarps);
    }
    mbar_init(drain0, 1);
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

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: one slot per (K block, term) holds that term's A and B tiles. A block's
    // terms are loaded highest first, the order in which the MMA issuer frees their slots.
    int slot = 0;
    uint32_t phase = 0;   // position in the slot ring, continued across tiles
    uint32_t issued = 0;  // slots loaded so far (the last min(issued, S) may still be in flight)
    bool ok = !p.stall_loads;
    for (uint32_t wi = blockIdx.x; wi < nwork && ok; wi += gridDim.x) {
      int32_t m0, n0;
      int kb0, kb1;
      work_item(wi, m0, n0, kb0, kb1);
      for (int kb = kb0; kb < kb1 && ok; ++kb) {
        for (int j = 0; j < T; ++j) {
          const int t = T - 1 - j;
          if (*abort_flag || !mbar_wait(empty0 + 8 * slot, phase ^ 1u, p.wait_ns, p.status, 11)) {
            *abort_flag = 1;
            ok = false;
            break;
          }
          const uint32_t sa = smem_u32(smem + slot * p.slot_bytes);
          const int32_t kx = kb * (kRowBytes / (kBF16 ? 2 : 4));
          mbar_expect_tx(full0 + 8 * slot, a_bytes + b_bytes);
          tma_load_2d(sa, &p.amap[t], kx, m0, full0 + 8 * slot);
          tma_load_2d(sa + a_bytes, &p.bmap[t], kx, n0, full0 + 8 * slot);
          ++issued;
          if (++slot == S) {
            slot = 0;
            phase ^= 1u;
          }
        }
      }
    }
    if (!ok && issued > 0) {
      // abort: before the CTA releases its shared memory, let the loads already issued land (the
      // last min(issued, S) slots; earlier ones were consumed), each wait bounded again
      const uint32_t first = issued > static_cast<uint32_t>(S) ? issued - S : 0u;
      for (uint32_t i = first; i < issued; ++i) {
        const uint32_t sl = i % static_cast<uint32_t>(S), ph = (i / static_cast<uint32_t>(S)) & 1u;
        mbar_wait(full0 + 8 * sl, ph, p.wait_ns, p.status, 15);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    bool ok = true;
    bool any = false;  // MMAs issued (an abort waits for them before TMEM is released)
    int buf = 0, slot = 0;
    uint32_t bphase = 0, phase = 0;  // ring positions, continued across tiles
    for (uint32_t wi = blockIdx.x; wi < nwork && ok; wi += gridDim.x) {
      int32_t m0, n0;
      int kb0, kb1;
      work_item(wi, m0, n0, kb0, kb1);
      for (int kb = kb0; kb < kb1; ++kb) {
        const int b = buf;
        if (*abort_flag || !mbar_wait(acce0 + 8 * b, bphase ^ 1u, p.wait_ns, p.status, 14)) {
          ok = false;
          break;
        }
        if (++buf == NB) {
          buf = 0;
          bphase ^= 1u;
        }
        // ring positions of the block's slots (the producer loads term T-1 first), then the slot
        // and phase of each term; all in scalars -- descriptors and slots kept in registers (a
        // dynamically indexed array would live in local memory and stall every MMA issue)
        int r0 = slot, r1 = 0, r2 = 0;
        uint32_t f0 = phase, f1 = 0u, f2 = 0u;
        auto advance = [&]() {
          if (++slot == S) {
            slot = 0;
            phase ^= 1u;
          }
        };
        advance();
        if (T > 1) {
          r1 = slot;
          f1 = phase;
          advance();
        }
        if (T > 2) {
          r2 = slot;
          f2 = phase;
          advance();
        }
        const int st0 = T == 3 ? r2 : (T == 2 ? r1 : r0), st1 = T == 3 ? r1 : r0, st2 = r0;
        const uint32_t ph0 = T == 3 ? f2 : (T == 2 ? f1 : f0), ph1 = T == 3 ? f1 : f0, ph2 = f0;
        const uint32_t base = smem_u32(smem);
        const uint64_t ad0 = smem_desc(base + st0 * p.slot_bytes), bd0 = smem_desc(base + st0 * p.slot_bytes + a_bytes);
        const uint64_t ad1 = smem_desc(base + st1 * p.slot_bytes), bd1 = smem_desc(base + st1 * p.slot_bytes + a_bytes);
        const uint64_t ad2 = smem_desc(base + st2 * p.slot_bytes), bd2 = smem_desc(base + st2 * p.slot_bytes + a_bytes);
        const uint32_t dst0 = tmem + static_cast<uint32_t>(2 * b * BN);  // P0: the leading product alone
        const uint32_t dst1 = dst0 + static_cast<uint32_t>(BN);          // P1: the correction products
        uint32_t acc = 0;
        // one product A_i . B_j over the block: 4 instructions, 32 bytes of K each (+2 in the
        // descriptor's 16-byte address field)
        auto product = [&](uint32_t dst, uint64_t ad, uint64_t bd) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            mma<kBF16>(dst, ad + 2 * kk, bd + 2 * kk, p.idesc, acc);
            acc = 1;
          }
        };
        auto arrived = [&](int sl, uint32_t ph) {
          const bool w = mbar_wait(full0 + 8 * sl, ph, p.wait_ns, p.status, 12);
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          return w;
        };
        // all of the block's terms are resident before its first MMA (a failed wait then leaves
        // nothing of this block in flight); the correction products go into P1 smallest first, the
        // leading product into P0, and a term's slot is released (commit: freed once the MMAs
        // issued so far complete) right after its last use
        const bool got = (T < 3 || arrived(st2, ph2)) && (T < 2 || arrived(st1, ph1)) && arrived(st0, ph0);
        if (!got) {
          ok = false;
          break;
        }
        any = true;
        if (T == 3) {
          product(dst1, ad0, bd2);
          product(dst1, ad1, bd1);
          product(dst1, ad2, bd0);
          mma_commit(empty0 + 8 * st2);
        }
        if (T >= 2) {
          product(dst1, ad0, bd1);
          product(dst1, ad1, bd0);
          mma_commit(empty0 + 8 * st1);
        }
        acc = 0;
        product(dst0, ad0, bd0);
        mma_commit(empty0 + 8 * st0);
        mma_commit(accf0 + 8 * b);
      }
    }
    if (!ok) {
      *abort_flag = 1;
      if (any) {
        // abort: wait (bounded) until every MMA issued so far has completed, so that none is
        // still writing TMEM or reading shared memory when they are released
        mma_commit(drain0);
        mbar_wait(drain0, 0u, p.wait_ns, p.status, 16);
      }
    }
  } else if (warp >= kEpiWarp0) {
    // ---- epilogue: promote partials into round-to-nearest FP32 registers, store FP64 per tile
    const int q = warp & 3, h = (warp - kEpiWarp0) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(32 * q) << 16;
    float acc[COLS];
    bool ok = true;
    int buf = 0;
    uint32_t bphase = 0;
    for (uint32_t wi = blockIdx.x; wi < nwork && ok; wi += gridDim.x) {
      int32_t m0, n0;
      int kb0, kb1;
      work_item(wi, m0, n0, kb0, kb1);
      const int64_t row = static_cast<int64_t>(m0) + 32 * q + lane;
      const int64_t col0 = static_cast<int64_t>(n0) + h * COLS;
      // rows/columns beyond M, N were zero-filled by TMA and are not stored; M and N are powers of
      // two >= 32 and >= 16, so a warp's 32 rows and COLS columns are all inside or all outside
      const bool mine = row < p.M && col0 < p.N;
      double* dbase = p.ksplit > 1 ? p.ws + static_cast<int64_t>(wi / tiles) * p.M * p.N : p.C;
#pragma unroll
      for (int j = 0; j < COLS; ++j) acc[j] = 0.0f;
      for (int kb = kb0; kb < kb1; ++kb) {
        const int b = buf;
        int w = 1;
        if (lane == 0) w = mbar_wait(accf0 + 8 * b, bphase, p.wait_ns, p.status, 13) ? 1 : 0;
        if (++buf == NB) {
          buf = 0;
          bphase ^= 1u;
        }
        ok = __shfl_sync(0xffffffffu, w, 0) != 0;
        if (!ok || *abort_flag) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t col = static_cast<uint32_t>(2 * b * BN + h * COLS);
#pragma unroll
        for (int c0 = 0; c0 < COLS; c0 += CH) {
          uint32_t r0[CH], r1[CH];
#pragma unroll
          for (int c1 = 0; c1 < CH; c1 += 16) tmem_ld16(tmem + lane_base + col + c0 + c1, r0 + c1);
          if (T > 1) {
#pragma unroll
            for (int c1 = 0; c1 < CH; c1 += 16) tmem_ld16(tmem + lane_base + col + BN + c0 + c1, r1 + c1);
          }
          tmem_wait_ld();
          if (T > 1) {
#pragma unroll
            for (int j = 0; j < CH; ++j) acc[c0 + j] += __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
          } else {
#pragma unroll
            for (int j = 0; j < CH; ++j) acc[c0 + j] += __uint_as_float(r0[j]);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(acce0 + 8 * b);
      }
      if (!ok) break;
      // the MMA warp is already filling the next buffers while this tile is written; FP32 -> FP64
      // is exact and runs on the integer pipe (GB300's FP64 rate would make a hardware conversion
      // per element a visible cost of the store)
      if (mine) {
        double2* dstp = reinterpret_cast<double2*>(dbase + row * p.N + col0);
#pragma unroll
        for (int j = 0; j < COLS / 2; ++j)
          dstp[j] = make_double2(f32_to_f64_scaled(acc[2 * j], 0, 1.0), f32_to_f64_scaled(acc[2 * j + 1], 0, 1.0));
      }
    }
    if (!ok) *abort_flag = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  // __syncthreads (bar.sync, the aligned form) must be executed by all threads of a warp
  // together; warps 0 and 1 get here diverged (lane 0 ran the producer / MMA loop, lanes 1-31 came
  // straight through), so they reconverge first. The barrier then orders warp 1's TMEM release
  // after every epilogue warp's last TMEM read and after the abort drains above.
  __syncwarp();
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

// SM count of the current device (queried once per device).
int sm_count() {
  static int counts[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (counts[dev] == 0) cudaDeviceGetAttribute(&counts[dev], cudaDevAttrMultiProcessorCount, dev);
  return counts[dev];
}

template <int BN, bool BF16>
void run_tile(const void* params, unsigned grid, size_t smem, cudaStream_t s) {
  k_gemm_tc<BN, BF16><<<grid, kThreads, smem, s>>>(*static_cast<const TcParams*>(params));
}

// Fill the tile geometry of `p` and the launch shape of `t` (host only; nothing is enqueued).
template <int BN, bool BF16>
cudaError_t prepare_tile(TcParams& p, TcPrepared* t, int64_t M, int64_t N) {
  p.slot_bytes = static_cast<uint32_t>((kBM + BN) * kRowBytes);
  p.slots = static_cast<int32_t>(kSmemBudget / p.slot_bytes);
  if (p.slots > kMaxSlots) p.slots = kMaxSlots;
  if (p.slots < p.terms) return cudaErrorInvalidValue;
  p.bufs = 256 / BN > kMaxBufs ? kMaxBufs : 256 / BN;  // each buffer: 2 partials x BN TMEM columns
  const size_t smem = size_t(p.slots) * p.slot_bytes + 1024 /* barriers */ + 1024 /* alignment */;
  const int64_t mt = (M + kBM - 1) / kBM, nt = (N + BN - 1) / BN;
  const int64_t tiles = mt * nt;
  if (mt > 0x7FFFFFFF || nt > 0x7FFFFFFF) return cudaErrorInvalidValue;
  p.ntn = static_cast<int32_t>(nt);
  p.mtn = static_cast<int32_t>(mt);
  p.group = static_cast<int32_t>(mt < 8 ? mt : 8);
  p.tiles = tiles;
  // persistent grid: one CTA per SM (the kernel holds 1 CTA/SM), each walking tiles with a stride
  const int sms = sm_count();
  if (sms <= 0) return cudaErrorInvalidDevice;
  // work items are (tile, K split) pairs: a GEMM with few tiles but many K splits still spreads
  // over every SM
  const int64_t work = tiles * static_cast<int64_t>(p.ksplit);
  const int64_t grid = work < sms ? work : sms;
  const uint32_t fmt = BF16 ? 1u : 2u;  // A/B type: TF32 = 2, BF16 = 1; D = F32; both K-major
  p.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(BN >> 3) << 17) |
            (static_cast<uint32_t>(kBM >> 4) << 24);
  // the shared-memory opt-in is a per-function attribute: set once per device (the size is the
  // same for every launch of one instantiation)
  static bool attr_set[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(k_gemm_tc<BN, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  t->grid = static_cast<unsigned>(grid);
  t->smem = smem;
  t->run = &run_tile<BN, BF16>;
  return cudaSuccess;
}

}  // namespace

// Shapes are powers of two (binary-index tensors). Tiles may overhang the matrices: TMA fills the
// rows of a box beyond M or N, and the K columns beyond the last full 128-byte row, with zeros, and
// the epilogue stores only rows < M and columns < N. Row strides must be multiples of 16 bytes.
bool tc_gemm_supported(int64_t M, int64_t N, int64_t K, int kind) {
  const int64_t es = kind == 1 ? 2 : 4;
  const bool pow2 = (M & (M - 1)) == 0 && (N & (N - 1)) == 0 && (K & (K - 1)) == 0;
  return pow2 && M >= 32 && N >= 16 && K * es >= 32 && M * N <= (int64_t(1) << 40) && K * es <= (int64_t(1) << 38);
}

int tc_gemm_splits(int64_t M, int64_t N, int64_t K, int kind) {
  const int64_t es = kind == 1 ? 2 : 4;
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
  // workspace of ksplit * M * N doubles: at most 8 GiB (beyond that, fewer and longer splits)
  while (ks > 1 && ks * M * N * 8 > (int64_t(8) << 30)) --ks;
  if (ks <= 1) return 1;
  const int64_t per = (kblocks + ks - 1) / ks;
  return static_cast<int>((kblocks + per - 1) / per);
}

namespace {

// C[i] = sum over splits s (in order) of W[s][i]
__global__ void __launch_bounds__(256) k_split_sum(const double* __restrict__ W, int ksplit, int64_t n,
                                                   double* __restrict__ C) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    double v = 0;
    for (int s = 0; s < ksplit; ++s) v += W[s * n + i];
    C[i] = v;
  }
}

}  // namespace

cudaError_t tc_gemm_prepare(TcPrepared* t, char* base, const int64_t* a_off, const int64_t* b_off, int terms,
                            double* C, int64_t M, int64_t N, int64_t K, int kind, double* ws, int ksplit,
                            int* d_status, unsigned long long wait_ns, int stall_loads) {
  static_assert(sizeof(TcParams) <= sizeof(t->params), "kernel parameters exceed the prepared-launch buffer");
  t->ready = false;
  if (!tc_gemm_supported(M, N, K, kind) || terms < 1 || terms > kMaxTerms) return cudaErrorNotSupported;
  if (ksplit < 1 || (ksplit > 1 && !ws)) return cudaErrorInvalidValue;
  const bool bf16 = kind == 1;
  // BN = 256 would need 128 FP32 accumulators per epilogue thread and spill at 320 threads.
  const int bn = N >= 128 ? 128 : (N >= 64 ? 64 : 32);
  TcParams p;
  std::memset(&p, 0, sizeof(p));
  for (int i = 0; i < terms; ++i) {
    if (!make_map(&p.amap[i], base + a_off[i], M, K, kBM, bf16)) return cudaErrorInvalidValue;
    if (!make_map(&p.bmap[i], base + b_off[i], N, K, static_cast<uint32_t>(bn), bf16)) return cudaErrorInvalidValue;
  }
  p.C = C;
  p.ws = ws;
  p.status = d_status;
  p.M = M;
  p.N = N;
  p.terms = terms;
  p.wait_ns = wait_ns;
  p.stall_loads = stall_loads;
  const int64_t row_elems = kRowBytes / (bf16 ? 2 : 4);
  p.kblocks = static_cast<int32_t>((K + row_elems - 1) / row_elems);
  p.kb_split = (p.kblocks + ksplit - 1) / ksplit;
  p.ksplit = (p.kblocks + p.kb_split - 1) / p.kb_split;
  if (p.ksplit != ksplit) return cudaErrorInvalidValue;  // the workspace was sized for `ksplit` splits
  cudaError_t e;
  if (bf16) {
    if (bn == 128) e = prepare_tile<128, true>(p, t, M, N);
    else if (bn == 64) e = prepare_tile<64, true>(p, t, M, N);
    else e = prepare_tile<32, true>(p, t, M, N);
  } else {
    if (bn == 128) e = prepare_tile<128, false>(p, t, M, N);
    else if (bn == 64) e = prepare_tile<64, false>(p, t, M, N);
    else e = prepare_tile<32, false>(p, t, M, N);
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
  k_split_sum<<<static_cast<unsigned>(blocks), 256, 0, s>>>(t.ws, t.ksplit, t.n, t.C);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(char* base, const int64_t* a_off, const int64_t* b_off, int terms, double* C, int64_t M,
                           int64_t N, int64_t K, int kind, double* ws, int ksplit, int* d_status, cudaStream_t s) {
  return launch_gemm_tc_ex(base, a_off, b_off, terms, C, M, N, K, kind, ws, ksplit, d_status, s, kWaitNs, 0);
}

cudaError_t launch_gemm_tc_ex(char* base, const int64_t* a_off, const int64_t* b_off, int terms, double* C, int64_t M,
                              int64_t N, int64_t K, int kind, double* ws, int ksplit, int* d_status, cudaStream_t s,
                              unsigned long long wait_ns, int stall_loads) {
  TcPrepared t;
  cudaError_t e = tc_gemm_prepare(&t, base, a_off, b_off, terms, C, M, N, K, kind, ws, ksplit, d_status, wait_ns,
                                  stall_loads);
  if (e != cudaSuccess) return e;
  return tc_gemm_run(t, s);
}

}  // namespace ajf
