// Device side of the tensor-core GEMM (sm_103a): kernel parameters, PTX wrappers (mbarrier, TMA,
// tcgen05), and the three roles of a 320-thread block over a range of work items. Included by
// tc_gemm.cu (the standalone persistent GEMM kernel) and by queue.cu (the persistent step
// interpreter, whose blocks run GEMM work items as tasks between other steps). The kernel's
// design and its accuracy argument are described at the top of tc_gemm.cu.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace ajf {
namespace tc {

constexpr int kBM = 128;             // rows per tile (UMMA M)
constexpr int kRowBytes = 128;       // bytes of K per tile row (one 128-byte swizzle span)
constexpr int kMaxSlots = 8;
constexpr int kMaxBufs = 4;
constexpr int kThreads = 320;        // producer warp, MMA warp, eight epilogue warps
constexpr int kEpiWarps = 8;
constexpr int kEpiWarp0 = 2;       // epilogue warps 2..9: warp w reads TMEM lanes 32 * (w % 4) .. + 31
// The FP32 register accumulation of promoted partials spans at most this many K blocks: longer
// contractions are split over K (FP32 partial tiles summed afterwards), so the small late
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
  float* C;                          // the product (FP32: each value is one promoted register sum)
  const float* sa;                   // scaled fp16 operands: A's scales [K block][M], B's [K block][N]
  const float* sb;
  int* status;
  int64_t M, N;
  int32_t terms, kblocks, ntn, slots, bufs;
  int32_t mtn;                       // tiles along M
  int32_t group;                     // M tiles per raster group (L2 reuse of B tiles)
  int32_t ksplit, kb_split;          // K splits and K blocks per split
  int64_t tiles;
  int32_t tmem_stride;               // TMEM columns per partial buffer (two partials of BN columns each)
  int32_t pad0;
  float* ws;                         // split partials [ksplit][M][N] (ksplit > 1)
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

// 1-D bulk copy global -> shared (16-byte aligned addresses, a multiple of 16 bytes).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
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

// Operand kinds: 0 TF32 (kind::tf32), 1 bf16, 2 fp16 scaled per row and K block (kind::f16; the
// instruction descriptor names the type).
template <int kKind>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (kKind != 0) {
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

// Shared-memory addresses of the GEMM's pipeline (slots and barriers) and its TMEM base.
struct TcShared {
  uint8_t* slots;                    // S slots of p.slot_bytes, 1024-byte aligned
  uint32_t full0, empty0, accf0, acce0, drain0;  // barrier arrays (8 bytes per barrier)
  uint32_t sfull0;                   // scaled fp16: the scales of TMEM buffer b have arrived
  float* scales;                     // scaled fp16: per TMEM buffer, 128 row scales then 128 column scales
  volatile int* abort_flag;
  float* stage;                      // epilogue store staging (see kStageCols)
  uint32_t tmem;
};
constexpr int kScaleFloats = 256;    // floats of scales per TMEM buffer
// The epilogue writes its FP32 tile through shared memory, kStageCols(kind) columns at a time: a
// thread owns one row, so storing straight from registers would touch 32 rows (32 cache lines) per
// warp store. Staged, each warp store covers whole row segments: 4 rows x 128 bytes (32 columns)
// for the TF32 and bf16 kinds, 8 rows x 64 bytes (16 columns) for the scaled fp16 kind, whose
// scale buffers take part of the space. (On GB300 a tile pattern written in 64-byte row pieces
// reached 3.4 TB/s, in 128-byte pieces 5.4 TB/s.) The 16-byte chunks of a staged row are
// XOR-swizzled so that the row-wise writes (8 rows per phase) and the read-back (one or two rows
// per 8 lanes) are both free of bank conflicts. The staging area starts at the scale buffers
// (unused by the TF32 and bf16 kinds) and holds kEpiWarps x 32 rows x 32 floats; the scaled fp16
// kind stages after its scale buffers, 16 columns wide (as does every kind when a thread holds
// only 16 columns, BN = 32).
__host__ __device__ constexpr int stage_cols(int kind) { return kind == 2 ? 16 : 32; }
constexpr uint32_t kTcStageBytes = kEpiWarps * 32 * 32 * 4;
static_assert(kMaxBufs * kScaleFloats * 4 + kEpiWarps * 32 * 16 * 4 <= kTcStageBytes, "staging layout");

// Ring positions of the three roles; they continue from one call of tc_gemm_items to the next
// (the barrier phases must), so a caller keeps one TcRing per thread for the block's lifetime.
struct TcRing {
  int slot = 0;                      // producer: next slot
  uint32_t phase = 0;
  uint32_t issued = 0;               // producer: slots loaded so far
  int mslot = 0;                     // MMA issuer: next slot and TMEM buffer
  uint32_t mphase = 0;
  int mbuf = 0;
  uint32_t mbphase = 0;
  bool any = false;                  // MMA issuer: MMAs issued so far
  uint32_t scopies = 0;              // MMA issuer: scale copies issued so far (scaled fp16)
  int ebuf = 0;                      // epilogue: next TMEM buffer
  uint32_t ebphase = 0;
};

// Layout of the pipeline's control region (kTcControlBytes from `bars`, 16-byte aligned): the
// barrier arrays, the TMEM address slot and the abort flag in the first 256 bytes, then
// kTcStageBytes shared by the scale buffers of the scaled fp16 kind (kMaxBufs x kScaleFloats
// floats) and the epilogue's staging buffers.
constexpr uint32_t kTcControlBytes = 256 + kTcStageBytes;
__device__ __forceinline__ uint32_t* tc_layout(uint8_t* slots, uint8_t* bars, TcShared& sh) {
  sh.slots = slots;
  sh.full0 = smem_u32(bars);
  sh.empty0 = sh.full0 + 8 * kMaxSlots;
  sh.accf0 = sh.empty0 + 8 * kMaxSlots;   // partial buffer b ready (MMA -> epilogue)
  sh.acce0 = sh.accf0 + 8 * kMaxBufs;     // partial buffer b drained (epilogue -> MMA)
  sh.drain0 = sh.acce0 + 8 * kMaxBufs;    // MMAs issued before an abort have completed
  sh.sfull0 = sh.drain0 + 8;              // scales of buffer b arrived
  sh.abort_flag = reinterpret_cast<volatile int*>(bars + 16 * kMaxSlots + 24 * kMaxBufs + 12);
  sh.scales = reinterpret_cast<float*>(bars + 256);
  sh.stage = reinterpret_cast<float*>(bars + 256);
  return reinterpret_cast<uint32_t*>(bars + 16 * kMaxSlots + 24 * kMaxBufs + 8);  // TMEM address slot
}

// Initialise the pipeline barriers (thread 0; the block synchronises afterwards).
__device__ __forceinline__ void tc_init_barriers(const TcShared& sh, int S, int NB) {
  for (int s = 0; s < S; ++s) {
    mbar_init(sh.full0 + 8 * s, 1);
    mbar_init(sh.empty0 + 8 * s, 1);
  }
  for (int b = 0; b < NB; ++b) {
    mbar_init(sh.accf0 + 8 * b, 1);
    mbar_init(sh.acce0 + 8 * b, kEpiWarps);
  }
  mbar_init(sh.drain0, 1);
  for (int b = 0; b < NB; ++b) mbar_init(sh.sfull0 + 8 * b, 1);
  *sh.abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Work items wi0, wi0 + step, ... (< wi1) of one GEMM, run by the block's three roles: warp 0
// lane 0 the TMA producer, warp 1 lane 0 the MMA issuer, warps 2..9 the epilogue; the other
// lanes of warps 0 and 1 pass straight through. Returns false in a role that gave up (a bounded
// wait expired, or another role set the abort flag); the roles' ring positions advance in `r`.
template <int BN, int kKind>
__device__ __forceinline__ bool tc_gemm_items(const TcParams& p, uint32_t wi0, uint32_t wi1, uint32_t step,
                                              const TcShared& sh, TcRing& r) {
  static_assert(BN == 32 || BN == 64 || BN == 128, "tile width");
  constexpr int COLS = BN / 2;                       // columns per epilogue thread (one TMEM lane = one row)
  constexpr int CH = COLS < 16 ? COLS : 16;          // columns per drain chunk
  constexpr uint32_t a_bytes = kBM * kRowBytes, b_bytes = BN * kRowBytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = p.slots, T = p.terms, NB = p.bufs;
  const uint32_t tmem = sh.tmem;
  // persistent tile loop: every role walks the same work items, and its ring positions (slots,
  // TMEM buffers) continue across items. Grouped raster: `group` M tiles sweep the N tiles
  // together, so concurrently running CTAs share each B tile through L2 instead of streaming all
  // of B once per M tile. Work item wi is tile wi % tiles of K split wi / tiles.
  const uint32_t tiles = static_cast<uint32_t>(p.tiles);
  auto work_item = [&](uint32_t wi, int32_t& m0, int32_t& n0, int& kb0, int& kb1) {
    const uint32_t tile = wi % tiles, ks = wi / tiles;
    const uint32_t per_group = static_cast<uint32_t>(p.group) * static_cast<uint32_t>(p.ntn);
    const uint32_t g = tile / per_group, rr = tile % per_group;
    const uint32_t first_m = g * static_cast<uint32_t>(p.group);
    const uint32_t left = static_cast<uint32_t>(p.mtn) - first_m;
    const uint32_t gm = left < static_cast<uint32_t>(p.group) ? left : static_cast<uint32_t>(p.group);
    m0 = static_cast<int32_t>((first_m + rr % gm) * kBM);
    n0 = static_cast<int32_t>((rr / gm) * BN);
    kb0 = static_cast<int>(ks) * p.kb_split;
    kb1 = kb0 + p.kb_split < p.kblocks ? kb0 + p.kb_split : p.kblocks;
  };
  bool ok = true;
  if (warp == 0 && lane == 0) {
    // ---- TMA producer: one slot per (K block, term) holds that term's A and B tiles. A block's
    // terms are loaded highest first, the order in which the MMA issuer frees their slots.
    int slot = r.slot;
    uint32_t phase = r.phase, issued = r.issued;
    ok = !p.stall_loads;
    for (uint32_t wi = wi0; wi < wi1 && ok; wi += step) {
      int32_t m0, n0;
      int kb0, kb1;
      work_item(wi, m0, n0, kb0, kb1);
      for (int kb = kb0; kb < kb1 && ok; ++kb) {
        for (int j = 0; j < T; ++j) {
          const int t = T - 1 - j;
          if (*sh.abort_flag || !mbar_wait(sh.empty0 + 8 * slot, phase ^ 1u, p.wait_ns, p.status, 11)) {
            *sh.abort_flag = 1;
            ok = false;
            break;
          }
          const uint32_t sa = smem_u32(sh.slots + slot * p.slot_bytes);
          const int32_t kx = kb * (kRowBytes / (kKind != 0 ? 2 : 4));
          mbar_expect_tx(sh.full0 + 8 * slot, a_bytes + b_bytes);
          tma_load_2d(sa, &p.amap[t], kx, m0, sh.full0 + 8 * slot);
          tma_load_2d(sa + a_bytes, &p.bmap[t], kx, n0, sh.full0 + 8 * slot);
          ++issued;
          if (++slot == S) {
            slot = 0;
            phase ^= 1u;
          }
        }
      }
    }
    r.slot = slot;
    r.phase = phase;
    r.issued = issued;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    int buf = r.mbuf, slot = r.mslot;
    uint32_t bphase = r.mbphase, phase = r.mphase;
    for (uint32_t wi = wi0; wi < wi1 && ok; wi += step) {
      int32_t m0, n0;
      int kb0, kb1;
      work_item(wi, m0, n0, kb0, kb1);
      for (int kb = kb0; kb < kb1; ++kb) {
        const int b = buf;
        if (*sh.abort_flag || !mbar_wait(sh.acce0 + 8 * b, bphase ^ 1u, p.wait_ns, p.status, 14)) {
          ok = false;
          break;
        }
        if (kKind == 2) {
          // the K block's row and column scales into buffer b's scale area (the epilogue has
          // released the buffer, so also its scales)
          const uint32_t rows = static_cast<uint32_t>(p.M - m0 < kBM ? p.M - m0 : kBM);
          const uint32_t cols = static_cast<uint32_t>(p.N - n0 < BN ? p.N - n0 : BN);
          const uint32_t sdst = smem_u32(sh.scales + b * kScaleFloats);
          mbar_expect_tx(sh.sfull0 + 8 * b, 4 * (rows + cols));
          bulk_load(sdst, p.sa + static_cast<int64_t>(kb) * p.M + m0, 4 * rows, sh.sfull0 + 8 * b);
          bulk_load(sdst + 4 * 128, p.sb + static_cast<int64_t>(kb) * p.N + n0, 4 * cols, sh.sfull0 + 8 * b);
          ++r.scopies;
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
        const uint32_t base = smem_u32(sh.slots);
        const uint64_t ad0 = smem_desc(base + st0 * p.slot_bytes), bd0 = smem_desc(base + st0 * p.slot_bytes + a_bytes);
        const uint64_t ad1 = smem_desc(base + st1 * p.slot_bytes), bd1 = smem_desc(base + st1 * p.slot_bytes + a_bytes);
        const uint64_t ad2 = smem_desc(base + st2 * p.slot_bytes), bd2 = smem_desc(base + st2 * p.slot_bytes + a_bytes);
        const uint32_t dst0 = tmem + static_cast<uint32_t>(b * p.tmem_stride);  // P0: the leading product alone
        const uint32_t dst1 = dst0 + static_cast<uint32_t>(BN);                 // P1: the correction products
        uint32_t acc = 0;
        // one product A_i . B_j over the block: 4 instructions, 32 bytes of K each (+2 in the
        // descriptor's 16-byte address field)
        auto product = [&](uint32_t dst, uint64_t ad, uint64_t bd) {
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            mma<kKind>(dst, ad + 2 * kk, bd + 2 * kk, p.idesc, acc);
            acc = 1;
          }
        };
        auto arrived = [&](int sl, uint32_t ph) {
          const bool w = mbar_wait(sh.full0 + 8 * sl, ph, p.wait_ns, p.status, 12);
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
        r.any = true;
        if (T == 3) {
          product(dst1, ad0, bd2);
          product(dst1, ad1, bd1);
          product(dst1, ad2, bd0);
          mma_commit(sh.empty0 + 8 * st2);
        }
        if (T >= 2) {
          product(dst1, ad0, bd1);
          product(dst1, ad1, bd0);
          mma_commit(sh.empty0 + 8 * st1);
        }
        acc = 0;
        product(dst0, ad0, bd0);
        mma_commit(sh.empty0 + 8 * st0);
        mma_commit(sh.accf0 + 8 * b);
      }
    }
    if (!ok) *sh.abort_flag = 1;
    r.mbuf = buf;
    r.mslot = slot;
    r.mbphase = bphase;
    r.mphase = phase;
  } else if (warp >= kEpiWarp0) {
    // ---- epilogue: promote partials into round-to-nearest FP32 registers, store FP32 per tile
    const int q = warp & 3, h = (warp - kEpiWarp0) >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(32 * q) << 16;
    float acc[COLS];
    int buf = r.ebuf;
    uint32_t bphase = r.ebphase;
    for (uint32_t wi = wi0; wi < wi1 && ok; wi += step) {
      int32_t m0, n0;
      int kb0, kb1;
      work_item(wi, m0, n0, kb0, kb1);
      const int64_t row = static_cast<int64_t>(m0) + 32 * q + lane;
      const int64_t col0 = static_cast<int64_t>(n0) + h * COLS;
      // rows/columns beyond M, N were zero-filled by TMA and are not stored; M and N are powers of
      // two >= 32 and >= 16, so a warp's 32 rows and COLS columns are all inside or all outside
      const bool mine = row < p.M && col0 < p.N;
      float* dbase = p.ksplit > 1 ? p.ws + static_cast<int64_t>(wi / tiles) * p.M * p.N : p.C;
#pragma unroll
      for (int j = 0; j < COLS; ++j) acc[j] = 0.0f;
      for (int kb = kb0; kb < kb1; ++kb) {
        const int b = buf;
        int w = 1;
        if (lane == 0) w = mbar_wait(sh.accf0 + 8 * b, bphase, p.wait_ns, p.status, 13) ? 1 : 0;
        if (++buf == NB) {
          buf = 0;
          bphase ^= 1u;
        }
        ok = __shfl_sync(0xffffffffu, w, 0) != 0;
        if (!ok || *sh.abort_flag) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t col = static_cast<uint32_t>(b * p.tmem_stride + h * COLS);
        float sa = 1.0f;
        const float* sbv = nullptr;
        if (kKind == 2) {
          // this K block's scales: the row's (per lane) and the columns' (the same for every lane)
          int ws = 1;
          if (lane == 0) ws = mbar_wait(sh.sfull0 + 8 * b, (bphase ^ (buf == 0 ? 1u : 0u)) & 1u, p.wait_ns, p.status,
                                        17) ? 1 : 0;
          if (!__shfl_sync(0xffffffffu, ws, 0)) {
            ok = false;
            break;
          }
          const float* sbuf = sh.scales + b * kScaleFloats;
          sa = sbuf[32 * q + lane];
          sbv = sbuf + 128 + h * COLS;
        }
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
          if (kKind == 2) {
            // the block's partial in units of q_row q_col: scale it back (powers of two, exact
            // while in the normal range) and accumulate with round-to-nearest
#pragma unroll
            for (int j = 0; j < CH; j += 4) {
              const float4 e = *reinterpret_cast<const float4*>(sbv + c0 + j);
              acc[c0 + j] += ((__uint_as_float(r0[j]) + __uint_as_float(r1[j])) * sa) * e.x;
              acc[c0 + j + 1] += ((__uint_as_float(r0[j + 1]) + __uint_as_float(r1[j + 1])) * sa) * e.y;
              acc[c0 + j + 2] += ((__uint_as_float(r0[j + 2]) + __uint_as_float(r1[j + 2])) * sa) * e.z;
              acc[c0 + j + 3] += ((__uint_as_float(r0[j + 3]) + __uint_as_float(r1[j + 3])) * sa) * e.w;
            }
          } else if (T > 1) {
#pragma unroll
            for (int j = 0; j < CH; ++j) acc[c0 + j] += __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
          } else {
#pragma unroll
            for (int j = 0; j < CH; ++j) acc[c0 + j] += __uint_as_float(r0[j]);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(sh.acce0 + 8 * b);
      }
      if (!ok) break;
      // the MMA warp is already filling the next buffers while this tile is written. `mine` is the
      // same for the whole warp.
      if (mine) {
        constexpr int SC = stage_cols(kKind) < COLS ? stage_cols(kKind) : COLS;  // staged columns: 32 or 16
        constexpr int CH16 = SC / 4;                      // 16-byte chunks per staged row: 8 or 4
        constexpr int RPI = 32 / CH16;                    // rows per warp store: 4 or 8
        float* st = sh.stage + (kKind == 2 ? kMaxBufs * kScaleFloats : 0) + (warp - kEpiWarp0) * 32 * SC;
        float4* srow = reinterpret_cast<float4*>(st + lane * SC);
        // chunk j of row r sits at position j ^ sw(r): sw = r % 8 for 8 chunks per row (128-byte
        // rows all start on bank 0), (r / 2) % 4 for 4 chunks (64-byte rows: even and odd rows
        // start on banks 0 and 16)
        const int wsw = CH16 == 8 ? (lane & 7) : ((lane >> 1) & 3);
        // read-back: warp store i covers rows RPI i .. RPI i + RPI - 1; lane l carries chunk
        // l % CH16 of row RPI i + l / CH16
        const int rr = lane / CH16, pc = lane % CH16;
        float* drow = dbase + (row - lane + rr) * p.N + col0 + 4 * pc;
#pragma unroll
        for (int c = 0; c < COLS; c += SC) {
#pragma unroll
          for (int j = 0; j < CH16; ++j)
            srow[j ^ wsw] = make_float4(acc[c + 4 * j], acc[c + 4 * j + 1], acc[c + 4 * j + 2], acc[c + 4 * j + 3]);
          __syncwarp();
#pragma unroll
          for (int i = 0; i < 32 / RPI; ++i) {
            const int rs = RPI * i + rr;
            const int rsw = CH16 == 8 ? (rs & 7) : ((rs >> 1) & 3);
            *reinterpret_cast<float4*>(drow + RPI * i * p.N + c) =
                reinterpret_cast<const float4*>(st + rs * SC)[pc ^ rsw];
          }
          __syncwarp();
        }
      }
    }
    if (!ok) *sh.abort_flag = 1;
    r.ebuf = buf;
    r.ebphase = bphase;
  }
  return ok;
}

// After an abort (the abort flag set), before the block releases its shared memory and TMEM: the
// producer waits (bounded) until the loads it issued have landed -- the last min(issued, S) slots;
// earlier ones were consumed -- and the MMA issuer until every MMA it issued has completed.
__device__ __forceinline__ void tc_drain_after_abort(int slots, int nbufs, unsigned long long wait_ns, int* status,
                                                     const TcShared& sh, const TcRing& r) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t S = static_cast<uint32_t>(slots);
  if (warp == 0 && lane == 0 && r.issued > 0) {
    const uint32_t first = r.issued > S ? r.issued - S : 0u;
    for (uint32_t i = first; i < r.issued; ++i) mbar_wait(sh.full0 + 8 * (i % S), (i / S) & 1u, wait_ns, status, 15);
  } else if (warp == 1 && lane == 0) {
    if (r.any) {
      mma_commit(sh.drain0);
      mbar_wait(sh.drain0, 0u, wait_ns, status, 16);
    }
    // scale copies issued: the last min(issued, NB) may still be landing
    const uint32_t NB = static_cast<uint32_t>(nbufs);
    const uint32_t first = r.scopies > NB ? r.scopies - NB : 0u;
    for (uint32_t i = first; i < r.scopies; ++i) mbar_wait(sh.sfull0 + 8 * (i % NB), (i / NB) & 1u, wait_ns, status, 18);
  }
}

}  // namespace tc
}  // namespace ajf
