// Device bodies of the contraction program's CUDA-core kernels (sm_103a), shared by the
// standalone kernels (kernels.cu: one launch per program step, block index = blockIdx.x) and the
// persistent step interpreter (queue.cu: one launch for many programs, whose thread blocks run
// these bodies as tasks with virtual block indices).
//
// Every body runs on kBodyThreads = 256 threads (threads 0..255 of the block) and synchronises
// them through the Sync policy: __syncthreads() in a standalone kernel, a named barrier of those
// 256 threads in the interpreter, whose blocks carry more warps. Shared-memory scratch comes in
// through pointers, so that the interpreter can place it in its own dynamic shared memory.
//
//  leaf_body        builds a leaf tensor of the miter network from the uploaded complex128
//                   gate/Kraus matrices (gate, conjugate, adjoint, transpose, Kraus stack with an
//                   open index, superoperator M_N = sum_k N_k (x) N_k^*; Sec. IV-A/IV-B).
//  small_body       small pairwise contractions, one gather per operand element through 8-bit
//                   offset tables (bits of any binary-index layout).
//  splitk_body      contractions with few outputs and a long contracted index: FP64 partial sums
//                   per block; splitk_done_body sums them in a fixed order (deterministic).
//  dot_body         tiled full contraction to a scalar (the trace of a closed network).
//  perm_body        gathers a complex tensor into a real, K-contiguous GEMM operand (the complex
//                   product C = A B becomes the real product [[Ar,-Ai],[Ai,Ar]] [Br;Bi] = [Cr;Ci]),
//                   in the operand format of the precision mode.
//  split_sum_body   sums the FP64 K-split partial tiles of a tensor-core GEMM in a fixed order.
//  open_body/final_body  the FP64 end of the path: t_i for Alg. I, sum |t_i|^2, F_J and 1 - F_J.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "device.h"

namespace ajf {

constexpr int kBodyThreads = 256;

// Barrier policies of the bodies.
struct SyncBlock {  // a standalone kernel of kBodyThreads threads
  __device__ __forceinline__ static void sync() { __syncthreads(); }
};
struct SyncBody {  // threads 0..kBodyThreads-1 of a larger block: named barrier 1
  __device__ __forceinline__ static void sync() { asm volatile("bar.sync 1, %0;" ::"n"(kBodyThreads) : "memory"); }
};

// ------------------------------------------------------------------ offset tables

__device__ __forceinline__ int nchunks(int nbits) { return (nbits + 7) >> 3; }

// Fill `tab` (nchunks * 256 entries) for map `m`; all threads of the block participate.
__device__ __forceinline__ void build_table(const BitMap& m, int64_t* tab) {
  const int nc = nchunks(m.nbits);
  for (int e = threadIdx.x; e < nc * 256; e += kBodyThreads) {
    const int c = e >> 8, v = e & 255;
    int64_t off = 0;
    for (int i = 0; i < 8; ++i) {
      const int bit = c * 8 + i;
      if (bit < m.nbits && ((v >> i) & 1) && m.pos[bit] >= 0) off += int64_t(1) << m.pos[bit];
    }
    tab[e] = off;
  }
}

__device__ __forceinline__ int64_t lookup(const int64_t* tab, int nc, int64_t idx) {
  int64_t off = 0;
  for (int c = 0; c < nc; ++c) off += tab[(c << 8) | ((idx >> (8 * c)) & 255)];
  return off;
}

// Operand `off` (element offset in its own type's units) of a step whose tensor is complex64 (f32:
// FP32 planes, the product of a reduced-precision GEMM) or complex128 (FP64 planes, every other
// tensor), and `arena` the arena as FP64 elements: calls fn with the typed pointer, so that each
// combination of operand types gets its own loop.
template <typename Fn>
__device__ __forceinline__ void with_operands(const double* arena, int64_t a, bool fa, int64_t b, bool fb, Fn&& fn) {
  const float* af = reinterpret_cast<const float*>(arena) + a;
  const float* bf = reinterpret_cast<const float*>(arena) + b;
  if (fa) {
    if (fb) fn(af, bf);
    else fn(af, arena + b);
  } else {
    if (fb) fn(arena + a, bf);
    else fn(arena + a, arena + b);
  }
}

// ------------------------------------------------------------------ leaves

// Element e of leaf L (complex, FP64) from the uploaded complex128 matrices.
__device__ __forceinline__ void leaf_value(const LeafDev& L, const double* __restrict__ in, int64_t e, double& re,
                                           double& im) {
  re = 0;
  im = 0;
  const int a = L.a;
  const int64_t dim = int64_t(1) << a;
  switch (L.kind) {
    case 0: case 1: case 2: case 3: {  // gate, conj, adjoint, transpose
      const int64_t r = e >> a, c = e & (dim - 1);
      const bool swap = (L.kind == 2 || L.kind == 3);
      const int64_t idx = swap ? (c * dim + r) : (r * dim + c);
      re = in[2 * (L.src + idx)];
      im = in[2 * (L.src + idx) + 1];
      if (L.kind == 1 || L.kind == 2) im = -im;
      break;
    }
    case 4: {  // Kraus stack with open index kappa above the 2a operator bits
      const int64_t kappa = e >> (2 * a);
      const int64_t rc = e & (dim * dim - 1);
      if (kappa < L.nk) {
        re = in[2 * (L.src + kappa * dim * dim + rc)];
        im = in[2 * (L.src + kappa * dim * dim + rc) + 1];
      }
      break;
    }
    case 5: {  // M_N over wires (q..., q'...): a = 2 * noise arity
      const int an = a / 2;
      const int64_t nd = int64_t(1) << an;
      const int64_t R = e >> a, C = e & (dim - 1);
      const int64_t o = R >> an, op = R & (nd - 1), i = C >> an, ip = C & (nd - 1);
      for (int k = 0; k < L.nk; ++k) {
        const int64_t base = L.src + int64_t(k) * nd * nd;
        const double xr = in[2 * (base + o * nd + i)], xi = in[2 * (base + o * nd + i) + 1];
        const double yr = in[2 * (base + op * nd + ip)], yi = -in[2 * (base + op * nd + ip) + 1];
        re += xr * yr - xi * yi;
        im += xr * yi + xi * yr;
      }
      break;
    }
    default:  // identity delta[out][in]
      re = (e == 0 || e == 3) ? 1.0 : 0.0;
      break;
  }
}

// Index into the full (unsliced) leaf of element e of a leaf whose sliced labels are fixed:
// e's bits fill the free positions from the lowest up, the sliced positions take fix_val.
__device__ __forceinline__ int64_t leaf_full_index(const LeafDev& L, int64_t e) {
  if (L.fix_mask == 0) return e;
  int64_t full = L.fix_val;
  int src = 0;
  for (int p = 0; p < 16 && src < L.bits; ++p) {
    if ((L.fix_mask >> p) & 1) continue;
    full |= ((e >> src) & 1) << p;
    ++src;
  }
  return full;
}

// One leaf per (virtual) block.
template <typename T>
__device__ __forceinline__ void leaf_body(const LeafDev* leaves, const double* __restrict__ in, T* __restrict__ arena,
                                          int vb) {
  const LeafDev L = leaves[vb];
  const int64_t n = int64_t(1) << L.bits;
  for (int64_t e = threadIdx.x; e < n; e += kBodyThreads) {
    double re, im;
    leaf_value(L, in, leaf_full_index(L, e), re, im);
    arena[L.off + e] = static_cast<T>(re);
    arena[L.off + L.plane + e] = static_cast<T>(im);
  }
}

// ------------------------------------------------------------------ small contractions

__device__ __forceinline__ int find_step(const StepDev* steps, int nsteps, int block) {
  int lo = 0, hi = nsteps - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (steps[mid].block0 <= block) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename T, typename Acc, typename Sync>
__device__ __forceinline__ void small_body(const StepDev* __restrict__ steps, int nsteps, int total_blocks,
                                           T* __restrict__ arena, int vb, int64_t* tab) {
  const int s = find_step(steps, nsteps, vb);
  const StepDev& st = steps[s];
  const int end = (s + 1 < nsteps) ? steps[s + 1].block0 : total_blocks;
  const int nb = end - st.block0;
  const int c_oa = nchunks(st.oa.nbits), c_ob = nchunks(st.ob.nbits);
  const int c_ka = nchunks(st.ka.nbits), c_kb = nchunks(st.kb.nbits);
  int64_t* t_oa = tab;
  int64_t* t_ob = t_oa + c_oa * 256;
  int64_t* t_ka = t_ob + c_ob * 256;
  int64_t* t_kb = t_ka + c_ka * 256;
  build_table(st.oa, t_oa);
  build_table(st.ob, t_ob);
  build_table(st.ka, t_ka);
  build_table(st.kb, t_kb);
  Sync::sync();
  const int64_t nout = int64_t(1) << st.rc, nk = int64_t(1) << st.rk;
  T* C = arena + st.c;
  with_operands(arena, st.a, st.fa, st.b, st.fb, [&](const auto* A, const auto* B) {
    for (int64_t o = int64_t(vb - st.block0) * kBodyThreads + threadIdx.x; o < nout;
         o += int64_t(nb) * kBodyThreads) {
      const int64_t oa = lookup(t_oa, c_oa, o), ob = lookup(t_ob, c_ob, o);
      Acc re = 0, im = 0;
      for (int64_t kk = 0; kk < nk; ++kk) {
        const int64_t ia = oa + lookup(t_ka, c_ka, kk), ib = ob + lookup(t_kb, c_kb, kk);
        const Acc ar = A[ia], ai = A[st.pa + ia], br = B[ib], bi = B[st.pb + ib];
        re += ar * br - ai * bi;
        im += ar * bi + ai * br;
      }
      C[o] = static_cast<T>(re);
      C[st.pc + o] = static_cast<T>(im);
    }
  });
}


template <typename T, typename Sync>
__device__ __forceinline__ void splitk_body(const StepDev* __restrict__ steps, int nsteps, const T* __restrict__ arena,
                                            double2* __restrict__ partial, int vb, int64_t* tab, double* red_re,
                                            double* red_im) {
  const int s = find_step(steps, nsteps, vb);
  const StepDev& st = steps[s];
  const int local = vb - st.block0;
  const int64_t o = local / st.nsplit;
  const int split = local % st.nsplit;
  const int c_oa = nchunks(st.oa.nbits), c_ob = nchunks(st.ob.nbits);
  const int c_ka = nchunks(st.ka.nbits), c_kb = nchunks(st.kb.nbits);
  int64_t* t_oa = tab;
  int64_t* t_ob = t_oa + c_oa * 256;
  int64_t* t_ka = t_ob + c_ob * 256;
  int64_t* t_kb = t_ka + c_ka * 256;
  build_table(st.oa, t_oa);
  build_table(st.ob, t_ob);
  build_table(st.ka, t_ka);
  build_table(st.kb, t_kb);
  Sync::sync();
  const int64_t nk = int64_t(1) << st.rk;
  const int64_t chunk = (nk + st.nsplit - 1) / st.nsplit;
  const int64_t k0 = int64_t(split) * chunk;
  const int64_t k1 = min(nk, k0 + chunk);
  const int64_t oa = lookup(t_oa, c_oa, o), ob = lookup(t_ob, c_ob, o);
  double re = 0, im = 0;
  with_operands(arena, st.a, st.fa, st.b, st.fb, [&](const auto* A, const auto* B) {
    for (int64_t kk = k0 + threadIdx.x; kk < k1; kk += kBodyThreads) {
      const int64_t ia = oa + lookup(t_ka, c_ka, kk), ib = ob + lookup(t_kb, c_kb, kk);
      const double ar = A[ia], ai = A[st.pa + ia], br = B[ib], bi = B[st.pb + ib];
      re += ar * br - ai * bi;
      im += ar * bi + ai * br;
    }
  });
  red_re[threadIdx.x] = re;
  red_im[threadIdx.x] = im;
  Sync::sync();
  for (int w = kBodyThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red_re[threadIdx.x] += red_re[threadIdx.x + w];
      red_im[threadIdx.x] += red_im[threadIdx.x + w];
    }
    Sync::sync();
  }
  if (threadIdx.x == 0) partial[st.poff + o * st.nsplit + split] = make_double2(red_re[0], red_im[0]);
}


// Full contraction S = sum_kk A[a(kk)] B[b(kk)] of two tensors (the trace of a closed network),
// tiled so that both operands are read along their contiguous bits. A tile fixes all contracted
// bits but ntl of them: the ones on A's lowest positions and the ones on B's lowest positions.
// Phase 1 stages the tile of A in shared memory in A order (lanes along A's contiguous bits);
// phase 2 streams the tile of B in B order and multiplies with the staged A values. FP64 partial
// sums per block; k_splitk_done adds them in a fixed order. kF32 (reduced-precision modes): the
// products of each tile are formed and summed in FP32 per thread (FP32 operands: complex64
// tensors as they are, complex128 ones rounded; relative error ~1e-7 per term) and the tile sums
// are accumulated in FP64.
// Asynchronous global -> shared copies (4 bytes, or 16 bytes with both addresses 16-byte aligned),
// committed in groups; cp_async_wait<N> returns once at most N of this thread's groups are pending.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T, bool kF32, typename Sync, bool kStaged = false>
__device__ __forceinline__ void dot_body(const StepDev* __restrict__ steps, int nsteps, const T* __restrict__ arena,
                                         double2* __restrict__ partial, int vb, int64_t* tab, double* red_re,
                                         double* red_im) {
  const int s = find_step(steps, nsteps, vb);
  const StepDev& st = steps[s];
  const int split = vb - st.block0;
  const int c_ka = nchunks(st.ka.nbits), c_kb = nchunks(st.kb.nbits);
  const int ntl = st.ntl, nt = 1 << ntl;
  int64_t* t_ka = tab;
  int64_t* t_kb = t_ka + c_ka * 256;
  int64_t* locA = t_kb + c_kb * 256;         // [nt] offset in A of tile-local index (A order)
  int64_t* locB = locA + nt;                 // [nt] offset in B of tile-local index (B order)
  // staged and register values: FP32 for FP32 products, FP64 otherwise
  using V = typename std::conditional<kF32, float, double>::type;
  V* sre = reinterpret_cast<V*>(locB + nt);
  V* sim = sre + nt;
  uint16_t* a_of_b = reinterpret_cast<uint16_t*>(sim + nt);  // B-order local index -> A-order
  uint64_t tilemask = 0;
  for (int i = 0; i < ntl; ++i) tilemask |= uint64_t(1) << st.tl[i];
  // the tile number's bits are the contracted bits outside the tile, lowest first: tables over the
  // tile number give a tile's base offsets in A and B with a few shared-memory reads (they have
  // at most as many chunks as the tables over all contracted bits, whose space they take)
  BitMap ta, tb;
  ta.nbits = tb.nbits = st.rk - ntl;
  for (int i = 0, j = 0; i < st.rk; ++i) {
    if ((tilemask >> i) & 1) continue;
    ta.pos[j] = st.ka.pos[i];
    tb.pos[j] = st.kb.pos[i];
    ++j;
  }
  const int c_ta = nchunks(ta.nbits);
  build_table(ta, t_ka);
  build_table(tb, t_kb);
  for (int l = threadIdx.x; l < nt; l += kBodyThreads) {
    int64_t oa = 0, ob = 0;
    uint64_t kk = 0;
    for (int i = 0; i < ntl; ++i) {
      if ((l >> i) & 1) {
        oa += int64_t(1) << st.ka.pos[st.tl[i]];
        ob += int64_t(1) << st.kb.pos[st.tlb[i]];
        kk |= uint64_t(1) << st.tlb[i];
      }
    }
    locA[l] = oa;
    locB[l] = ob;
    int la = 0;  // A-order local index of the contracted-index value kk
    for (int i = 0; i < ntl; ++i)
      if ((kk >> st.tl[i]) & 1) la |= 1 << i;
    a_of_b[l] = static_cast<uint16_t>(la);
  }
  Sync::sync();
  const int64_t ntiles = int64_t(1) << (st.rk - ntl);
  // vector form: both operands FP32 with their two lowest positions the tile's two lowest bits in
  // both orders (always so for a full contraction, whose tile holds each operand's five lowest
  // positions) and 16-byte aligned planes: a thread's 4 consecutive tile-local indices are then 4
  // consecutive elements of A (A order) and of B (B order), one 16-byte load per plane
  const bool vec = kF32 && st.fa && st.fb && ntl == 10 && st.ka.pos[st.tl[0]] == 0 && st.ka.pos[st.tl[1]] == 1 &&
                   st.kb.pos[st.tlb[0]] == 0 && st.kb.pos[st.tlb[1]] == 1 &&
                   ((st.a | st.pa | st.b | st.pb) & 3) == 0;
  double re = 0, im = 0;
  with_operands(arena, st.a, st.fa, st.b, st.fb, [&](const auto* A, const auto* B) {
    // the tile's base offsets in A and B
    auto tile_base = [&](int64_t t, int64_t& ba, int64_t& bb) {
      ba = lookup(t_ka, c_ta, t);
      bb = lookup(t_kb, c_ta, t);
    };
    using TA = typename std::remove_cv<typename std::remove_pointer<decltype(A)>::type>::type;
    using TB = typename std::remove_cv<typename std::remove_pointer<decltype(B)>::type>::type;
    if constexpr (kF32 && std::is_same<TA, float>::value && std::is_same<TB, float>::value) {
      if (vec) {
        // thread t owns tile-local indices 4t .. 4t + 3 in both orders; the next tile's four
        // 16-byte loads are in flight while the current tile is multiplied. A is staged at
        // l ^ ((l >> 5) & 31) as below; each B element then reads its A partner there.
        const int l0 = 4 * threadIdx.x;
        const int64_t oA = locA[l0], oB = locB[l0];
        const int k5 = (l0 >> 5) & 31;
        int sa[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int la = a_of_b[l0 + j];
          sa[j] = la ^ ((la >> 5) & 31);
        }
        if constexpr (kStaged) {
          // Staged form: asynchronous copies into three shared-memory stages, two tiles ahead of
          // the one being multiplied, with no registers held for them. A stage is four arrays of
          // 1024 floats (A re, A im at the swizzled positions above, B re, B im in B order); 6 of
          // the 12 arrays overlay locA .. sim (24 KB, free once this thread's offsets and A
          // positions are in registers), the other 6 follow the layout (dot_smem_bytes).
          float* const R = reinterpret_cast<float*>(locA);
          float* const X = reinterpret_cast<float*>(reinterpret_cast<char*>(locA) + nt * 34);
          auto arr = [&](int k) -> float* { return k < 6 ? R + k * 1024 : X + (k - 6) * 1024; };
          Sync::sync();  // every thread has read locA, locB and a_of_b
          auto issue = [&](int sg, int64_t t) {
            int64_t ba, bb;
            tile_base(t, ba, bb);
            float* const dr = arr(4 * sg);
            float* const di = arr(4 * sg + 1);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              cp_async4(dr + ((l0 + j) ^ k5), A + ba + oA + j);
              cp_async4(di + ((l0 + j) ^ k5), A + st.pa + ba + oA + j);
            }
            cp_async16(arr(4 * sg + 2) + l0, B + bb + oB);
            cp_async16(arr(4 * sg + 3) + l0, B + st.pb + bb + oB);
          };
          const int64_t ns = st.nsplit;
          int64_t t = split;
          if (t < ntiles) issue(0, t);
          cp_async_commit();
          if (t + ns < ntiles) issue(1, t + ns);
          cp_async_commit();
          int sg = 0;
          while (t < ntiles) {
            cp_async_wait<1>();  // this thread's copies of tile t have landed
            Sync::sync();        // everyone's have, and stage (sg + 2) % 3 is no longer read
            if (t + 2 * ns < ntiles) issue(sg == 0 ? 2 : sg - 1, t + 2 * ns);
            cp_async_commit();
            const float* const xr = arr(4 * sg);
            const float* const xi = arr(4 * sg + 1);
            const float4 br = *reinterpret_cast<const float4*>(arr(4 * sg + 2) + l0);
            const float4 bi = *reinterpret_cast<const float4*>(arr(4 * sg + 3) + l0);
            const float cb[8] = {br.x, br.y, br.z, br.w, bi.x, bi.y, bi.z, bi.w};
            float fre = 0.0f, fim = 0.0f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float ar = xr[sa[j]], ai = xi[sa[j]];
              fre += ar * cb[j] - ai * cb[4 + j];
              fim += ar * cb[4 + j] + ai * cb[j];
            }
            re += fre;
            im += fim;
            t += ns;
            sg = sg == 2 ? 0 : sg + 1;
          }
          cp_async_wait<0>();
          return;
        }
        float4 ar, ai, br, bi;
        auto load4 = [&](int64_t t) {
          int64_t ba, bb;
          tile_base(t, ba, bb);
          ar = *reinterpret_cast<const float4*>(A + ba + oA);
          ai = *reinterpret_cast<const float4*>(A + st.pa + ba + oA);
          br = *reinterpret_cast<const float4*>(B + bb + oB);
          bi = *reinterpret_cast<const float4*>(B + st.pb + bb + oB);
        };
        int64_t t = split;
        if (t < ntiles) load4(t);
        while (t < ntiles) {
          sre[(l0 + 0) ^ k5] = ar.x;
          sre[(l0 + 1) ^ k5] = ar.y;
          sre[(l0 + 2) ^ k5] = ar.z;
          sre[(l0 + 3) ^ k5] = ar.w;
          sim[(l0 + 0) ^ k5] = ai.x;
          sim[(l0 + 1) ^ k5] = ai.y;
          sim[(l0 + 2) ^ k5] = ai.z;
          sim[(l0 + 3) ^ k5] = ai.w;
          const float cb[8] = {br.x, br.y, br.z, br.w, bi.x, bi.y, bi.z, bi.w};
          Sync::sync();
          const int64_t tn = t + st.nsplit;
          if (tn < ntiles) load4(tn);
          float fre = 0.0f, fim = 0.0f;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float xr = sre[sa[j]], xi = sim[sa[j]];
            fre += xr * cb[j] - xi * cb[4 + j];
            fim += xr * cb[4 + j] + xi * cb[j];
          }
          re += fre;
          im += fim;
          Sync::sync();
          t = tn;
        }
        return;
      }
    }
    // Software pipeline: the A and B values of the next tile (kPer per thread; tiles hold at most
    // 2^10 = 256 * kPer elements) are loaded into registers while the current tile is multiplied,
    // so the loads of two tiles are in flight. Staged A values sit at index l ^ ((l >> 5) & 31):
    // B-ordered reads that stride across A's index (B's low bits on A's high bits) then fall into
    // distinct shared-memory banks.
    constexpr int kPer = 4;
    V are[kPer], aim[kPer], bre[kPer], bim[kPer];
    auto load_tile = [&](int64_t t) {
      int64_t ba, bb;
      tile_base(t, ba, bb);
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int l = threadIdx.x + q * kBodyThreads;
        if (l < nt) {
          are[q] = static_cast<V>(A[ba + locA[l]]);
          aim[q] = static_cast<V>(A[st.pa + ba + locA[l]]);
          bre[q] = static_cast<V>(B[bb + locB[l]]);
          bim[q] = static_cast<V>(B[st.pb + bb + locB[l]]);
        }
      }
    };
    int64_t t = split;
    if (t < ntiles) load_tile(t);
    while (t < ntiles) {
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int l = threadIdx.x + q * kBodyThreads;
        if (l < nt) {
          const int sl = l ^ ((l >> 5) & 31);
          sre[sl] = are[q];
          sim[sl] = aim[q];
        }
      }
      V cbr[kPer], cbi[kPer];
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        cbr[q] = bre[q];
        cbi[q] = bim[q];
      }
      Sync::sync();
      const int64_t tn = t + st.nsplit;
      if (tn < ntiles) load_tile(tn);
      if (kF32) {
        float fre = 0.0f, fim = 0.0f;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
          const int l = threadIdx.x + q * kBodyThreads;
          if (l < nt) {
            const int la = a_of_b[l];
            const int sl = la ^ ((la >> 5) & 31);
            const float ar = static_cast<float>(sre[sl]), ai = static_cast<float>(sim[sl]);
            const float br = static_cast<float>(cbr[q]), bi = static_cast<float>(cbi[q]);
            fre += ar * br - ai * bi;
            fim += ar * bi + ai * br;
          }
        }
        re += fre;
        im += fim;
      } else {
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
          const int l = threadIdx.x + q * kBodyThreads;
          if (l < nt) {
            const int la = a_of_b[l];
            const int sl = la ^ ((la >> 5) & 31);
            const double ar = sre[sl], ai = sim[sl], br = cbr[q], bi = cbi[q];
            re += ar * br - ai * bi;
            im += ar * bi + ai * br;
          }
        }
      }
      Sync::sync();
      t = tn;
    }
  });
  red_re[threadIdx.x] = re;
  red_im[threadIdx.x] = im;
  Sync::sync();
  for (int w = kBodyThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red_re[threadIdx.x] += red_re[threadIdx.x + w];
      red_im[threadIdx.x] += red_im[threadIdx.x + w];
    }
    Sync::sync();
  }
  if (threadIdx.x == 0) partial[st.poff + split] = make_double2(red_re[0], red_im[0]);
}


// Sum the split-K partials of every output in a fixed order (deterministic): with many splits a
// whole block reduces each output (strided per-thread sums, then a tree), otherwise one thread
// sums one output's splits.
template <typename T, typename Sync>
__device__ __forceinline__ void splitk_done_body(const StepDev* __restrict__ steps, const double2* __restrict__ partial,
                                                 T* __restrict__ arena, double2* __restrict__ scalars, int vb,
                                                 double* red_re, double* red_im) {
  const StepDev& st = steps[vb];
  const int64_t nout = int64_t(1) << st.rc;
  auto emit = [&](int64_t o, double re, double im) {
    if (st.scalar_slot >= 0) {
      scalars[st.scalar_slot] = make_double2(re, im);
    } else {
      arena[st.c + o] = static_cast<T>(re);
      arena[st.c + st.pc + o] = static_cast<T>(im);
    }
  };
  if (st.nsplit >= 64) {
    for (int64_t o = 0; o < nout; ++o) {
      double re = 0, im = 0;
      for (int sp = threadIdx.x; sp < st.nsplit; sp += kBodyThreads) {
        const double2 v = partial[st.poff + o * st.nsplit + sp];
        re += v.x;
        im += v.y;
      }
      red_re[threadIdx.x] = re;
      red_im[threadIdx.x] = im;
      Sync::sync();
      for (int w = kBodyThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
          red_re[threadIdx.x] += red_re[threadIdx.x + w];
          red_im[threadIdx.x] += red_im[threadIdx.x + w];
        }
        Sync::sync();
      }
      if (threadIdx.x == 0) emit(o, red_re[0], red_im[0]);
      Sync::sync();
    }
    return;
  }
  for (int64_t o = threadIdx.x; o < nout; o += kBodyThreads) {
    double re = 0, im = 0;
    for (int sp = 0; sp < st.nsplit; ++sp) {
      const double2 v = partial[st.poff + o * st.nsplit + sp];
      re += v.x;
      im += v.y;
    }
    emit(o, re, im);
  }
}


// ------------------------------------------------------------------ GEMM operand preparation

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// The six-product bf16 split makes its leading term a fixed-point number: an integer multiple of
// q = 2^qexp with |x_0 / q| <= 2^8, q fixed per operand row and 128-byte K block (64 elements).
// Then every product of leading terms within one K block is a multiple of q_a q_b below
// 2^16 q_a q_b, and their block sum of 64 stays below 2^24 q_a q_b, so the tensor core's FP32
// accumulation of the leading product is exact (it truncates nothing). The remainder x - x_0
// (exact in FP32, |.| <= q/2) is split into the middle and low terms in floating point, which
// keeps x to 2^-26 of the block's largest entry. The two-term splits keep a floating leading term:
// with a fixed-point one their single correction term would leave entries far below the block's
// largest with only its 8 or 11 bits.
//
// The scaled fp16 split (OPM_F16X2S) stores x / q instead: hi = rint(x / q), an integer of at most
// 2^9 (exact in fp16), and lo = fp16(x / q - hi), with q kept per row and K block in a scale array
// that the GEMM's epilogue applies to each K block's partial sums. 512^2 * 64 = 2^24 bounds the
// block sum of the leading products, so their accumulation is exact as well.
__device__ __forceinline__ bool split_mode(int mode) { return mode == OPM_BF16X3 || mode == OPM_F16X2S; }
__device__ __forceinline__ int lead_bits(int mode) { return mode == OPM_BF16X3 ? 8 : (mode == OPM_F16X2S ? 9 : 0); }

// qexp for a row block whose largest magnitude is m: q = 2^(floor(log2 m) + 1 - lead bits), so
// that m / q < 2^lead bits; clamped to the normal FP32 range (zero blocks take the floor).
__device__ __forceinline__ int quantum_exp(float m, int lead) {
  const int e = static_cast<int>((__float_as_uint(m) >> 23) & 0xFFu) - 127;  // floor(log2 m), m normal
  const int qe = e + 1 - lead;
  return qe < -126 ? -126 : qe;
}

__device__ __forceinline__ float pow2f(int e) { return __uint_as_float(static_cast<uint32_t>(127 + e) << 23); }

// Leading term of x: rint(x / q) q, exact (power-of-two scalings of a float with |x / q| < 2^9).
__device__ __forceinline__ float lead_term(float x, int qexp) { return rintf(x * pow2f(-qexp)) * pow2f(qexp); }

// Two consecutive operand elements (idx even) of the FP64 operand mode.
__device__ __forceinline__ void store_operand2_f64(const PermDev& p, char* base, int64_t idx, double v0, double v1) {
  *reinterpret_cast<double2*>(reinterpret_cast<double*>(base + p.dst[0]) + idx) = make_double2(v0, v1);
}

// Two consecutive operand elements (idx even, same row and K block) of an FP32-based operand mode
// (the values already rounded to FP32), with one vector store per split term. qexp: the block's
// leading-term quantum (six-product split only).
__device__ __forceinline__ void store_operand2(const PermDev& p, char* base, int64_t idx, float x0, float x1,
                                               int qexp) {
  switch (p.mode) {
    case OPM_F32:
      *reinterpret_cast<float2*>(reinterpret_cast<float*>(base + p.dst[0]) + idx) = make_float2(x0, x1);
      break;
    case OPM_TF32:
      *reinterpret_cast<float2*>(reinterpret_cast<float*>(base + p.dst[0]) + idx) =
          make_float2(to_tf32(x0), to_tf32(x1));
      break;
    case OPM_TF32X2: {  // floating split: hi = tf32(x), lo = tf32(x - hi)
      const float h0 = to_tf32(x0), h1 = to_tf32(x1);
      *reinterpret_cast<float2*>(reinterpret_cast<float*>(base + p.dst[0]) + idx) = make_float2(h0, h1);
      *reinterpret_cast<float2*>(reinterpret_cast<float*>(base + p.dst[1]) + idx) =
          make_float2(to_tf32(x0 - h0), to_tf32(x1 - h1));
      break;
    }
    case OPM_BF16X2: {  // floating split: hi = bf16(x), lo = bf16(x - hi)
      const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
      const float2 hf = __bfloat1622float2(h);
      *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(base + p.dst[0]) + idx) = h;
      *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(base + p.dst[1]) + idx) =
          __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
      break;
    }
    case OPM_F16X2S: {  // x / q in fp16: an integer leading term and the remainder
      const float sc = pow2f(-qexp);
      const float y0 = x0 * sc, y1 = x1 * sc;
      const float h0 = rintf(y0), h1 = rintf(y1);
      *reinterpret_cast<__half2*>(reinterpret_cast<__half*>(base + p.dst[0]) + idx) = __floats2half2_rn(h0, h1);
      *reinterpret_cast<__half2*>(reinterpret_cast<__half*>(base + p.dst[1]) + idx) =
          __floats2half2_rn(y0 - h0, y1 - h1);
      break;
    }
    default: {  // OPM_BF16X3: fixed-point leading term, floating middle and low terms
      const float h0 = lead_term(x0, qexp), h1 = lead_term(x1, qexp);
      const float r0 = x0 - h0, r1 = x1 - h1;
      const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
      const float2 mf = __bfloat1622float2(m);
      *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(base + p.dst[0]) + idx) =
          __floats2bfloat162_rn(h0, h1);
      *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(base + p.dst[1]) + idx) = m;
      *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(base + p.dst[2]) + idx) =
          __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
      break;
    }
  }
}

// Tile of 32 rows x TK k per iteration, 256 threads; TK = 32, or for the six-product bf16 split
// 64 = one 128-byte K block of the operand (the leading-term quantum is fixed per row and block).
// The tile is staged in shared memory in S: double for the FP64 operand mode, float for every
// other mode (which splits the FP32 rounding of each value), so that a 32 x 64 float tile takes
// the space of a 32 x 32 double one. The source offsets of the tile's rows and columns are
// computed once per tile; loads run with lanes along whichever index is contiguous in the source,
// stores with lanes along k and two elements per vector store.
// Shared-memory scratch of one gather block (the tile in S, row and column offsets, quanta).
template <typename S>
struct PermSmem {
  static constexpr int TKMAX = sizeof(S) == 8 ? 32 : 64;
  S tre[32][TKMAX + 1], tim[32][TKMAX + 1];
  int64_t roff[32], koff[TKMAX];
  int qre[32], qim[32];
};

// The three bf16 terms of 8 consecutive values of one row block (OPM_BF16X3, quantum 2^qexp),
// packed 8 per 16 bytes; the same arithmetic, in the same order, as store_operand2.
__device__ __forceinline__ void split8_bf16x3(const float (&x)[8], int qexp, uint4& hi, uint4& mid, uint4& lo) {
  uint32_t h[4], m[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float h0 = lead_term(x[2 * j], qexp), h1 = lead_term(x[2 * j + 1], qexp);
    const float r0 = x[2 * j] - h0, r1 = x[2 * j + 1] - h1;
    const __nv_bfloat162 mb = __floats2bfloat162_rn(r0, r1);
    const float2 mf = __bfloat1622float2(mb);
    const __nv_bfloat162 hb = __floats2bfloat162_rn(h0, h1);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
    h[j] = *reinterpret_cast<const uint32_t*>(&hb);
    m[j] = *reinterpret_cast<const uint32_t*>(&mb);
    l[j] = *reinterpret_cast<const uint32_t*>(&lb);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  mid = make_uint4(m[0], m[1], m[2], m[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ uint4 neg_bf16x8(uint4 v) {
  return make_uint4(v.x ^ 0x80008000u, v.y ^ 0x80008000u, v.z ^ 0x80008000u, v.w ^ 0x80008000u);
}

// The six-product bf16 split over whole 32-row x 64-k tiles (R >= 32, K >= 64). Each thread splits
// 8 consecutive k of one row -- the row's quantum from a max over the row's 8 threads (lanes of
// one aligned group of 8) -- and writes every term with 16-byte stores; the embedded side's
// second copies reuse the split (-Im is Im with the sign bits flipped). Two barriers per tile.
// The values are those of the general loop below, which handles every other case.
template <typename Sync>
__device__ __forceinline__ void perm_tiles_bf16x3(const PermDev& p, const double* __restrict__ arena,
                                                  char* __restrict__ base, int vb, int vg, const int64_t* t_r,
                                                  int c_r, const int64_t* t_k, int c_k, PermSmem<float>& sm,
                                                  PermSmem<float>* sm2) {
  const int64_t R = int64_t(1) << p.rbits, K = int64_t(1) << p.kbits;
  const int64_t ntk = K / 64, ntiles = (R / 32) * ntk;
  const double* src = arena + p.src;
  const float* srcf = reinterpret_cast<const float*>(arena) + p.src;
  const int64_t ld = 2 * K;
  const int lead = lead_bits(OPM_BF16X3);
  uint4* d0 = reinterpret_cast<uint4*>(base + p.dst[0]);
  uint4* d1 = reinterpret_cast<uint4*>(base + p.dst[1]);
  uint4* d2 = reinterpret_cast<uint4*>(base + p.dst[2]);
  // split phase: row i of the tile, k chunk c (k = 8c .. 8c + 7)
  const int i = threadIdx.x >> 3, c = threadIdx.x & 7;
  auto store3 = [&](int64_t idx, const uint4& a, const uint4& b, const uint4& e) {
    d0[idx >> 3] = a;
    d1[idx >> 3] = b;
    d2[idx >> 3] = e;
  };
  // the source offsets of a tile's 32 rows and 64 k (threads 0..95)
  auto lookups = [&](PermSmem<float>& b, int64_t tile) {
    const int64_t r0 = (tile / ntk) * 32, k0 = (tile % ntk) * 64;
    if (threadIdx.x < 32) b.roff[threadIdx.x] = lookup(t_r, c_r, r0 + threadIdx.x);
    else if (threadIdx.x < 96) b.koff[threadIdx.x - 32] = lookup(t_k, c_k, k0 + threadIdx.x - 32);
  };
  // thread element q (of 8): tile row rr and column kk, lanes along the source-contiguous index
  auto elem = [&](int q, int& rr, int& kk) {
    const int l = threadIdx.x + 256 * q;
    rr = p.rows_fast ? (l & 31) : (l >> 6);
    kk = p.rows_fast ? (l >> 5) : (l & 63);
  };
  // split and store a staged tile
  auto split_tile = [&](const PermSmem<float>& b, int64_t tile) {
    const int64_t r = (tile / ntk) * 32 + i, k = (tile % ntk) * 64 + 8 * c;
    uint4 h, m, l;
    {
      float x[8];
      float mx = 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        x[j] = b.tre[i][8 * c + j];
        mx = fmaxf(mx, fabsf(x[j]));
      }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      split8_bf16x3(x, quantum_exp(mx, lead), h, m, l);
    }
    store3(r * ld + k, h, m, l);                                  // (s=0, t=0) or Y side: Re
    if (p.embed) store3((R + r) * ld + K + k, h, m, l);           // (s=1, t=1): Re
    {
      float x[8];
      float mx = 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        x[j] = b.tim[i][8 * c + j];
        mx = fmaxf(mx, fabsf(x[j]));
      }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      split8_bf16x3(x, quantum_exp(mx, lead), h, m, l);
    }
    if (p.embed) {
      store3((R + r) * ld + k, h, m, l);                                       // (s=1, t=0):  Im
      store3(r * ld + K + k, neg_bf16x8(h), neg_bf16x8(m), neg_bf16x8(l));     // (s=0, t=1): -Im
    } else {
      store3(r * ld + K + k, h, m, l);                                         // Y side: Im
    }
  };
  if (sm2 != nullptr && p.src_f32) {
    // Complex64 source and a second tile buffer: the next tile's values are copied
    // asynchronously into the other buffer while this one is split, so a tile's load latency
    // overlaps the previous tile's split and stores instead of following it.
    PermSmem<float>* const buf[2] = {&sm, sm2};
    auto issue = [&](PermSmem<float>& b) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        int rr, kk;
        elem(q, rr, kk);
        const int64_t off = b.roff[rr] + b.koff[kk];
        cp_async4(&b.tre[rr][kk], srcf + off);
        cp_async4(&b.tim[rr][kk], srcf + p.plane + off);
      }
    };
    int64_t tile = vb;
    if (tile < ntiles) lookups(*buf[0], tile);
    Sync::sync();
    if (tile < ntiles) issue(*buf[0]);
    cp_async_commit();
    int cur = 0;
    for (; tile < ntiles; tile += vg) {
      const int64_t next = tile + vg;
      // buf[cur ^ 1]'s offsets were last read by the copies of two tiles back, issued before the
      // previous barrier
      if (next < ntiles) lookups(*buf[cur ^ 1], next);
      cp_async_wait<0>();
      Sync::sync();  // this tile's values and the next tile's offsets are visible; every thread
                     // has split the previous tile, whose buffer the next copies overwrite
      if (next < ntiles) issue(*buf[cur ^ 1]);
      cp_async_commit();
      split_tile(*buf[cur], tile);
      cur ^= 1;
    }
    cp_async_wait<0>();
    Sync::sync();
    return;
  }
  for (int64_t tile = vb; tile < ntiles; tile += vg) {
    lookups(sm, tile);
    Sync::sync();
    {
      // all loads (x 2 planes) of a thread are issued before its shared-memory stores
      float vr[8], vi[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        int rr, kk;
        elem(q, rr, kk);
        const int64_t off = sm.roff[rr] + sm.koff[kk];
        if (p.src_f32) {
          vr[q] = srcf[off];
          vi[q] = srcf[p.plane + off];
        } else {
          vr[q] = static_cast<float>(src[off]);
          vi[q] = static_cast<float>(src[p.plane + off]);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        int rr, kk;
        elem(q, rr, kk);
        sm.tre[rr][kk] = vr[q];
        sm.tim[rr][kk] = vi[q];
      }
    }
    Sync::sync();
    split_tile(sm, tile);
  }
  Sync::sync();
}

template <typename S, typename Sync>
__device__ __forceinline__ void perm_body(const PermDev* __restrict__ perms, const double* __restrict__ arena,
                                          char* __restrict__ base, int vb, int vg, int vy, int64_t* tab,
                                          PermSmem<S>& sm, PermSmem<float>* sm2 = nullptr) {
  constexpr int TKMAX = PermSmem<S>::TKMAX;
  auto& tre = sm.tre;
  auto& tim = sm.tim;
  auto& roff = sm.roff;
  auto& koff = sm.koff;
  auto& qre = sm.qre;
  auto& qim = sm.qim;
  const PermDev& p = perms[vy];
  const int c_r = nchunks(p.rows.nbits), c_k = nchunks(p.cols.nbits);
  int64_t* t_r = tab;
  int64_t* t_k = tab + c_r * 256;
  build_table(p.rows, t_r);
  build_table(p.cols, t_k);
  Sync::sync();
  if constexpr (sizeof(S) == 4) {
    if (p.mode == OPM_BF16X3 && p.rbits >= 5 && p.kbits >= 6) {
      perm_tiles_bf16x3<Sync>(p, arena, base, vb, vg, t_r, c_r, t_k, c_k, sm, sm2);
      return;
    }
  }
  const bool split = sizeof(S) == 4 && split_mode(p.mode);
  const int lead = lead_bits(p.mode);
  // K block of the six-product split in complex k: 64 elements of one plane; with K below that,
  // one block holds both planes of the row (Re and -Im, or Im and Re, or Re and Im)
  const int W = split ? 64 : 32;
  const int TR = p.rbits >= 5 ? 32 : (1 << p.rbits);
  const int TK = p.kbits >= 6 && W == 64 ? 64 : (p.kbits >= 5 ? 32 : (1 << p.kbits));
  const bool joint = (int64_t(1) << p.kbits) < W;  // the quantum spans both planes
  const int KW = TK > 32 ? 64 : 32;                // k extent of the thread mapping
  const int64_t R = int64_t(1) << p.rbits, K = int64_t(1) << p.kbits;
  const int64_t ntr = R / TR, ntk = K / TK;
  // the source: complex64 (p.src_f32, a reduced-precision GEMM's product) or complex128
  const double* src = arena + p.src;
  const float* srcf = reinterpret_cast<const float*>(arena) + p.src;
  const int64_t ld = 2 * K;
  for (int64_t tile = vb; tile < ntr * ntk; tile += vg) {
    const int64_t r0 = (tile / ntk) * TR, k0 = (tile % ntk) * TK;
    if (threadIdx.x < 32) roff[threadIdx.x] = threadIdx.x < TR ? lookup(t_r, c_r, r0 + threadIdx.x) : 0;
    else if (threadIdx.x < 32 + TKMAX)
      koff[threadIdx.x - 32] = threadIdx.x - 32 < TK ? lookup(t_k, c_k, k0 + threadIdx.x - 32) : 0;
    Sync::sync();
    // all loads (x 2 planes) of a thread are issued before its shared-memory stores
    S vr[8], vi[8];
#pragma unroll
    for (int q = 0; q < TKMAX / 8; ++q) {
      if (q < KW / 8) {
        const int l = threadIdx.x + 256 * q;
        const int rr = p.rows_fast ? (l & 31) : l / KW, kk = p.rows_fast ? (l >> 5) : (l & (KW - 1));
        if (rr < TR && kk < TK) {
          const int64_t off = roff[rr] + koff[kk];
          if (p.src_f32) {
            vr[q] = srcf[off];
            vi[q] = srcf[p.plane + off];
          } else {
            vr[q] = static_cast<S>(src[off]);
            vi[q] = static_cast<S>(src[p.plane + off]);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < TKMAX / 8; ++q) {
      if (q < KW / 8) {
        const int l = threadIdx.x + 256 * q;
        const int rr = p.rows_fast ? (l & 31) : l / KW, kk = p.rows_fast ? (l >> 5) : (l & (KW - 1));
        if (rr < TR && kk < TK) {
          tre[rr][kk] = vr[q];
          tim[rr][kk] = vi[q];
        }
      }
    }
    Sync::sync();
    if (split) {
      // per row: the largest |Re| and |Im| of the tile's k range (of the FP32 values that are
      // split), one warp per four rows
      const int wp = threadIdx.x >> 5, ln = threadIdx.x & 31;
      for (int i = wp; i < TR; i += 8) {
        float mr = 0.f, mi = 0.f;
        for (int k = ln; k < TK; k += 32) {
          mr = fmaxf(mr, fabsf(static_cast<float>(tre[i][k])));
          mi = fmaxf(mi, fabsf(static_cast<float>(tim[i][k])));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          mr = fmaxf(mr, __shfl_xor_sync(0xffffffffu, mr, o));
          mi = fmaxf(mi, __shfl_xor_sync(0xffffffffu, mi, o));
        }
        if (ln == 0) {
          if (joint) mr = mi = fmaxf(mr, mi);
          qre[i] = quantum_exp(mr, lead);
          qim[i] = quantum_exp(mi, lead);
        }
      }
      Sync::sync();
      if (p.mode == OPM_F16X2S && threadIdx.x < TR) {
        // the scales q of this tile's rows, [K block][row] over the operand's rows (2R embedded):
        // t = 0 holds Re (s = 0) or Im (s = 1), t = 1 holds -Im (s = 0) or Re (s = 1); a K below
        // one block puts both halves of a row in block 0 with a joint quantum
        const int i = threadIdx.x;
        const int64_t r = r0 + i, Rt = p.embed ? 2 * R : R;
        float* sc = reinterpret_cast<float*>(base + p.dst[2]);
        const float fr = pow2f(qre[i]), fi = pow2f(qim[i]);
        const int64_t kb0 = joint ? 0 : k0 / 64, kb1 = joint ? 0 : (K + k0) / 64;
        if (p.embed) {
          sc[kb0 * Rt + r] = fr;
          sc[kb0 * Rt + R + r] = fi;
          if (!joint) {
            sc[kb1 * Rt + r] = fi;
            sc[kb1 * Rt + R + r] = fr;
          }
        } else {
          sc[kb0 * Rt + r] = fr;
          if (!joint) sc[kb1 * Rt + r] = fi;
        }
      }
    }
    const int pairs = TK >> 1;
    for (int w = threadIdx.x; w < TR * pairs; w += kBodyThreads) {
      const int i = w / pairs, j = 2 * (w % pairs);
      const int64_t r = r0 + i, k = k0 + j;
      if constexpr (sizeof(S) == 8) {
        const double re0 = tre[i][j], re1 = tre[i][j + 1], im0 = tim[i][j], im1 = tim[i][j + 1];
        if (p.embed) {
          store_operand2_f64(p, base, r * ld + k, re0, re1);             // (s=0, t=0):  Re
          store_operand2_f64(p, base, r * ld + K + k, -im0, -im1);       // (s=0, t=1): -Im
          store_operand2_f64(p, base, (R + r) * ld + k, im0, im1);       // (s=1, t=0):  Im
          store_operand2_f64(p, base, (R + r) * ld + K + k, re0, re1);   // (s=1, t=1):  Re
        } else {
          store_operand2_f64(p, base, r * ld + k, re0, re1);
          store_operand2_f64(p, base, r * ld + K + k, im0, im1);
        }
      } else {
        const float re0 = tre[i][j], re1 = tre[i][j + 1], im0 = tim[i][j], im1 = tim[i][j + 1];
        const int qr = split ? qre[i] : 0, qi = split ? qim[i] : 0;
        if (p.embed) {
          store_operand2(p, base, r * ld + k, re0, re1, qr);             // (s=0, t=0):  Re
          store_operand2(p, base, r * ld + K + k, -im0, -im1, qi);       // (s=0, t=1): -Im
          store_operand2(p, base, (R + r) * ld + k, im0, im1, qi);       // (s=1, t=0):  Im
          store_operand2(p, base, (R + r) * ld + K + k, re0, re1, qr);   // (s=1, t=1):  Re
        } else {
          store_operand2(p, base, r * ld + k, re0, re1, qr);
          store_operand2(p, base, r * ld + K + k, im0, im1, qi);
        }
      }
    }
    Sync::sync();
  }
}


// ------------------------------------------------------------------ final FP64 reduction

template <typename T, typename Sync>
__device__ __forceinline__ void open_body(const FinalDev* __restrict__ fd, const T* __restrict__ arena,
                                          const double2* __restrict__ scalars, double* __restrict__ traces,
                                          double* __restrict__ partial, int vb, int vg, int64_t* tab, double* red) {
  const FinalDev& f = *fd;
  // common factor: product of scalar components and 2 per untouched wire
  double sr = ldexp(1.0, f.loops), si = 0;
  for (int i = 0; i < f.n_scalars; ++i) {
    const double2 v = scalars[i];
    const double nr = sr * v.x - si * v.y, ni = sr * v.y + si * v.x;
    sr = nr;
    si = ni;
  }
  const int c = nchunks(f.open_map.nbits);
  build_table(f.open_map, tab);
  Sync::sync();
  const int64_t n = int64_t(1) << f.open_bits;
  double acc = 0;
  for (int64_t j = int64_t(vb) * kBodyThreads + threadIdx.x; j < n; j += int64_t(vg) * kBodyThreads) {
    double tr = 1, ti = 0;
    if (f.open_off >= 0) {
      const int64_t off = lookup(tab, c, j);
      if (f.open_f32) {  // the product of a reduced-precision GEMM (complex64)
        const float* of = reinterpret_cast<const float*>(arena) + f.open_off;
        tr = of[off];
        ti = of[f.open_plane + off];
      } else {
        tr = static_cast<double>(arena[f.open_off + off]);
        ti = static_cast<double>(arena[f.open_off + f.open_plane + off]);
      }
    }
    const double vr = tr * sr - ti * si, vi = tr * si + ti * sr;
    traces[2 * j] = vr;
    traces[2 * j + 1] = vi;
    acc += vr * vr + vi * vi;
  }
  red[threadIdx.x] = acc;
  Sync::sync();
  for (int w = kBodyThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    Sync::sync();
  }
  if (threadIdx.x == 0) partial[vb] = red[0];
}

// Thread 0 only.
__device__ __forceinline__ void final_body(const FinalDev* __restrict__ fd, const double2* __restrict__ scalars,
                                           const double* __restrict__ partial, double* __restrict__ result) {
  const FinalDev& f = *fd;
  double S = 0;
  if (f.alg == 2) {
    double sr = ldexp(1.0, f.loops), si = 0;
    for (int i = 0; i < f.n_scalars; ++i) {
      const double2 v = scalars[i];
      const double nr = sr * v.x - si * v.y, ni = sr * v.y + si * v.x;
      sr = nr;
      si = ni;
    }
    S = sr;
  } else {
    for (int b = 0; b < f.nblocks; ++b) S += partial[b];
  }
  const double d2 = ldexp(1.0, 2 * f.n_qubits);
  result[0] = S;
  result[1] = S / d2;
  result[2] = (d2 - S) / d2;
}

// C[i] = sum over splits s (in order) of W[s][i], block vb of vg: the FP32 partials of a K-split
// tensor-core GEMM, added in FP32 with Kahan's compensation (the sum's error stays within a few
// units in the last place of the largest partial, whatever the number of splits; no FP64
// arithmetic, which GB300 runs at a small fraction of its FP32 rate).
__device__ __forceinline__ void split_sum_body(const float* __restrict__ W, int ksplit, int64_t n,
                                               float* __restrict__ C, int vb, int vg) {
  for (int64_t i = int64_t(vb) * kBodyThreads + threadIdx.x; i < n; i += int64_t(vg) * kBodyThreads) {
    float s = 0.0f, comp = 0.0f;
    for (int k = 0; k < ksplit; ++k) {
      const float y = W[k * n + i] - comp;
      const float t = s + y;
      comp = (t - s) - y;
      s = t;
    }
    C[i] = s;
  }
}

}  // namespace ajf
