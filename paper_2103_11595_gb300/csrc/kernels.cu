// CUDA-core kernels of the contraction program (sm_103a).
//
//  k_leaf        builds every leaf tensor of the miter network from the uploaded complex128
//                gate/Kraus matrices (gate, conjugate, adjoint, transpose, Kraus stack with an
//                open index, superoperator M_N = sum_k N_k (x) N_k^*; Sec. IV-A/IV-B).
//  k_small       many independent small pairwise contractions in one launch, one gather per
//                operand element through 8-bit offset tables (bits of any binary-index layout).
//  k_splitk      contractions with few outputs and a long contracted index (including the final
//                full contraction to the trace): FP64 partial sums per block, then k_splitk_done
//                sums them in a fixed order (deterministic).
//  k_perm        gathers a complex tensor into a real, K-contiguous GEMM operand (the complex
//                product C = A B becomes the real product [[Ar,-Ai],[Ai,Ar]] [Br;Bi] = [Cr;Ci]),
//                with the operand format of the precision mode (FP64, FP32, TF32, split TF32,
//                split bf16).
//  k_gemm_simt   real "TN" GEMM on CUDA cores (FP32 or FP64) writing the planar result.
//  k_open/k_final  the FP64 end of the path: t_i for Alg. I, sum |t_i|^2, F_J and 1 - F_J.
#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bodies.cuh"
#include "device.h"
#include "kernels.h"

namespace ajf {

// ------------------------------------------------------------------ standalone kernels
// (the bodies are in bodies.cuh; one launch per program step, 256 threads per block)

template <typename T>
__global__ void __launch_bounds__(kBodyThreads) k_leaf(const LeafDev* leaves, const double* __restrict__ in,
                                                       T* __restrict__ arena) {
  leaf_body<T>(leaves, in, arena, blockIdx.x);
}

template <typename T, typename Acc>
__global__ void __launch_bounds__(kBodyThreads) k_small(const StepDev* __restrict__ steps, int nsteps,
                                                        int total_blocks, T* __restrict__ arena) {
  extern __shared__ int64_t tab[];
  small_body<T, Acc, SyncBlock>(steps, nsteps, total_blocks, arena, blockIdx.x, tab);
}

template <typename T>
__global__ void __launch_bounds__(kBodyThreads) k_splitk(const StepDev* __restrict__ steps, int nsteps,
                                                         const T* __restrict__ arena, double2* __restrict__ partial) {
  extern __shared__ int64_t tab[];
  __shared__ double red_re[kBodyThreads], red_im[kBodyThreads];
  splitk_body<T, SyncBlock>(steps, nsteps, arena, partial, blockIdx.x, tab, red_re, red_im);
}

// 4 blocks per SM (64 registers): the tiled trace is bound by memory latency, and its grid is
// sized for 4 blocks per SM (3 for the staged FP32 form, whose stages take more shared memory)
template <typename T, bool kF32>
__global__ void __launch_bounds__(kBodyThreads, 4) k_dot(const StepDev* __restrict__ steps, int nsteps,
                                                      const T* __restrict__ arena, double2* __restrict__ partial) {
  extern __shared__ int64_t tab[];
  __shared__ double red_re[kBodyThreads], red_im[kBodyThreads];
  dot_body<T, kF32, SyncBlock, kF32>(steps, nsteps, arena, partial, blockIdx.x, tab, red_re, red_im);
}

template <typename T>
__global__ void __launch_bounds__(kBodyThreads) k_splitk_done(const StepDev* __restrict__ steps, int nsteps,
                                                              const double2* __restrict__ partial,
                                                              T* __restrict__ arena, double2* __restrict__ scalars) {
  (void)nsteps;
  __shared__ double red_re[kBodyThreads], red_im[kBodyThreads];
  splitk_done_body<T, SyncBlock>(steps, partial, arena, scalars, blockIdx.x, red_re, red_im);
}

// 4 blocks per SM (64 registers): the gather is bound by memory latency; measured on GB300 with
// 98 registers (2 blocks per SM) a large gather reached 1.2-1.3 TB/s. S: staging type (FP64 for
// the FP64 operand mode, FP32 otherwise).
template <typename S>
__global__ void __launch_bounds__(kBodyThreads, 4) k_perm(const PermDev* __restrict__ perms,
                                                       const double* __restrict__ arena, char* __restrict__ base) {
  extern __shared__ int64_t tab[];
  __shared__ PermSmem<S> sm;
  if constexpr (sizeof(S) == 4) {
    __shared__ PermSmem<float> sm2;  // second tile buffer of the six-product split's copy pipeline
    perm_body<S, SyncBlock>(perms, arena, base, blockIdx.x, gridDim.x, blockIdx.y, tab, sm, &sm2);
  } else {
    perm_body<S, SyncBlock>(perms, arena, base, blockIdx.x, gridDim.x, blockIdx.y, tab, sm);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBodyThreads) k_open(const FinalDev* __restrict__ fd, const T* __restrict__ arena,
                                                       const double2* __restrict__ scalars,
                                                       double* __restrict__ traces, double* __restrict__ partial) {
  extern __shared__ int64_t tab[];
  __shared__ double red[kBodyThreads];
  open_body<T, SyncBlock>(fd, arena, scalars, traces, partial, blockIdx.x, gridDim.x, tab, red);
}

__global__ void k_final(const FinalDev* __restrict__ fd, const double2* __restrict__ scalars,
                        const double* __restrict__ partial, double* __restrict__ result) {
  if (threadIdx.x == 0) final_body(fd, scalars, partial, result);
}

// ------------------------------------------------------------------ CUDA-core GEMM

// C[M][N] (row-major, ldc = N) = A[M][K] . B[N][K]^T with A and B row-major, K contiguous;
// operands, accumulation and result in T (FP32 or FP64).
template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) k_gemm_simt(const T* __restrict__ A, const T* __restrict__ B,
                                                                     T* __restrict__ C, int64_t M, int64_t N,
                                                                     int64_t K) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tr = tid / (BN / TN), tc = tid % (BN / TN);
  const int64_t nbn = (N + BN - 1) / BN;
  const int64_t m0 = (int64_t(blockIdx.x) / nbn) * BM, n0 = (int64_t(blockIdx.x) % nbn) * BN;
  // FP64: one accumulator per output. FP32: the products of each BK-long K tile are summed in
  // FP32, and the tile sums are added into a compensated (Kahan) FP32 accumulator, so that long
  // contractions do not lose the small late addends of a plain FP32 running sum.
  constexpr bool kComp = sizeof(T) == 4;
  T acc[TM][TN], comp[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = comp[i][j] = 0;
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += NT) {
      const int r = e / BK, k = e % BK;
      const int64_t gm = m0 + r, gk = k0 + k;
      As[k][r] = (gm < M && gk < K) ? A[gm * K + gk] : T(0);
    }
    for (int e = tid; e < BN * BK; e += NT) {
      const int r = e / BK, k = e % BK;
      const int64_t gn = n0 + r, gk = k0 + k;
      Bs[k][r] = (gn < N && gk < K) ? B[gn * K + gk] : T(0);
    }
    __syncthreads();
    T part[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) part[i][j] = 0;
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[k][tr * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[k][tc * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) part[i][j] += a[i] * b[j];
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        if (kComp) {
          const T y = part[i][j] - comp[i][j];
          const T t = acc[i][j] + y;
          comp[i][j] = (t - acc[i][j]) - y;
          acc[i][j] = t;
        } else {
          acc[i][j] += part[i][j];
        }
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gm = m0 + tr * TM + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gn = n0 + tc * TN + j;
      if (gn < N) C[gm * N + gn] = acc[i][j];
    }
  }
}

// ------------------------------------------------------------------ persistent kernel

// offset(idx) = sum over the map's bits set in idx of 2^pos (bits with pos < 0 address nothing)
__device__ __forceinline__ int64_t map_offset(const BitMap& m, int64_t idx) {
  int64_t off = 0;
  for (int i = 0; i < m.nbits; ++i)
    if (((idx >> i) & 1) && m.pos[i] >= 0) off += int64_t(1) << m.pos[i];
  return off;
}

// First local index handled by this thread when the flat index space continues from `base`
// (thread t takes the flat indices congruent to t modulo the block size).
__device__ __forceinline__ int64_t first_local(int64_t base, int unit, int nunits) {
  return ((unit - base % nunits) % nunits + nunits) % nunits;
}

// One thread block per network runs the network's whole program: leaves, every step in level
// order (one block barrier per level), the FP64 trace and F. The work region (all tensors) is
// kept in shared memory when it fits (job.smem), otherwise it stays in the arena. Steps of one
// level are independent; a level's outputs are spread over the threads (LK_SMALL: a thread per
// output element; LK_SPLITK: a warp per output element, lanes along the contracted index,
// summed in a fixed shuffle order).
__global__ void __launch_bounds__(256) k_persistent(const InterpJob* __restrict__ jobs,
                                                    const InterpOp* __restrict__ ops) {
  extern __shared__ double swork[];
  __shared__ double red[256];
  const InterpJob J = jobs[blockIdx.x];
  double* arena = reinterpret_cast<double*>(J.base);
  double* W = J.smem ? swork : arena;
  const int64_t w0 = J.smem ? J.work0 : 0;
  const int tid = threadIdx.x, nt = blockDim.x;

  // leaves
  {
    const LeafDev* leaves = reinterpret_cast<const LeafDev*>(J.base + J.off_leaves);
    const double* in = reinterpret_cast<const double*>(J.base + J.off_inputs);
    int64_t base = 0;
    for (int l = 0; l < J.n_leaves; ++l) {
      const LeafDev L = leaves[l];
      const int64_t n = int64_t(1) << L.bits;
      for (int64_t e = first_local(base, tid, nt); e < n; e += nt) {
        double re, im;
        leaf_value(L, in, leaf_full_index(L, e), re, im);
        W[L.off - w0 + e] = re;
        W[L.off - w0 + L.plane + e] = im;
      }
      base += n;
    }
  }
  __syncthreads();

  const StepDev* steps = reinterpret_cast<const StepDev*>(J.base + J.off_steps);
  double2* scalars = reinterpret_cast<double2*>(J.base + J.off_scalars);
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  for (int q = 0; q < J.n_ops; ++q) {
    const InterpOp op = ops[J.op0 + q];
    int64_t base = 0;
    for (int s = op.first; s < op.first + op.count; ++s) {
      const StepDev& st = steps[s];
      const int64_t nout = int64_t(1) << st.rc, nk = int64_t(1) << st.rk;
      const double* A = W + (st.a - w0);
      const double* B = W + (st.b - w0);
      if (op.kind == 0) {
        double* C = W + (st.c - w0);
        for (int64_t o = first_local(base, tid, nt); o < nout; o += nt) {
          const int64_t oa = map_offset(st.oa, o), ob = map_offset(st.ob, o);
          double re = 0, im = 0;
          for (int64_t kk = 0; kk < nk; ++kk) {
            const int64_t ia = oa + map_offset(st.ka, kk), ib = ob + map_offset(st.kb, kk);
            const double ar = A[ia], ai = A[st.pa + ia], br = B[ib], bi = B[st.pb + ib];
            re += ar * br - ai * bi;
            im += ar * bi + ai * br;
          }
          C[o] = re;
          C[st.pc + o] = im;
        }
      } else {
        for (int64_t o = first_local(base, warp, nw); o < nout; o += nw) {
          const int64_t oa = map_offset(st.oa, o), ob = map_offset(st.ob, o);
          double re = 0, im = 0;
          for (int64_t kk = lane; kk < nk; kk += 32) {
            const int64_t ia = oa + map_offset(st.ka, kk), ib = ob + map_offset(st.kb, kk);
            const double ar = A[ia], ai = A[st.pa + ia], br = B[ib], bi = B[st.pb + ib];
            re += ar * br - ai * bi;
            im += ar * bi + ai * br;
          }
          for (int w = 16; w > 0; w >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, w);
            im += __shfl_xor_sync(0xffffffffu, im, w);
          }
          if (lane == 0) {
            if (st.scalar_slot >= 0) {
              scalars[st.scalar_slot] = make_double2(re, im);
            } else {
              W[st.c - w0 + o] = re;
              W[st.c - w0 + st.pc + o] = im;
            }
          }
        }
      }
      base += nout;
    }
    __syncthreads();
  }

  // FP64 end: common factor, traces (Alg. I), sum |t|^2, F and 1 - F
  const FinalDev& f = *reinterpret_cast<const FinalDev*>(J.base + J.off_final);
  double sr = ldexp(1.0, f.loops), si = 0;
  for (int i = 0; i < f.n_scalars; ++i) {
    const double2 v = scalars[i];
    const double nr = sr * v.x - si * v.y, ni = sr * v.y + si * v.x;
    sr = nr;
    si = ni;
  }
  double* traces = reinterpret_cast<double*>(J.base + J.off_traces);
  const int64_t n = int64_t(1) << f.open_bits;
  double acc = 0;
  for (int64_t j = tid; j < n; j += nt) {
    double tr = 1, ti = 0;
    if (f.open_off >= 0) {
      const int64_t off = map_offset(f.open_map, j);
      tr = W[f.open_off - w0 + off];
      ti = W[f.open_off - w0 + f.open_plane + off];
    }
    const double vr = tr * sr - ti * si, vi = tr * si + ti * sr;
    traces[2 * j] = vr;
    traces[2 * j + 1] = vi;
    acc += vr * vr + vi * vi;
  }
  red[tid] = acc;
  __syncthreads();
  for (int w = nt / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) {
    const double S = f.alg == 2 ? sr : red[0];
    const double d2 = ldexp(1.0, 2 * f.n_qubits);
    double* result = reinterpret_cast<double*>(J.base + J.off_result);
    result[0] = S;
    result[1] = S / d2;
    result[2] = (d2 - S) / d2;
    if (J.out) {
      J.out[0] = S;
      J.out[1] = S / d2;
      J.out[2] = (d2 - S) / d2;
    }
  }
}

// ------------------------------------------------------------------ launch wrappers

static size_t table_bytes(const BitMap* const* maps, int n) {
  size_t b = 0;
  for (int i = 0; i < n; ++i) b += size_t((maps[i]->nbits + 7) / 8) * 256 * sizeof(int64_t);
  return b;
}

cudaError_t launch_leaves(const LeafDev* d_leaves, int n, const double* d_in, void* arena, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_leaf<double><<<n, kBodyThreads, 0, s>>>(d_leaves, d_in, static_cast<double*>(arena));
  return cudaGetLastError();
}

cudaError_t launch_small(const StepDev* d_steps, int nsteps, int total_blocks, size_t smem, void* arena,
                         cudaStream_t s) {
  if (nsteps == 0) return cudaSuccess;
  k_small<double, double><<<total_blocks, 256, smem, s>>>(d_steps, nsteps, total_blocks, static_cast<double*>(arena));
  return cudaGetLastError();
}

cudaError_t launch_splitk(const StepDev* d_steps, int nsteps, int total_blocks, size_t smem, void* arena,
                          double2* partial, double2* scalars, cudaStream_t s) {
  if (nsteps == 0) return cudaSuccess;
  k_splitk<double><<<total_blocks, 256, smem, s>>>(d_steps, nsteps, static_cast<const double*>(arena), partial);
  k_splitk_done<double><<<nsteps, 256, 0, s>>>(d_steps, nsteps, partial, static_cast<double*>(arena), scalars);
  return cudaGetLastError();
}

bool dot_staged(const StepDev& st, bool f32_products) { return f32_products && st.fa && st.fb && st.ntl == 10; }

size_t dot_smem_bytes(const StepDev& st, bool f32_products) {
  const BitMap* maps[2] = {&st.ka, &st.kb};
  const size_t nt = size_t(1) << st.ntl;
  // the staged form adds 6 of its 12 stage arrays (nt floats each) after the layout below; the
  // other 6 overlay the offset and staging arrays once their values are in registers
  return table_bytes(maps, 2) + nt * (8 + 8 + 8 + 8 + 2) + 16 + (dot_staged(st, f32_products) ? 6 * nt * 4 : 0);
}

cudaError_t launch_dot(const StepDev* d_steps, int nsteps, int total_blocks, size_t smem, const void* arena,
                       double2* partial, double2* scalars, bool f32_products, cudaStream_t s) {
  if (nsteps == 0) return cudaSuccess;
  if (f32_products)
    k_dot<double, true><<<total_blocks, 256, smem, s>>>(d_steps, nsteps, static_cast<const double*>(arena), partial);
  else
    k_dot<double, false><<<total_blocks, 256, smem, s>>>(d_steps, nsteps, static_cast<const double*>(arena), partial);
  k_splitk_done<double><<<nsteps, 256, 0, s>>>(d_steps, nsteps, partial, static_cast<double*>(const_cast<void*>(arena)),
                                               scalars);
  return cudaGetLastError();
}

cudaError_t launch_perm(const PermDev* d_perms, int nperm, int grid_x, size_t smem, const void* arena, void* base,
                        bool op_f64, cudaStream_t s) {
  if (nperm == 0) return cudaSuccess;
  dim3 grid(grid_x, nperm);
  // the operand format (FP64 or a reduced one) is in each PermDev, and every PermDev of one launch
  // has the same one; each source is complex128, or complex64 when a reduced-precision GEMM made it
  if (op_f64)
    k_perm<double><<<grid, 256, smem, s>>>(d_perms, static_cast<const double*>(arena), static_cast<char*>(base));
  else
    k_perm<float><<<grid, 256, smem, s>>>(d_perms, static_cast<const double*>(arena), static_cast<char*>(base));
  return cudaGetLastError();
}

cudaError_t launch_gemm_simt(const void* A, const void* B, void* C, int64_t M, int64_t N, int64_t K, bool f64,
                             cudaStream_t s) {
  if (f64) {
    const unsigned grid = unsigned(((N + 63) / 64) * ((M + 63) / 64));
    k_gemm_simt<double, 64, 64, 8, 4, 4><<<grid, 256, 0, s>>>(static_cast<const double*>(A), static_cast<const double*>(B),
                                                             static_cast<double*>(C), M, N, K);
  } else {
    const unsigned grid = unsigned(((N + 63) / 64) * ((M + 127) / 128));
    k_gemm_simt<float, 128, 64, 8, 8, 4><<<grid, 256, 0, s>>>(static_cast<const float*>(A), static_cast<const float*>(B),
                                                             static_cast<float*>(C), M, N, K);
  }
  return cudaGetLastError();
}

cudaError_t launch_final(const FinalDev* d_fd, int open_bits_nchunks, int nblocks, const void* arena,
                         const double2* scalars, double* traces, double* partial, double* result, cudaStream_t s) {
  const size_t smem = size_t(open_bits_nchunks) * 256 * sizeof(int64_t);
  k_open<double><<<nblocks, 256, smem, s>>>(d_fd, static_cast<const double*>(arena), scalars, traces, partial);
  k_final<<<1, 32, 0, s>>>(d_fd, scalars, partial, result);
  return cudaGetLastError();
}

size_t step_table_bytes(const StepDev& st) {
  const BitMap* maps[4] = {&st.oa, &st.ob, &st.ka, &st.kb};
  return table_bytes(maps, 4);
}

size_t perm_table_bytes(const PermDev& p) {
  const BitMap* maps[2] = {&p.rows, &p.cols};
  return table_bytes(maps, 2);
}

cudaError_t set_kernel_smem_limits() {
  const int big = 96 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_small<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_splitk<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dot<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dot<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_perm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_perm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_open<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  return e;
}

}  // namespace ajf

namespace ajf {

cudaError_t launch_persistent(const InterpJob* d_jobs, int n_jobs, const InterpOp* d_ops, size_t smem, int threads,
                              cudaStream_t s) {
  if (n_jobs == 0) return cudaSuccess;
  // block size: a power of two from one warp to the kernel's 256 (its reduction buffer)
  if (threads < 32 || threads > 256 || (threads & (threads - 1))) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  k_persistent<<<n_jobs, threads, smem, s>>>(d_jobs, d_ops);
  return cudaGetLastError();
}

}  // namespace ajf
