// C ABI of libajf (see include/ajf.h): context, input validation, planning, upload and the
// executor that enqueues a lowered program on the context's stream.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <map>
#include <string>
#include <vector>

#include "ajf_internal.h"
#include "kernels.h"
#include "mlp.h"
#include "program.h"

using namespace ajf;

namespace {

// NVTX range for profilers (Nsight Systems / Compute): header-only NVTX3, inert when no tool is
// attached. Ranges: plan, upload, program run (graph replay or enqueue), result read-back,
// sliced evaluations and batches.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

struct GateData {
  int arity;
  int q[3];
  std::vector<double> mat;  // complex128 interleaved
};

struct NoiseData {
  int after, arity, nk;
  int q[3];
  std::vector<double> kraus;
};

}  // namespace

struct ajf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  int n = 0;
  bool has_ideal = false, has_impl = false;
  std::vector<GateData> ideal, impl;
  std::vector<NoiseData> noises;
  // plan
  bool planned = false;
  int alg = 0;
  ajf_plan_opts opts{};
  Inputs in;
  Network net;
  Path path;
  Program prog;
  ajf_plan_info info{};
  std::vector<char> desc_image;
  // device memory
  char* arena = nullptr;
  size_t arena_cap = 0;
  bool own_arena = true;
  void* user_ws = nullptr;
  size_t user_ws_bytes = 0;
  bool uploaded = false;
  char* pinned = nullptr;
  size_t pinned_cap = 0;
  cudaGraphExec_t graph = nullptr;
  bool tc_device = false;
  bool have_alg1 = false;
  // sliced Alg. I plan: noises with a fixed Kraus index and their leaves; traces gathered per slice
  std::vector<int> slice_noises, slice_leaves;
  std::vector<double> slice_traces;
  // progress of a sliced Alg. I evaluation: slices done (in the plan's order), their sum |t|^2,
  // traces done, and whether slice_traces holds every trace done (false after a restore)
  int64_t slice_next = 0, slice_done = 0;
  double slice_S = 0;
  bool slice_traces_valid = true;
  // bond slicing: the sliced labels, and for each leaf that carries one, the positions of its
  // sliced labels in the full leaf index with the label's index into bond_labels
  std::vector<int> bond_labels;
  struct BondLeaf {
    int leaf;
    std::vector<std::pair<int, int>> bits;  // (position in the full leaf index, sliced label)
  };
  std::vector<BondLeaf> bond_leaves;
  std::vector<double> bond_traces;  // Alg. I: FP64 sums of the slices' traces (padded order)
  // structural plan cache: the path is reused when the network's shape and options repeat
  // (path_full: the unsliced path; path: the one lowered, restricted to the sliced network)
  Path path_full;
  std::vector<int64_t> plan_key;
  bool path_valid = false;
  // lowered-program cache: a re-plan of the same structure, precision and lowering keeps the
  // program, its descriptor image and its CUDA graph; only the packed input values change
  std::vector<int64_t> prog_key;
  bool prog_valid = false;
  int64_t prog_gen = 0;  // bumped whenever a new program is lowered
  // tensor-core GEMM launches prepared on the host for (program, arena); index = launch index.
  // One set for the context's own arena, one for the fixed arena of ajf_fidelity_noalloc, so
  // that alternating the two paths re-encodes nothing.
  struct TcPrepSet {
    std::vector<ajf::TcPrepared> prep;
    int64_t gen = -1;
    char* arena = nullptr;
  };
  TcPrepSet tc_own, tc_static;
  // device address of the fixed arena of ajf_fidelity_noalloc, resolved by ajf_create
  char* static_arena = nullptr;
  // step-interpreter launches led by this context: phase/task tables, GEMM parameter blocks,
  // counters and status word in one device buffer, the CUDA graph of the launch, and what they
  // were built for
  char* q_dev = nullptr;
  size_t q_cap = 0;
  std::vector<uintptr_t> q_key;
  int q_nphases = 0, q_ntasks = 0;
  size_t q_off_phases = 0, q_off_tasks = 0, q_off_counters = 0, q_off_status = 0;
  cudaGraphExec_t q_graph = nullptr;
  double q_flops = 0, q_bytes = 0;
  // profiling
  struct ProfRec {
    cudaEvent_t a, b;
    int cls;
    double flops, bytes;
  };
  bool profiling = false;
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> event_pool;
  ajf_kernel_stats stats[8] = {};
  // learned merge scorer
  std::vector<float> mlp_weights;
  int64_t mlp_version = 0;
  ajf::MlpScorer mlp_scorer;
  // persistent launches led by this context: job/op table (device) and what it was built for
  int64_t plan_gen = 0;
  char* pers_dev = nullptr;
  size_t pers_cap = 0;
  std::vector<char> pers_host;
  std::vector<uintptr_t> pers_key;
  size_t pers_smem = 0;
  int pers_threads = 256;  // block size of the persistent launch (autotuned per batch)
  cudaEvent_t sync_ev = nullptr;  // cross-stream ordering of persistent launches
};

namespace {

// Process-wide cache of planned paths, keyed by the structural plan key (bounded, oldest out).
struct SharedPaths {
  std::mutex m;
  std::map<std::vector<int64_t>, Path> paths;
  std::deque<std::vector<int64_t>> order;
};
constexpr size_t kSharedPathsMax = 512;
SharedPaths& shared_paths() {
  static SharedPaths sp;
  return sp;
}
bool shared_path_lookup(const std::vector<int64_t>& key, Path* out) {
  SharedPaths& sp = shared_paths();
  std::lock_guard<std::mutex> lock(sp.m);
  auto it = sp.paths.find(key);
  if (it == sp.paths.end()) return false;
  *out = it->second;
  return true;
}
void shared_path_store(const std::vector<int64_t>& key, const Path& path) {
  SharedPaths& sp = shared_paths();
  std::lock_guard<std::mutex> lock(sp.m);
  if (sp.paths.count(key)) return;
  sp.paths.emplace(key, path);
  sp.order.push_back(key);
  while (sp.order.size() > kSharedPathsMax) {
    sp.paths.erase(sp.order.front());
    sp.order.pop_front();
  }
}

ajf_status fail(ajf_ctx* c, ajf_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

ajf_status cuda_fail(ajf_ctx* c, cudaError_t e, const char* what) {
  return fail(c, AJF_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(ctx, call)                                       \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);    \
  } while (0)

using cd = std::complex<double>;

// ||M^dagger M - I||_F for a row-major complex matrix (validation of Sec. II inputs).
double unitarity_error(const double* m, int dim) {
  double err = 0;
  for (int i = 0; i < dim; ++i)
    for (int j = 0; j < dim; ++j) {
      cd s = 0;
      for (int k = 0; k < dim; ++k) s += std::conj(cd(m[2 * (k * dim + i)], m[2 * (k * dim + i) + 1])) *
                                         cd(m[2 * (k * dim + j)], m[2 * (k * dim + j) + 1]);
      if (i == j) s -= 1.0;
      err += std::norm(s);
    }
  return std::sqrt(err);
}

double tp_error(const double* ks, int nk, int dim) {
  double err = 0;
  for (int i = 0; i < dim; ++i)
    for (int j = 0; j < dim; ++j) {
      cd s = 0;
      for (int k = 0; k < nk; ++k) {
        const double* m = ks + 2 * size_t(k) * dim * dim;
        for (int r = 0; r < dim; ++r) s += std::conj(cd(m[2 * (r * dim + i)], m[2 * (r * dim + i) + 1])) *
                                           cd(m[2 * (r * dim + j)], m[2 * (r * dim + j) + 1]);
      }
      if (i == j) s -= 1.0;
      err += std::norm(s);
    }
  return std::sqrt(err);
}

// The CUDA graph of a context replays its current program on its current arena; it is dropped
// when either changes.
void drop_graph(ajf_ctx* c) {
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
}

void invalidate(ajf_ctx* c) {
  c->planned = false;
  c->uploaded = false;
  c->have_alg1 = false;
}

// Pack the caller's matrices into one complex128 buffer and fill the index structures.
void pack_inputs(ajf_ctx* c) {
  Inputs& in = c->in;
  in = Inputs();
  in.n = c->n;
  in.has_ideal = c->has_ideal;
  in.has_impl = c->has_impl;
  auto add_gates = [&](const std::vector<GateData>& src, std::vector<GateIn>& dst) {
    for (auto& g : src) {
      GateIn gi;
      gi.arity = g.arity;
      for (int i = 0; i < 3; ++i) gi.q[i] = g.q[i];
      gi.mat_off = static_cast<int64_t>(in.packed.size() / 2);
      in.packed.insert(in.packed.end(), g.mat.begin(), g.mat.end());
      dst.push_back(gi);
    }
  };
  add_gates(c->ideal, in.ideal);
  if (c->has_impl) add_gates(c->impl, in.impl);
  for (auto& nz : c->noises) {
    NoiseIn ni;
    ni.after = nz.after;
    ni.arity = nz.arity;
    for (int i = 0; i < 3; ++i) ni.q[i] = nz.q[i];
    ni.nk = nz.nk;
    ni.kbits = 0;
    while ((1 << ni.kbits) < nz.nk) ni.kbits++;
    ni.kraus_off = static_cast<int64_t>(in.packed.size() / 2);
    in.packed.insert(in.packed.end(), nz.kraus.begin(), nz.kraus.end());
    in.noises.push_back(ni);
  }
}

ajf_status ensure_arena(ajf_ctx* c) {
  const size_t need = c->prog.arena_bytes;
  if (c->user_ws) {
    if (c->user_ws_bytes < need)
      return fail(c, AJF_E_NOMEM, "workspace of " + std::to_string(c->user_ws_bytes) + " bytes < " +
                                       std::to_string(need) + " needed");
    if (c->arena != static_cast<char*>(c->user_ws)) drop_graph(c);
    c->arena = static_cast<char*>(c->user_ws);
    return AJF_OK;
  }
  if (c->own_arena && c->arena && c->arena_cap >= need) return AJF_OK;
  drop_graph(c);
  if (c->own_arena && c->arena) {
    cudaFree(c->arena);
    c->arena = nullptr;
    c->arena_cap = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, AJF_E_NOMEM, "cudaMalloc of " + std::to_string(need) + " bytes failed");
  }
  c->arena = static_cast<char*>(p);
  c->arena_cap = need;
  c->own_arena = true;
  return AJF_OK;
}

ajf_status ensure_pinned(ajf_ctx* c, size_t bytes) {
  if (c->pinned_cap >= bytes) return AJF_OK;
  if (c->pinned) cudaFreeHost(c->pinned);
  c->pinned = nullptr;
  c->pinned_cap = 0;
  void* p = nullptr;
  cudaError_t e = cudaMallocHost(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, AJF_E_NOMEM, "cudaMallocHost failed");
  }
  c->pinned = static_cast<char*>(p);
  c->pinned_cap = bytes;
  return AJF_OK;
}

cudaEvent_t pool_event(ajf_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Profiling: events around one launch (no-op unless profiling is on).
struct ProfScope {
  ajf_ctx* c;
  cudaStream_t s;
  int cls;
  double flops, bytes;
  cudaEvent_t a = nullptr;
  ProfScope(ajf_ctx* c_, cudaStream_t s_, int cls_, double f, double b) : c(c_), s(s_), cls(cls_), flops(f), bytes(b) {
    if (c->profiling) {
      a = pool_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = pool_event(c);
    cudaEventRecord(b, s);
    c->prof_pending.push_back({a, b, cls, flops, bytes});
  }
};

void drain_profile(ajf_ctx* c) {
  for (auto& r : c->prof_pending) {
    float ms = 0;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      c->stats[r.cls].launches++;
      c->stats[r.cls].ms += ms;
      c->stats[r.cls].flops += r.flops;
      c->stats[r.cls].bytes += r.bytes;
    }
    c->event_pool.push_back(r.a);
    c->event_pool.push_back(r.b);
  }
  c->prof_pending.clear();
}

// Enqueue the device program: leaves, contraction launches, FP64 final reduction.
// Host set-up of the program's tensor-core GEMM launches (tensor maps, tiling, kernel parameters)
// for the context's current arena, kept in `tc` until the program or the arena changes.
ajf_status prepare_tc_set(ajf_ctx* c, ajf_ctx::TcPrepSet* tc) {
  const Program& P = c->prog;
  char* base = c->arena;
  if (tc->gen == c->prog_gen && tc->arena == base && tc->prep.size() == P.launches.size()) return AJF_OK;
  int* status = reinterpret_cast<int*>(base + P.off_status);
  tc->prep.assign(P.launches.size(), TcPrepared{});
  for (size_t i = 0; i < P.launches.size(); ++i) {
    const Launch& ln = P.launches[i];
    if (ln.kind != LK_GEMM_TC) continue;
    const cudaError_t e = tc_gemm_prepare(&tc->prep[i], base, ln.a_off, ln.b_off, ln.npass,
                                          reinterpret_cast<float*>(base + ln.c_off), ln.M, ln.N, ln.K, ln.tc_kind,
                                          reinterpret_cast<float*>(base + ln.ws_off), ln.ksplit, status, kTcWaitNs, 0);
    if (e != cudaSuccess) {
      tc->gen = -1;
      return cuda_fail(c, e, "tensor-core GEMM set-up");
    }
  }
  tc->gen = c->prog_gen;
  tc->arena = base;
  return AJF_OK;
}

ajf_status enqueue_program(ajf_ctx* c, cudaStream_t s, ajf_ctx::TcPrepSet* tc = nullptr) {
  const Program& P = c->prog;
  char* base = c->arena;
  if (!tc) tc = &c->tc_own;
  void* arena = base;
  cudaError_t e;
  {
    ProfScope ps(c, s, 0, 0, 0);
    e = launch_leaves(reinterpret_cast<const LeafDev*>(base + P.off_leaves), static_cast<int>(P.leaves.size()),
                      reinterpret_cast<const double*>(base + P.off_inputs), arena, s);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "leaf kernel");
  const StepDev* steps = reinterpret_cast<const StepDev*>(base + P.off_steps);
  const PermDev* perms = reinterpret_cast<const PermDev*>(base + P.off_perms);
  double2* partial = reinterpret_cast<double2*>(base + P.off_partial);
  double2* scalars = reinterpret_cast<double2*>(base + P.off_scalars);
  // tensor-core GEMM set-up (tensor maps, tiling) is done on the host once per program and arena,
  // outside the timed launches
  {
    const ajf_status st = prepare_tc_set(c, tc);
    if (st != AJF_OK) return st;
  }
  for (size_t li = 0; li < P.launches.size(); ++li) {
    const Launch& ln = P.launches[li];
    static const int kClass[6] = {1, 2, 3, 4, 5, 2};
    ProfScope ps(c, s, kClass[ln.kind], ln.flops, ln.bytes);
    switch (ln.kind) {
      case LK_DOT:
        e = launch_dot(steps + ln.first, ln.count, ln.blocks, ln.smem, arena, partial, scalars, ln.op_f64 == 0, s);
        break;
      case LK_SMALL:
        e = launch_small(steps + ln.first, ln.count, ln.blocks, ln.smem, arena, s);
        break;
      case LK_SPLITK:
        e = launch_splitk(steps + ln.first, ln.count, ln.blocks, ln.smem, arena, partial, scalars, s);
        break;
      case LK_PERM:
        e = launch_perm(perms + ln.first, ln.count, ln.blocks, ln.smem, arena, base, ln.op_f64 != 0, s);
        break;
      case LK_GEMM_SIMT:
        e = launch_gemm_simt(base + ln.a_off[0], base + ln.b_off[0], base + ln.c_off, ln.M, ln.N, ln.K, ln.op_f64 != 0,
                             s);
        break;
      case LK_GEMM_TC:
        e = tc_gemm_run(tc->prep[li], s);
        break;
      default:
        e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "contraction launch");
  }
  {
    ProfScope ps(c, s, 6, 0, 0);
    e = launch_final(reinterpret_cast<const FinalDev*>(base + P.off_final), P.final_nchunks, P.final_blocks, arena,
                     scalars, reinterpret_cast<double*>(base + P.off_traces),
                     reinterpret_cast<double*>(base + P.off_open_partial), reinterpret_cast<double*>(base + P.off_result),
                     s);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "final reduction");
  return AJF_OK;
}

ajf_status run_program(ajf_ctx* c) {
  Range nvtx_range("ajf run program");
  if (c->opts.use_graph && !c->profiling) {
    if (!c->graph) {
      cudaGraph_t g = nullptr;
      CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      ajf_status st = enqueue_program(c, c->stream);
      cudaError_t e = cudaStreamEndCapture(c->stream, &g);
      if (st != AJF_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&c->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    CUDA_TRY(c, cudaGraphLaunch(c->graph, c->stream));
    return AJF_OK;
  }
  return enqueue_program(c, c->stream);
}

ajf_status do_upload(ajf_ctx* c) {
  Range nvtx_range("ajf upload");
  if (!c->planned) return fail(c, AJF_E_STATE, "ajf_upload: no plan");
  ajf_status st = ensure_arena(c);
  if (st != AJF_OK) return st;
  const Program& P = c->prog;
  const size_t total = c->desc_image.size() + P.input_bytes;
  st = ensure_pinned(c, std::max<size_t>(total, 64));
  if (st != AJF_OK) return st;
  // the pinned image is filled before any copy is enqueued; wait for earlier copies to finish
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  std::memcpy(c->pinned, c->desc_image.data(), c->desc_image.size());
  std::memcpy(c->pinned + c->desc_image.size(), c->in.packed.data(), P.input_bytes);
  CUDA_TRY(c, cudaMemcpyAsync(c->arena + P.off_desc, c->pinned, c->desc_image.size(), cudaMemcpyHostToDevice,
                              c->stream));
  if (P.input_bytes)
    CUDA_TRY(c, cudaMemcpyAsync(c->arena + P.off_inputs, c->pinned + c->desc_image.size(), P.input_bytes,
                                cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->arena + P.off_status, 0, 16 * sizeof(int32_t), c->stream));
  c->uploaded = true;
  return AJF_OK;
}

ajf_status check_status_words(ajf_ctx* c) {
  int status[4] = {0, 0, 0, 0};
  CUDA_TRY(c, cudaMemcpy(status, c->arena + c->prog.off_status, sizeof(status), cudaMemcpyDeviceToHost));
  if (status[0] != 0) {
    cudaMemsetAsync(c->arena + c->prog.off_status, 0, 16 * sizeof(int32_t), c->stream);
    return fail(c, AJF_E_TIMEOUT, "a bounded device-side wait expired (code " + std::to_string(status[0]) + ")");
  }
  return AJF_OK;
}

int64_t real_combinations(const ajf_ctx* c) {
  int64_t n = 1;
  for (auto& nz : c->noises) n *= nz.nk;
  return n;
}

bool is_sliced(const ajf_ctx* c) { return c->planned && !c->slice_noises.empty(); }
bool bond_sliced(const ajf_ctx* c) { return c->planned && !c->bond_labels.empty(); }
// plans that run the program more than once per evaluation (Kraus-index or bond slices)
bool multi_run(const ajf_ctx* c) { return is_sliced(c) || bond_sliced(c); }

// Sliced Alg. I (the remark after Alg. I on stopping early): one run of the program per
// combination of the fixed Kraus indices, heaviest first; each run's sum |t|^2 is added in FP64
// and its traces are scattered into the full, lexicographically ordered trace array.
// Runs up to max_slices (<= 0: all) further slices from the context's progress (reset: from the
// first); stops early once the partial F exceeds 1 - eps (eps >= 0).
ajf_status run_slices(ajf_ctx* c, double eps, int64_t max_slices, bool reset, ajf_result* out) {
  Range nvtx_range("ajf Alg. I Kraus slices");
  const Program& P = c->prog;
  const auto& nz = c->in.noises;
  const int m = static_cast<int>(nz.size());
  const int ns = static_cast<int>(c->slice_noises.size());
  std::vector<char> fixed(m, 0);
  for (int j : c->slice_noises) fixed[j] = 1;
  // weight of Kraus operator k of noise j: ||K||_F^2 / 2^a (these sum to 1 over k for a channel)
  auto weight = [&](int j, int k) {
    const int d = 1 << nz[j].arity;
    const double* K = c->in.packed.data() + 2 * (nz[j].kraus_off + static_cast<int64_t>(k) * d * d);
    double w = 0;
    for (int i = 0; i < 2 * d * d; ++i) w += K[i] * K[i];
    return w / d;
  };
  struct Slice {
    std::vector<int> k;
    double w;
  };
  std::vector<Slice> slices(1, Slice{std::vector<int>(ns, 0), 1.0});
  for (int i = 0; i < ns; ++i) {
    std::vector<Slice> next;
    const int j = c->slice_noises[i];
    for (auto& sl : slices)
      for (int k = 0; k < nz[j].nk; ++k) {
        Slice t = sl;
        t.k[i] = k;
        t.w *= weight(j, k);
        next.push_back(t);
      }
    slices.swap(next);
  }
  std::stable_sort(slices.begin(), slices.end(), [](const Slice& a, const Slice& b) { return a.w > b.w; });
  // trace layout: full index = lexicographic over all noises (last fastest); the program's padded
  // index holds the open (unfixed) noises' Kraus indices, the last-added noise in the lowest bits
  std::vector<int64_t> radix(m, 1);
  for (int j = m - 2; j >= 0; --j) radix[j] = radix[j + 1] * nz[j + 1].nk;
  std::vector<int> shift(m, 0);
  for (int j = m - 1, acc = 0; j >= 0; --j) {
    shift[j] = acc;
    if (!fixed[j]) acc += nz[j].kbits;
  }
  const int64_t total = real_combinations(c);
  int64_t per_slice = 1;
  for (int j = 0; j < m; ++j)
    if (!fixed[j]) per_slice *= nz[j].nk;
  if (reset) {
    c->slice_next = 0;
    c->slice_done = 0;
    c->slice_S = 0;
    c->slice_traces_valid = true;
    c->slice_traces.assign(2 * static_cast<size_t>(total), 0.0);
  }
  std::vector<double> padded(2 * static_cast<size_t>(P.n_traces));
  const size_t leaves_at = P.off_leaves - P.off_desc;
  const int nsq = 2 * c->n;
  const int64_t n_slices = static_cast<int64_t>(slices.size());
  for (int64_t ran = 0; c->slice_next < n_slices && (max_slices <= 0 || ran < max_slices); ++ran) {
    if (eps >= 0 && std::ldexp(c->slice_S, -nsq) > 1.0 - eps) break;  // already decided
    const Slice& sl = slices[c->slice_next];
    for (int i = 0; i < ns; ++i) {
      const int j = c->slice_noises[i];
      const int d = 1 << nz[j].arity;
      const int64_t src = nz[j].kraus_off + static_cast<int64_t>(sl.k[i]) * d * d;
      std::memcpy(c->desc_image.data() + leaves_at + c->slice_leaves[i] * sizeof(LeafDev) + offsetof(LeafDev, src),
                  &src, sizeof(src));
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->arena + P.off_leaves, c->desc_image.data() + leaves_at,
                                P.leaves.size() * sizeof(LeafDev), cudaMemcpyHostToDevice, c->stream));
    ajf_status st = run_program(c);
    if (st != AJF_OK) return st;
    double res[3];
    CUDA_TRY(c, cudaMemcpyAsync(res, c->arena + P.off_result, sizeof(res), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(padded.data(), c->arena + P.off_traces, padded.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    st = check_status_words(c);
    if (st != AJF_OK) return st;
    c->slice_S += res[0];
    // scatter: odometer over the open noises' Kraus indices
    std::vector<int> digit(m, 0);
    for (int i = 0; i < ns; ++i) digit[c->slice_noises[i]] = sl.k[i];
    for (int64_t t = 0; t < per_slice; ++t) {
      int64_t idx = 0, pidx = 0;
      for (int j = 0; j < m; ++j) {
        idx += digit[j] * radix[j];
        if (!fixed[j]) pidx |= int64_t(digit[j]) << shift[j];
      }
      c->slice_traces[2 * idx] = padded[2 * pidx];
      c->slice_traces[2 * idx + 1] = padded[2 * pidx + 1];
      for (int j = m - 1; j >= 0; --j) {
        if (fixed[j]) continue;
        if (++digit[j] < nz[j].nk) break;
        digit[j] = 0;
      }
    }
    c->slice_done += per_slice;
    c->slice_next++;
  }
  const double S = c->slice_S;
  const bool all = c->slice_next == n_slices;
  out->S = S;
  out->F = std::ldexp(S, -nsq);
  out->one_minus_F = std::ldexp(std::ldexp(1.0, nsq) - S, -nsq);
  out->traces_done = c->slice_done;
  // decided "yes" by any partial sum above 1 - eps; "no" only once every slice is in
  out->equivalent = eps < 0 ? -1 : (out->F > 1.0 - eps ? 1 : (all ? 0 : -1));
  out->reserved = 0;
  c->have_alg1 = all && c->slice_traces_valid;
  return AJF_OK;
}

ajf_status fidelity_sliced(ajf_ctx* c, double eps, ajf_result* out) { return run_slices(c, eps, 0, true, out); }

// Bond-sliced plan: one run of the program per assignment of the sliced labels, the leaves that
// carry them taking the assignment's bits (fix_val; only the leaf descriptors change between
// runs, which also holds under CUDA-graph replay). Alg. II adds the runs' real scalars, Alg. I
// the runs' complex traces before |t|^2 is formed: both are linear in the runs, F is not.
// Bond-sliced runs: each run's leaf descriptors are staged in a pinned slot and its result (and
// Alg. I traces) read back into the same slot asynchronously, so runs are enqueued back to back
// with one synchronisation per chunk of runs.
struct BondLayout {
  size_t lb = 0, tr_bytes = 0, per_run = 0;
  int64_t chunk = 1;
};

BondLayout bond_layout(const ajf_ctx* c, int alg, int64_t count) {
  auto a16 = [](size_t x) { return (x + 15) / 16 * 16; };
  BondLayout L;
  L.lb = c->bond_leaves.empty() ? 0 : a16(c->prog.leaves.size() * sizeof(LeafDev));
  L.tr_bytes = alg == 1 ? 2 * static_cast<size_t>(c->prog.n_traces) * sizeof(double) : 0;
  L.per_run = L.lb + 32 + a16(L.tr_bytes);
  L.chunk = std::max<int64_t>(1, std::min<int64_t>(count, static_cast<int64_t>((size_t(256) << 20) / L.per_run)));
  return L;
}

// Stage and enqueue runs [v0, v0 + n) (n <= L.chunk) into pinned slots 0..n-1.
ajf_status enqueue_bond_runs(ajf_ctx* c, int alg, int64_t v0, int64_t n, const BondLayout& L) {
  const Program& P = c->prog;
  const size_t leaves_at = P.off_leaves - P.off_desc;
  const size_t leaves_bytes = P.leaves.size() * sizeof(LeafDev);
  for (int64_t r = 0; r < n; ++r) {
    char* slot = c->pinned + static_cast<size_t>(r) * L.per_run;
    const int64_t v = v0 + r;
    if (L.lb) {
      for (auto& bl : c->bond_leaves) {
        uint16_t val = 0;
        for (auto& pb : bl.bits)
          if ((v >> pb.second) & 1) val = static_cast<uint16_t>(val | (1u << pb.first));
        std::memcpy(c->desc_image.data() + leaves_at + bl.leaf * sizeof(LeafDev) + offsetof(LeafDev, fix_val), &val,
                    sizeof(val));
      }
      std::memcpy(slot, c->desc_image.data() + leaves_at, leaves_bytes);
      CUDA_TRY(c, cudaMemcpyAsync(c->arena + P.off_leaves, slot, leaves_bytes, cudaMemcpyHostToDevice, c->stream));
    }
    ajf_status st = run_program(c);
    if (st != AJF_OK) return st;
    CUDA_TRY(c, cudaMemcpyAsync(slot + L.lb, c->arena + P.off_result, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
    if (alg == 1)
      CUDA_TRY(c, cudaMemcpyAsync(slot + L.lb + 32, c->arena + P.off_traces, L.tr_bytes, cudaMemcpyDeviceToHost,
                                  c->stream));
  }
  return AJF_OK;
}

// After the stream has drained: add the n slots' results in run order (Alg. II: Neumaier sum of
// the scalars into S/comp; Alg. I: traces into bond_traces).
void collect_bond_runs(ajf_ctx* c, int alg, int64_t n, const BondLayout& L, double& S, double& comp) {
  for (int64_t r = 0; r < n; ++r) {
    const char* slot = c->pinned + static_cast<size_t>(r) * L.per_run;
    if (alg == 2) {
      double x;
      std::memcpy(&x, slot + L.lb, sizeof(x));
      const double t = S + x;
      comp += std::fabs(S) >= std::fabs(x) ? (S - t) + x : (x - t) + S;
      S = t;
    } else {
      const double* tr = reinterpret_cast<const double*>(slot + L.lb + 32);
      for (size_t i = 0; i < c->bond_traces.size(); ++i) c->bond_traces[i] += tr[i];
    }
  }
}

// run_bonds runs assignments [first, first + count) (a plan without bond slicing has the one
// assignment 0): Alg. II returns the Neumaier-compensated FP64 sum of the runs' scalars in
// *S_out, Alg. I adds the runs' traces to bond_traces (padded order) in run order.
ajf_status run_bonds(ajf_ctx* c, int alg, int64_t first, int64_t count, double* S_out) {
  const BondLayout L = bond_layout(c, alg, count);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // the staging buffer may still feed an upload
  ajf_status st = ensure_pinned(c, L.per_run * static_cast<size_t>(L.chunk));
  if (st != AJF_OK) return st;
  double S = 0, comp = 0;
  for (int64_t v0 = first; v0 < first + count; v0 += L.chunk) {
    const int64_t n = std::min(L.chunk, first + count - v0);
    st = enqueue_bond_runs(c, alg, v0, n, L);
    if (st != AJF_OK) return st;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    st = check_status_words(c);
    if (st != AJF_OK) return st;
    collect_bond_runs(c, alg, n, L, S, comp);
  }
  if (S_out) *S_out = S + comp;
  return AJF_OK;
}

// The result of a whole bond-sliced evaluation: S from the Alg. II sum, or from the summed
// Alg. I traces (|t|^2 is formed only after the sum over slices).
void finish_bonds(ajf_ctx* c, int alg, double S, double eps, ajf_result* out) {
  if (alg == 1) {
    double comp = 0;
    S = 0;
    for (size_t i = 0; i < c->bond_traces.size(); i += 2) {
      const double x = c->bond_traces[i] * c->bond_traces[i] + c->bond_traces[i + 1] * c->bond_traces[i + 1];
      const double t = S + x;
      comp += S >= x ? (S - t) + x : (x - t) + S;
      S = t;
    }
    S += comp;
  }
  const int nsq = 2 * c->n;
  out->S = S;
  out->F = std::ldexp(S, -nsq);
  out->one_minus_F = std::ldexp(std::ldexp(1.0, nsq) - S, -nsq);
  out->traces_done = alg == 1 ? real_combinations(c) : 0;
  out->equivalent = eps < 0 ? -1 : (out->F > 1.0 - eps ? 1 : 0);
  out->reserved = 0;
  if (alg == 1) c->have_alg1 = true;
}

ajf_status fidelity_bonds(ajf_ctx* c, int alg, double eps, ajf_result* out) {
  Range nvtx_range("ajf bond slices");
  const int nb = static_cast<int>(c->bond_labels.size());
  if (alg == 1) c->bond_traces.assign(2 * static_cast<size_t>(c->prog.n_traces), 0.0);
  double S = 0;
  ajf_status st = run_bonds(c, alg, 0, int64_t(1) << nb, &S);
  if (st != AJF_OK) return st;
  finish_bonds(c, alg, S, eps, out);
  return AJF_OK;
}

int64_t slice_count(const ajf_ctx* c) {
  int64_t n = 1;
  for (int j : c->slice_noises) n *= c->in.noises[j].nk;
  return n;
}

// Signature of a sliced plan and its input values (FNV-1a over the plan key and the packed
// matrices): a checkpoint resumes only where the same slices would sum the same traces.
uint64_t slice_signature(const ajf_ctx* c) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  mix(c->prog_key.data(), c->prog_key.size() * sizeof(int64_t));
  mix(c->in.packed.data(), c->in.packed.size() * sizeof(double));
  return h;
}

ajf_status fidelity(ajf_ctx* c, int alg, double eps, ajf_result* out) {
  Range nvtx_range("ajf fidelity");
  if (!c) return AJF_E_ARG;
  if (!out) return fail(c, AJF_E_ARG, "out is NULL");
  if (!c->planned || c->alg != alg) return fail(c, AJF_E_STATE, "no Alg. " + std::to_string(alg) + " plan");
  if (c->device < 0) return fail(c, AJF_E_STATE, "host-only context (device -1) cannot run the contraction");
  if (eps > 1.0) return fail(c, AJF_E_ARG, "eps > 1");
  CUDA_TRY(c, cudaSetDevice(c->device));
  if (!c->uploaded) {
    ajf_status st = do_upload(c);
    if (st != AJF_OK) return st;
  }
  if (alg == 1 && is_sliced(c)) return fidelity_sliced(c, eps, out);
  if (bond_sliced(c)) return fidelity_bonds(c, alg, eps, out);
  ajf_status st = run_program(c);
  if (st != AJF_OK) return st;
  double res[3];
  CUDA_TRY(c, cudaMemcpyAsync(res, c->arena + c->prog.off_result, sizeof(res), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  st = check_status_words(c);
  if (st != AJF_OK) return st;
  out->S = res[0];
  out->F = res[1];
  out->one_minus_F = res[2];
  out->traces_done = alg == 1 ? real_combinations(c) : 0;
  out->equivalent = eps < 0 ? -1 : (out->F > 1.0 - eps ? 1 : 0);
  out->reserved = 0;
  if (alg == 1) c->have_alg1 = true;
  return AJF_OK;
}

}  // namespace

extern "C" {

const char* ajf_version(void) { return "ajf 0.1 sm_103a"; }

ajf_status ajf_create(ajf_ctx** out, int device, void* cuda_stream) {
  if (!out) return AJF_E_ARG;
  *out = nullptr;
  auto c = std::make_unique<ajf_ctx>();
  c->device = device;
  if (device < 0) {  // host-only context: validation and planning, no device work
    c->tc_device = true;
    *out = c.release();
    return AJF_OK;
  }
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return AJF_E_CUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return AJF_E_CUDA;
  c->tc_device = prop.major >= 10;
  if (set_kernel_smem_limits() != cudaSuccess) return AJF_E_CUDA;
  // The fixed arena of ajf_fidelity_noalloc: its module is loaded (and the array reserved) here,
  // at set-up, so that the no-allocation call itself never triggers the reservation. Looked up
  // for every context, so a context created after a device reset sees the current address.
  {
    void* sa = nullptr;
    if (static_arena_address(device, &sa) != cudaSuccess) {
      cudaGetLastError();
      return AJF_E_CUDA;
    }
    c->static_arena = static_cast<char*>(sa);
  }
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return AJF_E_CUDA;
    c->own_stream = true;
  }
  *out = c.release();
  return AJF_OK;
}

void ajf_destroy(ajf_ctx* c) {
  if (!c) return;
  if (c->device < 0) {
    delete c;
    return;
  }
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  drain_profile(c);
  for (auto e : c->event_pool) cudaEventDestroy(e);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->own_arena && c->arena && !c->user_ws) cudaFree(c->arena);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->pers_dev) cudaFree(c->pers_dev);
  if (c->q_graph) cudaGraphExecDestroy(c->q_graph);
  if (c->q_dev) cudaFree(c->q_dev);
  if (c->sync_ev) cudaEventDestroy(c->sync_ev);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* ajf_last_error(const ajf_ctx* c) { return c ? c->err.c_str() : "null context"; }

ajf_status ajf_load_circuit(ajf_ctx* c, int role, int n_qubits, int n_gates, const int32_t* arity,
                            const int32_t* qubits, const double* mats) {
  if (!c) return AJF_E_ARG;
  if (role != AJF_IDEAL && role != AJF_IMPL) return fail(c, AJF_E_ARG, "role must be AJF_IDEAL or AJF_IMPL");
  if (n_qubits < 1 || n_qubits > 62) return fail(c, AJF_E_ARG, "n_qubits must be in [1, 62]");
  if (n_gates < 0) return fail(c, AJF_E_ARG, "n_gates < 0");
  if (n_gates > 0 && (!arity || !qubits || !mats)) return fail(c, AJF_E_ARG, "NULL array");
  if (role == AJF_IMPL && (!c->has_ideal || n_qubits != c->n))
    return fail(c, AJF_E_ARG, "AJF_IMPL needs a loaded AJF_IDEAL circuit on the same qubits");
  std::vector<GateData> gates;
  gates.reserve(n_gates);
  size_t qi = 0, mi = 0;
  for (int g = 0; g < n_gates; ++g) {
    GateData gd;
    gd.arity = arity[g];
    if (gd.arity < 1 || gd.arity > 3) return fail(c, AJF_E_ARG, "gate " + std::to_string(g) + ": arity not in {1,2,3}");
    for (int i = 0; i < 3; ++i) gd.q[i] = 0;
    for (int i = 0; i < gd.arity; ++i) {
      const int q = qubits[qi + i];
      if (q < 0 || q >= n_qubits) return fail(c, AJF_E_ARG, "gate " + std::to_string(g) + ": qubit out of range");
      for (int j = 0; j < i; ++j)
        if (gd.q[j] == q) return fail(c, AJF_E_ARG, "gate " + std::to_string(g) + ": repeated qubit");
      gd.q[i] = q;
    }
    qi += gd.arity;
    const int dim = 1 << gd.arity;
    gd.mat.assign(mats + mi, mats + mi + 2 * dim * dim);
    mi += 2 * dim * dim;
    const double err = unitarity_error(gd.mat.data(), dim);
    if (!(err <= 1e-10))
      return fail(c, AJF_E_NOT_UNITARY, "gate " + std::to_string(g) + " is not unitary (||G^+G-I||_F = " +
                                            std::to_string(err) + ")");
    gates.push_back(std::move(gd));
  }
  if (role == AJF_IDEAL) {
    c->n = n_qubits;
    c->ideal = std::move(gates);
    c->has_ideal = true;
    c->impl.clear();
    c->has_impl = false;
    c->noises.clear();
  } else {
    c->impl = std::move(gates);
    c->has_impl = true;
  }
  invalidate(c);
  c->err.clear();
  return AJF_OK;
}

ajf_status ajf_add_noise(ajf_ctx* c, int32_t after_gate, int32_t arity, const int32_t* qubits, int32_t n_kraus,
                         const double* kraus) {
  if (!c) return AJF_E_ARG;
  if (!c->has_ideal) return fail(c, AJF_E_STATE, "ajf_add_noise before ajf_load_circuit");
  const int nsk = static_cast<int>(c->has_impl ? c->impl.size() : c->ideal.size());
  if (after_gate < -1 || after_gate >= nsk) return fail(c, AJF_E_ARG, "after_gate out of range");
  if (arity < 1 || arity > 3) return fail(c, AJF_E_ARG, "noise arity not in {1,2,3}");
  if (n_kraus < 1 || n_kraus > 256) return fail(c, AJF_E_ARG, "n_kraus not in [1, 256]");
  if (!qubits || !kraus) return fail(c, AJF_E_ARG, "NULL array");
  NoiseData nd;
  nd.after = after_gate;
  nd.arity = arity;
  nd.nk = n_kraus;
  for (int i = 0; i < 3; ++i) nd.q[i] = 0;
  for (int i = 0; i < arity; ++i) {
    if (qubits[i] < 0 || qubits[i] >= c->n) return fail(c, AJF_E_ARG, "noise qubit out of range");
    for (int j = 0; j < i; ++j)
      if (nd.q[j] == qubits[i]) return fail(c, AJF_E_ARG, "noise: repeated qubit");
    nd.q[i] = qubits[i];
  }
  const int dim = 1 << arity;
  nd.kraus.assign(kraus, kraus + 2 * size_t(n_kraus) * dim * dim);
  const double err = tp_error(nd.kraus.data(), n_kraus, dim);
  if (!(err <= 1e-10))
    return fail(c, AJF_E_NOT_TP, "Kraus set is not trace preserving (||sum K^+K - I||_F = " + std::to_string(err) + ")");
  c->noises.push_back(std::move(nd));
  invalidate(c);
  c->err.clear();
  return AJF_OK;
}

ajf_status ajf_clear_noise(ajf_ctx* c) {
  if (!c) return AJF_E_ARG;
  c->noises.clear();
  invalidate(c);
  return AJF_OK;
}

namespace {

ajf_status plan_one(ajf_ctx* c, int alg, const ajf_plan_opts* opts, ajf_plan_info* info) {
  Range nvtx_range("ajf plan");
  if (!c) return AJF_E_ARG;
  if (!c->has_ideal) return fail(c, AJF_E_STATE, "ajf_plan before ajf_load_circuit");
  if (alg != 1 && alg != 2) return fail(c, AJF_E_ARG, "alg must be 0, 1 or 2");
  ajf_plan_opts o{};
  o.planner = AJF_PLANNER_AUTO;
  o.precision = AJF_PREC_F64;
  o.trials = 32;
  if (opts) o = *opts;
  if (o.trials <= 0) o.trials = 32;
  if (o.planner < AJF_PLANNER_AUTO || o.planner > AJF_PLANNER_LEARNED) return fail(c, AJF_E_ARG, "bad planner");
  if (o.precision < AJF_PREC_F64 || o.precision > AJF_PREC_F16X3) return fail(c, AJF_E_ARG, "bad precision");
  for (int i = 0; i < 4; ++i)
    if (o.reserved[i] != 0) return fail(c, AJF_E_ARG, "reserved fields must be zero");
  if (o.slice_bonds < AJF_SLICE_AUTO || o.slice_bonds > AJF_MAX_SLICE_BONDS)
    return fail(c, AJF_E_ARG, "slice_bonds must be AJF_SLICE_AUTO or between 0 and AJF_MAX_SLICE_BONDS");
  if (o.slice_bonds != 0 && o.alg1_slices > 0)
    return fail(c, AJF_E_ARG, "slice_bonds and alg1_slices cannot be combined");
  if (o.slice_bonds != 0 && o.lowering == AJF_LOWER_PERSISTENT)
    return fail(c, AJF_E_ARG, "a bond-sliced plan cannot use the persistent lowering");
  if (o.alg1_slices < 0 || o.alg1_slices > static_cast<int>(c->noises.size()))
    return fail(c, AJF_E_ARG, "alg1_slices must be between 0 and the number of noises");
  if (o.alg1_slices > 0 && alg != 1) return fail(c, AJF_E_ARG, "alg1_slices applies to Alg. I only");
  if (o.alg1_slices > 0 && o.lowering == AJF_LOWER_PERSISTENT)
    return fail(c, AJF_E_ARG, "a sliced Alg. I plan cannot use the persistent lowering");
  if (o.simplify & ~(AJF_SIMPLIFY_SWAP | AJF_SIMPLIFY_CANCEL)) return fail(c, AJF_E_ARG, "unknown simplify flags");
  if (o.lowering != AJF_LOWER_DEFAULT && o.lowering != AJF_LOWER_PERSISTENT) return fail(c, AJF_E_ARG, "bad lowering");
  if (o.lowering == AJF_LOWER_PERSISTENT && o.precision != AJF_PREC_F64)
    return fail(c, AJF_E_ARG, "the persistent lowering computes in FP64: precision must be AJF_PREC_F64");
  const int nsk = static_cast<int>(c->has_impl ? c->impl.size() : c->ideal.size());
  for (auto& nz : c->noises)
    if (nz.after >= nsk) return fail(c, AJF_E_ARG, "a noise is placed after a gate the skeleton does not have");
  if (c->device >= 0) CUDA_TRY(c, cudaSetDevice(c->device));
  if (o.precision >= AJF_PREC_TF32 && !c->tc_device)
    return fail(c, AJF_E_UNSUPPORTED, "tensor-core precision modes need tcgen05 (sm_100 or newer)");
  invalidate(c);
  const auto t0 = std::chrono::steady_clock::now();
  pack_inputs(c);
  // sliced noises: the alg1_slices noises with the most Kraus operators (earlier first on ties)
  std::vector<int> slice_noises;
  std::vector<char> sliced(c->in.noises.size(), 0);
  if (o.alg1_slices > 0) {
    std::vector<int> order(c->in.noises.size());
    for (size_t j = 0; j < order.size(); ++j) order[j] = static_cast<int>(j);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return c->in.noises[x].nk > c->in.noises[y].nk; });
    slice_noises.assign(order.begin(), order.begin() + o.alg1_slices);
    std::sort(slice_noises.begin(), slice_noises.end());
    for (int j : slice_noises) sliced[j] = 1;
  }
  if (alg == 1) {
    int open_bits = 0;
    for (size_t j = 0; j < c->in.noises.size(); ++j)
      if (!sliced[j]) open_bits += c->in.noises[j].kbits;
    if (open_bits > 40)
      return fail(c, AJF_E_BUDGET, "Alg. I result tensor would hold 2^" + std::to_string(open_bits) +
                                       " traces (more than 2^40); use Alg. II or slice more noises");
  }
  std::vector<int64_t> key = {alg, c->n, c->has_impl, o.planner, o.precision, o.trials, static_cast<int64_t>(o.seed),
                              c->mlp_version};
  auto key_gates = [&](const std::vector<GateData>& gs) {
    key.push_back(static_cast<int64_t>(gs.size()));
    for (auto& g : gs) key.insert(key.end(), {g.arity, g.q[0], g.q[1], g.q[2]});
  };
  key_gates(c->ideal);
  if (c->has_impl) key_gates(c->impl);
  for (auto& nz : c->noises) key.insert(key.end(), {nz.after, nz.arity, nz.q[0], nz.q[1], nz.q[2], nz.nk});
  // a simplified sequence depends on the matrices: it becomes part of the structure
  const Sequence seq = compose_sequence(c->in, o.simplify);
  key.push_back(o.simplify);
  key.push_back(o.alg1_slices);
  key.insert(key.end(), slice_noises.begin(), slice_noises.end());
  if (o.simplify) {
    key.push_back(static_cast<int64_t>(seq.ops.size()));
    for (auto& op : seq.ops) key.insert(key.end(), {op.kind, op.index, op.w[0], op.w[1], op.w[2]});
    key.insert(key.end(), seq.closure.begin(), seq.closure.end());
  }
  double budget = o.mem_budget_bytes;
  if (budget <= 0 && c->device < 0) budget = 1e18;
  if (budget <= 0) {
    size_t fr = 0, tot = 0;
    CUDA_TRY(c, cudaMemGetInfo(&fr, &tot));
    budget = 0.6 * static_cast<double>(fr) + (c->own_arena ? static_cast<double>(c->arena_cap) : 0.0);
  }
  // the lowered program depends on the structure, the precision, the lowering, the device and
  // the slicing (under AJF_SLICE_AUTO also the budget it was sized for)
  std::vector<int64_t> pkey = key;
  pkey.push_back(o.lowering);
  pkey.push_back(c->tc_device ? 1 : 0);
  pkey.push_back(o.slice_bonds);
  if (o.slice_bonds == AJF_SLICE_AUTO) pkey.push_back(static_cast<int64_t>(budget));
  const bool prog_hit = c->prog_valid && pkey == c->prog_key;
  bool cached = prog_hit;
  if (!prog_hit) {
    drop_graph(c);
    c->prog_valid = false;
    cached = c->path_valid && key == c->plan_key;
    const Network full = (alg == 1) ? build_alg1(c->in, seq, sliced) : build_alg2(c->in, seq);
    c->net = full;
    PlanParams pp;
    pp.planner = o.planner;
    pp.precision = o.precision;
    pp.trials = o.trials;
    pp.seed = o.seed;
    pp.elem_bytes = o.precision == AJF_PREC_F64 ? 16 : 8;
    pp.tensor_cores = c->tc_device;
    switch (o.precision) {
      case AJF_PREC_F64: pp.peak_flops = 1.0e12; break;
      case AJF_PREC_F32: pp.peak_flops = 40e12; break;
      case AJF_PREC_TF32: pp.peak_flops = 500e12; break;
      case AJF_PREC_BF16X3: pp.peak_flops = 400e12; break;
      default: pp.peak_flops = 200e12; break;
    }
    cudaError_t score_err = cudaSuccess;
    if (o.planner == AJF_PLANNER_LEARNED && static_cast<int>(c->mlp_weights.size()) == kMlpParams) {
      pp.mlp = c->mlp_weights.data();
      if (c->device >= 0) {
        pp.scorer = [c, &score_err](const float* w, const float* x, int n, float* out) {
          const cudaError_t e = c->mlp_scorer.score(w, x, n, out);
          if (e != cudaSuccess) {
            score_err = e;
            for (int i = 0; i < n; ++i) out[i] = 0.0f;
          }
        };
      } else {
        pp.scorer = [](const float* w, const float* x, int n, float* out) {
          for (int i = 0; i < n; ++i) out[i] = mlp_score_host(w, x + static_cast<size_t>(i) * kMlpFeatures);
        };
      }
    }
    try {
      if (!cached) {
        c->path_valid = false;
        // process-wide cache: every context planning the same structure with the same options
        // gets the same path (the planners are deterministic given their seed); learned plans
        // depend on the context's model and are not shared
        const bool shared = o.planner != AJF_PLANNER_LEARNED;
        if (!shared || !shared_path_lookup(key, &c->path_full)) {
          c->path_full = plan_path(full, pp);
          if (shared) shared_path_store(key, c->path_full);
        }
        c->plan_key = key;
        c->path_valid = true;
      }
      // bond slicing: `count` labels of the full path; under AJF_SLICE_AUTO one more at a time
      // until the lowered arena fits the budget (starting where the widest tensor is addressable)
      auto apply_slices = [&](int count) {
        c->bond_labels = count > 0 ? choose_slice_labels(full, c->path_full, count) : std::vector<int>{};
        if (c->bond_labels.empty()) {
          c->net = full;
          c->path = c->path_full;
        } else {
          c->net = slice_network(full, c->bond_labels);
          c->path = restrict_path(c->net, c->path_full, c->bond_labels, pp);
        }
      };
      bool lowered = false;
      if (score_err == cudaSuccess) {
        int count = o.slice_bonds > 0 ? o.slice_bonds : 0;
        if (o.slice_bonds == AJF_SLICE_AUTO) count = std::max(0, c->path_full.width - (kMaxBits - 2));
        for (;;) {
          apply_slices(std::min(count, static_cast<int>(AJF_MAX_SLICE_BONDS)));
          lowered = c->path.width <= kMaxBits - 2;
          if (lowered)
            c->prog = lower(c->net, c->path, o.precision, c->in.packed.size() / 2, c->tc_device,
                            o.lowering == AJF_LOWER_PERSISTENT);
          if (o.slice_bonds != AJF_SLICE_AUTO) break;
          if (lowered && static_cast<double>(c->prog.arena_bytes) <= budget) break;
          if (count >= AJF_MAX_SLICE_BONDS || static_cast<int>(c->bond_labels.size()) < count) break;
          ++count;
        }
      }
      c->bond_leaves.clear();
      for (size_t l = 0; l < full.leaf_labels.size(); ++l) {
        ajf_ctx::BondLeaf bl{static_cast<int>(l), {}};
        for (size_t p = 0; p < full.leaf_labels[l].size(); ++p)
          for (size_t j = 0; j < c->bond_labels.size(); ++j)
            if (full.leaf_labels[l][p] == c->bond_labels[j]) bl.bits.emplace_back(static_cast<int>(p), static_cast<int>(j));
        if (!bl.bits.empty()) c->bond_leaves.push_back(bl);
      }
      if (score_err == cudaSuccess && !lowered) {
        // too wide to address: report the path's cost and width with the budget error
        ajf_plan_info pi{};
        pi.cmacs = c->path.cmacs;
        pi.flops = 8.0 * c->path.cmacs;
        pi.width = c->path.width;
        pi.n_steps = static_cast<int32_t>(c->path.steps.size());
        pi.n_leaves = static_cast<int32_t>(c->net.leaf_labels.size());
        pi.n_open_bits = static_cast<int32_t>(c->net.open_labels.size());
        pi.planner_used = c->path.planner;
        pi.arena_bytes = std::ldexp(1.0, c->path.width) * pp.elem_bytes;
        pi.n_sliced_bonds = static_cast<int32_t>(c->bond_labels.size());
        pi.cmacs = std::ldexp(pi.cmacs, pi.n_sliced_bonds);
        pi.flops = std::ldexp(pi.flops, pi.n_sliced_bonds);
        pi.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        c->info = pi;
        if (info) *info = pi;
        return fail(c, AJF_E_BUDGET, "planned width 2^" + std::to_string(c->path.width) +
                                         " elements is beyond what one device can hold");
      }
    } catch (const std::exception& ex) {
      return fail(c, AJF_E_BUDGET, std::string("planning failed: ") + ex.what());
    }
    if (score_err != cudaSuccess) {
      c->path_valid = false;
      return cuda_fail(c, score_err, "learned merge scorer");
    }
    c->prog_key = pkey;
    c->prog_valid = true;
    c->prog_gen++;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  // descriptor image
  const Program& P = c->prog;
  c->desc_image.assign(P.desc_bytes, 0);
  if (!P.leaves.empty())
    std::memcpy(c->desc_image.data() + (P.off_leaves - P.off_desc), P.leaves.data(), P.leaves.size() * sizeof(LeafDev));
  if (!P.steps.empty())
    std::memcpy(c->desc_image.data() + (P.off_steps - P.off_desc), P.steps.data(), P.steps.size() * sizeof(StepDev));
  if (!P.perms.empty())
    std::memcpy(c->desc_image.data() + (P.off_perms - P.off_desc), P.perms.data(), P.perms.size() * sizeof(PermDev));
  std::memcpy(c->desc_image.data() + (P.off_final - P.off_desc), &P.fin, sizeof(FinalDev));
  ajf_plan_info pi{};
  const int nb = static_cast<int>(c->bond_labels.size());
  pi.cmacs = std::ldexp(c->path.cmacs, nb);
  pi.flops = std::ldexp(P.flops, nb);
  pi.bytes = std::ldexp(P.bytes, nb);
  pi.gemm_flops = std::ldexp(P.gemm_flops, nb);
  pi.gemm_bytes = std::ldexp(P.gemm_bytes, nb);
  pi.n_sliced_bonds = nb;
  pi.arena_bytes = static_cast<double>(P.arena_bytes);
  pi.plan_seconds = secs;
  pi.width = c->path.width;
  pi.n_steps = static_cast<int32_t>(c->path.steps.size());
  pi.n_gemm_steps = P.n_gemm;
  pi.n_leaves = static_cast<int32_t>(c->net.leaf_labels.size());
  pi.n_open_bits = static_cast<int32_t>(c->net.open_labels.size());
  pi.planner_used = c->path.planner;
  pi.n_launches = 3;  // leaves + final pass + final sum
  for (auto& ln : P.launches)
    pi.n_launches += (ln.kind == LK_SPLITK || ln.kind == LK_DOT || (ln.kind == LK_GEMM_TC && ln.ksplit > 1)) ? 2 : 1;
  pi.n_tc_gemms = P.tensor_cores;
  pi.plan_cached = cached ? 1 : 0;
  pi.n_removed = seq.removed;
  pi.upload_bytes = static_cast<double>(P.desc_bytes + P.input_bytes);
  c->info = pi;
  if (info) *info = pi;
  if (static_cast<double>(P.arena_bytes) > budget)
    return fail(c, AJF_E_BUDGET, "plan needs " + std::to_string(P.arena_bytes) + " bytes, budget " +
                                     std::to_string(static_cast<size_t>(budget)) + " (width " +
                                     std::to_string(c->path.width) + ", " + std::to_string(nb) +
                                     " sliced labels)");
  c->opts = o;
  c->alg = alg;
  c->slice_noises = slice_noises;
  c->slice_next = c->slice_done = 0;
  c->slice_S = 0;
  c->slice_traces_valid = true;
  c->slice_traces.clear();
  c->slice_leaves.clear();
  for (int j : slice_noises) c->slice_leaves.push_back(c->net.noise_leaf[j]);
  c->planned = true;
  c->plan_gen++;
  c->err.clear();
  return AJF_OK;
}

}  // namespace

ajf_status ajf_plan(ajf_ctx* c, int alg, const ajf_plan_opts* opts, ajf_plan_info* info) {
  if (!c) return AJF_E_ARG;
  if (alg != AJF_ALG_AUTO) return plan_one(c, alg, opts, info);
  // AJF_ALG_AUTO: the cheaper of the two by the planner's time model (a sliced Alg. I plan runs
  // once per slice). Alg. II is planned first; Alg. I only when its result tensor is addressable.
  ajf_plan_opts o2{};
  o2.planner = AJF_PLANNER_AUTO;
  o2.precision = AJF_PREC_F64;
  o2.trials = 32;
  if (opts) o2 = *opts;
  o2.alg1_slices = 0;
  ajf_plan_info i2{};
  ajf_status st = plan_one(c, 2, &o2, &i2);
  const bool have2 = st == AJF_OK;
  const double t2 = have2 ? std::ldexp(c->path.est_seconds, static_cast<int>(c->bond_labels.size())) : 0.0;
  if (st != AJF_OK && st != AJF_E_BUDGET) return st;
  ajf_plan_info i1{};
  const ajf_status st1 = plan_one(c, 1, opts, &i1);
  if (st1 == AJF_OK) {
    double slices = 1;
    for (int j : c->slice_noises) slices *= c->noises[j].nk;
    if (!have2 || std::ldexp(c->path.est_seconds, static_cast<int>(c->bond_labels.size())) * slices <= t2) {
      if (info) *info = i1;
      return AJF_OK;
    }
  } else if (!have2) {
    return st1;
  }
  st = plan_one(c, 2, &o2, &i2);  // Alg. II was cheaper: plan it again (its path is recomputed)
  if (info) *info = i2;
  return st;
}

ajf_status ajf_planned_alg(const ajf_ctx* c, int* alg) {
  if (!c || !alg) return AJF_E_ARG;
  if (!c->planned) return AJF_E_STATE;
  *alg = c->alg;
  return AJF_OK;
}

ajf_status ajf_set_workspace(ajf_ctx* c, void* dev_ptr, size_t bytes) {
  if (!c) return AJF_E_ARG;
  if (dev_ptr && (reinterpret_cast<uintptr_t>(dev_ptr) % 256) != 0)
    return fail(c, AJF_E_ARG, "workspace must be 256-byte aligned");
  if (c->own_arena && c->arena && !c->user_ws) {
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->arena);
    c->arena_cap = 0;
  }
  c->arena = nullptr;
  c->user_ws = dev_ptr;
  c->user_ws_bytes = dev_ptr ? bytes : 0;
  c->own_arena = dev_ptr == nullptr;
  c->uploaded = false;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return AJF_OK;
}

ajf_status ajf_workspace_size(const ajf_ctx* c, size_t* bytes) {
  if (!c || !bytes) return AJF_E_ARG;
  if (!c->planned) return AJF_E_STATE;
  *bytes = c->prog.arena_bytes;
  return AJF_OK;
}

ajf_status ajf_upload(ajf_ctx* c) {
  if (!c) return AJF_E_ARG;
  if (c->device < 0) return fail(c, AJF_E_STATE, "host-only context");
  CUDA_TRY(c, cudaSetDevice(c->device));
  return do_upload(c);
}

ajf_status ajf_fidelity_alg1(ajf_ctx* c, double eps, ajf_result* out) { return fidelity(c, 1, eps, out); }

ajf_status ajf_fidelity_alg2(ajf_ctx* c, double eps, ajf_result* out) { return fidelity(c, 2, eps, out); }

ajf_status ajf_alg1_continue(ajf_ctx* c, double eps, int64_t max_slices, ajf_result* out) {
  if (!c) return AJF_E_ARG;
  if (!out) return fail(c, AJF_E_ARG, "out is NULL");
  if (!c->planned || c->alg != 1 || !is_sliced(c)) return fail(c, AJF_E_STATE, "needs a sliced Alg. I plan");
  if (c->device < 0) return fail(c, AJF_E_STATE, "host-only context (device -1) cannot run the contraction");
  if (eps > 1.0) return fail(c, AJF_E_ARG, "eps > 1");
  CUDA_TRY(c, cudaSetDevice(c->device));
  if (!c->uploaded) {
    ajf_status st = do_upload(c);
    if (st != AJF_OK) return st;
  }
  const bool fresh = c->slice_next == 0 && c->slice_traces.empty();
  return run_slices(c, eps, max_slices, fresh, out);
}

ajf_status ajf_alg1_checkpoint(const ajf_ctx* c, ajf_alg1_state* st) {
  if (!c || !st) return AJF_E_ARG;
  if (!c->planned || c->alg != 1 || !is_sliced(c)) return AJF_E_STATE;
  st->next_slice = c->slice_next;
  st->n_slices = slice_count(c);
  st->S = c->slice_S;
  st->traces_done = c->slice_done;
  st->plan_sig = slice_signature(c);
  return AJF_OK;
}

ajf_status ajf_alg1_restore(ajf_ctx* c, const ajf_alg1_state* st) {
  if (!c) return AJF_E_ARG;
  if (!st) return fail(c, AJF_E_ARG, "state is NULL");
  if (!c->planned || c->alg != 1 || !is_sliced(c)) return fail(c, AJF_E_STATE, "needs a sliced Alg. I plan");
  const int64_t n = slice_count(c);
  if (st->plan_sig != slice_signature(c) || st->n_slices != n)
    return fail(c, AJF_E_ARG, "checkpoint is of another plan or other input values");
  if (st->next_slice < 0 || st->next_slice > n || !(st->S >= 0) || st->traces_done < 0)
    return fail(c, AJF_E_ARG, "checkpoint fields out of range");
  c->slice_next = st->next_slice;
  c->slice_S = st->S;
  c->slice_done = st->traces_done;
  c->slice_traces.assign(2 * static_cast<size_t>(real_combinations(c)), 0.0);
  c->slice_traces_valid = st->next_slice == 0;  // the traces of earlier slices are not in a checkpoint
  c->have_alg1 = false;
  return AJF_OK;
}

ajf_status ajf_check_plan(ajf_ctx* c) {
  if (!c) return AJF_E_ARG;
  if (!c->planned) return fail(c, AJF_E_STATE, "no plan");
  const std::string why = check_program(c->prog);
  if (!why.empty()) return fail(c, AJF_E_STATE, "plan check: " + why);
  c->err.clear();
  return AJF_OK;
}

ajf_status ajf_selftest_check_plan(ajf_ctx* c, int mutation) {
  if (!c) return AJF_E_ARG;
  if (!c->planned) return fail(c, AJF_E_STATE, "no plan");
  Program P = c->prog;  // a copy: the context's program is not touched
  auto first_step = [&](auto pred) -> StepDev* {
    for (auto& ln : P.launches)
      if (ln.kind == LK_SMALL || ln.kind == LK_SPLITK || ln.kind == LK_DOT)
        for (int k = ln.first; k < ln.first + ln.count; ++k)
          if (pred(P.steps[k])) return &P.steps[k];
    return nullptr;
  };
  // Point the reads of the complex128 tensor at element offset `from` (plane `plane`, written
  // before launch `first`) to `to`: launches from `first` on, until one writes over its old place.
  auto redirect = [&](int64_t from, int64_t plane, size_t first, int64_t to) {
    const int64_t lo = from, hi = from + 2 * plane;
    auto hits = [&](int64_t o, int64_t p) { return o < hi && lo < o + 2 * p; };
    for (size_t li = first; li < P.launches.size(); ++li) {
      const Launch& ln = P.launches[li];
      bool overwritten = false;
      if (ln.kind == LK_SMALL || ln.kind == LK_SPLITK || ln.kind == LK_DOT) {
        for (int k = ln.first; k < ln.first + ln.count; ++k) {
          StepDev& d = P.steps[k];
          if (d.a == from && d.pa == plane && !d.fa) d.a = to;
          if (d.b == from && d.pb == plane && !d.fb) d.b = to;
        }
        for (int k = ln.first; k < ln.first + ln.count; ++k)
          overwritten = overwritten || (P.steps[k].scalar_slot < 0 && hits(P.steps[k].c, P.steps[k].pc));
      } else if (ln.kind == LK_PERM) {
        for (int k = ln.first; k < ln.first + ln.count; ++k)
          if (P.perms[k].src == from && P.perms[k].plane == plane && !P.perms[k].src_f32) P.perms[k].src = to;
      } else {
        // the GEMM's result, in FP64 units (complex64 from a reduced-precision GEMM)
        const int64_t ce = ln.op_f64 ? 8 : 4;
        overwritten = hits(ln.c_off / 8, ln.M * ln.N * ce / 16);
      }
      if (overwritten) return;
    }
    if (P.fin.open_off == from && P.fin.open_plane == plane && !P.fin.open_f32) P.fin.open_off = to;
  };
  switch (mutation) {
    case 1:  // a leaf placed past the end of the work region
      if (P.leaves.empty()) return fail(c, AJF_E_ARG, "no leaves");
      P.leaves[0].off = static_cast<int64_t>((P.off_work + P.work_bytes) / P.elem);
      break;
    case 2: {  // an index-map position beyond the operand's bits
      StepDev* d = first_step([](const StepDev& x) { return x.rk > 0; });
      if (!d) return fail(c, AJF_E_ARG, "no step with a contracted index");
      int bits = 0;
      while ((int64_t(1) << bits) < d->pa) ++bits;
      d->ka.pos[0] = static_cast<int8_t>(bits);
      break;
    }
    case 3: {  // a step writing over its own input (its readers follow it)
      StepDev* d = first_step([](const StepDev& x) { return x.scalar_slot < 0 && x.pc <= x.pa; });
      if (!d) return fail(c, AJF_E_ARG, "no step with a tensor output");
      const size_t li = static_cast<size_t>(std::find_if(P.launches.begin(), P.launches.end(), [&](const Launch& l) {
                          return (l.kind == LK_SMALL || l.kind == LK_SPLITK || l.kind == LK_DOT) && l.first <= d - P.steps.data() &&
                                 d - P.steps.data() < l.first + l.count;
                        }) - P.launches.begin());
      redirect(d->c, d->pc, li + 1, d->a);
      d->c = d->a;
      break;
    }
    case 4: {  // a read of memory no launch wrote (the operand shifted by one element)
      StepDev* d = first_step([](const StepDev&) { return true; });
      if (!d) return fail(c, AJF_E_ARG, "no pairwise step");
      d->a += 1;
      break;
    }
    case 5: {  // two leaves of one size in the same place (the second one's readers follow it)
      for (size_t j = 1; j < P.leaves.size(); ++j)
        if (P.leaves[j].bits == P.leaves[0].bits) {
          redirect(P.leaves[j].off, P.leaves[j].plane, 0, P.leaves[0].off);
          P.leaves[j].off = P.leaves[0].off;
          break;
        }
      break;
    }
    case 6: {  // a step of the first launch writing over a leaf that a later launch still reads
      const Launch& l0 = P.launches.empty() ? Launch{} : P.launches[0];
      if (P.launches.empty() || l0.kind != LK_SMALL) return fail(c, AJF_E_ARG, "first launch is not a small-step launch");
      std::vector<char> early(P.leaves.size(), 0);  // leaves the first launch reads
      for (int k = l0.first; k < l0.first + l0.count; ++k)
        for (size_t l = 0; l < P.leaves.size(); ++l)
          if (P.steps[k].a == P.leaves[l].off || P.steps[k].b == P.leaves[l].off) early[l] = 1;
      StepDev* d = nullptr;
      for (int k = l0.first; k < l0.first + l0.count && !d; ++k)
        if (P.steps[k].scalar_slot < 0) d = &P.steps[k];
      size_t x = 0;  // a leaf the first launch does not read, of another size than d's output
      while (x < P.leaves.size() && d && (early[x] || P.leaves[x].plane == d->pc)) ++x;
      if (!d || x == P.leaves.size()) return fail(c, AJF_E_ARG, "no step / late leaf to use");
      redirect(d->c, d->pc, 1, P.leaves[x].off);
      d->c = P.leaves[x].off;
      break;
    }
    case 7: {  // an operand bit that no map addresses (an output bit dropped from A's map)
      StepDev* d = first_step([](const StepDev& x) {
        for (int i = 0; i < x.oa.nbits; ++i)
          if (x.oa.pos[i] >= 0) return true;
        return false;
      });
      if (!d) return fail(c, AJF_E_ARG, "no step with an output bit of A");
      for (int i = 0; i < d->oa.nbits; ++i)
        if (d->oa.pos[i] >= 0) {
          d->oa.pos[i] = -1;
          break;
        }
      break;
    }
    case 8: {  // a GEMM whose K is twice its gathers' (it would read past their operand terms)
      Launch* g = nullptr;
      for (auto& ln : P.launches)
        if (!g && (ln.kind == LK_GEMM_TC || ln.kind == LK_GEMM_SIMT)) g = &ln;
      if (!g) return fail(c, AJF_E_ARG, "no GEMM launch");
      g->K *= 2;
      break;
    }
    default:
      return fail(c, AJF_E_ARG, "unknown mutation");
  }
  const std::string why = check_program(P);
  if (why.empty()) return fail(c, AJF_E_STATE, "planted mistake " + std::to_string(mutation) + " was not caught");
  c->err = "caught: " + why;
  return AJF_OK;
}

ajf_status ajf_slice_count(const ajf_ctx* c, int64_t* n) {
  if (!c || !n) return AJF_E_ARG;
  if (!c->planned) return AJF_E_STATE;
  *n = is_sliced(c) ? slice_count(c) : (int64_t(1) << c->bond_labels.size());
  return AJF_OK;
}

ajf_status ajf_alg2_slice_range(ajf_ctx* c, int64_t first, int64_t count, double* S_part) {
  if (!c) return AJF_E_ARG;
  if (!S_part) return fail(c, AJF_E_ARG, "S_part is NULL");
  if (!c->planned || c->alg != 2) return fail(c, AJF_E_STATE, "needs an Alg. II plan");
  if (c->device < 0) return fail(c, AJF_E_STATE, "host-only context (device -1) cannot run the contraction");
  const int64_t n = int64_t(1) << c->bond_labels.size();
  if (first < 0 || count < 0 || first > n || count > n - first)
    return fail(c, AJF_E_ARG, "slice range outside [0, " + std::to_string(n) + ")");
  *S_part = 0;
  if (count == 0) return AJF_OK;
  CUDA_TRY(c, cudaSetDevice(c->device));
  if (!c->uploaded) {
    ajf_status st = do_upload(c);
    if (st != AJF_OK) return st;
  }
  return run_bonds(c, 2, first, count, S_part);
}

ajf_status ajf_shard_units(const ajf_ctx* c, int32_t* kind, int64_t* n_units) {
  if (!c || !kind || !n_units) return AJF_E_ARG;
  if (!c->planned) return AJF_E_STATE;
  if (c->alg == 1 && is_sliced(c)) {
    *kind = AJF_UNITS_KRAUS_SLICES;
    *n_units = slice_count(c);
  } else if (c->alg == 2) {
    *kind = AJF_UNITS_BOND_SLICES;
    *n_units = int64_t(1) << c->bond_labels.size();
  } else {
    *kind = AJF_UNITS_WHOLE;
    *n_units = 1;
  }
  return AJF_OK;
}

ajf_status ajf_fidelity_from_sum(int n_qubits, double S, double eps, int64_t traces_done, ajf_result* out) {
  if (!out || n_qubits < 1 || n_qubits > 62 || !std::isfinite(S) || S < 0 || eps > 1.0 || std::isnan(eps))
    return AJF_E_ARG;
  const int nsq = 2 * n_qubits;
  out->S = S;
  out->F = std::ldexp(S, -nsq);
  out->one_minus_F = std::ldexp(std::ldexp(1.0, nsq) - S, -nsq);
  out->traces_done = traces_done;
  out->equivalent = eps < 0 ? -1 : (out->F > 1.0 - eps ? 1 : 0);
  out->reserved = 0;
  return AJF_OK;
}

ajf_status ajf_fidelity(ajf_ctx* c, double eps, ajf_result* out) {
  if (!c) return AJF_E_ARG;
  if (!c->planned) return fail(c, AJF_E_STATE, "no plan");
  return fidelity(c, c->alg, eps, out);
}

ajf_status ajf_fidelity_noalloc(ajf_ctx* c, int alg, double eps, ajf_result* out) {
  if (!c) return AJF_E_ARG;
  if (!out) return fail(c, AJF_E_ARG, "out is NULL");
  if (alg != 1 && alg != 2) return fail(c, AJF_E_ARG, "alg must be 1 or 2");
  if (!c->planned || c->alg != alg) return fail(c, AJF_E_STATE, "no Alg. " + std::to_string(alg) + " plan");
  if (c->device < 0) return fail(c, AJF_E_STATE, "host-only context (device -1) cannot run the contraction");
  if (eps > 1.0) return fail(c, AJF_E_ARG, "eps > 1");
  if (multi_run(c)) return fail(c, AJF_E_STATE, "a sliced plan runs through ajf_fidelity_alg1/2 / ajf_fidelity only");
  const Program& P = c->prog;
  if (P.arena_bytes > kStaticArenaBytes)
    return fail(c, AJF_E_NOMEM, "plan needs " + std::to_string(P.arena_bytes) + " bytes of device memory; the fixed " +
                                    "arena of ajf_fidelity_noalloc holds " + std::to_string(kStaticArenaBytes) + " bytes");
  if (!c->static_arena) return fail(c, AJF_E_STATE, "the fixed arena was not resolved when the context was created");
  CUDA_TRY(c, cudaSetDevice(c->device));
  // Run the same device program with the fixed arena as its base; the context's own arena, its
  // CUDA graph, its prepared tensor-core launches and its profiling state are left untouched.
  char* const own_arena = c->arena;
  const bool own_profiling = c->profiling;
  c->arena = c->static_arena;
  c->profiling = false;
  ajf_status st = AJF_OK;
  double res[3] = {0, 0, 0};
  int status[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(c->arena + P.off_desc, c->desc_image.data(), c->desc_image.size(),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && P.input_bytes)
    e = cudaMemcpyAsync(c->arena + P.off_inputs, c->in.packed.data(), P.input_bytes, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->arena + P.off_status, 0, 16 * sizeof(int32_t), c->stream);
  if (e != cudaSuccess) st = cuda_fail(c, e, "ajf_fidelity_noalloc upload");
  if (st == AJF_OK) st = enqueue_program(c, c->stream, &c->tc_static);
  if (st == AJF_OK) {
    e = cudaMemcpyAsync(res, c->arena + P.off_result, sizeof(res), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(status, c->arena + P.off_status, sizeof(status), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = cuda_fail(c, e, "ajf_fidelity_noalloc read-back");
  }
  c->arena = own_arena;
  c->profiling = own_profiling;
  if (st != AJF_OK) return st;
  if (status[0] != 0)
    return fail(c, AJF_E_TIMEOUT, "a bounded device-side wait expired (code " + std::to_string(status[0]) + ")");
  out->S = res[0];
  out->F = res[1];
  out->one_minus_F = res[2];
  out->traces_done = alg == 1 ? real_combinations(c) : 0;
  out->equivalent = eps < 0 ? -1 : (out->F > 1.0 - eps ? 1 : 0);
  out->reserved = 0;
  return AJF_OK;
}

ajf_status ajf_alg1_traces(ajf_ctx* c, double* traces, int64_t count) {
  if (!c) return AJF_E_ARG;
  if (!c->have_alg1 || !c->planned || c->alg != 1) return fail(c, AJF_E_STATE, "no Alg. I result");
  if (!traces) return fail(c, AJF_E_ARG, "traces is NULL");
  const int64_t real = real_combinations(c);
  if (count != real) return fail(c, AJF_E_ARG, "count must be " + std::to_string(real));
  if (is_sliced(c)) {  // gathered on the host slice by slice
    std::memcpy(traces, c->slice_traces.data(), 2 * static_cast<size_t>(real) * sizeof(double));
    return AJF_OK;
  }
  std::vector<double> padded;
  if (bond_sliced(c)) {  // summed on the host over the bond slices
    padded = c->bond_traces;
  } else {
    CUDA_TRY(c, cudaSetDevice(c->device));
    padded.resize(2 * static_cast<size_t>(c->prog.n_traces));
    CUDA_TRY(c, cudaMemcpyAsync(padded.data(), c->arena + c->prog.off_traces, padded.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  // padded index: noise j's Kraus index shifted by the bits of the noises added after it
  const int m = static_cast<int>(c->in.noises.size());
  std::vector<int> shift(m, 0);
  int acc = 0;
  for (int j = m - 1; j >= 0; --j) {
    shift[j] = acc;
    acc += c->in.noises[j].kbits;
  }
  std::vector<int> digit(m, 0);
  for (int64_t idx = 0; idx < real; ++idx) {
    int64_t pidx = 0;
    for (int j = 0; j < m; ++j) pidx |= int64_t(digit[j]) << shift[j];
    traces[2 * idx] = padded[2 * pidx];
    traces[2 * idx + 1] = padded[2 * pidx + 1];
    for (int j = m - 1; j >= 0; --j) {
      if (++digit[j] < c->in.noises[j].nk) break;
      digit[j] = 0;
    }
  }
  return AJF_OK;
}

ajf_status ajf_launch(ajf_ctx* c, double* dev_result) {
  if (!c) return AJF_E_ARG;
  if (!c->planned || !c->uploaded || c->device < 0)
    return fail(c, AJF_E_STATE, "ajf_launch needs a plan and uploaded inputs on a device context");
  if (multi_run(c)) return fail(c, AJF_E_STATE, "a sliced plan runs through ajf_fidelity_alg1/2 / ajf_fidelity only");
  CUDA_TRY(c, cudaSetDevice(c->device));
  ajf_status st = run_program(c);
  if (st != AJF_OK) return st;
  if (dev_result)
    CUDA_TRY(c, cudaMemcpyAsync(dev_result, c->arena + c->prog.off_result, 3 * sizeof(double), cudaMemcpyDeviceToDevice,
                                c->stream));
  return AJF_OK;
}

ajf_status ajf_selftest_gemm(int device, int kind, int npass, int64_t M, int64_t N, int64_t K, const void* A,
                             const void* B, double* C) {
  if (!A || !B || !C || npass < 1 || npass > 3 || (kind != 0 && kind != 1) || M <= 0 || N <= 0 || K <= 0)
    return AJF_E_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return AJF_E_CUDA;
  if (!tc_gemm_supported(M, N, K, kind)) return AJF_E_UNSUPPORTED;
  const size_t es = kind == 1 ? 2 : 4;
  const size_t abytes = size_t(npass) * M * K * es, bbytes = size_t(npass) * N * K * es, cbytes = size_t(M) * N * 4;
  const int ksplit = tc_gemm_splits(M, N, K, kind);
  const size_t wbytes = ksplit > 1 ? size_t(ksplit) * cbytes : 0;
  char* d = nullptr;
  const size_t off_b = (abytes + 255) / 256 * 256, off_c = off_b + (bbytes + 255) / 256 * 256;
  const size_t off_w = off_c + (cbytes + 255) / 256 * 256;
  const size_t off_s = off_w + (wbytes + 255) / 256 * 256;
  if (cudaMalloc(&d, off_s + 256) != cudaSuccess) return AJF_E_NOMEM;
  ajf_status st = AJF_OK;
  int status = 0;
  int64_t ao[6], bo[6];
  for (int p = 0; p < npass; ++p) {
    ao[p] = static_cast<int64_t>(p * M * K * es);
    bo[p] = static_cast<int64_t>(off_b + p * N * K * es);
  }
  if (cudaMemcpy(d, A, abytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d + off_b, B, bbytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(d + off_s, 0, 256) != cudaSuccess)
    st = AJF_E_CUDA;
  if (st == AJF_OK && launch_gemm_tc(d, ao, bo, npass, reinterpret_cast<float*>(d + off_c), M, N, K, kind,
                                     reinterpret_cast<float*>(d + off_w), ksplit, reinterpret_cast<int*>(d + off_s),
                                     0) != cudaSuccess)
    st = AJF_E_CUDA;
  if (st == AJF_OK && cudaDeviceSynchronize() != cudaSuccess) st = AJF_E_CUDA;
  std::vector<float> cf(size_t(M) * N);
  if (st == AJF_OK && (cudaMemcpy(cf.data(), d + off_c, cbytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
                       cudaMemcpy(&status, d + off_s, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess))
    st = AJF_E_CUDA;
  if (st == AJF_OK)
    for (size_t i = 0; i < cf.size(); ++i) C[i] = cf[i];  // FP32 -> FP64, exact
  if (st == AJF_OK && status != 0) st = AJF_E_TIMEOUT;
  cudaFree(d);
  return st;
}

ajf_status ajf_selftest_queue_timeout(int device, double wait_ms, int32_t* code) {
  if (!code || !(wait_ms > 0) || wait_ms > 10000) return AJF_E_ARG;
  *code = 0;
  if (cudaSetDevice(device) != cudaSuccess) return AJF_E_CUDA;
  // phase 0 declares two tasks but the queue holds one of them, so the task of phase 1, which
  // waits for phase 0 to complete, waits for a count that never arrives
  const size_t off_tasks = 1024, off_counters = 2048, off_status = 3072, off_data = 4096;
  char* d = nullptr;
  if (cudaMalloc(&d, off_data + 1024) != cudaSuccess) return AJF_E_NOMEM;
  QPhase ph[2];
  std::memset(ph, 0, sizeof(ph));
  for (int i = 0; i < 2; ++i) {
    ph[i].kind = QK_SPLIT_SUM;
    ph[i].nblocks = 1;
    ph[i].n = 1;
    ph[i].ksplit = 1;
    ph[i].p0 = reinterpret_cast<double*>(d + off_data);
    ph[i].p1 = reinterpret_cast<double*>(d + off_data + 512);
  }
  ph[0].ntasks = 2;
  ph[0].prev = -1;
  ph[1].ntasks = 1;
  ph[1].prev = 0;
  QTask tk[2] = {{0, 0, 1, 0}, {1, 0, 1, 0}};
  ajf_status st = AJF_OK;
  if (cudaMemcpy(d, ph, sizeof(ph), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d + off_tasks, tk, sizeof(tk), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(d + off_status, 0, 1024) != cudaSuccess || cudaMemset(d + off_data, 0, 1024) != cudaSuccess)
    st = AJF_E_CUDA;
  if (st == AJF_OK &&
      launch_queue(reinterpret_cast<const QPhase*>(d), 2, reinterpret_cast<const QTask*>(d + off_tasks), 2,
                   reinterpret_cast<int*>(d + off_counters), reinterpret_cast<int*>(d + off_status), 2, 0,
                   static_cast<unsigned long long>(wait_ms * 1e6)) != cudaSuccess)
    st = AJF_E_CUDA;
  if (st == AJF_OK && cudaDeviceSynchronize() != cudaSuccess) st = AJF_E_CUDA;
  int status = 0;
  if (st == AJF_OK && cudaMemcpy(&status, d + off_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    st = AJF_E_CUDA;
  cudaFree(d);
  if (st != AJF_OK) return st;
  *code = status;
  return status != 0 ? AJF_E_TIMEOUT : AJF_OK;
}

ajf_status ajf_selftest_split_gemm(int device, int precision, int64_t M, int64_t N, int64_t K, const double* A,
                                   const double* B, double* C) {
  if (!A || !B || !C) return AJF_E_ARG;
  int mode = 0, terms = 0;
  switch (precision) {
    case AJF_PREC_TF32: mode = OPM_TF32; terms = 1; break;
    case AJF_PREC_TF32X3: mode = OPM_TF32X2; terms = 2; break;
    case AJF_PREC_BF16X3: mode = OPM_BF16X2; terms = 2; break;
    case AJF_PREC_BF16X6: mode = OPM_BF16X3; terms = 3; break;
    case AJF_PREC_F16X3: mode = OPM_F16X2S; terms = 2; break;
    default: return AJF_E_ARG;
  }
  auto log2i = [](int64_t x) {
    int b = 0;
    while ((int64_t(1) << b) < x) ++b;
    return (int64_t(1) << b) == x ? b : -1;
  };
  const int mb = log2i(M), nb = log2i(N), kb = log2i(K);
  if (mb < 4 || nb < 4 || kb < 3 || mb + kb > 30 || nb + kb > 30) return AJF_E_UNSUPPORTED;
  const int kind = mode == OPM_F16X2S ? 2 : (mode >= OPM_BF16X2 ? 1 : 0);
  const int64_t Mt = 2 * M, Kt = 2 * K;
  if (!tc_gemm_supported(Mt, N, Kt, kind)) return AJF_E_UNSUPPORTED;
  if (cudaSetDevice(device) != cudaSuccess) return AJF_E_CUDA;
  const size_t eb = kind != 0 ? 2 : 4;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  // device layout: A and B as planar complex64 tensors (FP32 planes, imaginary planes zero; the
  // tensors of the reduced-precision modes), operand terms, C (FP32), K-split workspace, status
  const size_t a_src = 0, b_src = al(2 * size_t(M) * K * 4);
  const size_t x0 = b_src + al(2 * size_t(N) * K * 4);
  const size_t xbytes = al(size_t(Mt) * Kt * eb), ybytes = al(size_t(N) * Kt * eb);
  const size_t y0 = x0 + terms * xbytes;
  const size_t c_off = y0 + terms * ybytes;
  const int ksplit = tc_gemm_splits(Mt, N, Kt, kind);
  const size_t cbytes = al(size_t(Mt) * N * 4);
  const size_t w_off = c_off + cbytes, s_off = w_off + (ksplit > 1 ? ksplit * cbytes : 0);
  const size_t p_off = s_off + 256;
  // scaled fp16: one FP32 scale per row and 128-byte K block of each operand
  const size_t kblk = kind == 2 ? (size_t(Kt) * eb + 127) / 128 : 0;
  const size_t xs_off = p_off + al(2 * sizeof(PermDev)), ys_off = xs_off + al(size_t(Mt) * kblk * 4);
  const size_t total = ys_off + al(size_t(N) * kblk * 4);
  char* d = nullptr;
  if (cudaMalloc(&d, total) != cudaSuccess) return AJF_E_NOMEM;
  std::vector<PermDev> pd(2);
  std::memset(pd.data(), 0, 2 * sizeof(PermDev));
  for (int side = 0; side < 2; ++side) {
    PermDev& q = pd[side];
    const int rb = side == 0 ? mb : nb;
    q.src = static_cast<int64_t>((side == 0 ? a_src : b_src) / 4);
    q.src_f32 = 1;
    q.plane = (int64_t(1) << rb) * K;
    q.rows.nbits = rb;
    for (int i = 0; i < rb; ++i) q.rows.pos[i] = static_cast<int8_t>(kb + i);
    q.cols.nbits = kb;
    for (int i = 0; i < kb; ++i) q.cols.pos[i] = static_cast<int8_t>(i);
    q.rbits = rb;
    q.kbits = kb;
    q.embed = side == 0 ? 1 : 0;
    q.rows_fast = 0;
    q.mode = mode;
    for (int t = 0; t < 3; ++t)
      q.dst[t] = static_cast<int64_t>((side == 0 ? x0 + t * xbytes : y0 + t * ybytes));
    if (kind == 2) q.dst[2] = static_cast<int64_t>(side == 0 ? xs_off : ys_off);
  }
  ajf_status st = AJF_OK;
  std::vector<float> planar(2 * size_t(std::max(M, N)) * K, 0.0f);
  auto upload = [&](const double* src, int64_t rows, size_t off) {
    std::fill(planar.begin(), planar.end(), 0.0f);
    for (size_t i = 0; i < size_t(rows) * K; ++i) planar[i] = static_cast<float>(src[i]);  // round to nearest
    return cudaMemcpy(d + off, planar.data(), 2 * size_t(rows) * K * sizeof(float), cudaMemcpyHostToDevice);
  };
  if (upload(A, M, a_src) != cudaSuccess || upload(B, N, b_src) != cudaSuccess ||
      cudaMemcpy(d + p_off, pd.data(), 2 * sizeof(PermDev), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(d + s_off, 0, 256) != cudaSuccess)
    st = AJF_E_CUDA;
  if (st == AJF_OK) {
    const int64_t tiles = std::max<int64_t>(int64_t(1) << std::max(0, mb + kb - 10), int64_t(1) << std::max(0, nb + kb - 10));
    const size_t smem = std::max(perm_table_bytes(pd[0]), perm_table_bytes(pd[1]));
    if (launch_perm(reinterpret_cast<const PermDev*>(d + p_off), 2, static_cast<int>(std::min<int64_t>(tiles, 2048)),
                    smem, d, d, false, 0) != cudaSuccess)
      st = AJF_E_CUDA;
  }
  int64_t ao[6] = {0, 0, 0, 0, 0, 0}, bo[6] = {0, 0, 0, 0, 0, 0};
  for (int t = 0; t < terms; ++t) {
    ao[t] = static_cast<int64_t>(x0 + t * xbytes);
    bo[t] = static_cast<int64_t>(y0 + t * ybytes);
  }
  if (kind == 2) {
    ao[2] = static_cast<int64_t>(xs_off);
    bo[2] = static_cast<int64_t>(ys_off);
  }
  if (st == AJF_OK && launch_gemm_tc(d, ao, bo, terms, reinterpret_cast<float*>(d + c_off), Mt, N, Kt, kind,
                                     reinterpret_cast<float*>(d + w_off), ksplit, reinterpret_cast<int*>(d + s_off),
                                     0) != cudaSuccess)
    st = AJF_E_CUDA;
  if (st == AJF_OK && cudaDeviceSynchronize() != cudaSuccess) st = AJF_E_CUDA;
  int status = 0;
  // the first M rows of C' = [[A, 0], [0, A]] [B | 0]^T hold A . B^T
  std::vector<float> cf(size_t(M) * N);
  if (st == AJF_OK && (cudaMemcpy(cf.data(), d + c_off, cf.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
                       cudaMemcpy(&status, d + s_off, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess))
    st = AJF_E_CUDA;
  if (st == AJF_OK)
    for (size_t i = 0; i < cf.size(); ++i) C[i] = cf[i];  // FP32 -> FP64, exact
  if (st == AJF_OK && status != 0) st = AJF_E_TIMEOUT;
  cudaFree(d);
  return st;
}

ajf_status ajf_plan_launches(const ajf_ctx* c, ajf_launch_info* out, int cap, int* n) {
  if (!c || !n || cap < 0 || (cap > 0 && !out)) return AJF_E_ARG;
  if (!c->planned) return AJF_E_STATE;
  std::vector<ajf_launch_info> v;
  auto add = [&](int kind, int terms, int64_t M, int64_t N, int64_t K, double f, double b) {
    ajf_launch_info li;
    li.kind = kind;
    li.terms = terms;
    li.M = M;
    li.N = N;
    li.K = K;
    li.flops = f;
    li.bytes = b;
    v.push_back(li);
  };
  add(0, 0, 0, 0, 0, 0, 0);
  static const int kClass[6] = {1, 2, 3, 4, 5, 2};
  for (const Launch& ln : c->prog.launches) {
    add(kClass[ln.kind], ln.kind == LK_GEMM_TC ? ln.npass : (ln.kind == LK_GEMM_SIMT ? 1 : 0), ln.M, ln.N, ln.K,
        ln.flops, ln.bytes);
    if (ln.kind == LK_SPLITK || ln.kind == LK_DOT) add(2, 0, 0, 0, 0, 0, 0);  // the deterministic final-sum launch
  }
  add(6, 0, 0, 0, 0, 0, 0);
  add(6, 0, 0, 0, 0, 0, 0);
  *n = static_cast<int>(v.size());
  for (int i = 0; i < cap && i < static_cast<int>(v.size()); ++i) out[i] = v[i];
  return AJF_OK;
}

ajf_status ajf_selftest_wait_timeout(int device, double wait_ms, int32_t* code) {
  if (!code || !(wait_ms > 0) || wait_ms > 10000) return AJF_E_ARG;
  *code = 0;
  if (cudaSetDevice(device) != cudaSuccess) return AJF_E_CUDA;
  const int64_t M = 128, N = 32, K = 32;
  char* d = nullptr;
  const size_t off_b = M * K * 4, off_c = off_b + N * K * 4, off_s = off_c + M * N * 8;
  if (cudaMalloc(&d, off_s + 256) != cudaSuccess) return AJF_E_NOMEM;
  ajf_status st = AJF_OK;
  const int64_t ao[1] = {0}, bo[1] = {static_cast<int64_t>(off_b)};
  if (cudaMemset(d, 0, off_s + 256) != cudaSuccess) st = AJF_E_CUDA;
  if (st == AJF_OK &&
      launch_gemm_tc_ex(d, ao, bo, 1, reinterpret_cast<float*>(d + off_c), M, N, K, 0, nullptr, 1,
                        reinterpret_cast<int*>(d + off_s), 0, static_cast<unsigned long long>(wait_ms * 1e6),
                        1) != cudaSuccess)
    st = AJF_E_CUDA;
  if (st == AJF_OK && cudaDeviceSynchronize() != cudaSuccess) st = AJF_E_CUDA;
  int status = 0;
  if (st == AJF_OK && cudaMemcpy(&status, d + off_s, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    st = AJF_E_CUDA;
  cudaFree(d);
  if (st != AJF_OK) return st;
  *code = status;
  return status != 0 ? AJF_E_TIMEOUT : AJF_OK;
}

int32_t ajf_learned_param_count(void) { return kMlpParams; }

ajf_status ajf_set_learned_model(ajf_ctx* c, const float* weights, int32_t n) {
  if (!c) return AJF_E_ARG;
  if (!weights) {
    c->mlp_weights.clear();
  } else {
    if (n != kMlpParams) return fail(c, AJF_E_ARG, "the merge scorer has " + std::to_string(kMlpParams) + " parameters");
    c->mlp_weights.assign(weights, weights + n);
  }
  c->mlp_version++;
  invalidate(c);
  return AJF_OK;
}

ajf_status ajf_learned_dataset(ajf_ctx* c, int alg, int32_t trials, uint64_t seed, int32_t negatives, float* out,
                               int64_t cap_pairs, int64_t* n_pairs) {
  if (!c || !n_pairs || cap_pairs < 0 || (cap_pairs > 0 && !out) || negatives < 1) return AJF_E_ARG;
  if (alg != 1 && alg != 2) return fail(c, AJF_E_ARG, "alg must be 1 or 2");
  if (!c->has_ideal) return fail(c, AJF_E_STATE, "no circuit loaded");
  pack_inputs(c);
  if (alg == 1) {
    int open_bits = 0;
    for (auto& nz : c->in.noises) open_bits += nz.kbits;
    if (open_bits > 40) return fail(c, AJF_E_BUDGET, "Alg. I result tensor too large");
  }
  const Sequence seq = compose_sequence(c->in, 0);
  const Network net = (alg == 1) ? build_alg1(c->in, seq) : build_alg2(c->in, seq);
  PlanParams pp;
  pp.planner = AJF_PLANNER_AUTO;
  pp.trials = std::max(1, trials);
  pp.seed = seed;
  pp.peak_flops = 200e12;
  pp.elem_bytes = 16;
  Path ref;
  std::vector<float> pairs;
  try {
    ref = plan_path(net, pp);
    learned_dataset(net, ref, seed + 7, negatives, pairs);
  } catch (const std::exception& ex) {
    return fail(c, AJF_E_BUDGET, std::string("planning failed: ") + ex.what());
  }
  const int64_t n = static_cast<int64_t>(pairs.size() / (2 * kMlpFeatures));
  *n_pairs = n;
  const int64_t m = std::min(n, cap_pairs);
  if (m > 0) std::memcpy(out, pairs.data(), static_cast<size_t>(m) * 2 * kMlpFeatures * sizeof(float));
  return AJF_OK;
}

ajf_status ajf_learned_train(int device, const float* pairs, int64_t n_pairs, int32_t epochs, int32_t batch, float lr,
                             uint64_t seed, float* weights, int32_t n_weights, double* final_loss) {
  if (!pairs || !weights || n_pairs < 1 || epochs < 1 || batch < 1 || n_weights != kMlpParams || n_pairs > (1 << 30))
    return AJF_E_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return AJF_E_CUDA;
  const cudaError_t e = mlp_train(pairs, static_cast<int>(n_pairs), epochs,
                                  static_cast<int>(std::min<int64_t>(batch, n_pairs)), lr, seed, weights, final_loss);
  if (e == cudaErrorMemoryAllocation) return AJF_E_NOMEM;
  return e == cudaSuccess ? AJF_OK : AJF_E_CUDA;
}

ajf_status ajf_profile_enable(ajf_ctx* c, int on) {
  if (!c) return AJF_E_ARG;
  if (c->device >= 0) {
    cudaSetDevice(c->device);
    drain_profile(c);
  }
  for (auto& s : c->stats) s = ajf_kernel_stats{};
  c->profiling = on != 0;
  return AJF_OK;
}

ajf_status ajf_profile_read(ajf_ctx* c, ajf_kernel_stats* stats, int cap) {
  if (!c || !stats || cap < 0) return AJF_E_ARG;
  if (c->device >= 0) {
    CUDA_TRY(c, cudaSetDevice(c->device));
    drain_profile(c);
  }
  for (int i = 0; i < cap && i < 8; ++i) stats[i] = c->stats[i];
  return AJF_OK;
}

ajf_status ajf_fidelity_batch(ajf_ctx* const* ctxs, int n_ctx, int alg, double eps, ajf_result* out) {
  Range nvtx_range("ajf batch");
  if (!ctxs || n_ctx < 1 || !out || (alg != 1 && alg != 2)) return AJF_E_ARG;
  for (int i = 0; i < n_ctx; ++i) {
    if (!ctxs[i]) return AJF_E_ARG;
    if (ctxs[i]->device != ctxs[0]->device || ctxs[i]->device < 0)
      return fail(ctxs[0], AJF_E_ARG, "contexts must share one device");
    if (!ctxs[i]->planned || ctxs[i]->alg != alg)
      return fail(ctxs[i], AJF_E_STATE, "context without an Alg. " + std::to_string(alg) + " plan");
    if (is_sliced(ctxs[i]))
      return fail(ctxs[i], AJF_E_STATE, "a sliced Alg. I plan runs through ajf_fidelity_alg1 / ajf_fidelity only");
    if (eps > 1.0) return fail(ctxs[0], AJF_E_ARG, "eps > 1");
  }
  // every context runs on its own stream so independent circuits overlap on the GPU; a
  // bond-sliced context enqueues all its runs at once when they fit one staging chunk
  std::vector<char> bonds_pending(n_ctx, 0);
  for (int i = 0; i < n_ctx; ++i) {
    ajf_ctx* c = ctxs[i];
    CUDA_TRY(c, cudaSetDevice(c->device));
    if (!c->uploaded) {
      ajf_status st = do_upload(c);
      if (st != AJF_OK) return st;
    }
    if (bond_sliced(c)) {
      const int64_t runs = int64_t(1) << c->bond_labels.size();
      const BondLayout L = bond_layout(c, alg, runs);
      if (L.chunk < runs) continue;  // run in the second pass, chunk by chunk
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      ajf_status st = ensure_pinned(c, L.per_run * static_cast<size_t>(runs));
      if (st == AJF_OK) st = enqueue_bond_runs(c, alg, 0, runs, L);
      if (st != AJF_OK) return st;
      bonds_pending[i] = 1;
      continue;
    }
    ajf_status st = run_program(c);
    if (st != AJF_OK) return st;
  }
  for (int i = 0; i < n_ctx; ++i) {
    ajf_ctx* c = ctxs[i];
    if (bond_sliced(c)) {
      ajf_status st;
      if (bonds_pending[i]) {
        const int64_t runs = int64_t(1) << c->bond_labels.size();
        const BondLayout L = bond_layout(c, alg, runs);
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        st = check_status_words(c);
        if (st != AJF_OK) return st;
        if (alg == 1) c->bond_traces.assign(2 * static_cast<size_t>(c->prog.n_traces), 0.0);
        double S = 0, comp = 0;
        collect_bond_runs(c, alg, runs, L, S, comp);
        finish_bonds(c, alg, S + comp, eps, &out[i]);
      } else {
        st = fidelity_bonds(c, alg, eps, &out[i]);
        if (st != AJF_OK) return st;
      }
      continue;
    }
    double res[3];
    CUDA_TRY(c, cudaMemcpyAsync(res, c->arena + c->prog.off_result, sizeof(res), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    ajf_status st = check_status_words(c);
    if (st != AJF_OK) return st;
    out[i].S = res[0];
    out[i].F = res[1];
    out[i].one_minus_F = res[2];
    out[i].traces_done = alg == 1 ? real_combinations(c) : 0;
    out[i].equivalent = eps < 0 ? -1 : (res[1] > 1.0 - eps ? 1 : 0);
    out[i].reserved = 0;
    if (alg == 1) c->have_alg1 = true;
  }
  return AJF_OK;
}

ajf_status ajf_fidelity_alg1_batch(ajf_ctx* const* ctxs, int n_ctx, double eps, ajf_result* out) {
  if (!ctxs || n_ctx < 1 || !out) return AJF_E_ARG;
  for (int i = 0; i < n_ctx; ++i) {
    if (!ctxs[i]) return AJF_E_ARG;
    if (ctxs[i]->device != ctxs[0]->device) return fail(ctxs[0], AJF_E_ARG, "contexts on different devices");
    if (!ctxs[i]->planned || ctxs[i]->alg != 1) return fail(ctxs[i], AJF_E_STATE, "context without an Alg. I plan");
    if (multi_run(ctxs[i])) return fail(ctxs[i], AJF_E_STATE, "a sliced plan runs through ajf_fidelity_alg1/2 / ajf_fidelity only");
    if (ctxs[i]->opts.precision != ctxs[0]->opts.precision) return fail(ctxs[0], AJF_E_ARG, "mixed precision");
  }
  // every context runs on its own stream so independent circuits overlap on the GPU
  for (int i = 0; i < n_ctx; ++i) {
    ajf_ctx* c = ctxs[i];
    CUDA_TRY(c, cudaSetDevice(c->device));
    if (!c->uploaded) {
      ajf_status st = do_upload(c);
      if (st != AJF_OK) return st;
    }
    ajf_status st = run_program(c);
    if (st != AJF_OK) return st;
  }
  for (int i = 0; i < n_ctx; ++i) {
    ajf_ctx* c = ctxs[i];
    double res[3];
    CUDA_TRY(c, cudaMemcpyAsync(res, c->arena + c->prog.off_result, sizeof(res), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    ajf_status st = check_status_words(c);
    if (st != AJF_OK) return st;
    out[i].S = res[0];
    out[i].F = res[1];
    out[i].one_minus_F = res[2];
    out[i].traces_done = real_combinations(c);
    out[i].equivalent = eps < 0 ? -1 : (res[1] > 1.0 - eps ? 1 : 0);
    out[i].reserved = 0;
    c->have_alg1 = true;
  }
  return AJF_OK;
}

}  // extern "C"

namespace {

ajf_status sync_event(ajf_ctx* c, cudaEvent_t* ev) {
  if (!c->sync_ev) CUDA_TRY(c, cudaEventCreateWithFlags(&c->sync_ev, cudaEventDisableTiming));
  *ev = c->sync_ev;
  return AJF_OK;
}

// Job and op table of a persistent launch over `ctxs`, kept in ctxs[0]'s device buffer and
// rebuilt only when a context, its arena, its plan or the result pointer changed.
// ---- block-size autotuning of the persistent launch
// A batch's signature is its device and the structures (plan keys) of its networks in order; the
// fastest block size measured for a signature is kept for the process and used by every later
// persistent launch of a batch with that signature (256 threads until one is measured).
std::mutex g_tune_mu;
std::map<std::vector<int64_t>, int> g_tuned_threads;

std::vector<int64_t> batch_signature(ajf_ctx* const* ctxs, int n) {
  std::vector<int64_t> sig = {ctxs[0]->device, n};
  for (int i = 0; i < n; ++i) {
    sig.push_back(static_cast<int64_t>(ctxs[i]->prog_key.size()));
    sig.insert(sig.end(), ctxs[i]->prog_key.begin(), ctxs[i]->prog_key.end());
  }
  return sig;
}

int tuned_threads(ajf_ctx* const* ctxs, int n) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned_threads.find(batch_signature(ctxs, n));
  return it == g_tuned_threads.end() ? 256 : it->second;
}

ajf_status persistent_table(ajf_ctx* const* ctxs, int n, double* dev_results) {
  ajf_ctx* lead = ctxs[0];
  std::vector<uintptr_t> key;
  key.reserve(3 * static_cast<size_t>(n) + 1);
  key.push_back(reinterpret_cast<uintptr_t>(dev_results));
  for (int i = 0; i < n; ++i) {
    key.push_back(reinterpret_cast<uintptr_t>(ctxs[i]));
    key.push_back(reinterpret_cast<uintptr_t>(ctxs[i]->arena));
    key.push_back(static_cast<uintptr_t>(ctxs[i]->plan_gen));
  }
  if (lead->pers_dev && key == lead->pers_key) return AJF_OK;
  std::vector<InterpJob> jobs(n);
  std::vector<InterpOp> ops;
  size_t smem = 0;
  for (int i = 0; i < n; ++i) {
    const ajf_ctx* c = ctxs[i];
    const Program& P = c->prog;
    InterpJob& J = jobs[i];
    std::memset(&J, 0, sizeof(J));
    J.base = c->arena;
    J.out = dev_results ? dev_results + 3 * static_cast<size_t>(i) : nullptr;
    J.off_leaves = static_cast<int64_t>(P.off_leaves);
    J.off_steps = static_cast<int64_t>(P.off_steps);
    J.off_final = static_cast<int64_t>(P.off_final);
    J.off_inputs = static_cast<int64_t>(P.off_inputs);
    J.off_scalars = static_cast<int64_t>(P.off_scalars);
    J.off_traces = static_cast<int64_t>(P.off_traces);
    J.off_result = static_cast<int64_t>(P.off_result);
    J.work0 = static_cast<int64_t>(P.off_work / P.elem);
    J.n_leaves = static_cast<int32_t>(P.leaves.size());
    J.op0 = static_cast<int32_t>(ops.size());
    J.n_ops = static_cast<int32_t>(P.launches.size());
    J.smem = P.work_bytes <= kPersistentSmemMax ? 1 : 0;
    if (J.smem) smem = std::max(smem, P.work_bytes);
    for (const Launch& ln : P.launches) {
      if (ln.kind != LK_SMALL && ln.kind != LK_SPLITK)
        return fail(ctxs[i], AJF_E_STATE, "internal: a persistent-lowered program holds a GEMM launch");
      ops.push_back(InterpOp{ln.kind, ln.first, ln.count, 0});
    }
  }
  lead->pers_threads = tuned_threads(ctxs, n);
  const size_t jb = (sizeof(InterpJob) * static_cast<size_t>(n) + 255) & ~size_t(255);
  const size_t bytes = jb + sizeof(InterpOp) * std::max<size_t>(1, ops.size());
  lead->pers_host.assign(bytes, 0);
  std::memcpy(lead->pers_host.data(), jobs.data(), sizeof(InterpJob) * static_cast<size_t>(n));
  if (!ops.empty()) std::memcpy(lead->pers_host.data() + jb, ops.data(), sizeof(InterpOp) * ops.size());
  if (bytes > lead->pers_cap) {
    if (lead->pers_dev) {
      CUDA_TRY(lead, cudaStreamSynchronize(lead->stream));
      cudaFree(lead->pers_dev);
      lead->pers_dev = nullptr;
      lead->pers_cap = 0;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(lead, AJF_E_NOMEM, "persistent job table");
    }
    lead->pers_dev = static_cast<char*>(p);
    lead->pers_cap = bytes;
  }
  CUDA_TRY(lead, cudaMemcpyAsync(lead->pers_dev, lead->pers_host.data(), bytes, cudaMemcpyHostToDevice, lead->stream));
  lead->pers_key = key;
  lead->pers_smem = smem;
  return AJF_OK;
}

size_t persistent_ops_offset(int n) { return (sizeof(InterpJob) * static_cast<size_t>(n) + 255) & ~size_t(255); }

ajf_status check_batch(ajf_ctx* const* ctxs, int n_ctx) {
  if (!ctxs || n_ctx < 1) return AJF_E_ARG;
  for (int i = 0; i < n_ctx; ++i) {
    if (!ctxs[i]) return AJF_E_ARG;
    if (ctxs[i]->device < 0 || ctxs[i]->device != ctxs[0]->device)
      return fail(ctxs[0], AJF_E_ARG, "contexts must share one device");
  }
  return AJF_OK;
}

// Enqueue one persistent launch over ctxs (all persistent-lowered, planned) on ctxs[0]'s stream.
ajf_status launch_persistent_ctxs(ajf_ctx* const* ctxs, int n_ctx, double* dev_results) {
  ajf_ctx* lead = ctxs[0];
  CUDA_TRY(lead, cudaSetDevice(lead->device));
  for (int i = 0; i < n_ctx; ++i) {
    if (!ctxs[i]->uploaded) {
      ajf_status st = do_upload(ctxs[i]);
      if (st != AJF_OK) return st;
    }
  }
  ajf_status st = persistent_table(ctxs, n_ctx, dev_results);
  if (st != AJF_OK) return st;
  cudaStream_t s0 = lead->stream;
  for (int i = 1; i < n_ctx; ++i) {
    if (ctxs[i]->stream == s0) continue;
    cudaEvent_t ev = nullptr;
    if ((st = sync_event(ctxs[i], &ev)) != AJF_OK) return st;
    CUDA_TRY(ctxs[i], cudaEventRecord(ev, ctxs[i]->stream));
    CUDA_TRY(lead, cudaStreamWaitEvent(s0, ev, 0));
  }
  {
    double fl = 0, by = 0;
    for (int i = 0; i < n_ctx; ++i) {
      fl += ctxs[i]->prog.flops;
      by += ctxs[i]->prog.bytes;
    }
    ProfScope ps(lead, s0, 7, fl, by);
    const cudaError_t e = launch_persistent(reinterpret_cast<const InterpJob*>(lead->pers_dev), n_ctx,
                                            reinterpret_cast<const InterpOp*>(lead->pers_dev + persistent_ops_offset(n_ctx)),
                                            lead->pers_smem, lead->pers_threads, s0);
    if (e != cudaSuccess) return cuda_fail(lead, e, "persistent kernel");
  }
  cudaEvent_t ev0 = nullptr;
  if ((st = sync_event(lead, &ev0)) != AJF_OK) return st;
  CUDA_TRY(lead, cudaEventRecord(ev0, s0));
  for (int i = 1; i < n_ctx; ++i)
    if (ctxs[i]->stream != s0) CUDA_TRY(ctxs[i], cudaStreamWaitEvent(ctxs[i]->stream, ev0, 0));
  for (int i = 0; i < n_ctx; ++i)
    if (ctxs[i]->alg == 1) ctxs[i]->have_alg1 = true;
  return AJF_OK;
}

// ---- persistent step interpreter: one launch for the default-lowered programs of many contexts
//
// Task granularity, the interpreter's tunable shape: GEMM work items per task, and the number of
// tasks a CUDA-core phase is cut into (at most; never more than its blocks). The process keeps the
// fastest measured setting per batch signature (ajf_autotune_queue).
struct QueueShape {
  int gemm_items = 2;
  int body_tasks = 304;
};
std::map<std::vector<int64_t>, QueueShape> g_tuned_queue;

QueueShape tuned_queue(ajf_ctx* const* ctxs, int n) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned_queue.find(batch_signature(ctxs, n));
  return it == g_tuned_queue.end() ? QueueShape{} : it->second;
}

int queue_sms(int device) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  return sms;
}

// Phase and task tables of an interpreter launch over ctxs, in ctxs[0]'s device buffer; rebuilt
// only when a context, its arena, its program, the result pointer or the shape changed.
ajf_status queue_table(ajf_ctx* const* ctxs, int n, double* dev_results, const QueueShape& shape) {
  ajf_ctx* lead = ctxs[0];
  std::vector<uintptr_t> key = {reinterpret_cast<uintptr_t>(dev_results), static_cast<uintptr_t>(shape.gemm_items),
                                static_cast<uintptr_t>(shape.body_tasks)};
  for (int i = 0; i < n; ++i) {
    key.push_back(reinterpret_cast<uintptr_t>(ctxs[i]));
    key.push_back(reinterpret_cast<uintptr_t>(ctxs[i]->arena));
    key.push_back(static_cast<uintptr_t>(ctxs[i]->prog_gen));
    key.push_back(static_cast<uintptr_t>(ctxs[i]->plan_gen));
  }
  if (lead->q_dev && key == lead->q_key) return AJF_OK;
  const size_t gp_bytes = queue_gemm_params_bytes();
  // per program: its phases in launch order (prev filled in below); GEMM parameter blocks
  std::vector<std::vector<QPhase>> progs(n);
  std::vector<std::vector<int>> gemm_param_index(n);  // per phase: index of its parameter block or -1
  std::vector<char> params;
  double flops = 0, bytes = 0;
  for (int i = 0; i < n; ++i) {
    ajf_ctx* c = ctxs[i];
    const Program& P = c->prog;
    char* base = c->arena;
    flops += P.flops;
    bytes += P.bytes;
    ajf_status st = prepare_tc_set(c, &c->tc_own);
    if (st != AJF_OK) return st;
    auto add = [&](QPhase ph, int gp) {
      ph.base = base;
      progs[i].push_back(ph);
      gemm_param_index[i].push_back(gp);
    };
    const StepDev* steps = reinterpret_cast<const StepDev*>(base + P.off_steps);
    const PermDev* perms = reinterpret_cast<const PermDev*>(base + P.off_perms);
    double* partial = reinterpret_cast<double*>(base + P.off_partial);
    double* scalars = reinterpret_cast<double*>(base + P.off_scalars);
    QPhase ph;
    std::memset(&ph, 0, sizeof(ph));
    ph.kind = QK_LEAVES;
    ph.nblocks = ph.count = static_cast<int32_t>(P.leaves.size());
    ph.desc = base + P.off_leaves;
    ph.p0 = reinterpret_cast<double*>(base + P.off_inputs);
    add(ph, -1);
    for (size_t li = 0; li < P.launches.size(); ++li) {
      const Launch& ln = P.launches[li];
      std::memset(&ph, 0, sizeof(ph));
      switch (ln.kind) {
        case LK_SMALL:
          ph.kind = QK_SMALL;
          ph.nblocks = ln.blocks;
          ph.count = ln.count;
          ph.desc = steps + ln.first;
          add(ph, -1);
          break;
        case LK_SPLITK:
        case LK_DOT: {
          ph.kind = ln.kind == LK_DOT ? QK_DOT : QK_SPLITK;
          ph.nblocks = ln.blocks;
          ph.count = ln.count;
          ph.flag = ln.op_f64 == 0 ? 1 : 0;
          ph.desc = steps + ln.first;
          ph.p0 = partial;
          add(ph, -1);
          QPhase d;
          std::memset(&d, 0, sizeof(d));
          d.kind = QK_SPLITK_DONE;
          d.nblocks = d.count = ln.count;
          d.desc = steps + ln.first;
          d.p0 = partial;
          d.p1 = scalars;
          add(d, -1);
          break;
        }
        case LK_PERM:
          if (ln.op_f64) return fail(c, AJF_E_UNSUPPORTED, "step interpreter: FP64 GEMM operands (use a tensor-core mode)");
          ph.kind = QK_PERM;
          ph.grid_x = ln.blocks;
          ph.count = ln.count;
          ph.nblocks = ln.blocks * ln.count;
          ph.desc = perms + ln.first;
          add(ph, -1);
          break;
        case LK_GEMM_TC: {
          int bn = 0, bf16 = 0, nwork = 0;
          const size_t at = params.size();
          params.resize(at + gp_bytes, 0);
          const cudaError_t e = queue_gemm_params(c->tc_own.prep[li], params.data() + at, &bn, &bf16, &nwork);
          if (e != cudaSuccess) return cuda_fail(c, e, "step interpreter: GEMM parameters");
          ph.kind = QK_GEMM;
          ph.nblocks = nwork;
          ph.flag = bf16;
          ph.bn = bn;
          add(ph, static_cast<int>(at / gp_bytes));
          if (ln.ksplit > 1) {
            QPhase d;
            std::memset(&d, 0, sizeof(d));
            d.kind = QK_SPLIT_SUM;
            d.n = ln.M * ln.N;
            d.nblocks = static_cast<int32_t>(std::min<int64_t>((d.n + 255) / 256, 4096));
            d.ksplit = ln.ksplit;
            d.p0 = reinterpret_cast<double*>(base + ln.ws_off);
            d.p1 = reinterpret_cast<double*>(base + ln.c_off);
            add(d, -1);
          }
          break;
        }
        default:
          return fail(c, AJF_E_UNSUPPORTED, "step interpreter: CUDA-core GEMM steps (use a tensor-core mode)");
      }
    }
    std::memset(&ph, 0, sizeof(ph));
    ph.kind = QK_OPEN;
    ph.nblocks = P.final_blocks;
    ph.desc = base + P.off_final;
    ph.p0 = scalars;
    ph.p1 = reinterpret_cast<double*>(base + P.off_traces);
    ph.p2 = reinterpret_cast<double*>(base + P.off_open_partial);
    add(ph, -1);
    QPhase f = ph;
    f.kind = QK_FINAL;
    f.nblocks = 1;
    f.p1 = reinterpret_cast<double*>(base + P.off_result);
    f.p3 = dev_results ? dev_results + 3 * static_cast<size_t>(i) : nullptr;
    add(f, -1);
  }
  // interleave the programs' phases (round r holds phase r of every program) and cut them into tasks
  const int sms = std::max(1, queue_sms(lead->device));
  std::vector<QPhase> phases;
  std::vector<QTask> tasks;
  std::vector<int> last(n, -1);
  std::vector<std::pair<int, int>> gemm_fix;  // (phase, parameter block)
  size_t rounds = 0;
  for (auto& v : progs) rounds = std::max(rounds, v.size());
  for (size_t r = 0; r < rounds; ++r) {
    for (int i = 0; i < n; ++i) {
      if (r >= progs[i].size()) continue;
      QPhase ph = progs[i][r];
      const int idx = static_cast<int>(phases.size());
      ph.prev = last[i];
      last[i] = idx;
      int per = 1;
      if (ph.kind == QK_GEMM) per = std::max(1, shape.gemm_items);
      else if (ph.kind != QK_FINAL) per = std::max(1, (ph.nblocks + shape.body_tasks - 1) / shape.body_tasks);
      ph.ntasks = 0;
      for (int b = 0; b < std::max(1, ph.nblocks); b += per) {
        tasks.push_back(QTask{idx, b, std::min(std::max(1, ph.nblocks), b + per), 0});
        ++ph.ntasks;
      }
      const int gp = gemm_param_index[i][r];
      if (gp >= 0) gemm_fix.push_back({idx, gp});
      phases.push_back(ph);
    }
  }
  (void)sms;
  // device buffer: GEMM parameter blocks (1024-byte aligned) | phases | tasks | counters | status
  auto al = [](size_t x) { return (x + 1023) / 1024 * 1024; };
  const size_t off_params = 0;
  const size_t off_phases = off_params + al(params.size());
  const size_t off_tasks = off_phases + al(sizeof(QPhase) * phases.size());
  const size_t off_counters = off_tasks + al(sizeof(QTask) * tasks.size());
  const size_t off_status = off_counters + al(sizeof(int) * (kQPhase0 + phases.size()));
  const size_t total = off_status + 1024;
  if (total > lead->q_cap) {
    if (lead->q_dev) {
      CUDA_TRY(lead, cudaStreamSynchronize(lead->stream));
      cudaFree(lead->q_dev);
      lead->q_dev = nullptr;
      lead->q_cap = 0;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, total) != cudaSuccess) {
      cudaGetLastError();
      return fail(lead, AJF_E_NOMEM, "step interpreter tables");
    }
    lead->q_dev = static_cast<char*>(p);
    lead->q_cap = total;
  }
  for (auto& [idx, gp] : gemm_fix) phases[idx].gemm = lead->q_dev + off_params + static_cast<size_t>(gp) * gp_bytes;
  std::vector<char> host(off_counters, 0);
  if (!params.empty()) std::memcpy(host.data() + off_params, params.data(), params.size());
  std::memcpy(host.data() + off_phases, phases.data(), sizeof(QPhase) * phases.size());
  std::memcpy(host.data() + off_tasks, tasks.data(), sizeof(QTask) * tasks.size());
  CUDA_TRY(lead, cudaMemcpyAsync(lead->q_dev, host.data(), host.size(), cudaMemcpyHostToDevice, lead->stream));
  CUDA_TRY(lead, cudaMemsetAsync(lead->q_dev + off_status, 0, 1024, lead->stream));
  CUDA_TRY(lead, cudaStreamSynchronize(lead->stream));  // `host` goes out of scope
  lead->q_key = key;
  lead->q_nphases = static_cast<int>(phases.size());
  lead->q_ntasks = static_cast<int>(tasks.size());
  lead->q_off_phases = off_phases;
  lead->q_off_tasks = off_tasks;
  lead->q_off_counters = off_counters;
  lead->q_off_status = off_status;
  lead->q_flops = flops;
  lead->q_bytes = bytes;
  if (lead->q_graph) {
    cudaGraphExecDestroy(lead->q_graph);
    lead->q_graph = nullptr;
  }
  return AJF_OK;
}

ajf_status check_queue_batch(ajf_ctx* const* ctxs, int n_ctx) {
  ajf_status st = check_batch(ctxs, n_ctx);
  if (st != AJF_OK) return st;
  for (int i = 0; i < n_ctx; ++i) {
    const ajf_ctx* c = ctxs[i];
    if (!c->planned || c->prog.persistent)
      return fail(ctxs[i], AJF_E_STATE, "step interpreter: context without a default-lowered plan");
    if (multi_run(c)) return fail(ctxs[i], AJF_E_STATE, "step interpreter: sliced plans run through ajf_fidelity_alg1/2");
    if (!c->tc_device) return fail(ctxs[i], AJF_E_UNSUPPORTED, "step interpreter needs a tcgen05 device");
  }
  return AJF_OK;
}

// Enqueue one interpreter launch over ctxs on ctxs[0]'s stream (after every context's stream).
ajf_status launch_queue_ctxs(ajf_ctx* const* ctxs, int n_ctx, double* dev_results, const QueueShape& shape) {
  ajf_ctx* lead = ctxs[0];
  CUDA_TRY(lead, cudaSetDevice(lead->device));
  for (int i = 0; i < n_ctx; ++i) {
    if (!ctxs[i]->uploaded) {
      ajf_status st = do_upload(ctxs[i]);
      if (st != AJF_OK) return st;
    }
  }
  ajf_status st = queue_table(ctxs, n_ctx, dev_results, shape);
  if (st != AJF_OK) return st;
  cudaStream_t s0 = lead->stream;
  for (int i = 1; i < n_ctx; ++i) {
    if (ctxs[i]->stream == s0) continue;
    cudaEvent_t ev = nullptr;
    if ((st = sync_event(ctxs[i], &ev)) != AJF_OK) return st;
    CUDA_TRY(ctxs[i], cudaEventRecord(ev, ctxs[i]->stream));
    CUDA_TRY(lead, cudaStreamWaitEvent(s0, ev, 0));
  }
  const int blocks = std::max(1, std::min(queue_sms(lead->device), lead->q_ntasks));
  auto enqueue = [&](cudaStream_t s) {
    return launch_queue(reinterpret_cast<const QPhase*>(lead->q_dev + lead->q_off_phases),
                        lead->q_nphases, reinterpret_cast<const QTask*>(lead->q_dev + lead->q_off_tasks),
                        lead->q_ntasks, reinterpret_cast<int*>(lead->q_dev + lead->q_off_counters),
                        reinterpret_cast<int*>(lead->q_dev + lead->q_off_status), blocks, s);
  };
  if (lead->profiling) {
    ProfScope ps(lead, s0, 7, lead->q_flops, lead->q_bytes);
    const cudaError_t e = launch_queue(
        reinterpret_cast<const QPhase*>(lead->q_dev + lead->q_off_phases), lead->q_nphases,
        reinterpret_cast<const QTask*>(lead->q_dev + lead->q_off_tasks), lead->q_ntasks,
        reinterpret_cast<int*>(lead->q_dev + lead->q_off_counters), reinterpret_cast<int*>(lead->q_dev + lead->q_off_status),
        blocks, s0, kTcWaitNs, reinterpret_cast<unsigned long long*>(lead->q_dev + lead->q_off_status + 256));
    if (e != cudaSuccess) return cuda_fail(lead, e, "step interpreter");
  } else {
    // the launch (counter reset + kernel) is captured once into a CUDA graph and replayed
    if (!lead->q_graph) {
      cudaGraph_t g = nullptr;
      CUDA_TRY(lead, cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
      const cudaError_t e = enqueue(s0);
      const cudaError_t e2 = cudaStreamEndCapture(s0, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(lead, e != cudaSuccess ? e : e2, "step interpreter graph capture");
      }
      const cudaError_t e3 = cudaGraphInstantiate(&lead->q_graph, g, 0);
      cudaGraphDestroy(g);
      if (e3 != cudaSuccess) return cuda_fail(lead, e3, "step interpreter graph");
    }
    CUDA_TRY(lead, cudaGraphLaunch(lead->q_graph, s0));
  }
  cudaEvent_t ev0 = nullptr;
  if ((st = sync_event(lead, &ev0)) != AJF_OK) return st;
  CUDA_TRY(lead, cudaEventRecord(ev0, s0));
  for (int i = 1; i < n_ctx; ++i)
    if (ctxs[i]->stream != s0) CUDA_TRY(ctxs[i], cudaStreamWaitEvent(ctxs[i]->stream, ev0, 0));
  for (int i = 0; i < n_ctx; ++i)
    if (ctxs[i]->alg == 1) ctxs[i]->have_alg1 = true;
  return AJF_OK;
}

ajf_status queue_status(ajf_ctx* lead) {
  int status = 0;
  CUDA_TRY(lead, cudaMemcpyAsync(&status, lead->q_dev + lead->q_off_status, sizeof(int), cudaMemcpyDeviceToHost,
                                 lead->stream));
  CUDA_TRY(lead, cudaStreamSynchronize(lead->stream));
  if (status != 0)
    return fail(lead, AJF_E_TIMEOUT, "step interpreter: a bounded device-side wait expired (code " +
                                         std::to_string(status) + ")");
  return AJF_OK;
}

}  // namespace

extern "C" {

ajf_status ajf_launch_queue(ajf_ctx* const* ctxs, int n_ctx, double* dev_results) {
  Range nvtx_range("ajf step interpreter launch");
  ajf_status st = check_queue_batch(ctxs, n_ctx);
  if (st != AJF_OK) return st;
  return launch_queue_ctxs(ctxs, n_ctx, dev_results, tuned_queue(ctxs, n_ctx));
}

ajf_status ajf_queue_profile(ajf_ctx* c, double* out, int cap, int reset) {
  if (!c || !out || cap < 0) return AJF_E_ARG;
  if (!c->q_dev) return fail(c, AJF_E_STATE, "no step-interpreter launch led by this context");
  unsigned long long v[3 * kQKinds] = {};
  CUDA_TRY(c, cudaSetDevice(c->device));
  CUDA_TRY(c, cudaMemcpyAsync(v, c->q_dev + c->q_off_status + 256, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
  if (reset) CUDA_TRY(c, cudaMemsetAsync(c->q_dev + c->q_off_status + 256, 0, sizeof(v), c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < cap && i < 3 * kQKinds; ++i) out[i] = static_cast<double>(v[i]) * (i % 3 == 2 ? 1.0 : 1e-9);
  return AJF_OK;
}

ajf_status ajf_fidelity_batch_queue(ajf_ctx* const* ctxs, int n_ctx, int alg, double eps, ajf_result* out) {
  ajf_status st = check_queue_batch(ctxs, n_ctx);
  if (st != AJF_OK) return st;
  if (!out || (alg != 1 && alg != 2)) return fail(ctxs[0], AJF_E_ARG, "bad alg or out");
  if (eps > 1.0) return fail(ctxs[0], AJF_E_ARG, "eps > 1");
  for (int i = 0; i < n_ctx; ++i)
    if (ctxs[i]->alg != alg) return fail(ctxs[i], AJF_E_STATE, "context without an Alg. " + std::to_string(alg) + " plan");
  st = launch_queue_ctxs(ctxs, n_ctx, nullptr, tuned_queue(ctxs, n_ctx));
  if (st != AJF_OK) return st;
  st = queue_status(ctxs[0]);
  if (st != AJF_OK) return st;
  for (int i = 0; i < n_ctx; ++i) {
    ajf_ctx* c = ctxs[i];
    double res[3];
    CUDA_TRY(c, cudaMemcpyAsync(res, c->arena + c->prog.off_result, sizeof(res), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    st = check_status_words(c);
    if (st != AJF_OK) return st;
    out[i].S = res[0];
    out[i].F = res[1];
    out[i].one_minus_F = res[2];
    out[i].traces_done = alg == 1 ? real_combinations(c) : 0;
    out[i].equivalent = eps < 0 ? -1 : (res[1] > 1.0 - eps ? 1 : 0);
    out[i].reserved = 0;
    if (alg == 1) c->have_alg1 = true;
  }
  return AJF_OK;
}

ajf_status ajf_autotune_queue(ajf_ctx* const* ctxs, int n_ctx, int reps, int32_t* gemm_items, int32_t* body_tasks) {
  ajf_status st = check_queue_batch(ctxs, n_ctx);
  if (st != AJF_OK) return st;
  if (reps < 1) return fail(ctxs[0], AJF_E_ARG, "reps < 1");
  ajf_ctx* lead = ctxs[0];
  CUDA_TRY(lead, cudaSetDevice(lead->device));
  const bool prof = lead->profiling;
  lead->profiling = false;
  // candidate shapes: GEMM work items per task x tasks per CUDA-core phase; a shape must beat the
  // best so far by 2% to replace it (timing noise)
  const int items[3] = {1, 2, 4};
  const int bodies[3] = {152, 304, 608};
  QueueShape best;
  float best_ms = -1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(lead, cudaEventCreate(&e0));
  CUDA_TRY(lead, cudaEventCreate(&e1));
  for (int gi : items) {
    for (int bt : bodies) {
      QueueShape sh;
      sh.gemm_items = gi;
      sh.body_tasks = bt;
      st = launch_queue_ctxs(ctxs, n_ctx, nullptr, sh);  // warm-up (tables, graph)
      if (st == AJF_OK) st = queue_status(lead);
      if (st != AJF_OK) break;
      cudaEventRecord(e0, lead->stream);
      for (int r = 0; r < reps && st == AJF_OK; ++r) st = launch_queue_ctxs(ctxs, n_ctx, nullptr, sh);
      cudaEventRecord(e1, lead->stream);
      if (st == AJF_OK) st = queue_status(lead);
      if (st != AJF_OK) break;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (best_ms < 0 || ms < 0.98f * best_ms) {
        best_ms = ms;
        best = sh;
      }
    }
    if (st != AJF_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  lead->profiling = prof;
  if (st != AJF_OK) return st;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned_queue[batch_signature(ctxs, n_ctx)] = best;
  }
  if (gemm_items) *gemm_items = best.gemm_items;
  if (body_tasks) *body_tasks = best.body_tasks;
  return AJF_OK;
}

ajf_status ajf_launch_persistent(ajf_ctx* const* ctxs, int n_ctx, double* dev_results) {
  Range nvtx_range("ajf persistent launch");
  ajf_status st = check_batch(ctxs, n_ctx);
  if (st != AJF_OK) return st;
  for (int i = 0; i < n_ctx; ++i)
    if (!ctxs[i]->planned || !ctxs[i]->prog.persistent)
      return fail(ctxs[i], AJF_E_STATE, "context without a plan made with AJF_LOWER_PERSISTENT");
  return launch_persistent_ctxs(ctxs, n_ctx, dev_results);
}

ajf_status ajf_autotune_persistent(ajf_ctx* const* ctxs, int n_ctx, int reps, int32_t* threads) {
  ajf_status st = check_batch(ctxs, n_ctx);
  if (st != AJF_OK) return st;
  if (reps < 1 || !threads) return fail(ctxs[0], AJF_E_ARG, "reps must be >= 1 and threads non-NULL");
  for (int i = 0; i < n_ctx; ++i)
    if (!ctxs[i]->planned || !ctxs[i]->prog.persistent)
      return fail(ctxs[i], AJF_E_STATE, "context without a plan made with AJF_LOWER_PERSISTENT");
  ajf_ctx* lead = ctxs[0];
  CUDA_TRY(lead, cudaSetDevice(lead->device));
  st = launch_persistent_ctxs(ctxs, n_ctx, nullptr);  // uploads, job table, first-launch costs
  if (st != AJF_OK) return st;
  cudaEvent_t e0, e1;
  CUDA_TRY(lead, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(lead, cudaGetLastError(), "cudaEventCreate");
  }
  int best = 256;
  float best_ms = 0;
  for (int t : {256, 128, 64}) {
    lead->pers_threads = t;
    st = launch_persistent_ctxs(ctxs, n_ctx, nullptr);  // warm-up at this block size
    cudaError_t e = cudaEventRecord(e0, lead->stream);
    for (int r = 0; st == AJF_OK && e == cudaSuccess && r < reps; ++r) {
      lead->pers_threads = t;
      st = launch_persistent_ctxs(ctxs, n_ctx, nullptr);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, lead->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (st == AJF_OK && e != cudaSuccess) st = cuda_fail(lead, e, "autotune timing");
    if (st != AJF_OK) break;
    if (t == 256 || ms < 0.97f * best_ms) {  // a smaller block must win clearly
      best = t;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != AJF_OK) {
    lead->pers_threads = tuned_threads(ctxs, n_ctx);
    return st;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned_threads[batch_signature(ctxs, n_ctx)] = best;
  }
  lead->pers_threads = best;
  *threads = best;
  return AJF_OK;
}

ajf_status ajf_fidelity_batch_persistent(ajf_ctx* const* ctxs, int n_ctx, int alg, double eps, ajf_result* out,
                                         int32_t* n_persistent) {
  ajf_status st = check_batch(ctxs, n_ctx);
  if (st != AJF_OK) return st;
  if (!out || (alg != 1 && alg != 2)) return fail(ctxs[0], AJF_E_ARG, "bad alg or out");
  if (eps > 1.0) return fail(ctxs[0], AJF_E_ARG, "eps > 1");
  std::vector<ajf_ctx*> pers, rest;
  for (int i = 0; i < n_ctx; ++i) {
    if (!ctxs[i]->planned || ctxs[i]->alg != alg)
      return fail(ctxs[i], AJF_E_STATE, "context without an Alg. " + std::to_string(alg) + " plan");
    if (multi_run(ctxs[i])) return fail(ctxs[i], AJF_E_STATE, "a sliced plan runs through ajf_fidelity_alg1/2 / ajf_fidelity only");
    (ctxs[i]->prog.persistent ? pers : rest).push_back(ctxs[i]);
  }
  CUDA_TRY(ctxs[0], cudaSetDevice(ctxs[0]->device));
  if (!pers.empty()) {
    st = launch_persistent_ctxs(pers.data(), static_cast<int>(pers.size()), nullptr);
    if (st != AJF_OK) return st;
  }
  for (ajf_ctx* c : rest) {
    if (!c->uploaded) {
      st = do_upload(c);
      if (st != AJF_OK) return st;
    }
    st = run_program(c);
    if (st != AJF_OK) return st;
  }
  for (int i = 0; i < n_ctx; ++i) {
    ajf_ctx* c = ctxs[i];
    double res[3];
    CUDA_TRY(c, cudaMemcpyAsync(res, c->arena + c->prog.off_result, sizeof(res), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    st = check_status_words(c);
    if (st != AJF_OK) return st;
    out[i].S = res[0];
    out[i].F = res[1];
    out[i].one_minus_F = res[2];
    out[i].traces_done = alg == 1 ? real_combinations(c) : 0;
    out[i].equivalent = eps < 0 ? -1 : (res[1] > 1.0 - eps ? 1 : 0);
    out[i].reserved = 0;
    if (alg == 1) c->have_alg1 = true;
  }
  if (n_persistent) *n_persistent = static_cast<int32_t>(pers.size());
  return AJF_OK;
}

}  // extern "C"
