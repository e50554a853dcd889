// Internal data structures of libajf (host side). Not part of the ABI.
#pragma once

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/ajf.h"

namespace ajf {

// ------------------------------------------------------------------ inputs (copied from the caller)

struct GateIn {
  int arity = 0;
  int q[3] = {0, 0, 0};
  int64_t mat_off = 0;  // complex offset into Inputs::packed
};

struct NoiseIn {
  int after = -1;
  int arity = 0;
  int q[3] = {0, 0, 0};
  int nk = 0;            // Kraus operators
  int kbits = 0;         // ceil(log2(nk)): bits of the open Kraus index (Alg. I)
  int64_t kraus_off = 0; // complex offset into Inputs::packed
};

struct Inputs {
  int n = 0;
  bool has_ideal = false, has_impl = false;
  std::vector<GateIn> ideal, impl;
  std::vector<NoiseIn> noises;
  std::vector<double> packed;  // complex128 interleaved; every matrix the caller passed
  const std::vector<GateIn>& skeleton() const { return has_impl ? impl : ideal; }
};

// ------------------------------------------------------------------ network

// How a leaf tensor's values are made on the device from the packed inputs.
enum LeafKind : int32_t {
  LEAF_GATE = 0,        // G[out][in]
  LEAF_GATE_CONJ = 1,   // G^*[out][in]
  LEAF_GATE_DAG = 2,    // (G^dagger)[out][in] = conj(G[in][out])
  LEAF_GATE_TRANS = 3,  // (G^T)[out][in] = G[in][out]
  LEAF_KRAUS_OPEN = 4,  // T[kappa][out][in] = K_kappa[out][in], zero for kappa >= nk
  LEAF_SUPEROP = 5,     // M_N[(o,o')][(i,i')] = sum_k K_k[o][i] conj(K_k[o'][i'])
  LEAF_IDENTITY = 6,    // delta[out][in], 2 x 2
};

struct LeafSpec {
  int32_t kind = 0;
  int32_t a = 0;        // wires of the operator (2a tensor bits before any Kraus bits)
  int64_t src = 0;      // complex offset of the source matrix / first Kraus operator
  int32_t nk = 0;       // Kraus operators (LEAF_KRAUS_OPEN, LEAF_SUPEROP)
  int32_t kbits = 0;    // open Kraus-index bits (LEAF_KRAUS_OPEN)
  uint32_t fix_mask = 0;  // bond slicing: bits of the full leaf index (before slicing) whose
                          // labels are sliced; their values are set per slice on the device
};

// A tensor's labels are listed from bit 0 (stride 1) upward: element index = sum_i bit_i * 2^i.
// Every label has dimension 2. A label occurs in exactly two leaves unless it is open.
struct Network {
  int alg = 0;
  int n_labels = 0;
  std::vector<std::vector<int>> leaf_labels;
  std::vector<LeafSpec> leaf_specs;
  std::vector<int> open_labels;  // bit order of the Alg. I result tensor t
  int loops = 0;                 // wires touched by no tensor: each a factor tr(I_2) = 2
  int n_qubits = 0;
  std::vector<int> noise_leaf;   // leaf of each noise (-1: removed or absent)
};

// ------------------------------------------------------------------ contraction path

struct PathStep {
  int a = -1, b = -1;     // tensor ids (leaves 0..L-1, then one new id per step)
  std::vector<int> out;   // labels of the result, unordered (layout is chosen at lowering)
};

struct Path {
  std::vector<PathStep> steps;      // each step creates tensor id L + index
  std::vector<int> final_ids;       // tensors left at the end (scalars and/or the open tensor)
  double cmacs = 0, max_size = 0, est_seconds = 0;
  int width = 0;
  int planner = 0;
};

struct PlanParams {
  int planner = AJF_PLANNER_AUTO;
  int precision = AJF_PREC_F64;
  int trials = 32;
  uint64_t seed = 0;
  double peak_flops = 1e12;   // contraction throughput of the chosen precision (time model)
  double peak_bw = 6.5e12;    // bytes/s
  double elem_bytes = 16;
  bool tensor_cores = true;   // GEMM-class steps of the TF32 / bf16 modes run on tcgen05
  // learned merge scorer: weights and a batched scoring function (device kernels or host)
  const float* mlp = nullptr;
  std::function<void(const float* w, const float* x, int n, float* out)> scorer;
  double learned_noise = 0.0;  // Gumbel noise on scores for randomised restarts
};

Path plan_path(const Network& net, const PlanParams& p);
// Estimated device time of a step (ranks of the operands, of their union and of the result).
double step_seconds(int ra, int rb, int runion, int rc, const PlanParams& p);
void evaluate_path(const Network& net, Path& path, const PlanParams& p);
Path plan_greedy(const Network& net, const PlanParams& p, uint64_t seed, double temperature);
Path plan_minfill(const Network& net, const PlanParams& p, uint64_t seed);
Path plan_learned(const Network& net, const PlanParams& p, uint64_t seed, bool* used);
// Subtree reconfiguration: every merge's subtree, cut at up to 8 inputs, is replaced by the
// cheapest binary tree over those inputs (dynamic programming over subsets, evaluate_path's cost
// model) when that is cheaper; `passes` sweeps over the forest. The result computes the same
// tensors at the roots.
Path reconfigure_path(const Network& net, const Path& path, const PlanParams& p, int passes);
// Bond slicing. choose_slice_labels: `count` closed labels to fix, picked greedily on `path` so
// that the widest tensors shrink first (labels whose removal would leave a leaf without labels
// are never picked). slice_network: the network with those labels removed from its leaves
// (LeafSpec::fix_mask marks where they were). restrict_path: `path` over the sliced network (a
// step that becomes a scalar joins the final tensors), with its cost evaluated.
std::vector<int> choose_slice_labels(const Network& net, const Path& path, int count);
Network slice_network(const Network& net, const std::vector<int>& labels);
Path restrict_path(const Network& sliced, const Path& path, const std::vector<int>& labels, const PlanParams& p);
// Replay `ref` and append (chosen merge, other candidate) feature pairs; returns the pair count.
int learned_dataset(const Network& net, const Path& ref, uint64_t seed, int negatives, std::vector<float>& out);

// ------------------------------------------------------------------ composed sequence

// One element of the closed composed sequence: an implementation gate, the adjoint of an ideal
// gate, or a noise, on wires w[0..arity) (rewired by SWAP elimination).
enum SeqKind : int32_t { SEQ_GATE = 0, SEQ_ADJ = 1, SEQ_NOISE = 2 };
struct SeqOp {
  int32_t kind = SEQ_GATE;
  int32_t index = 0;  // skeleton gate (SEQ_GATE), ideal gate (SEQ_ADJ) or noise (SEQ_NOISE)
  int32_t arity = 0;
  int32_t w[3] = {0, 0, 0};
};
struct Sequence {
  std::vector<SeqOp> ops;    // time order: implementation, then the ideal circuit's adjoint
  std::vector<int> closure;  // closure[w]: the input wire joined to output wire w
  int removed = 0;           // gates removed by the simplifications
};
// The sequence of `in`, simplified by AJF_SIMPLIFY_* `flags`.
Sequence compose_sequence(const Inputs& in, int flags);

// ------------------------------------------------------------------ network builders

// `sliced[j]` (may be empty): noise j gets a single-operator leaf (its first Kraus operator; the
// caller points the leaf at another one per slice) and no open index.
Network build_alg1(const Inputs& in, const Sequence& seq, const std::vector<char>& sliced = {});
Network build_alg2(const Inputs& in, const Sequence& seq);

}  // namespace ajf
