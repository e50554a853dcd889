// Contraction-path planners (host side).
//
// A path is a sequence of pairwise merges. Every label has dimension 2, so a merge of tensors
// with label sets a and b costs 2^{|a u b|} complex multiply-adds (M*N*K) and produces a tensor
// of 2^{|a ^ b|} elements.
//
//  * Greedy: repeatedly merge the pair sharing a label with the smallest "memory removed" cost
//    size(out) - size(a) - size(b); randomised restarts perturb the cost (in log scale) with
//    Gumbel noise of a chosen temperature.
//  * Min-fill (Sec. IV-C orders contractions by a tree decomposition of the network's line graph,
//    whose vertices are the network's labels, with an edge between labels of one tensor):
//    eliminate labels in min-fill order -- the vertex whose neighbourhood needs the fewest new
//    edges to become a clique, random tie-breaks -- and contract, for each eliminated label, the
//    two tensors that carry it. Elimination orders and tree decompositions are equivalent
//    (the width of the decomposition bounds the largest intermediate).
//  * Learned: an MLP scores candidate merges (planner_learned.cpp); the greedy planner is its
//    fallback and judge.
// The AUTO planner runs restarts of both and keeps the path with the smallest estimated time
// (step_seconds: a model of the lowered kernels on GB300), after subtree reconfiguration.
#include <algorithm>
#include <array>
#include <bitset>
#include <chrono>
#include <functional>
#include <limits>
#include <unordered_set>
#include <cmath>
#include <cstring>
#include <queue>
#include <unordered_map>

#include "ajf_internal.h"

namespace ajf {
namespace {

struct Rng {
  uint64_t s;
  explicit Rng(uint64_t seed) : s(seed * 0x9E3779B97F4A7C15ull + 0x1234567ull) {}
  uint64_t next() {  // splitmix64
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double gumbel() { return -std::log(-std::log(uniform())); }
};

using Labels = std::vector<int>;  // sorted

Labels sorted(std::vector<int> v) {
  std::sort(v.begin(), v.end());
  return v;
}

// Symmetric difference and intersection size of two sorted label sets.
Labels sym_diff(const Labels& a, const Labels& b, int* shared) {
  Labels out;
  out.reserve(a.size() + b.size());
  size_t i = 0, j = 0;
  int sh = 0;
  while (i < a.size() || j < b.size()) {
    if (j == b.size() || (i < a.size() && a[i] < b[j])) out.push_back(a[i++]);
    else if (i == a.size() || b[j] < a[i]) out.push_back(b[j++]);
    else { ++sh; ++i; ++j; }
  }
  if (shared) *shared = sh;
  return out;
}

// Merge whatever is left when no two tensors share a label: tensors with open labels are joined
// by outer products (smallest first); scalars stay separate and are multiplied at the end.
void finish_components(std::vector<Labels>& ts, std::vector<char>& alive, Path& path) {
  std::vector<int> open_ids;
  for (size_t i = 0; i < ts.size(); ++i)
    if (alive[i]) {
      if (ts[i].empty()) path.final_ids.push_back(static_cast<int>(i));
      else open_ids.push_back(static_cast<int>(i));
    }
  while (open_ids.size() > 1) {
    std::sort(open_ids.begin(), open_ids.end(),
              [&](int x, int y) { return ts[x].size() < ts[y].size(); });
    const int a = open_ids[0], b = open_ids[1];
    PathStep st;
    st.a = a;
    st.b = b;
    st.out = sym_diff(ts[a], ts[b], nullptr);
    alive[a] = alive[b] = 0;
    ts.push_back(st.out);
    alive.push_back(1);
    path.steps.push_back(st);
    open_ids.erase(open_ids.begin(), open_ids.begin() + 2);
    open_ids.push_back(static_cast<int>(ts.size()) - 1);
  }
  if (!open_ids.empty()) path.final_ids.push_back(open_ids[0]);
}

}  // namespace

// Estimated device time of one pairwise step with operand ranks ra, rb and result rank rc (labels
// of dimension 2; runion = |a u b|, so K = 2^(ra + rb - runion)), following the lowering's choice
// of kernel class (program.cpp) and GB300's rates: tensors are complex128 in HBM in the FP64 mode
// and complex64 in the reduced-precision modes (p.elem_bytes per complex element), the
// gate-absorption, split-K and trace kernels compute in FP64 on the CUDA cores, GEMM-class steps
// gather both operands into the precision's operand terms and run one real GEMM of
// 2M x N x 2K on the tensor cores (or on the CUDA cores in the FP64 / FP32 modes), and every
// GEMM-class step carries a fixed cost of its two launches. A GEMM whose output tiles cannot
// occupy every SM runs proportionally slower.
double step_seconds(int ra, int rb, int runion, int rc, const PlanParams& p) {
  constexpr double kBw = 5.0e12;        // achieved HBM bandwidth of the streaming kernels (B/s)
  constexpr double kGatherBw = 3.4e12;  // achieved bandwidth of the operand gather (permuted reads, ncu)
  constexpr double kFp64 = 1.0e12;      // FP64 CUDA-core rate (flop/s)
  constexpr double kFp32 = 40e12;       // FP32 CUDA-core rate
  constexpr double kSMs = 152;
  const int rk = ra + rb - runion;
  const double flops = 8.0 * std::ldexp(1.0, runion);  // 8 per complex multiply-add
  const double io = (std::ldexp(1.0, ra) + std::ldexp(1.0, rb) + std::ldexp(1.0, rc)) * p.elem_bytes;
  if (rc == 0) return std::max(io / kBw, flops / (p.precision == AJF_PREC_F64 ? kFp64 : kFp32)) + 3e-6;
  const int ma = ra - rk, nb = rb - rk;
  const bool gemm = ma >= 4 && nb >= 4 && rk >= 3 && ma + nb + rk >= 18;
  if (!gemm) {
    if (rc <= 12 && rk >= 10) return std::max(io / kBw, flops / kFp64) + 3e-6;  // split-K
    return std::max(io / kBw, flops / kFp64) + 1e-6;                            // one thread per output
  }
  // GEMM class: X (the smaller operand) embedded as 2M x 2K, Y as N x 2K
  const int m = ra <= rb ? ma : nb, n = ra <= rb ? nb : ma;
  const double Mt = std::ldexp(1.0, m + 1), Nt = std::ldexp(1.0, n), Kt = std::ldexp(1.0, rk + 1);
  const bool tc = p.tensor_cores && p.precision >= AJF_PREC_TF32;
  int terms = 1, passes = 1;
  double eb = 8, rate = kFp64, tm = 64, tn = 64;
  if (p.precision == AJF_PREC_F32) {
    eb = 4;
    rate = kFp32;
    tm = 128;
  } else if (tc) {
    const bool bf16 = p.precision == AJF_PREC_BF16X3 || p.precision == AJF_PREC_BF16X6 || p.precision == AJF_PREC_F16X3;
    terms = p.precision == AJF_PREC_TF32 ? 1 : (p.precision == AJF_PREC_BF16X6 ? 3 : 2);
    passes = p.precision == AJF_PREC_TF32 ? 1 : (p.precision == AJF_PREC_BF16X6 ? 6 : 3);
    eb = bf16 ? 2 : 4;
    rate = bf16 ? 1.1e15 : 0.55e15;  // sustained tensor rate of the split GEMM's hardware products
    tm = 128;
    tn = Nt >= 128 ? 128 : Nt;
  }
  const double operands = terms * eb * (Mt * Kt + Nt * Kt);
  const double gather = (std::ldexp(1.0, ra) + std::ldexp(1.0, rb)) * p.elem_bytes + operands;
  const double out = Mt * Nt * p.elem_bytes / 2;  // real planes of the complex result
  double tiles = std::ceil(Mt / tm) * std::ceil(Nt / tn);
  if (tc) tiles *= std::max(1.0, std::min(std::ceil(kSMs / tiles) * 2.0, Kt * eb / 1024.0));  // K splits
  const double eff = std::min(1.0, tiles / kSMs);
  return gather / kGatherBw + std::max(passes * flops / (rate * eff), (operands + out) / kBw) + 14e-6;
}

void evaluate_path(const Network& net, Path& path, const PlanParams& p) {
  std::vector<int> rank;
  for (auto& l : net.leaf_labels) rank.push_back(static_cast<int>(l.size()));
  double cm = 0, secs = 0, maxsz = 0;
  int width = 0;
  for (int r : rank) width = std::max(width, r);
  for (auto& st : path.steps) {
    const int ra = rank[st.a], rb = rank[st.b], rc = static_cast<int>(st.out.size());
    const int k = (ra + rb - rc) / 2;
    const double c = std::ldexp(1.0, ra + rb - k);
    cm += c;
    secs += step_seconds(ra, rb, ra + rb - k, rc, p);
    rank.push_back(rc);
    width = std::max(width, rc);
    maxsz = std::max(maxsz, std::ldexp(1.0, rc));
  }
  path.cmacs = cm;
  path.width = width;
  path.max_size = maxsz;
  path.est_seconds = secs;
}

// ------------------------------------------------------------------ bond slicing
//
// Slicing a closed label b writes the contraction as the sum of two contractions, one with b
// fixed to 0 and one with b fixed to 1 in both tensors that carry it: the full contraction is a
// sum over every label assignment, so fixing some labels and summing over their values is the
// same sum in another order. s sliced labels give 2^s independent contractions whose tensors are
// all at most 2^s times smaller.

std::vector<int> choose_slice_labels(const Network& net, const Path& path, int count) {
  const int L = static_cast<int>(net.leaf_labels.size());
  std::vector<Labels> ts;
  for (auto& l : net.leaf_labels) ts.push_back(sorted(l));
  for (auto& st : path.steps) ts.push_back(sorted(st.out));
  std::vector<char> open(net.n_labels, 0), cut(net.n_labels, 0);
  for (int x : net.open_labels) open[x] = 1;
  // leaves carrying each label, to keep every leaf at one label at least
  std::vector<std::vector<int>> holders(net.n_labels);
  for (int i = 0; i < L; ++i)
    for (int x : ts[i]) holders[x].push_back(i);
  std::vector<int> left(L);
  for (int i = 0; i < L; ++i) left[i] = static_cast<int>(ts[i].size());
  std::vector<int> chosen;
  for (int round = 0; round < count; ++round) {
    std::vector<int> rank(ts.size());
    int w = 0;
    for (size_t i = 0; i < ts.size(); ++i) {
      int r = 0;
      for (int x : ts[i]) r += cut[x] ? 0 : 1;
      rank[i] = r;
      w = std::max(w, r);
    }
    // score: tensors of the largest rank that carry the label, then the summed size of every
    // tensor that carries it (the memory and work that halve). When the largest tensors carry
    // no closed label (an Alg. I result made of open indices), the volume alone decides.
    std::vector<double> in_widest(net.n_labels, 0), mass(net.n_labels, 0);
    for (size_t i = 0; i < ts.size(); ++i)
      for (int x : ts[i]) {
        if (cut[x]) continue;
        if (rank[i] == w) in_widest[x] += 1;
        mass[x] += std::ldexp(1.0, rank[i]);
      }
    int best = -1;
    for (int x = 0; x < net.n_labels; ++x) {
      if (open[x] || cut[x] || mass[x] == 0) continue;
      bool keeps = true;
      for (int h : holders[x]) keeps = keeps && left[h] > 1;
      if (!keeps) continue;
      if (best < 0 || in_widest[x] > in_widest[best] || (in_widest[x] == in_widest[best] && mass[x] > mass[best]))
        best = x;
    }
    if (best < 0) break;  // nothing left to slice
    cut[best] = 1;
    for (int h : holders[best]) --left[h];
    chosen.push_back(best);
  }
  std::sort(chosen.begin(), chosen.end());
  return chosen;
}

Network slice_network(const Network& net, const std::vector<int>& labels) {
  Network out = net;
  std::vector<char> cut(net.n_labels, 0);
  for (int x : labels) cut[x] = 1;
  for (size_t i = 0; i < out.leaf_labels.size(); ++i) {
    const std::vector<int>& full = net.leaf_labels[i];
    std::vector<int> kept;
    uint32_t mask = 0;
    for (size_t p = 0; p < full.size(); ++p) {
      if (cut[full[p]]) mask |= 1u << p;
      else kept.push_back(full[p]);
    }
    out.leaf_labels[i] = kept;
    out.leaf_specs[i].fix_mask = mask;
  }
  return out;
}

Path restrict_path(const Network& sliced, const Path& path, const std::vector<int>& labels, const PlanParams& p) {
  std::vector<char> cut;
  for (int x : labels) {
    if (x >= static_cast<int>(cut.size())) cut.resize(x + 1, 0);
    cut[x] = 1;
  }
  auto is_cut = [&](int x) { return x < static_cast<int>(cut.size()) && cut[x]; };
  const int L = static_cast<int>(sliced.leaf_labels.size());
  // id[old] = new tensor id, or -1 for a scalar that is already among the final tensors
  std::vector<int> id(L + path.steps.size(), -1);
  for (int i = 0; i < L; ++i) id[i] = i;
  Path r;
  r.planner = path.planner;
  int next = L;
  for (size_t s = 0; s < path.steps.size(); ++s) {
    const PathStep& st = path.steps[s];
    const int a = id[st.a], b = id[st.b];
    if (a < 0 || b < 0) {  // merging with a scalar: the scalar stays a final factor
      id[L + s] = a < 0 ? b : a;
      continue;
    }
    PathStep ns;
    ns.a = a;
    ns.b = b;
    for (int x : st.out)
      if (!is_cut(x)) ns.out.push_back(x);
    r.steps.push_back(ns);
    const int mine = next++;
    if (ns.out.empty()) {
      r.final_ids.push_back(mine);
      id[L + s] = -1;
    } else {
      id[L + s] = mine;
    }
  }
  for (int f : path.final_ids)
    if (id[f] >= 0 && std::find(r.final_ids.begin(), r.final_ids.end(), id[f]) == r.final_ids.end())
      r.final_ids.push_back(id[f]);
  evaluate_path(sliced, r, p);
  return r;
}

Path plan_greedy(const Network& net, const PlanParams& p, uint64_t seed, double temperature) {
  Rng rng(seed);
  const int L = static_cast<int>(net.leaf_labels.size());
  std::vector<Labels> ts;
  std::vector<char> alive(L, 1);
  std::vector<int> version(L, 0);
  for (auto& l : net.leaf_labels) ts.push_back(sorted(l));
  // label -> tensors carrying it (at most two)
  std::vector<std::array<int, 2>> owner(net.n_labels, {-1, -1});
  auto add_owner = [&](int lab, int t) {
    if (owner[lab][0] < 0) owner[lab][0] = t;
    else owner[lab][1] = t;
  };
  auto drop_owner = [&](int lab, int t) {
    if (owner[lab][0] == t) owner[lab][0] = owner[lab][1];
    else if (owner[lab][1] != t) return;
    owner[lab][1] = -1;
  };
  for (int t = 0; t < L; ++t)
    for (int lab : ts[t]) add_owner(lab, t);

  struct Cand {
    double key;
    int a, b, va, vb;
    bool operator<(const Cand& o) const { return key > o.key; }  // min-heap
  };
  std::priority_queue<Cand> pq;
  auto push_pair = [&](int a, int b) {
    int sh = 0;
    const Labels out = sym_diff(ts[a], ts[b], &sh);
    const double cost = std::ldexp(1.0, static_cast<int>(out.size())) -
                        std::ldexp(1.0, static_cast<int>(ts[a].size())) -
                        std::ldexp(1.0, static_cast<int>(ts[b].size()));
    double key = (cost >= 0 ? 1.0 : -1.0) * std::log2(1.0 + std::fabs(cost));
    if (temperature > 0) key -= temperature * rng.gumbel();
    pq.push({key, a, b, version[a], version[b]});
  };
  {
    std::unordered_set<uint64_t> seen;
    for (int lab = 0; lab < net.n_labels; ++lab) {
      const int a = owner[lab][0], b = owner[lab][1];
      if (a < 0 || b < 0) continue;
      const uint64_t key = (static_cast<uint64_t>(std::min(a, b)) << 32) | static_cast<uint32_t>(std::max(a, b));
      if (seen.insert(key).second) push_pair(std::min(a, b), std::max(a, b));
    }
  }

  Path path;
  while (!pq.empty()) {
    Cand c = pq.top();
    pq.pop();
    if (!alive[c.a] || !alive[c.b] || version[c.a] != c.va || version[c.b] != c.vb) continue;
    PathStep st;
    st.a = c.a;
    st.b = c.b;
    st.out = sym_diff(ts[c.a], ts[c.b], nullptr);
    for (int lab : ts[c.a]) drop_owner(lab, c.a);
    for (int lab : ts[c.b]) drop_owner(lab, c.b);
    alive[c.a] = alive[c.b] = 0;
    const int id = static_cast<int>(ts.size());
    ts.push_back(st.out);
    alive.push_back(1);
    version.push_back(0);
    for (int lab : st.out) add_owner(lab, id);
    path.steps.push_back(st);
    // new candidates: neighbours of the new tensor
    std::vector<int> nbs;
    for (int lab : ts[id]) {
      const int o = owner[lab][0] == id ? owner[lab][1] : owner[lab][0];
      if (o >= 0) nbs.push_back(o);
    }
    std::sort(nbs.begin(), nbs.end());
    nbs.erase(std::unique(nbs.begin(), nbs.end()), nbs.end());
    for (int o : nbs) push_pair(std::min(o, id), std::max(o, id));
  }
  finish_components(ts, alive, path);
  path.planner = AJF_PLANNER_GREEDY;
  evaluate_path(net, path, p);
  return path;
}

Path plan_minfill(const Network& net, const PlanParams& p, uint64_t seed) {
  Rng rng(seed);
  const int V = net.n_labels;
  const int W = (V + 63) / 64;
  std::vector<uint64_t> adj(static_cast<size_t>(V) * W, 0);
  auto row = [&](int v) { return adj.data() + static_cast<size_t>(v) * W; };
  auto has = [&](int u, int v) { return (row(u)[v >> 6] >> (v & 63)) & 1ull; };
  auto set_edge = [&](int u, int v) {
    row(u)[v >> 6] |= 1ull << (v & 63);
    row(v)[u >> 6] |= 1ull << (u & 63);
  };
  std::vector<char> present(V, 0), is_open(V, 0);
  for (int lab : net.open_labels) is_open[lab] = 1;
  for (auto& l : net.leaf_labels) {
    for (int x : l) present[x] = 1;
    for (size_t i = 0; i < l.size(); ++i)
      for (size_t j = i + 1; j < l.size(); ++j) set_edge(l[i], l[j]);
  }
  std::vector<std::vector<int>> nbr(V);
  auto refresh_nbr = [&](int v) {
    nbr[v].clear();
    const uint64_t* r = row(v);
    for (int w = 0; w < W; ++w) {
      uint64_t x = r[w];
      while (x) {
        const int b = __builtin_ctzll(x);
        nbr[v].push_back(w * 64 + b);
        x &= x - 1;
      }
    }
  };
  auto fill = [&](int v) {
    long f = 0;
    const auto& nb = nbr[v];
    for (size_t i = 0; i < nb.size(); ++i)
      for (size_t j = i + 1; j < nb.size(); ++j)
        if (!has(nb[i], nb[j])) ++f;
    return f;
  };
  std::vector<long> score(V, 0);
  std::vector<double> tie(V, 0);
  std::vector<char> alive(V, 0);
  int remaining = 0;
  for (int v = 0; v < V; ++v)
    if (present[v]) {
      refresh_nbr(v);
      alive[v] = 1;
      tie[v] = rng.uniform();
      if (!is_open[v]) ++remaining;
    }
  for (int v = 0; v < V; ++v)
    if (alive[v]) score[v] = fill(v);

  std::vector<int> order;
  order.reserve(remaining);
  std::vector<int> mark(V, -1);
  for (int it = 0; it < remaining; ++it) {
    int best = -1;
    for (int v = 0; v < V; ++v) {
      if (!alive[v] || is_open[v]) continue;
      if (best < 0 || score[v] < score[best] || (score[v] == score[best] && tie[v] < tie[best]))
        best = v;
    }
    const int v = best;
    const std::vector<int> nb = nbr[v];
    for (size_t i = 0; i < nb.size(); ++i)
      for (size_t j = i + 1; j < nb.size(); ++j) set_edge(nb[i], nb[j]);
    for (int u : nb) row(u)[v >> 6] &= ~(1ull << (v & 63));
    std::memset(row(v), 0, W * sizeof(uint64_t));
    alive[v] = 0;
    order.push_back(v);
    // neighbourhoods changed for nb; fill counts may change within two hops
    std::vector<int> touched;
    for (int u : nb) {
      refresh_nbr(u);
      if (mark[u] != it) { mark[u] = it; touched.push_back(u); }
    }
    for (int u : nb)
      for (int w : nbr[u])
        if (mark[w] != it) { mark[w] = it; touched.push_back(w); }
    for (int u : touched)
      if (alive[u]) score[u] = fill(u);
  }

  // Contract along the elimination order.
  const int L = static_cast<int>(net.leaf_labels.size());
  std::vector<Labels> ts;
  std::vector<char> talive(L, 1);
  for (auto& l : net.leaf_labels) ts.push_back(sorted(l));
  std::vector<std::array<int, 2>> owner(V, {-1, -1});
  auto add_owner = [&](int lab, int t) {
    if (owner[lab][0] < 0) owner[lab][0] = t;
    else owner[lab][1] = t;
  };
  auto drop_owner = [&](int lab, int t) {
    if (owner[lab][0] == t) owner[lab][0] = owner[lab][1];
    else if (owner[lab][1] != t) return;
    owner[lab][1] = -1;
  };
  for (int t = 0; t < L; ++t)
    for (int lab : ts[t]) add_owner(lab, t);
  Path path;
  for (int x : order) {
    const int a = owner[x][0], b = owner[x][1];
    if (a < 0 || b < 0) continue;
    PathStep st;
    st.a = std::min(a, b);
    st.b = std::max(a, b);
    st.out = sym_diff(ts[st.a], ts[st.b], nullptr);
    for (int lab : ts[st.a]) drop_owner(lab, st.a);
    for (int lab : ts[st.b]) drop_owner(lab, st.b);
    talive[st.a] = talive[st.b] = 0;
    const int id = static_cast<int>(ts.size());
    ts.push_back(st.out);
    talive.push_back(1);
    for (int lab : st.out) add_owner(lab, id);
    path.steps.push_back(st);
  }
  finish_components(ts, talive, path);
  path.planner = AJF_PLANNER_MINFILL;
  evaluate_path(net, path, p);
  return path;
}

// ---------------------------------------------------------------- subtree reconfiguration
//
// A path is a forest of binary merge trees. For a merge node v, cut its subtree at a frontier of
// up to kReconfInputs tensors (expanding the largest internal tensor first); every binary tree
// over those inputs computes the same tensor, out(v). Dynamic programming over subsets of the
// frontier finds the tree of least estimated time (the cost model of evaluate_path): the labels of
// the tensor made from a subset S are those of S's inputs that also occur in the rest of the
// frontier or in out(v). If it beats the current subtree, it replaces it. All merge nodes are
// visited, a few passes over the forest.
namespace {

constexpr int kReconfInputs = 8;
constexpr size_t kReconfCandidates = 16;  // candidate paths that get reconfigured (the best by estimate)
constexpr int kReconfPasses = 4;
constexpr int kReconfLabels = 512;
using LSet = std::bitset<kReconfLabels>;

struct Forest {
  int L = 0;
  std::vector<int> ca, cb;            // children (-1 for leaves)
  std::vector<Labels> lab;            // sorted labels of every node
  std::vector<int> roots;
};

Forest to_forest(const Network& net, const Path& path) {
  Forest f;
  f.L = static_cast<int>(net.leaf_labels.size());
  for (int i = 0; i < f.L; ++i) {
    f.ca.push_back(-1);
    f.cb.push_back(-1);
    f.lab.push_back(sorted(net.leaf_labels[i]));
  }
  for (auto& st : path.steps) {
    f.ca.push_back(st.a);
    f.cb.push_back(st.b);
    f.lab.push_back(sorted(st.out));
  }
  f.roots = path.final_ids;
  return f;
}

Path from_forest(const Forest& f) {
  Path out;
  std::vector<int> id(f.ca.size(), -1);
  for (int i = 0; i < f.L; ++i) id[i] = i;
  // post-order, iterative
  for (int r : f.roots) {
    std::vector<std::pair<int, bool>> stack{{r, false}};
    while (!stack.empty()) {
      auto [v, expanded] = stack.back();
      stack.pop_back();
      if (id[v] >= 0) continue;
      if (!expanded) {
        stack.push_back({v, true});
        stack.push_back({f.cb[v], false});
        stack.push_back({f.ca[v], false});
      } else {
        PathStep st;
        st.a = id[f.ca[v]];
        st.b = id[f.cb[v]];
        st.out = f.lab[v];
        id[v] = f.L + static_cast<int>(out.steps.size());
        out.steps.push_back(st);
      }
    }
    out.final_ids.push_back(id[r]);
  }
  return out;
}

// One reconfiguration of the subtree at merge node v; true if it was replaced by a cheaper one.
bool reconfigure_node(Forest& f, int v, const PlanParams& p) {
  // frontier: expand the internal node with the most labels until kReconfInputs inputs
  std::vector<int> front{f.ca[v], f.cb[v]};
  std::vector<int> inner{v};
  while (static_cast<int>(front.size()) < kReconfInputs) {
    int best = -1;
    for (int i = 0; i < static_cast<int>(front.size()); ++i)
      if (f.ca[front[i]] >= 0 && (best < 0 || f.lab[front[i]].size() > f.lab[front[best]].size())) best = i;
    if (best < 0) break;
    const int u = front[best];
    inner.push_back(u);
    front[best] = f.ca[u];
    front.push_back(f.cb[u]);
  }
  const int k = static_cast<int>(front.size());
  if (k < 3) return false;
  // current cost of the subtree between v and the frontier; every tree over k inputs has k - 1
  // merges, so only the work part can improve: skip subtrees with under a microsecond of it
  double cur = 0;
  for (int u : inner) {
    int sh = 0;
    const int ru = static_cast<int>(sym_diff(f.lab[f.ca[u]], f.lab[f.cb[u]], &sh).size()) + sh;
    cur += step_seconds(static_cast<int>(f.lab[f.ca[u]].size()), static_cast<int>(f.lab[f.cb[u]].size()), ru,
                        static_cast<int>(f.lab[u].size()), p);
  }
  if (cur < 1e-6 + 1e-6 * static_cast<double>(inner.size())) return false;
  // local label numbering
  std::unordered_map<int, int> local;
  auto loc = [&](int x) {
    auto it = local.find(x);
    if (it != local.end()) return it->second;
    const int n = static_cast<int>(local.size());
    local.emplace(x, n);
    return n;
  };
  std::vector<LSet> in(k);
  for (int i = 0; i < k; ++i)
    for (int x : f.lab[front[i]]) {
      const int l = loc(x);
      if (l >= kReconfLabels) return false;
      in[i].set(l);
    }
  LSet ext;
  for (int x : f.lab[v]) {
    auto it = local.find(x);
    if (it != local.end()) ext.set(it->second);
  }
  const int full = (1 << k) - 1;
  std::vector<LSet> uni(1 << k);
  for (int s = 1; s <= full; ++s) {
    const int low = s & -s;
    uni[s] = uni[s ^ low] | in[__builtin_ctz(low)];
  }
  std::vector<int> rank(1 << k);
  std::vector<LSet> tl(1 << k);
  for (int s = 1; s <= full; ++s) {
    tl[s] = uni[s] & (uni[full ^ s] | ext);
    rank[s] = static_cast<int>(tl[s].count());
  }
  std::vector<double> cost(1 << k, 0.0);
  std::vector<int> split(1 << k, 0);
  for (int s = 1; s <= full; ++s) {
    if ((s & (s - 1)) == 0) continue;  // single input
    const int low = s & -s;
    double best = std::numeric_limits<double>::infinity();
    int bsplit = 0;
    // s1 contains the lowest input of s; s2 = s ^ s1 nonempty
    for (int s1 = (s - 1) & s; s1 > 0; s1 = (s1 - 1) & s) {
      if (!(s1 & low)) continue;
      const int s2 = s ^ s1;
      const int ru = static_cast<int>((tl[s1] | tl[s2]).count());
      const double c = cost[s1] + cost[s2] + step_seconds(rank[s1], rank[s2], ru, rank[s], p);
      if (c < best) {
        best = c;
        bsplit = s1;
      }
    }
    cost[s] = best;
    split[s] = bsplit;
  }
  if (!(cost[full] < cur * (1.0 - 1e-9))) return false;
  // rebuild: the node for subset s (inputs are frontier nodes, v is the root)
  std::vector<int> label_of(local.size());
  for (auto& kv : local) label_of[kv.second] = kv.first;
  std::function<int(int)> build = [&](int s) -> int {
    if ((s & (s - 1)) == 0) return front[__builtin_ctz(s)];
    const int a = build(split[s]), b = build(s ^ split[s]);
    if (s == full) {
      f.ca[v] = a;
      f.cb[v] = b;
      return v;
    }
    Labels lb;
    for (size_t i = 0; i < label_of.size(); ++i)
      if (tl[s].test(i)) lb.push_back(label_of[i]);
    std::sort(lb.begin(), lb.end());
    f.ca.push_back(a);
    f.cb.push_back(b);
    f.lab.push_back(lb);
    return static_cast<int>(f.ca.size()) - 1;
  };
  build(full);
  return true;
}

}  // namespace

Path reconfigure_path(const Network& net, const Path& path, const PlanParams& p, int passes) {
  Forest f = to_forest(net, path);
  for (int pass = 0; pass < passes; ++pass) {
    bool changed = false;
    // visit merge nodes reachable from the roots, largest tensors first
    Path cur = from_forest(f);
    Forest g = to_forest(net, cur);
    std::vector<int> order;
    for (int v = g.L; v < static_cast<int>(g.ca.size()); ++v) order.push_back(v);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return g.lab[x].size() > g.lab[y].size(); });
    for (int v : order) changed |= reconfigure_node(g, v, p);
    f = std::move(g);
    if (!changed) break;
  }
  Path out = from_forest(f);
  out.planner = path.planner;
  evaluate_path(net, out, p);
  return out;
}

Path plan_path(const Network& net, const PlanParams& p) {
  const int trials = std::max(1, p.trials);
  Path best;
  bool have = false;
  auto consider = [&](Path&& cand) {
    if (!have || cand.est_seconds < best.est_seconds ||
        (cand.est_seconds == best.est_seconds && cand.cmacs < best.cmacs)) {
      best = std::move(cand);
      have = true;
    }
  };
  if (net.leaf_labels.empty()) {
    Path empty;
    empty.planner = p.planner;
    return empty;
  }
  std::vector<Path> cands;
  if (p.planner == AJF_PLANNER_LEARNED) {
    bool used = false;
    PlanParams q = p;
    for (int t = 0; t < trials; ++t) {
      q.learned_noise = t == 0 ? 0.0 : 0.25;
      cands.push_back(plan_learned(net, q, p.seed * 1000003ull + static_cast<uint64_t>(t), &used));
      if (!used) break;  // no model: plan_learned returned the greedy path
    }
    // the greedy planner judges: keep the learned path only if it is no worse
    cands.push_back(plan_greedy(net, p, p.seed, 0.0));
  } else {
    // restarts of both planners
    const bool do_greedy = p.planner == AJF_PLANNER_AUTO || p.planner == AJF_PLANNER_GREEDY;
    const bool do_minfill = p.planner == AJF_PLANNER_AUTO || p.planner == AJF_PLANNER_MINFILL;
    for (int t = 0; t < trials; ++t) {
      const uint64_t s = p.seed * 1000003ull + static_cast<uint64_t>(t);
      if (do_greedy) cands.push_back(plan_greedy(net, p, s, t == 0 ? 0.0 : (t % 3 == 1 ? 0.5 : 1.0)));
      if (do_minfill) cands.push_back(plan_minfill(net, p, s));
    }
  }
  // the best candidates are improved by subtree reconfiguration (the cheapest order of every
  // small subtree); the best path by estimated time is kept
  std::stable_sort(cands.begin(), cands.end(), [](const Path& x, const Path& y) {
    return x.est_seconds < y.est_seconds || (x.est_seconds == y.est_seconds && x.cmacs < y.cmacs);
  });
  const size_t top = std::min<size_t>(cands.size(), kReconfCandidates);
  for (size_t i = 0; i < top; ++i) consider(reconfigure_path(net, cands[i], p, kReconfPasses));
  for (auto& c : cands) consider(std::move(c));
  return best;
}

}  // namespace ajf
