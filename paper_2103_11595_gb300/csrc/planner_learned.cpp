// Learned merge scorer: planning with an MLP that scores candidate pairwise merges, and the
// training data that teaches it (host side; the MLP's kernels are in mlp.cu).
//
// The planner state is the set of tensors (label sets). A candidate is a pair of tensors sharing a
// label. When a candidate appears (at the start, or when a merge creates a tensor) it is described
// by 16 features of its operands, its result and the state (below) and scored once; the planner
// then repeatedly performs the best-scored live candidate. Training data comes from replaying a
// reference path -- the best path the greedy and min-fill planners find with restarts -- through
// the same bookkeeping: at every step the reference merge is paired with up to eight other live
// candidates, and the MLP learns to rank it first (mlp.cu). The greedy planner stays the fallback
// (no model loaded) and the judge (plan_path keeps the learned path only if it is no worse).
#include <algorithm>
#include <array>
#include <cmath>
#include <queue>
#include <unordered_set>

#include "ajf_internal.h"
#include "mlp.h"

namespace ajf {
namespace {

using Labels = std::vector<int>;

struct SplitMix {
  uint64_t s;
  explicit SplitMix(uint64_t seed) : s(seed * 0x9E3779B97F4A7C15ull + 77) {}
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
};

Labels sym_diff(const Labels& a, const Labels& b, int* shared) {
  Labels out;
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

// Network state with label ownership and per-tensor neighbour counts.
struct State {
  std::vector<Labels> ts;
  std::vector<char> alive;
  std::vector<std::array<int, 2>> owner;
  std::vector<char> open;
  int n_leaves = 0, steps = 0, total = 1, maxw = 0;

  explicit State(const Network& net) {
    n_leaves = static_cast<int>(net.leaf_labels.size());
    owner.assign(net.n_labels, {-1, -1});
    open.assign(net.n_labels, 0);
    for (int x : net.open_labels) open[x] = 1;
    for (auto& l : net.leaf_labels) {
      Labels s = l;
      std::sort(s.begin(), s.end());
      const int id = static_cast<int>(ts.size());
      ts.push_back(s);
      alive.push_back(1);
      for (int x : s) add_owner(x, id);
      maxw = std::max(maxw, static_cast<int>(s.size()));
    }
    total = std::max(1, n_leaves - 1);
  }
  void add_owner(int x, int t) {
    if (owner[x][0] < 0) owner[x][0] = t;
    else owner[x][1] = t;
  }
  void drop_owner(int x, int t) {
    if (owner[x][0] == t) owner[x][0] = owner[x][1];
    else if (owner[x][1] != t) return;
    owner[x][1] = -1;
  }
  std::vector<int> neighbours(int t) const {
    std::vector<int> nb;
    for (int x : ts[t]) {
      const int o = owner[x][0] == t ? owner[x][1] : owner[x][0];
      if (o >= 0) nb.push_back(o);
    }
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    return nb;
  }
  int merge(int a, int b) {
    Labels out = sym_diff(ts[a], ts[b], nullptr);
    for (int x : ts[a]) drop_owner(x, a);
    for (int x : ts[b]) drop_owner(x, b);
    alive[a] = alive[b] = 0;
    const int id = static_cast<int>(ts.size());
    for (int x : out) add_owner(x, id);
    maxw = std::max(maxw, static_cast<int>(out.size()));
    ts.push_back(std::move(out));
    alive.push_back(1);
    ++steps;
    return id;
  }
  // 16 features of merging a and b in the current state (the larger operand first).
  void features(int a, int b, float* f) const {
    if (ts[a].size() < ts[b].size() || (ts[a].size() == ts[b].size() && a > b)) std::swap(a, b);
    int sh = 0;
    const Labels out = sym_diff(ts[a], ts[b], &sh);
    const double ra = static_cast<double>(ts[a].size()), rb = static_cast<double>(ts[b].size());
    const double ro = static_cast<double>(out.size());
    int n_open = 0;
    for (int x : out) n_open += open[x];
    const double cost = std::ldexp(1.0, static_cast<int>(ro)) - std::ldexp(1.0, static_cast<int>(ra)) -
                        std::ldexp(1.0, static_cast<int>(rb));
    const double lc = (cost >= 0 ? 1.0 : -1.0) * std::log2(1.0 + std::fabs(cost));
    f[0] = static_cast<float>(ra / 32);
    f[1] = static_cast<float>(rb / 32);
    f[2] = static_cast<float>(ro / 32);
    f[3] = static_cast<float>(sh / 16.0);
    f[4] = static_cast<float>((ro - ra) / 16);
    f[5] = static_cast<float>((ra + rb - sh) / 48);
    f[6] = static_cast<float>(neighbours(a).size() / 16.0);
    f[7] = static_cast<float>(neighbours(b).size() / 16.0);
    f[8] = a < n_leaves ? 1.f : 0.f;
    f[9] = b < n_leaves ? 1.f : 0.f;
    f[10] = static_cast<float>(static_cast<double>(steps) / total);
    f[11] = static_cast<float>(n_open / 16.0);
    f[12] = static_cast<float>(maxw / 32.0);
    f[13] = static_cast<float>((ro - maxw) / 16);
    f[14] = static_cast<float>(lc / 32);
    f[15] = static_cast<float>((ra - rb) / 32);
  }
};

struct Cand {
  double key;
  int a, b;
  bool operator<(const Cand& o) const { return key < o.key; }  // max-heap
};

std::vector<std::pair<int, int>> initial_pairs(const State& s) {
  std::vector<std::pair<int, int>> out;
  std::unordered_set<uint64_t> seen;
  for (const auto& ow : s.owner) {
    if (ow[0] < 0 || ow[1] < 0) continue;
    const int a = std::min(ow[0], ow[1]), b = std::max(ow[0], ow[1]);
    if (seen.insert((uint64_t(a) << 32) | uint32_t(b)).second) out.push_back({a, b});
  }
  return out;
}

void finish(State& s, Path& path) {
  std::vector<int> open_ids;
  for (size_t i = 0; i < s.ts.size(); ++i)
    if (s.alive[i]) {
      if (s.ts[i].empty()) path.final_ids.push_back(static_cast<int>(i));
      else open_ids.push_back(static_cast<int>(i));
    }
  while (open_ids.size() > 1) {
    std::sort(open_ids.begin(), open_ids.end(), [&](int x, int y) { return s.ts[x].size() < s.ts[y].size(); });
    const int a = open_ids[0], b = open_ids[1];
    PathStep st;
    st.a = a;
    st.b = b;
    st.out = sym_diff(s.ts[a], s.ts[b], nullptr);
    s.merge(a, b);
    path.steps.push_back(st);
    open_ids.erase(open_ids.begin(), open_ids.begin() + 2);
    open_ids.push_back(static_cast<int>(s.ts.size()) - 1);
  }
  if (!open_ids.empty()) path.final_ids.push_back(open_ids[0]);
}

}  // namespace

Path plan_learned(const Network& net, const PlanParams& p, uint64_t seed, bool* used) {
  if (!p.mlp || !p.scorer) {
    if (used) *used = false;
    return plan_greedy(net, p, seed, 0.0);
  }
  if (used) *used = true;
  SplitMix rng(seed);
  State s(net);
  std::priority_queue<Cand> pq;
  std::vector<float> feats;
  std::vector<float> scores;
  auto push_scored = [&](const std::vector<std::pair<int, int>>& pairs) {
    if (pairs.empty()) return;
    feats.resize(pairs.size() * kMlpFeatures);
    scores.resize(pairs.size());
    for (size_t i = 0; i < pairs.size(); ++i) s.features(pairs[i].first, pairs[i].second, &feats[i * kMlpFeatures]);
    p.scorer(p.mlp, feats.data(), static_cast<int>(pairs.size()), scores.data());
    for (size_t i = 0; i < pairs.size(); ++i) {
      double key = scores[i];
      if (p.learned_noise > 0) key += p.learned_noise * -std::log(-std::log(rng.uniform()));
      pq.push({key, pairs[i].first, pairs[i].second});
    }
  };
  push_scored(initial_pairs(s));
  Path path;
  while (!pq.empty()) {
    const Cand c = pq.top();
    pq.pop();
    if (!s.alive[c.a] || !s.alive[c.b]) continue;
    PathStep st;
    st.a = c.a;
    st.b = c.b;
    st.out = sym_diff(s.ts[c.a], s.ts[c.b], nullptr);
    const int id = s.merge(c.a, c.b);
    path.steps.push_back(st);
    std::vector<std::pair<int, int>> fresh;
    for (int o : s.neighbours(id)) fresh.push_back({std::min(o, id), std::max(o, id)});
    push_scored(fresh);
  }
  finish(s, path);
  path.planner = AJF_PLANNER_LEARNED;
  evaluate_path(net, path, p);
  return path;
}

int learned_dataset(const Network& net, const Path& ref, uint64_t seed, int negatives, std::vector<float>& out) {
  SplitMix rng(seed);
  State s(net);
  // live candidates with their creation-time features
  struct Live {
    int a, b;
    std::array<float, kMlpFeatures> f;
  };
  std::vector<Live> live;
  auto add = [&](int a, int b) {
    Live l;
    l.a = std::min(a, b);
    l.b = std::max(a, b);
    s.features(l.a, l.b, l.f.data());
    live.push_back(l);
  };
  for (auto& pr : initial_pairs(s)) add(pr.first, pr.second);
  int emitted = 0;
  for (const PathStep& st : ref.steps) {
    const int a = std::min(st.a, st.b), b = std::max(st.a, st.b);
    if (a >= static_cast<int>(s.ts.size()) || b >= static_cast<int>(s.ts.size()) || !s.alive[a] || !s.alive[b]) break;
    // drop dead candidates
    live.erase(std::remove_if(live.begin(), live.end(), [&](const Live& l) { return !s.alive[l.a] || !s.alive[l.b]; }),
               live.end());
    int chosen = -1;
    for (size_t i = 0; i < live.size(); ++i)
      if (live[i].a == a && live[i].b == b) chosen = static_cast<int>(i);
    if (chosen >= 0 && live.size() > 1) {
      for (int k = 0; k < negatives; ++k) {
        int o = static_cast<int>(rng.next() % live.size());
        if (o == chosen) continue;
        out.insert(out.end(), live[chosen].f.begin(), live[chosen].f.end());
        out.insert(out.end(), live[o].f.begin(), live[o].f.end());
        ++emitted;
      }
    }
    const int id = s.merge(a, b);
    for (int o : s.neighbours(id)) add(o, id);
  }
  return emitted;
}

}  // namespace ajf
