// Miter-network builders (host side).
//
// Sec. IV (Fig. 3): the trace of a circuit's matrix is its gate network with every qubit's
// output wire joined to its input wire. Both builders walk the composed sequence (the noisy
// implementation in time order, then the ideal circuit's adjoint; see simplify.cpp) and close the
// wires -- output wire w to input wire closure[w], the identity unless SWAPs were eliminated.
//
// Alg. I (Sec. IV-A): one wire per qubit. Noisy gate k becomes one tensor holding all of its Kraus
// operators, indexed by an extra open index kappa_k (padded to a power of two with zero
// operators), so a single contraction yields t[kappa_1..kappa_m] = tr(U^dagger E_kappa) for every
// combination -- the enumeration of Alg. I done as one network whose noise-independent parts are
// contracted once (the role the shared computed table plays in Sec. IV-C).
//
// Alg. II (Sec. IV-B, steps 1-4): wires q and q' (numbered q + n). Gate V becomes V on q and V^*
// on q'; noisy gate {N_k} becomes M_N = sum_k N_k (x) N_k^* on (q..., q'...); the adjoint of the
// doubled ideal circuit puts V^dagger on q and V^T = (V^dagger)^* on q'.
//
// Tensor bit layout of a leaf on wires w_0..w_{a-1} (w_0 most significant): element index =
// row * 2^a + col of the operator matrix, so bit i < a is the input label of wire w_{a-1-i} and
// bit a + i is the output label of wire w_{a-1-i}; Kraus-index bits (Alg. I) sit above them.
#include <algorithm>
#include <map>

#include "ajf_internal.h"

namespace ajf {
namespace {

struct Builder {
  Network& net;
  std::vector<int> start, cur, nops;

  Builder(Network& n, int wires) : net(n), start(wires), cur(wires), nops(wires, 0) {
    for (int w = 0; w < wires; ++w) start[w] = cur[w] = net.n_labels++;
  }

  int new_label() { return net.n_labels++; }

  // Adds a leaf acting on `wires`; returns the labels of its extra (Kraus) bits.
  std::vector<int> op(const LeafSpec& spec, const std::vector<int>& wires, int extra_bits) {
    const int a = static_cast<int>(wires.size());
    std::vector<int> labels(2 * a + extra_bits);
    for (int i = 0; i < a; ++i) {
      const int w = wires[a - 1 - i];
      labels[i] = cur[w];
      const int o = new_label();
      labels[a + i] = o;
    }
    for (int i = 0; i < a; ++i) {
      const int w = wires[a - 1 - i];
      cur[w] = labels[a + i];
      nops[w]++;
    }
    std::vector<int> extra;
    for (int e = 0; e < extra_bits; ++e) {
      labels[2 * a + e] = new_label();
      extra.push_back(labels[2 * a + e]);
    }
    net.leaf_labels.push_back(std::move(labels));
    net.leaf_specs.push_back(spec);
    return extra;
  }

  // Join each wire's last label to the first label of wire closure[w]. A wire closed on itself
  // with one operation would make that leaf carry the same label twice, and a permuted closure
  // could join a leaf's output to its own input: an identity leaf delta[last][first] keeps labels
  // pairwise in both cases (a permuted closure always joins through one).
  void close(const std::vector<int>& closure) {
    std::map<int, int> rename;
    std::vector<std::pair<int, int>> deltas;
    for (size_t w = 0; w < start.size(); ++w) {
      const size_t to = static_cast<size_t>(closure[w]);
      if (to != w) {
        deltas.push_back({cur[w], start[to]});
      } else if (nops[w] == 0) {
        net.loops++;
      } else if (nops[w] == 1) {
        deltas.push_back({cur[w], start[w]});
      } else {
        rename[cur[w]] = start[w];
      }
    }
    for (auto& labels : net.leaf_labels)
      for (auto& x : labels) {
        auto it = rename.find(x);
        if (it != rename.end()) x = it->second;
      }
    for (auto& d : deltas) {
      LeafSpec s;
      s.kind = LEAF_IDENTITY;
      s.a = 1;
      net.leaf_labels.push_back({d.first, d.second});
      net.leaf_specs.push_back(s);
    }
  }
};

std::vector<int> op_wires(const SeqOp& op, int offset) {
  std::vector<int> w(op.arity);
  for (int i = 0; i < op.arity; ++i) w[i] = op.w[i] + offset;
  return w;
}

LeafSpec gate_spec(const GateIn& g, int kind) {
  LeafSpec s;
  s.kind = kind;
  s.a = g.arity;
  s.src = g.mat_off;
  return s;
}

}  // namespace

Network build_alg1(const Inputs& in, const Sequence& seq, const std::vector<char>& sliced) {
  Network net;
  net.alg = 1;
  net.n_qubits = in.n;
  net.noise_leaf.assign(in.noises.size(), -1);
  Builder b(net, in.n);
  std::vector<std::vector<int>> kappa(in.noises.size());
  const auto& sk = in.skeleton();
  for (const SeqOp& op : seq.ops) {
    if (op.kind == SEQ_GATE) {
      b.op(gate_spec(sk[op.index], LEAF_GATE), op_wires(op, 0), 0);
    } else if (op.kind == SEQ_ADJ) {
      b.op(gate_spec(in.ideal[op.index], LEAF_GATE_DAG), op_wires(op, 0), 0);
    } else {
      const NoiseIn& nz = in.noises[op.index];
      const bool fixed = !sliced.empty() && sliced[op.index];
      LeafSpec s;
      s.kind = LEAF_KRAUS_OPEN;
      s.a = nz.arity;
      s.src = nz.kraus_off;
      s.nk = fixed ? 1 : nz.nk;
      s.kbits = fixed ? 0 : nz.kbits;
      net.noise_leaf[op.index] = static_cast<int>(net.leaf_specs.size());
      kappa[op.index] = b.op(s, op_wires(op, 0), s.kbits);
    }
  }
  b.close(seq.closure);
  // Result layout: the last-added noise's Kraus index in the lowest bits, so the linear index of
  // t follows Alg. I's lexicographic enumeration (after removing the zero padding).
  for (int j = static_cast<int>(in.noises.size()) - 1; j >= 0; --j)
    for (int lab : kappa[j]) net.open_labels.push_back(lab);
  return net;
}

Network build_alg2(const Inputs& in, const Sequence& seq) {
  Network net;
  net.alg = 2;
  net.n_qubits = in.n;
  const int n = in.n;
  Builder b(net, 2 * n);
  const auto& sk = in.skeleton();
  for (const SeqOp& op : seq.ops) {
    if (op.kind == SEQ_GATE) {
      b.op(gate_spec(sk[op.index], LEAF_GATE), op_wires(op, 0), 0);
      b.op(gate_spec(sk[op.index], LEAF_GATE_CONJ), op_wires(op, n), 0);
    } else if (op.kind == SEQ_ADJ) {
      b.op(gate_spec(in.ideal[op.index], LEAF_GATE_DAG), op_wires(op, 0), 0);
      b.op(gate_spec(in.ideal[op.index], LEAF_GATE_TRANS), op_wires(op, n), 0);
    } else {
      const NoiseIn& nz = in.noises[op.index];
      LeafSpec s;
      s.kind = LEAF_SUPEROP;
      s.a = 2 * nz.arity;
      s.src = nz.kraus_off;
      s.nk = nz.nk;
      std::vector<int> w = op_wires(op, 0);
      for (int i = 0; i < op.arity; ++i) w.push_back(op.w[i] + n);
      b.op(s, w, 0);
    }
  }
  // the q' wires close like their q wires
  std::vector<int> closure(2 * n);
  for (int w = 0; w < n; ++w) {
    closure[w] = seq.closure[w];
    closure[w + n] = seq.closure[w] + n;
  }
  b.close(closure);
  return net;
}

}  // namespace ajf
