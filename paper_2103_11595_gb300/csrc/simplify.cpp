// The closed composed sequence of a miter and its two local simplifications (Sec. IV-C).
//
// Both miters contract the trace of one operator sequence: the noisy implementation in time
// order (noises placed after gate g follow g; after = -1 comes first), then the ideal circuit's
// adjoint (gates in reverse order, each conjugate-transposed), with every output wire joined to
// an input wire. Alg. II doubles each element of the same sequence (V on q and V^* on q'; a noise
// becomes M_N), so a simplification of the sequence serves both algorithms.
//
// "SWAP elimination" (Sec. IV-C): a SWAP gate on wires (x, y) is dropped and every later element
// has x and y exchanged; what the SWAP did is then done by the closure, which joins output wire x
// to the input wire that y led to and vice versa. With several SWAPs the closure is the product of
// their transpositions (the first SWAP's applied last): closure[w] = input wire joined to output w.
//
// "Local optimisations" (Sec. IV-C): two unitary elements A (earlier) and B (later) on the same
// ordered wires, with nothing in between acting on any of those wires, are removed when
// B . A = I. Under the trace the sequence is cyclic, so the search for B continues past the end of
// the sequence into its beginning ("both ends of the composed circuit"), the wires passing through
// the closure. Single elements equal to the identity are removed too. Noise elements are not
// unitary and are never removed; they block cancellation across them on their wires.
//
// A matrix counts as the identity (or SWAP) when every entry is within 1e-12 of it: exact inverse
// pairs such as H . H or V^dagger . V of the same packed matrix differ by rounding only.
#include <cmath>
#include <complex>

#include "ajf_internal.h"

namespace ajf {
namespace {

using cd = std::complex<double>;
constexpr double kIdentityTol = 1e-12;

// The operator of a unitary element (row-major 2^a x 2^a; first listed wire most significant).
std::vector<cd> element_matrix(const Inputs& in, const SeqOp& op) {
  const GateIn& g = op.kind == SEQ_GATE ? in.skeleton()[op.index] : in.ideal[op.index];
  const int d = 1 << g.arity;
  std::vector<cd> m(static_cast<size_t>(d) * d);
  const double* p = in.packed.data() + 2 * g.mat_off;
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) {
      const cd v(p[2 * (r * d + c)], p[2 * (r * d + c) + 1]);
      if (op.kind == SEQ_GATE)
        m[r * d + c] = v;
      else
        m[c * d + r] = std::conj(v);  // adjoint
    }
  return m;
}

bool near(const std::vector<cd>& m, const std::vector<cd>& ref) {
  for (size_t i = 0; i < m.size(); ++i)
    if (std::abs(m[i] - ref[i]) > kIdentityTol) return false;
  return true;
}

std::vector<cd> identity(int d) {
  std::vector<cd> m(static_cast<size_t>(d) * d, 0.0);
  for (int i = 0; i < d; ++i) m[i * d + i] = 1.0;
  return m;
}

bool is_swap(const std::vector<cd>& m) {
  std::vector<cd> s(16, 0.0);
  s[0 * 4 + 0] = s[1 * 4 + 2] = s[2 * 4 + 1] = s[3 * 4 + 3] = 1.0;
  return near(m, s);
}

// B . A for d x d matrices.
std::vector<cd> product(const std::vector<cd>& b, const std::vector<cd>& a, int d) {
  std::vector<cd> m(static_cast<size_t>(d) * d, 0.0);
  for (int r = 0; r < d; ++r)
    for (int k = 0; k < d; ++k)
      for (int c = 0; c < d; ++c) m[r * d + c] += b[r * d + k] * a[k * d + c];
  return m;
}

bool touches(const SeqOp& op, const std::vector<int>& wires) {
  for (int i = 0; i < op.arity; ++i)
    for (int w : wires)
      if (op.w[i] == w) return true;
  return false;
}

bool unitary(const SeqOp& op) { return op.kind != SEQ_NOISE; }

}  // namespace

Sequence compose_sequence(const Inputs& in, int flags) {
  Sequence s;
  s.closure.resize(in.n);
  for (int w = 0; w < in.n; ++w) s.closure[w] = w;
  auto add_gate = [&](int kind, int index, const GateIn& g) {
    SeqOp op;
    op.kind = kind;
    op.index = index;
    op.arity = g.arity;
    for (int i = 0; i < 3; ++i) op.w[i] = g.q[i];
    s.ops.push_back(op);
  };
  const auto& sk = in.skeleton();
  auto add_noise = [&](int j) {
    SeqOp op;
    op.kind = SEQ_NOISE;
    op.index = j;
    op.arity = in.noises[j].arity;
    for (int i = 0; i < 3; ++i) op.w[i] = in.noises[j].q[i];
    s.ops.push_back(op);
  };
  for (size_t j = 0; j < in.noises.size(); ++j)
    if (in.noises[j].after < 0) add_noise(static_cast<int>(j));
  for (size_t g = 0; g < sk.size(); ++g) {
    add_gate(SEQ_GATE, static_cast<int>(g), sk[g]);
    for (size_t j = 0; j < in.noises.size(); ++j)
      if (in.noises[j].after == static_cast<int>(g)) add_noise(static_cast<int>(j));
  }
  for (int g = static_cast<int>(in.ideal.size()) - 1; g >= 0; --g) add_gate(SEQ_ADJ, g, in.ideal[g]);
  if (!(flags & (AJF_SIMPLIFY_SWAP | AJF_SIMPLIFY_CANCEL))) return s;

  const Sequence original = s;
  std::vector<char> alive(s.ops.size(), 1);
  if (flags & AJF_SIMPLIFY_SWAP) {
    for (size_t t = 0; t < s.ops.size(); ++t) {
      const SeqOp& op = s.ops[t];
      if (!unitary(op) || op.arity != 2 || !is_swap(element_matrix(in, op))) continue;
      const int x = op.w[0], y = op.w[1];
      alive[t] = 0;
      for (size_t u = t + 1; u < s.ops.size(); ++u)
        for (int i = 0; i < s.ops[u].arity; ++i) {
          if (s.ops[u].w[i] == x)
            s.ops[u].w[i] = y;
          else if (s.ops[u].w[i] == y)
            s.ops[u].w[i] = x;
        }
      std::swap(s.closure[x], s.closure[y]);  // closure := closure o (x y)
    }
  }
  if (flags & AJF_SIMPLIFY_CANCEL) {
    const int n_ops = static_cast<int>(s.ops.size());
    for (int i = 0; i < n_ops; ++i)
      if (alive[i] && unitary(s.ops[i]) && near(element_matrix(in, s.ops[i]), identity(1 << s.ops[i].arity)))
        alive[i] = 0;
    bool changed = true;
    while (changed) {
      changed = false;
      for (int i = 0; i < n_ops; ++i) {
        if (!alive[i] || !unitary(s.ops[i])) continue;
        const SeqOp& a = s.ops[i];
        std::vector<int> wires(a.w, a.w + a.arity);
        bool wrapped = false;
        int j = i + 1;
        for (;;) {
          if (j == n_ops) {
            if (wrapped) break;
            wrapped = true;
            j = 0;
            for (int& w : wires) w = s.closure[w];  // continue through the closure
          }
          if (j == i) break;  // all the way round: nothing else on these wires
          if (alive[j] && touches(s.ops[j], wires)) {
            const SeqOp& b = s.ops[j];
            bool same = unitary(b) && b.arity == a.arity;
            for (int k = 0; same && k < a.arity; ++k) same = b.w[k] == wires[k];
            if (same) {
              const int d = 1 << a.arity;
              if (near(product(element_matrix(in, b), element_matrix(in, a), d), identity(d))) {
                alive[i] = alive[j] = 0;
                changed = true;
              }
            }
            break;
          }
          ++j;
        }
      }
    }
  }
  std::vector<SeqOp> kept;
  for (size_t t = 0; t < s.ops.size(); ++t)
    if (alive[t]) kept.push_back(s.ops[t]);
  if (kept.empty()) return original;  // keep a network to contract (a noiseless, fully cancelled pair)
  s.removed = static_cast<int>(s.ops.size() - kept.size());
  s.ops = std::move(kept);
  return s;
}

}  // namespace ajf
