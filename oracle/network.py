"""O2: Alg. I and Alg. II as closed miter tensor networks, contracted on the CPU (test infrastructure).

Sec. IV (Fig. 3): the trace of a circuit's matrix is the tensor network of its gates with every
output wire joined to the input wire of the same qubit.

Alg. I (Sec. IV-A): for one Kraus choice (j_1..j_m), the network is the implementation with noisy
gate k replaced by N^k_{j_k}, followed by U^dagger -- every ideal gate replaced by its Hermitian
conjugate, in reverse order -- with all n wires closed. Contracting it gives tr(U^dagger E_i);
F_J accumulates |tr|^2 over all choices.

Alg. II (Sec. IV-B), in the paper's four steps:
  1. each qubit q gets an auxiliary qubit q';
  2. every unitary gate V on q_{j1..jl} of the ideal circuit gets a copy V^* on q'_{j1..jl};
  3. the implementation is treated the same way, and every noisy gate {N_k} on q_{j1..jl}
     becomes one tensor M_N = sum_k N_k (x) N_k^* on (q_{j1..jl}, q'_{j1..jl});
  4. the doubled implementation is followed by the adjoint of the doubled ideal circuit
     (V^dagger on q, V^T on q', in reverse order) and all 2n wires are closed.
Contracting it gives sum_i |tr(U^dagger E_i)|^2 in one network.

Contraction: numpy.tensordot, one pair at a time, in one of three orders:
  "greedy"  -- the pair sharing a wire whose result has the fewest indices goes first;
  "random"  -- any pair sharing a wire (order-invariance tests);
  "minfill" -- Sec. IV-C orders the contraction by a tree decomposition of the network's line
               graph (a vertex per wire, an edge between wires of one tensor). Here the
               decomposition comes from min-fill elimination (fewest fill edges first, ties broken
               by a seeded random draw, best of a few draws by contraction cost); wires are then
               contracted in elimination order.
A wire that no tensor touches is a closed loop and contributes a factor tr(I_2) = 2.
All arithmetic is complex128.
"""
from __future__ import annotations

import math

import numpy as np

from .dense import combinations, timeline


class _Builder:
    def __init__(self, n_wires: int):
        self.next_label = 0
        self.tensors = []  # list of [array, labels]
        self.start = [self.new() for _ in range(n_wires)]
        self.cur = list(self.start)

    def new(self) -> int:
        self.next_label += 1
        return self.next_label - 1

    def op(self, mat: np.ndarray, wires) -> None:
        """Add a tensor T[out_1..out_a, in_1..in_a] = mat[out, in] on the given wires."""
        a = len(wires)
        outs = [self.new() for _ in wires]
        ins = [self.cur[w] for w in wires]
        self.tensors.append([np.asarray(mat, dtype=np.complex128).reshape((2,) * (2 * a)),
                             outs + ins])
        for w, o in zip(wires, outs):
            self.cur[w] = o

    def close(self):
        """Join every wire's last label to its first (the trace); returns (tensors, loops)."""
        loops = 0
        rename = {}
        for w, (s, c) in enumerate(zip(self.start, self.cur)):
            if s == c:
                loops += 1
            else:
                rename[c] = s
        out = []
        for arr, labels in self.tensors:
            labels = [rename.get(x, x) for x in labels]
            arr, labels = _self_trace(arr, labels)
            out.append((arr, labels))
        return out, loops


def _self_trace(arr, labels):
    """Sum over labels that occur twice in one tensor (a gate whose own output closes onto its
    own input)."""
    while True:
        seen = {}
        dup = None
        for i, x in enumerate(labels):
            if x in seen:
                dup = (seen[x], i)
                break
            seen[x] = i
        if dup is None:
            return arr, labels
        i, j = dup
        arr = np.trace(arr, axis1=i, axis2=j)
        labels = [x for k, x in enumerate(labels) if k not in (i, j)]


def alg1_network(inst, choice):
    """Closed single-layer miter for one Kraus choice (Sec. IV-A, Fig. 4)."""
    b = _Builder(inst.n)
    for kind, idx in timeline(inst):
        if kind == "gate":
            g = inst.skeleton[idx]
            b.op(g.mat, g.qubits)
        else:
            nz = inst.noises[idx]
            b.op(nz.kraus[choice[idx]], nz.qubits)
    for g in reversed(inst.ideal):
        b.op(np.conj(g.mat).T, g.qubits)
    return b.close()


def alg2_network(inst):
    """Closed doubled miter (Sec. IV-B steps 1-4, Fig. 5). Wire q' is numbered q + n."""
    n = inst.n
    b = _Builder(2 * n)
    for kind, idx in timeline(inst):
        if kind == "gate":
            g = inst.skeleton[idx]
            b.op(g.mat, g.qubits)
            b.op(np.conj(g.mat), [q + n for q in g.qubits])
        else:
            nz = inst.noises[idx]
            MN = sum(np.kron(K, np.conj(K)) for K in nz.kraus)
            b.op(MN, list(nz.qubits) + [q + n for q in nz.qubits])
    for g in reversed(inst.ideal):
        gd = np.conj(g.mat).T
        b.op(gd, g.qubits)
        b.op(np.conj(gd), [q + n for q in g.qubits])
    return b.close()


def _line_graph(tensors):
    adj = {}
    for _, labels in tensors:
        for x in labels:
            adj.setdefault(x, set())
        for x in labels:
            for y in labels:
                if x != y:
                    adj[x].add(y)
    return adj


def _fill(adj, v):
    nb = list(adj[v])
    c = 0
    for i in range(len(nb)):
        ai = adj[nb[i]]
        for j in range(i + 1, len(nb)):
            if nb[j] not in ai:
                c += 1
    return c


def minfill_order(tensors, rng=None):
    """Min-fill elimination order of the line graph's vertices (wires)."""
    adj = {x: set(s) for x, s in _line_graph(tensors).items()}
    score = {v: _fill(adj, v) for v in adj}
    tie = {v: (rng.random() if rng is not None else 0.0) for v in adj}
    order = []
    while adj:
        v = min(adj, key=lambda u: (score[u], tie[u], u))
        nb = list(adj[v])
        for i in range(len(nb)):
            for j in range(i + 1, len(nb)):
                adj[nb[i]].add(nb[j])
                adj[nb[j]].add(nb[i])
        for u in nb:
            adj[u].discard(v)
        del adj[v]
        order.append(v)
        touched = set(nb)
        for u in nb:
            touched |= adj[u]
        for u in touched:
            score[u] = _fill(adj, u)
    return order


def _elimination_cost(tensors, order):
    owner = {}
    ts = {i: set(l) for i, (_, l) in enumerate(tensors)}
    for i, l in ts.items():
        for x in l:
            owner.setdefault(x, set()).add(i)
    nid, cost = len(ts), 0
    for x in order:
        ids = [i for i in owner.get(x, ()) if i in ts]
        if len(ids) < 2:
            continue
        i, j = ids
        li, lj = ts.pop(i), ts.pop(j)
        sh = li & lj
        cost += 2 ** (len(li) + len(lj) - len(sh))
        out = (li | lj) - sh
        for y in li | lj:
            owner[y].discard(i)
            owner[y].discard(j)
        for y in out:
            owner[y].add(nid)
        ts[nid] = out
        nid += 1
    return cost


def best_minfill_order(tensors, trials: int = 4, seed: int = 0):
    rng = np.random.default_rng(seed)
    best = None
    for t in range(trials):
        order = minfill_order(tensors, rng if t else None)
        c = _elimination_cost(tensors, order)
        if best is None or c < best[0]:
            best = (c, order)
    return best[1]


def contract(tensors, loops: int = 0, order: str = "greedy", rng=None, trials: int = 4):
    """Contract a closed network to a scalar. Returns (value, max_rank_seen)."""
    if order == "minfill":
        return _contract_by_elimination(tensors, loops, best_minfill_order(tensors, trials))
    ts = {i: (a, list(l)) for i, (a, l) in enumerate(tensors)}
    next_id = len(ts)
    max_rank = max((len(l) for _, l in ts.values()), default=0)
    while len(ts) > 1:
        where = {}
        for tid, (_, labels) in ts.items():
            for x in labels:
                where.setdefault(x, []).append(tid)
        pairs = set()
        for ids in where.values():
            if len(ids) == 2:
                pairs.add((min(ids), max(ids)))
        if not pairs:
            ids = sorted(ts)
            pair = (ids[0], ids[1])
        elif order == "random":
            plist = sorted(pairs)
            pair = plist[int(rng.integers(len(plist)))]
        else:
            best = None
            for (i, j) in sorted(pairs):
                li, lj = ts[i][1], ts[j][1]
                shared = len(set(li) & set(lj))
                r = len(li) + len(lj) - 2 * shared
                key = (r, len(li) + len(lj))
                if best is None or key < best[0]:
                    best = (key, (i, j))
            pair = best[1]
        i, j = pair
        ai, li = ts.pop(i)
        aj, lj = ts.pop(j)
        shared = [x for x in li if x in set(lj)]
        res = np.tensordot(ai, aj, axes=([li.index(x) for x in shared],
                                         [lj.index(x) for x in shared]))
        labels = [x for x in li if x not in shared] + [x for x in lj if x not in shared]
        max_rank = max(max_rank, len(labels))
        ts[next_id] = (res, labels)
        next_id += 1
    (arr, labels), = ts.values() if ts else [(np.array(1.0 + 0j), [])]
    assert not labels, "network was not closed"
    return complex(arr) * (2.0 ** loops), max_rank


def _pair(ai, li, aj, lj):
    sj = set(lj)
    shared = [x for x in li if x in sj]
    res = np.tensordot(ai, aj, axes=([li.index(x) for x in shared], [lj.index(x) for x in shared]))
    labels = [x for x in li if x not in shared] + [x for x in lj if x not in shared]
    return res, labels


def _contract_by_elimination(tensors, loops, order):
    ts = {i: (a, list(l)) for i, (a, l) in enumerate(tensors)}
    owner = {}
    for i, (_, l) in ts.items():
        for x in l:
            owner.setdefault(x, set()).add(i)
    nid = len(ts)
    max_rank = max((len(l) for _, l in ts.values()), default=0)
    for x in order:
        ids = [i for i in owner.get(x, ()) if i in ts]
        if len(ids) < 2:
            continue
        i, j = ids
        (ai, li), (aj, lj) = ts.pop(i), ts.pop(j)
        res, labels = _pair(ai, li, aj, lj)
        for y in li + lj:
            owner[y].discard(i)
            owner[y].discard(j)
        for y in labels:
            owner[y].add(nid)
        max_rank = max(max_rank, len(labels))
        ts[nid] = (res, labels)
        nid += 1
    val = 1.0 + 0j
    for arr, labels in ts.values():  # disconnected components end as scalars
        assert not labels, "network was not closed"
        val *= complex(arr)
    return val * (2.0 ** loops), max_rank


def alg1_trace(inst, choice, order="greedy", rng=None) -> complex:
    tensors, loops = alg1_network(inst, choice)
    return contract(tensors, loops, order, rng)[0]


def alg1_fidelity(inst, order="greedy", rng=None) -> dict:
    """Alg. I: enumerate all choices, contract each miter, accumulate |tr|^2."""
    t = np.array([alg1_trace(inst, c, order, rng) for c in combinations(inst)],
                 dtype=np.complex128)
    d2 = float(4 ** inst.n)
    S = math.fsum(float(abs(x) ** 2) for x in t)
    return {"F": S / d2, "one_minus_F": (d2 - S) / d2, "S": S, "traces": t}


def alg2_fidelity(inst, order="greedy", rng=None) -> dict:
    """Alg. II: one doubled network; its value is sum_i |tr(U^dagger E_i)|^2."""
    tensors, loops = alg2_network(inst)
    val, w = contract(tensors, loops, order, rng)
    d2 = float(4 ** inst.n)
    S = val.real
    return {"F": S / d2, "one_minus_F": (d2 - S) / d2, "S": S, "S_imag": val.imag, "width": w}
