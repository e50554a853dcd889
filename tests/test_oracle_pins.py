"""Pins for the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage it follows. Together they are chosen so that a plausible slip in the
oracle -- a dropped noise, N^dagger in place of N^*, U^T in place of U^dagger, a transposed gate,
a wrong qubit order -- fails at least one of them (see the planted-mistake tests at the end).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import dense, network, superop
from paper_2103_11595_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "qft2_examples.json")


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


# --------------------------------------------------------------------------- Examples 3 and 4


@pytest.mark.parametrize("case", golden()["cases"], ids=lambda c: f"p={c['p']}")
def test_example3_alg1_traces(case):
    """Example 3 (Sec. IV-A): traces (4p, 0, 0, 0) and F_J = p^2 for the noisy QFT_2."""
    inst = W.qft2_noisy(case["p"])
    for res in (dense.fidelity(inst), network.alg1_fidelity(inst)):
        np.testing.assert_allclose(res["traces"], case["traces"], atol=1e-13)
        assert res["F"] == pytest.approx(case["F"], abs=1e-13)


@pytest.mark.parametrize("case", golden()["cases"], ids=lambda c: f"p={c['p']}")
def test_example4_alg2_value(case):
    """Example 4 (Sec. IV-B): the doubled network contracts to 16 p^2."""
    inst = W.qft2_noisy(case["p"])
    assert superop.alg2_sum(inst).real == pytest.approx(case["alg2"], abs=1e-12)
    for order in ("greedy", "minfill"):
        assert network.alg2_fidelity(inst, order=order)["S"] == pytest.approx(case["alg2"], abs=1e-12)


def test_example4_noise_matrices():
    """Example 4: M_N = p I(x)I + (1-p) X(x)X and M_N' = p I(x)I + (1-p) Z(x)Z."""
    p = 0.3
    inst = W.qft2_noisy(p)
    mn = [sum(np.kron(K, np.conj(K)) for K in nz.kraus) for nz in inst.noises]
    np.testing.assert_allclose(mn[0], p * np.eye(4) + (1 - p) * np.kron(W.X, W.X), atol=1e-15)
    np.testing.assert_allclose(mn[1], p * np.eye(4) + (1 - p) * np.kron(W.Z, W.Z), atol=1e-15)


def test_early_exit_remark():
    """After Example 3: p=0.95, eps=0.1 -- the first trace alone gives (4p)^2/4^2 = 0.9025 > 0.9."""
    g = golden()["early_exit"]
    t = dense.traces(W.qft2_noisy(g["p"]))
    partial = abs(t[0]) ** 2 / 16
    assert partial == pytest.approx(g["partial_F_after_first_trace"], abs=1e-14)
    assert partial > 1 - g["epsilon"]


# --------------------------------------------------------------------------- closed forms


def _all_forms(inst, tol=1e-12, superop_ok=True):
    """Every oracle route on one instance; returns the dense F after checking agreement."""
    f = dense.fidelity(inst)["F"]
    assert network.alg1_fidelity(inst)["F"] == pytest.approx(f, abs=tol)
    assert network.alg2_fidelity(inst)["F"] == pytest.approx(f, abs=tol)
    assert network.alg2_fidelity(inst, order="minfill")["F"] == pytest.approx(f, abs=tol)
    if superop_ok:
        assert superop.alg2_sum(inst).real / 4 ** inst.n == pytest.approx(f, abs=tol)
    return f


@pytest.mark.parametrize("seed", range(4))
def test_noiseless_is_one(seed):
    """F_J(U, U) = |tr(U^dagger U)|^2 / d^2 = 1 (Sec. III)."""
    inst = W.random_small(seed, n=3, n_gates=12, n_noises=0)
    assert _all_forms(inst) == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("p", [0.0, 1e-4, 0.01, 0.3, 1.0])
def test_depolarising_on_identity(p):
    """One depolarising channel (error p) on the identity: F_J = 1 - 3p/4; with Example 2's
    parametrisation (p = probability of no error) F_J = p."""
    inst = W.identity_with_noises(1, [W.Noise(0, (0,), W.depolarising(p))])
    assert _all_forms(inst) == pytest.approx(1 - 0.75 * p, abs=1e-14)
    inst = W.identity_with_noises(1, [W.Noise(0, (0,), W.paper_depolarising(1 - p))])
    assert _all_forms(inst) == pytest.approx(1 - p, abs=1e-14)


@pytest.mark.parametrize("gamma", [0.0, 1e-3, 0.2, 1.0])
def test_amplitude_damping_on_identity(gamma):
    """Amplitude damping: |tr K0|^2/4 = (1 + sqrt(1-gamma))^2 / 4, tr K1 = 0."""
    inst = W.identity_with_noises(2, [W.Noise(1, (1,), W.amplitude_damping(gamma))])
    assert _all_forms(inst) == pytest.approx((1 + math.sqrt(1 - gamma)) ** 2 / 4, abs=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_single_noise_anywhere(seed):
    """With a single noise in an otherwise ideal circuit, the gates cancel under the cyclic trace:
    tr(U^dagger E_k) = tr(V^dagger K_k V) = 2^{n-a} tr(K_k), so F_J = sum_k |tr K_k|^2 / 4^a."""
    rng = np.random.default_rng(seed)
    inst = W.random_small(seed, n=3, n_gates=10, n_noises=0)
    if seed % 2 == 0:
        kr = np.stack([W.haar_unitary(rng, 2) * math.sqrt(w) for w in (0.7, 0.3)])
        a = 1
        qs = (int(rng.integers(3)),)
    else:
        kr = W.two_qubit_depolarising(0.1)
        a = 2
        qs = (0, 2)
    inst.noises = [W.Noise(int(rng.integers(len(inst.ideal))), qs, kr)]
    expect = sum(abs(np.trace(K)) ** 2 for K in kr) / 4 ** a
    assert _all_forms(inst) == pytest.approx(expect, abs=1e-12)


def test_disjoint_noises_multiply():
    """Noises on disjoint qubits of the identity: F_J factorises (tr of a tensor product)."""
    ps = [0.01, 0.2, 0.5]
    nz = [W.Noise(q, (q,), W.depolarising(p)) for q, p in enumerate(ps)]
    nz.append(W.Noise(0, (0,), W.amplitude_damping(0.3)))
    inst = W.identity_with_noises(4, nz[:3] + [W.Noise(3, (3,), W.amplitude_damping(0.3))])
    expect = np.prod([1 - 0.75 * p for p in ps]) * (1 + math.sqrt(0.7)) ** 2 / 4
    assert _all_forms(inst) == pytest.approx(expect, abs=1e-13)


def test_depolarising_composition():
    """Two depolarising channels in a row on one qubit compose to one with 1-p = (1-p1)(1-p2)."""
    p1, p2 = 0.1, 0.25
    inst = W.identity_with_noises(1, [W.Noise(0, (0,), W.depolarising(p1)),
                                      W.Noise(0, (0,), W.depolarising(p2))])
    p = 1 - (1 - p1) * (1 - p2)
    assert _all_forms(inst) == pytest.approx(1 - 0.75 * p, abs=1e-14)


# --------------------------------------------------------------------------- definitions


@pytest.mark.parametrize("seed", range(3))
def test_trace_formula_equals_state_fidelity(seed):
    """Sec. III: F_J(E,U) is the fidelity of the Jamiolkowski states; the trace formula must agree
    with that definition computed from density matrices and PSD square roots."""
    inst = W.random_small(seed, n=2 if seed < 2 else 3, n_gates=6, n_noises=2)
    f = dense.fidelity(inst)["F"]
    assert superop.jamiolkowski_fidelity(inst) == pytest.approx(f, abs=2e-6)


@pytest.mark.parametrize("seed", range(4))
def test_alg2_identity_bruteforce(seed):
    """Sec. IV-B: sum_i |tr(U^dagger E_i)|^2 = tr((U^dagger (x) U^T) M_E), dense, n <= 4."""
    inst = W.random_small(seed, n=2 + seed % 3, n_gates=8, n_noises=2 + seed % 2,
                          two_qubit_noise=(seed == 3))
    S = dense.fidelity(inst)["S"]
    val = superop.alg2_sum(inst)
    assert val.real == pytest.approx(S, rel=1e-12, abs=1e-12)
    assert abs(val.imag) < 1e-10


def _stabiliser_states():
    s = 1 / math.sqrt(2)
    return [np.array(v, dtype=np.complex128) for v in
            ([1, 0], [0, 1], [s, s], [s, -s], [s, 1j * s], [s, -1j * s])]


@pytest.mark.parametrize("seed", range(3))
def test_average_fidelity_relation(seed):
    """Sec. III: the Haar average of F(E(psi), U|psi>) equals (d F_J + 1)/(d + 1). For one qubit
    the six stabiliser states form a 2-design, so their mean is exact."""
    inst = W.random_small(seed, n=1, n_gates=4, n_noises=2)
    U = dense.circuit_matrix(1, inst.ideal)
    Es = [dense.kraus_of_circuit(inst, c) for c in dense.combinations(inst)]
    vals = []
    for psi in _stabiliser_states():
        up = U @ psi
        vals.append(sum(abs(np.vdot(up, E @ psi)) ** 2 for E in Es))
    fj = dense.fidelity(inst)["F"]
    assert np.mean(vals) == pytest.approx((2 * fj + 1) / 3, abs=1e-13)


@pytest.mark.parametrize("seed", range(3))
def test_stability_idle_qubits(seed):
    """Sec. III, stability: F_J(E (x) I, U (x) I) = F_J(E, U) -- idle qubits change nothing."""
    inst = W.random_small(seed, n=2, n_gates=6, n_noises=2)
    bigger = W.Instance(4, inst.ideal, inst.noises, name="padded")
    f = dense.fidelity(inst)["F"]
    assert dense.fidelity(bigger)["F"] == pytest.approx(f, abs=1e-13)
    assert network.alg1_fidelity(bigger)["F"] == pytest.approx(f, abs=1e-13)
    assert network.alg2_fidelity(bigger)["F"] == pytest.approx(f, abs=1e-13)


@pytest.mark.parametrize("seed", range(4))
def test_chaining_inequality(seed):
    """Sec. III, chaining: C_J(E1 o E2, U1 U2) <= C_J(E1, U1) + C_J(E2, U2), C_J = sqrt(1-F_J)."""
    a = W.random_small(10 + seed, n=2, n_gates=5, n_noises=2)
    b = W.random_small(20 + seed, n=2, n_gates=5, n_noises=2)
    shift = len(a.ideal)
    both = W.Instance(2, a.ideal + b.ideal,
                      a.noises + [W.Noise(nz.after_gate + shift, nz.qubits, nz.kraus) for nz in b.noises])
    c = lambda inst: math.sqrt(max(0.0, dense.fidelity(inst)["one_minus_F"]))
    assert c(both) <= c(a) + c(b) + 1e-12


# --------------------------------------------------------------------------- cross-agreement


@pytest.mark.parametrize("seed", range(6))
def test_networks_match_dense(seed):
    """O2 (Alg. I and Alg. II networks) against O1 (dense definition) on random instances with
    mixed noises, a 2-qubit noise, and an implementation skeleton different from the ideal."""
    inst = W.random_small(seed, n=3 + seed % 2, n_gates=10, n_noises=2 + seed % 2,
                          two_qubit_noise=(seed % 3 == 0))
    if seed % 2 == 1:
        rng = np.random.default_rng(seed)
        impl = list(inst.ideal)
        impl[0] = W.Gate(impl[0].qubits, W.haar_unitary(rng, 2 ** impl[0].arity))
        inst.impl = impl
    d = dense.fidelity(inst)
    a1 = network.alg1_fidelity(inst)
    np.testing.assert_allclose(a1["traces"], d["traces"], atol=1e-12)
    assert network.alg2_fidelity(inst)["S"] == pytest.approx(d["S"], rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_order_invariance(seed):
    """The contracted value does not depend on the pairwise order (tensor-network algebra)."""
    inst = W.random_small(seed, n=3, n_gates=12, n_noises=2)
    ref = network.alg2_fidelity(inst)["S"]
    rng = np.random.default_rng(seed)
    for _ in range(3):
        assert network.alg2_fidelity(inst, order="random", rng=rng)["S"] == pytest.approx(ref, rel=1e-12)
    tensors, loops = network.alg2_network(inst)
    for s in range(2):
        order = network.minfill_order(tensors, np.random.default_rng(s))
        val, _ = network._contract_by_elimination(tensors, loops, order)
        assert val.real == pytest.approx(ref, rel=1e-12)


def test_untouched_wires_are_loops():
    """A qubit no gate touches closes into a loop worth tr(I_2) = 2 per wire."""
    inst = W.Instance(3, [W.Gate((0,), W.H)], [W.Noise(0, (0,), W.depolarising(0.2))])
    assert network.alg2_fidelity(inst)["F"] == pytest.approx(1 - 0.15, abs=1e-14)
    assert network.alg1_fidelity(inst)["F"] == pytest.approx(1 - 0.15, abs=1e-14)


def test_tiny_config_all_routes():
    """n=3, 20-gate tiny workload: every route agrees to 1e-12."""
    for seed in range(3):
        _all_forms(W.tiny(seed))


# --------------------------------------------------------------------------- planted mistakes


def test_planted_mistake_dagger_instead_of_conjugate(monkeypatch):
    """Building M_N with N^dagger instead of N^* (Sec. IV-B step 3) must break Alg. II agreement."""
    rng = np.random.default_rng(7)
    kr = np.stack([W.haar_unitary(rng, 2) * math.sqrt(w) for w in (0.6, 0.4)])
    inst = W.random_small(1, n=2, n_gates=6, n_noises=0)
    inst.noises = [W.Noise(2, (0,), kr), W.Noise(4, (1,), W.amplitude_damping(0.3))]
    good = dense.fidelity(inst)["S"]
    assert network.alg2_fidelity(inst)["S"] == pytest.approx(good, rel=1e-12)
    real_kron = np.kron
    monkeypatch.setattr(network.np, "kron", lambda a, b: real_kron(a, np.conj(b).T))
    assert network.alg2_fidelity(inst)["S"] != pytest.approx(good, rel=1e-6)


def test_planted_mistake_dropped_noise(monkeypatch):
    """Dropping a noise from the timeline must break Example 3."""
    orig = dense.timeline
    monkeypatch.setattr(dense, "timeline", lambda inst: [op for op in orig(inst) if op != ("noise", 1)])
    inst = W.qft2_noisy(0.3)
    assert dense.fidelity(inst)["F"] != pytest.approx(0.09, abs=1e-6)


def test_planted_mistake_transposed_ideal():
    """Using U^T instead of U^dagger (Alg. I) breaks the noiseless F_J = 1 pin."""
    inst = W.random_small(2, n=2, n_gates=6, n_noises=0)
    U = dense.circuit_matrix(2, inst.ideal)
    wrong = abs(np.sum(U * U)) ** 2 / 16  # tr(U^T U) in place of tr(U^dagger U)
    assert wrong != pytest.approx(1.0, abs=1e-6)
    assert dense.fidelity(inst)["F"] == pytest.approx(1.0, abs=1e-12)


def test_gate_qubit_order_matters():
    """The first listed qubit of a gate is its most significant factor. With the ideal circuit
    H(0); CX(0->1); T(1) and an implementation using CX(1->0), tr(U^dagger V) = tr(CX_01 CX_10) = 1
    (a 3-cycle on |01>,|10>,|11> fixes only |00>), so F_J = 1/16; an oracle that ignored the
    gate's qubit order would report 1."""
    ideal = [W.Gate((0,), W.H), W.Gate((0, 1), W.CX), W.Gate((1,), W.T)]
    impl = [W.Gate((0,), W.H), W.Gate((1, 0), W.CX), W.Gate((1,), W.T)]
    inst = W.Instance(2, ideal, [], impl=impl)
    assert _all_forms(inst) == pytest.approx(1 / 16, abs=1e-14)


# --------------------------------------------------------------------------- one-operation wires


def _count_self_traces(monkeypatch):
    """Wrap the oracle's self-trace so a test can assert that a repeated label was really summed."""
    calls = {"n": 0}
    real = network._self_trace

    def counting(arr, labels):
        calls["n"] += len(labels) - len(set(labels))
        return real(arr, labels)

    monkeypatch.setattr(network, "_self_trace", counting)
    return calls


def _random_kraus(rng, a, weights):
    """A Kraus set of unequal, non-symmetric operators: sqrt(w) times Haar unitaries."""
    return np.stack([W.haar_unitary(rng, 2 ** a) * math.sqrt(w) for w in weights])


@pytest.mark.parametrize("seed", range(3))
def test_noise_on_gate_free_qubit(seed, monkeypatch):
    """A noise on a qubit that no gate touches: its wire holds one operation, whose output closes
    onto its own input, so each term is tr(K_k) (Sec. IV, the trace closes every wire). With the
    gates cancelling on the other qubits, F_J = sum_k |tr K_k|^2 / 4 (a single noise anywhere)."""
    rng = np.random.default_rng(40 + seed)
    gates = [W.Gate((0,), W.haar_unitary(rng, 2)) for _ in range(3)]
    kr = _random_kraus(rng, 1, (0.5, 0.3, 0.2))
    inst = W.Instance(2, gates, [W.Noise(1, (1,), kr)])
    expect = sum(abs(np.trace(K)) ** 2 for K in kr) / 4
    calls = _count_self_traces(monkeypatch)
    assert _all_forms(inst) == pytest.approx(expect, abs=1e-13)
    assert calls["n"] > 0


@pytest.mark.parametrize("busy", [False, True])
def test_two_qubit_noise_on_idle_wires(busy, monkeypatch):
    """A 2-qubit noise whose two wires (or one of them, `busy`) carry no other operation: one
    tensor closes onto itself on both label pairs (or on one, a partial trace). F_J must be the
    single-noise closed form sum_k |tr K_k|^2 / 16 for a non-symmetric Kraus set, so pairing an
    output with the wrong input, or a missing sum, fails."""
    rng = np.random.default_rng(7)
    kr = _random_kraus(rng, 2, (0.6, 0.4))
    gates = [W.Gate((0,), W.haar_unitary(rng, 2)), W.Gate((0,), W.haar_unitary(rng, 2))]
    if busy:
        gates.append(W.Gate((1,), W.haar_unitary(rng, 2)))
        nz = W.Noise(2, (1, 2), kr)
    else:
        nz = W.Noise(1, (1, 2), kr)
    inst = W.Instance(3, gates, [nz])
    expect = sum(abs(np.trace(K)) ** 2 for K in kr) / 16
    calls = _count_self_traces(monkeypatch)
    assert _all_forms(inst) == pytest.approx(expect, abs=1e-13)
    assert calls["n"] > 0


def test_one_operation_implementation_wire(monkeypatch):
    """Problem 1 allows an implementation that differs from U. Here the ideal circuit leaves
    qubit 1 idle and the implementation puts one gate G there: that wire is G alone, closed onto
    itself (tr G in Alg. I; tr G and tr G^* on q, q' in Alg. II), so
    F_J = |tr G|^2 / 4 * (1 - 3p/4) with a depolarising noise on qubit 0."""
    rng = np.random.default_rng(3)
    u = W.haar_unitary(rng, 2)
    g = W.haar_unitary(rng, 2)
    p = 0.2
    ideal = [W.Gate((0,), u)]
    impl = [W.Gate((0,), u), W.Gate((1,), g)]
    inst = W.Instance(2, ideal, [W.Noise(0, (0,), W.depolarising(p))], impl=impl)
    expect = abs(np.trace(g)) ** 2 / 4 * (1 - 0.75 * p)
    calls = _count_self_traces(monkeypatch)
    assert _all_forms(inst) == pytest.approx(expect, abs=1e-13)
    assert calls["n"] > 0


def _wrong_pair_self_trace(arr, labels):
    """Planted mistake: with two repeated labels, trace each first occurrence against the OTHER
    label's second occurrence."""
    pos = {}
    for i, x in enumerate(labels):
        pos.setdefault(x, []).append(i)
    dups = [v for v in pos.values() if len(v) == 2]
    if len(dups) < 2:
        return network._real_self_trace(arr, labels)
    (i1, j1), (i2, j2) = dups[0], dups[1]
    pairs = [(i1, j2), (i2, j1)]
    keep = [k for k in range(len(labels)) if k not in (i1, j1, i2, j2)]
    letters = "abcdefghijklmnopqrstuvwxyz"
    sub = [letters[k] for k in range(len(labels))]
    for a, b in pairs:
        sub[b] = sub[a]
    out = "".join(sub[k] for k in keep)
    return np.einsum("".join(sub) + "->" + out, arr), [labels[k] for k in keep]


def _no_sum_self_trace(arr, labels):
    """Planted mistake: keep only the diagonal element 0 of a repeated label instead of summing."""
    seen = {}
    for i, x in enumerate(labels):
        if x in seen:
            j0 = seen[x]
            idx = [slice(None)] * arr.ndim
            idx[j0] = 0
            idx[i] = 0
            return _no_sum_self_trace(arr[tuple(idx)], [y for k, y in enumerate(labels) if k not in (j0, i)])
        seen[x] = i
    return arr, labels


@pytest.mark.parametrize("mistake", [_wrong_pair_self_trace, _no_sum_self_trace], ids=["wrong_pair", "no_sum"])
def test_planted_mistake_self_trace(mistake, monkeypatch):
    """A self-trace that pairs the wrong axes or drops the sum must fail the idle-wire pin."""
    rng = np.random.default_rng(7)
    kr = _random_kraus(rng, 2, (0.6, 0.4))
    gates = [W.Gate((0,), W.haar_unitary(rng, 2)), W.Gate((0,), W.haar_unitary(rng, 2))]
    inst = W.Instance(3, gates, [W.Noise(1, (1, 2), kr)])
    expect = sum(abs(np.trace(K)) ** 2 for K in kr) / 16
    assert network.alg1_fidelity(inst)["F"] == pytest.approx(expect, abs=1e-13)
    monkeypatch.setattr(network, "_real_self_trace", network._self_trace, raising=False)
    monkeypatch.setattr(network, "_self_trace", mistake)
    assert network.alg1_fidelity(inst)["F"] != pytest.approx(expect, abs=1e-6)
