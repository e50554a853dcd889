"""SWAP elimination and local optimisations of the closed composed sequence (Sec. IV-C).

The simplifications must leave F_J unchanged (GPU tests: every flag setting against the oracle,
which contracts the sequence as given). The CPU tests pin what is removed: Example 5 of the paper
(the noisy QFT_2 of Fig. 1/2 with the ideal circuit given explicitly) loses its two SWAP gates and
its four H gates, leaving the bit flip, CS, the phase flip and CS^dagger (Fig. 5(b)).
"""
import numpy as np
import pytest

from paper_2103_11595_gb300 import ajf
from paper_2103_11595_gb300 import workloads as W


def _plan_host(inst, alg=1, **kw):
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, inst)
        return ajf.ajf_plan(c.handle, alg, trials=2, **kw)


def _swap_through_noise():
    """A phase flip on q1 first; H(0); SWAP; a bit flip on q0 after the SWAP. A noise then sits
    between the two SWAPs both ways round the closed sequence, so cancellation alone removes only
    the two H gates (across the closed trace); SWAP elimination rewires the SWAPs away."""
    gates = [W.Gate((0,), W.H, "H"), W.Gate((0, 1), W.SWAP, "SWAP")]
    noises = [W.Noise(-1, (1,), W.phase_flip(0.8), "pf"), W.Noise(1, (0,), W.bit_flip(0.9), "bf")]
    return W.Instance(2, gates, noises, name="swap_through_noise")


def _odd_swap(seed=0):
    """The implementation ends with a SWAP the ideal circuit does not have: one SWAP is left to the
    closure, which then joins output q0 to input q1 and vice versa (identity leaves)."""
    rng = np.random.default_rng(seed)
    ideal = [W.Gate((0,), W.haar_unitary(rng, 2)), W.Gate((0, 1), W.CX), W.Gate((2,), W.H),
             W.Gate((1, 2), W.haar_unitary(rng, 4))]
    impl = ideal + [W.Gate((0, 1), W.SWAP, "SWAP")]
    noises = [W.Noise(1, (1,), W.depolarising(0.9), "dep"), W.Noise(-1, (0,), W.amplitude_damping(0.05), "ad")]
    return W.Instance(3, ideal, noises, impl=impl, name=f"odd_swap({seed})")


def _padded(seed, n=4, pad=3):
    """A random small instance with `pad` random gates and their inverses inserted (in reverse
    order) before and after its gates, and SWAP pairs of random qubits around them."""
    inst = W.random_small(seed, n=n, n_gates=12, n_noises=2)
    rng = np.random.default_rng(1000 + seed)
    head, tail = [], []
    for _ in range(pad):
        a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
        g = W.Gate((a, b), W.haar_unitary(rng, 4), "U")
        head.append(g)
        tail.insert(0, W.Gate((a, b), g.mat.conj().T.copy(), "Udg"))
    a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
    sw = W.Gate((a, b), W.SWAP, "SWAP")
    gates = [sw] + head + tail + [sw] + list(inst.ideal)
    shift = len(gates) - len(inst.ideal)
    noises = [W.Noise(nz.after_gate + shift if nz.after_gate >= 0 else -1, nz.qubits, nz.kraus, nz.name)
              for nz in inst.noises]
    return W.Instance(n, gates, noises, name=f"padded({seed})")


def test_example5_counts():
    """Example 5: both SWAPs and all four H gates go; four tensors are left (Fig. 5(b))."""
    inst = W.qft2_noisy(0.9)
    none = _plan_host(inst)
    assert none["n_removed"] == 0 and none["n_leaves"] == 10
    for alg in (1, 2):
        full = _plan_host(inst, alg, simplify="all")
        assert full["n_removed"] == 6
        assert full["n_leaves"] == (4 if alg == 1 else 6)  # Alg. II: V and V^* per gate, one M_N per noise
    # the SWAPs are adjacent in the composed sequence here, so cancellation alone also removes them
    assert _plan_host(inst, simplify="cancel")["n_removed"] == 6
    assert _plan_host(inst, simplify="swap")["n_removed"] == 2


def test_swap_elimination_reaches_past_a_noise():
    inst = _swap_through_noise()
    assert _plan_host(inst, simplify="cancel")["n_removed"] == 2   # H . H across the closed trace
    full = _plan_host(inst, simplify="all")
    assert full["n_removed"] == 4                                    # + both SWAPs
    assert full["n_leaves"] == 2                                     # the two noises; q0 is an empty loop


def test_padding_is_removed():
    for seed in range(4):
        inst = _padded(seed)
        r = _plan_host(inst, simplify="all")
        # the 2 x 3 inserted gates and their adjoints in U^dagger cancel, and so do the SWAPs
        assert r["n_removed"] >= 2 * (2 * 3 + 2)


def test_odd_swap_closes_through_identities():
    inst = _odd_swap()
    r0 = _plan_host(inst, 2)
    r = _plan_host(inst, 2, simplify="swap")
    assert r["n_removed"] == 1
    # 4 wires of the doubled network are joined across (q0 <-> q1, q0' <-> q1') by identity leaves
    assert r["n_leaves"] == r0["n_leaves"] - 2 + 4


def test_noiseless_identity_keeps_a_network():
    """A noiseless circuit equal to its ideal would cancel completely; the sequence is then kept."""
    inst = W.Instance(2, [W.Gate((0,), W.H), W.Gate((0, 1), W.CX)], [])
    r = _plan_host(inst, 2, simplify="all")
    assert r["n_removed"] == 0 and r["n_leaves"] > 0


def test_simplify_flags_and_cache():
    inst = W.qft2_noisy(0.9)
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, inst)
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_plan(c.handle, 1, simplify=4)
        assert e.value.status == ajf.AJF_E_ARG
        a = ajf.ajf_plan(c.handle, 1, simplify="all", trials=2)
        b = ajf.ajf_plan(c.handle, 1, simplify="all", trials=2)
        assert b["plan_cached"] == 1 and b["n_removed"] == a["n_removed"] == 6
    # new matrix values that stop a cancellation change the simplified structure: no cached path
    changed = W.qft2_noisy(0.9)
    changed.impl = list(changed.ideal)
    changed.impl[2] = W.Gate((1,), W.S, "S")  # H(q2) -> S(q2) in the implementation
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, inst)
        ajf.ajf_plan(c.handle, 1, simplify="all", trials=2)
        ajf.load_instance(c.handle, changed)
        r = ajf.ajf_plan(c.handle, 1, simplify="all", trials=2)
        assert r["plan_cached"] == 0 and r["n_removed"] < 6


# --------------------------------------------------------------------------- GPU


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _fidelity(inst, alg, simplify, precision="f64", lowering="default"):
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, inst)
        info = ajf.ajf_plan(c.handle, alg, trials=4, simplify=simplify, precision=precision, lowering=lowering)
        r = ajf.ajf_fidelity_alg1(c.handle) if alg == 1 else ajf.ajf_fidelity_alg2(c.handle)
        traces = ajf.ajf_alg1_traces(c.handle, inst.n_combinations()) if alg == 1 else None
    return r, traces, info


@pytest.mark.gpu
@pytest.mark.parametrize("p", [0.3, 0.999])
def test_examples_3_to_5_values(gpu, p):
    """Simplified Example 5 network: traces (4p, 0, 0, 0), F = p^2, Alg. II value 16 p^2."""
    inst = W.qft2_noisy(p)
    r1, t, info = _fidelity(inst, 1, "all")
    assert info["n_removed"] == 6
    np.testing.assert_allclose(t, [4 * p, 0, 0, 0], atol=1e-12)
    assert r1["F"] == pytest.approx(p * p, abs=1e-13)
    r2, _, _ = _fidelity(inst, 2, "all")
    assert r2["S"] == pytest.approx(16 * p * p, abs=1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("simplify", ["swap", "cancel", "all"])
def test_invariance_against_oracle(gpu, simplify):
    from oracle import dense
    insts = ([W.tiny(s) for s in range(6)] + [_padded(s) for s in range(4)] + [_swap_through_noise()]
             + [_odd_swap(s) for s in range(3)])
    for inst in insts:
        ref = dense.fidelity(inst)
        for alg in (1, 2):
            r, t, _ = _fidelity(inst, alg, simplify)
            assert abs(r["F"] - ref["F"]) <= 1e-12, (inst.name, alg)
            if alg == 1:
                np.testing.assert_allclose(t, ref["traces"], atol=1e-12 * 2 ** inst.n)


@pytest.mark.gpu
def test_persistent_lowering_with_simplify(gpu):
    from oracle import dense
    insts = [_padded(s) for s in range(3)]
    refs = [dense.fidelity(i)["F"] for i in insts]
    ctxs = []
    try:
        for inst in insts:
            c = ajf.Context(0)
            ajf.load_instance(c.handle, inst)
            ajf.ajf_plan(c.handle, 2, trials=4, simplify="all", lowering="persistent")
            ctxs.append(c)
        res, n_p = ajf.ajf_fidelity_batch_persistent([c.handle for c in ctxs], 2)
        assert n_p == len(insts)
        for r, f in zip(res, refs):
            assert abs(r["F"] - f) <= 1e-12
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.gpu
def test_mid_instance_fewer_flops_same_value(gpu):
    """n = 16, 200 gates, 10 noises: the gates outside the noisy span cancel against U^dagger; F_J
    is the unsimplified FP64 value."""
    inst = W.mid(0)
    r0, _, i0 = _fidelity(inst, 2, "none")
    r1, _, i1 = _fidelity(inst, 2, "all")
    assert i1["n_removed"] > 0 and i1["flops"] <= i0["flops"]
    assert abs(r1["F"] - r0["F"]) <= 1e-12
