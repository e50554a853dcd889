"""Sliced Alg. I with the early exit, and automatic choice between Alg. I and Alg. II.

Sec. IV-A remarks that an affirmative answer needs only part of the traces: every term of
F_J = (1/d^2) sum |t_i|^2 is non-negative, so a partial sum above 1 - eps decides equivalence.
Its example (Example 3 with p = 0.95, eps = 0.1): tr(U^dagger E_{1,1}) = 4p alone gives
F_J >= (4p)^2 / 4^2 = 0.9025 > 0.9. A sliced plan fixes the Kraus index of some noises and runs
the network once per combination, heaviest first; that example stops after its first trace.
"""
import numpy as np
import pytest

from paper_2103_11595_gb300 import ajf
from paper_2103_11595_gb300 import workloads as W


def _host_plan(inst, alg, **kw):
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, inst)
        info = ajf.ajf_plan(c.handle, alg, trials=2, **kw)
        return info, ajf.ajf_planned_alg(c.handle)


def _mixed(seed):
    """3 qubits; a depolarising noise (4 Kraus operators) and two amplitude dampings (2 each)."""
    rng = np.random.default_rng(seed)
    gates = [W.Gate((q,), W.haar_unitary(rng, 2)) for q in range(3)] + [W.Gate((0, 1), W.CX), W.Gate((1, 2), W.CX)]
    noises = [W.Noise(0, (0,), W.amplitude_damping(0.02), "ad"), W.Noise(3, (1,), W.depolarising(0.03), "dep"),
              W.Noise(4, (2,), W.amplitude_damping(0.05), "ad")]
    return W.Instance(3, gates, noises, name=f"mixed({seed})")


def test_slices_remove_open_bits_of_the_largest_noises():
    inst = _mixed(0)
    full, _ = _host_plan(inst, 1)
    assert full["n_open_bits"] == 1 + 2 + 1
    one, _ = _host_plan(inst, 1, alg1_slices=1)
    assert one["n_open_bits"] == 2          # the depolarising noise (4 operators) is fixed first
    two, _ = _host_plan(inst, 1, alg1_slices=2)
    assert two["n_open_bits"] == 1          # then the earlier amplitude damping
    allf, _ = _host_plan(inst, 1, alg1_slices=3)
    assert allf["n_open_bits"] == 0


def test_slice_option_checks():
    inst = _mixed(0)
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, inst)
        for kw in ({"alg1_slices": 4}, {"alg1_slices": -1}):
            with pytest.raises(ajf.AjfError) as e:
                ajf.ajf_plan(c.handle, 1, **kw)
            assert e.value.status == ajf.AJF_E_ARG
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_plan(c.handle, 2, alg1_slices=1)
        assert e.value.status == ajf.AJF_E_ARG
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_plan(c.handle, 1, alg1_slices=1, lowering="persistent")
        assert e.value.status == ajf.AJF_E_ARG


def test_auto_selects_by_estimated_time():
    """Sec. V: Alg. I is the faster with few noises, Alg. II once the noises are many. Here Alg. I
    keeps every noise's Kraus index open in one network, so it loses only once those open bits
    outgrow the doubling of Alg. II: the n = 16 mid instance with 10 noises (13 open bits) still
    plans Alg. I about 30x cheaper, 6 qubits with 12 depolarising noises (24 open bits) do not."""
    one_noise = W.Instance(12, W.line_u3_cx(np.random.default_rng(1), 12, 60),
                           [W.Noise(30, (5,), W.depolarising(0.01), "dep")])
    assert _host_plan(one_noise, ajf.AJF_ALG_AUTO)[1] == 1
    assert _host_plan(W.mid(0), ajf.AJF_ALG_AUTO)[1] == 1
    rng = np.random.default_rng(3)
    gates = W.line_u3_cx(rng, 6, 30)
    noises = [W.Noise(int(g), (int(rng.integers(6)),), W.depolarising(0.01), "dep")
              for g in sorted(rng.choice(30, 12, replace=False))]
    info, alg = _host_plan(W.Instance(6, gates, noises), ajf.AJF_ALG_AUTO)
    assert alg == 2 and info["n_open_bits"] == 0


# --------------------------------------------------------------------------- GPU


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _run(inst, eps=-1.0, alg=1, **kw):
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, inst)
        ajf.ajf_plan(c.handle, alg, trials=4, **kw)
        r = ajf.ajf_fidelity(c.handle, eps)
        try:
            t = ajf.ajf_alg1_traces(c.handle, inst.n_combinations())
        except ajf.AjfError as e:
            t = e.status
        return r, t, ajf.ajf_planned_alg(c.handle)


@pytest.mark.gpu
def test_paper_example_stops_after_one_trace(gpu):
    inst = W.qft2_noisy(0.95)
    r, t, _ = _run(inst, eps=0.1, alg1_slices=2)
    assert r["traces_done"] == 1 and r["equivalent"] == 1
    assert r["F"] == pytest.approx(0.95 ** 2, abs=1e-13)  # (4p)^2 / 16 = 0.9025 > 0.9
    assert t == ajf.AJF_E_STATE                            # the other traces were never computed
    # eps = 0.05: 0.9025 does not reach 0.95, all four traces are needed and decide "no"
    r, t, _ = _run(inst, eps=0.05, alg1_slices=2)
    assert r["traces_done"] == 4 and r["equivalent"] == 0
    np.testing.assert_allclose(t, [4 * 0.95, 0, 0, 0], atol=1e-12)


@pytest.mark.gpu
@pytest.mark.parametrize("slices", [1, 2, 3])
def test_sliced_equals_unsliced(gpu, slices):
    from oracle import dense
    insts = [_mixed(s) for s in range(3)] + [W.random_small(s, n=4, n_gates=14, n_noises=3, two_qubit_noise=True)
                                             for s in range(3)]
    for inst in insts:
        ref = dense.fidelity(inst)
        r, t, _ = _run(inst, alg1_slices=min(slices, len(inst.noises)))
        assert abs(r["F"] - ref["F"]) <= 1e-12
        assert abs(r["one_minus_F"] - ref["one_minus_F"]) <= 1e-12
        assert r["traces_done"] == inst.n_combinations()
        np.testing.assert_allclose(t, ref["traces"], atol=1e-12 * 2 ** inst.n)


@pytest.mark.gpu
def test_early_exit_is_a_certified_lower_bound(gpu):
    from oracle import dense
    for s in range(3):
        inst = _mixed(s)
        ref = dense.fidelity(inst)["F"]
        r, t, _ = _run(inst, eps=0.2, alg1_slices=3)
        assert r["equivalent"] == 1 and r["traces_done"] < inst.n_combinations()
        assert 0.8 < r["F"] <= ref + 1e-12
        assert t == ajf.AJF_E_STATE


@pytest.mark.gpu
def test_sliced_plan_rejected_by_single_run_paths(gpu):
    inst = _mixed(0)
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, inst)
        ajf.ajf_plan(c.handle, 1, trials=2, alg1_slices=1)
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_fidelity_batch([c.handle], 1)
        assert e.value.status == ajf.AJF_E_STATE
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_fidelity_noalloc(c.handle, 1)
        assert e.value.status == ajf.AJF_E_STATE


@pytest.mark.gpu
def test_auto_matches_both_algorithms(gpu):
    from oracle import dense
    for inst in [W.tiny(0), W.tiny(1), _mixed(1)]:
        ref = dense.fidelity(inst)["F"]
        r, _, alg = _run(inst, alg=ajf.AJF_ALG_AUTO)
        assert alg in (1, 2) and abs(r["F"] - ref) <= 1e-12


def test_checkpoint_of_a_host_plan():
    inst = _mixed(0)
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, inst)
        ajf.ajf_plan(c.handle, 1, trials=2, alg1_slices=2)
        st = ajf.ajf_alg1_checkpoint(c.handle)
        assert st["next_slice"] == 0 and st["n_slices"] == 4 * 2 and st["S"] == 0
        ajf.ajf_alg1_restore(c.handle, dict(st, next_slice=3, S=1.5, traces_done=6))
        assert ajf.ajf_alg1_checkpoint(c.handle)["next_slice"] == 3
        for bad in (dict(st, plan_sig=st["plan_sig"] ^ 1), dict(st, next_slice=9), dict(st, n_slices=5)):
            with pytest.raises(ajf.AjfError) as e:
                ajf.ajf_alg1_restore(c.handle, bad)
            assert e.value.status == ajf.AJF_E_ARG
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_alg1_continue(c.handle)
        assert e.value.status == ajf.AJF_E_STATE  # host-only context
        # other input values: the checkpoint does not apply
        other = _mixed(1)
        ajf.load_instance(c.handle, other)
        ajf.ajf_plan(c.handle, 1, trials=2, alg1_slices=2)
        with pytest.raises(ajf.AjfError):
            ajf.ajf_alg1_restore(c.handle, st)
        # an unsliced plan has no progress to checkpoint
        ajf.ajf_plan(c.handle, 1, trials=2)
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_alg1_checkpoint(c.handle)
        assert e.value.status == ajf.AJF_E_STATE


@pytest.mark.gpu
def test_resume_from_checkpoint_in_a_new_context(gpu):
    """Slices 0..2 in one context, a checkpoint, the rest in another context: the same F, S and
    1 - F as one full evaluation (and as the oracle)."""
    from oracle import dense
    for s in range(3):
        inst = _mixed(s)
        ref = dense.fidelity(inst)
        with ajf.Context(0) as a:
            ajf.load_instance(a.handle, inst)
            ajf.ajf_plan(a.handle, 1, trials=2, alg1_slices=2)
            part = ajf.ajf_alg1_continue(a.handle, max_slices=3)
            assert part["equivalent"] == -1 and part["traces_done"] == 3 * 2
            st = ajf.ajf_alg1_checkpoint(a.handle)
            assert st["next_slice"] == 3
        with ajf.Context(0) as b:
            ajf.load_instance(b.handle, inst)
            ajf.ajf_plan(b.handle, 1, trials=2, alg1_slices=2)
            ajf.ajf_alg1_restore(b.handle, st)
            r = ajf.ajf_alg1_continue(b.handle, eps=1e-9)
            assert r["traces_done"] == inst.n_combinations() and r["equivalent"] == 0
            assert abs(r["F"] - ref["F"]) <= 1e-12 and abs(r["one_minus_F"] - ref["one_minus_F"]) <= 1e-12
            with pytest.raises(ajf.AjfError) as e:
                ajf.ajf_alg1_traces(b.handle, inst.n_combinations())
            assert e.value.status == ajf.AJF_E_STATE
            # the same context, continued in single slices without a restore, keeps its traces
            full = ajf.ajf_fidelity_alg1(b.handle)
            assert abs(full["F"] - ref["F"]) <= 1e-12
            np.testing.assert_allclose(ajf.ajf_alg1_traces(b.handle, inst.n_combinations()), ref["traces"], atol=1e-12 * 8)
