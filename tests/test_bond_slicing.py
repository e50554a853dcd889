"""Bond slicing: plans over the memory budget run as 2^s contractions of a smaller network.

A closed network contracts to the sum, over every assignment of its labels, of the product of
its tensors' entries (the trace of Sec. III written out index by index). Fixing s labels and
summing the 2^s contractions over their values is the same sum in another order, so F_J is
unchanged: Alg. II adds the slices' scalars, Alg. I adds the slices' traces t_i before forming
sum |t_i|^2. The paper contracts each network whole (Sec. IV-C); slicing has no counterpart
there. The CPU tests check the plans (width, arena, work, options); the GPU tests check F_J and
the traces against the oracle.
"""
import numpy as np
import pytest

from paper_2103_11595_gb300 import ajf
from paper_2103_11595_gb300 import workloads as W


def _host_plans(inst, alg, variants, trials=4):
    out = []
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, inst)
        for kw in variants:
            out.append(ajf.ajf_plan(c.handle, alg, trials=trials, **kw))
    return out


@pytest.mark.parametrize("alg", [1, 2])
def test_slicing_shrinks_the_widest_tensor_and_costs_work(alg):
    """mid instance (n = 16, 200 gates, 10 noises): each sliced label halves the tensors that
    carry it; the evaluation's total work (all slices) grows, and Alg. I keeps its open indices."""
    variants = [{}] + [{"slice_bonds": s} for s in (1, 2, 4, 8)]
    plans = _host_plans(W.mid(0), alg, variants)
    base = plans[0]
    assert base["n_sliced_bonds"] == 0
    prev = base
    for s, p in zip((1, 2, 4, 8), plans[1:]):
        assert p["n_sliced_bonds"] == s
        assert p["width"] <= prev["width"]
        assert p["arena_bytes"] <= prev["arena_bytes"]
        assert p["flops"] >= base["flops"] * (1 - 1e-12)
        assert p["n_open_bits"] == base["n_open_bits"]
        prev = p
    assert plans[-1]["width"] <= base["width"] - 4
    assert plans[-1]["arena_bytes"] < base["arena_bytes"] / 8


def test_auto_slices_only_as_far_as_the_budget_needs():
    inst = W.mid(0)
    base, roomy = _host_plans(inst, 2, [{}, {"slice_bonds": "auto", "mem_budget_bytes": 1e12}])
    assert roomy["n_sliced_bonds"] == 0 and roomy["width"] == base["width"]
    budget = base["arena_bytes"] / 5
    (tight,) = _host_plans(inst, 2, [{"slice_bonds": "auto", "mem_budget_bytes": budget}])
    assert 1 <= tight["n_sliced_bonds"] <= 8
    assert tight["arena_bytes"] <= budget
    # one label fewer would not fit
    (fewer,) = _host_plans(inst, 2, [{"slice_bonds": tight["n_sliced_bonds"] - 1}])
    assert fewer["arena_bytes"] > budget


def test_auto_reports_budget_error_when_slicing_cannot_fit():
    """The tiny network's arena is mostly descriptors and inputs: no slicing brings it to 1 KB."""
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, W.tiny(0))
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_plan(c.handle, 2, trials=2, slice_bonds="auto", mem_budget_bytes=1024)
        assert e.value.status == ajf.AJF_E_BUDGET
        assert "sliced labels" in str(e.value)


def test_slice_option_checks():
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, W.tiny(1))
        for kw in ({"slice_bonds": ajf.AJF_MAX_SLICE_BONDS + 1}, {"slice_bonds": -2},
                   {"slice_bonds": 1, "alg1_slices": 1}, {"slice_bonds": 1, "lowering": "persistent"}):
            alg = 1 if "alg1_slices" in kw else 2
            with pytest.raises(ajf.AjfError) as e:
                ajf.ajf_plan(c.handle, alg, trials=2, **kw)
            assert e.value.status == ajf.AJF_E_ARG, kw


def test_leaves_keep_a_label():
    """Asking for more labels than can be sliced stops early: a leaf is never left without
    labels, and the Alg. I open Kraus indices are never sliced. The noisy QFT_2 of Example 3
    (10 leaves in Alg. I, 18 in Alg. II) runs out before 24 labels."""
    for alg, leaves, open_bits in ((1, 10, 2), (2, 18, 0)):
        base, p = _host_plans(W.qft2_noisy(0.9), alg, [{}, {"slice_bonds": ajf.AJF_MAX_SLICE_BONDS}])
        assert base["n_leaves"] == leaves
        assert 0 < p["n_sliced_bonds"] <= leaves < ajf.AJF_MAX_SLICE_BONDS
        assert p["n_open_bits"] == open_bits
        assert p["width"] >= max(1, open_bits)


def _sliced_sum(tensors, loops, cut):
    """Sum over every assignment of the labels in `cut` of the contraction with those labels fixed
    in every tensor that carries them (the oracle's own networks and contraction)."""
    from oracle import network
    total = 0
    for v in range(2 ** len(cut)):
        fixed = {x: (v >> j) & 1 for j, x in enumerate(cut)}
        ts = [(arr[tuple(fixed[x] if x in fixed else slice(None) for x in ls)], [x for x in ls if x not in fixed])
              for arr, ls in tensors]
        total += network.contract(ts, loops, order="greedy")[0]
    return total


@pytest.mark.parametrize("seed", range(3))
def test_slicing_identity_on_the_oracle_networks(seed):
    """The identity bond slicing rests on, checked with the oracle's networks and no library code:
    fixing s labels in both tensors that carry them and adding the 2^s contractions gives the full
    contraction (the doubled network's S of Sec. IV-B and one Alg. I trace of Sec. IV-A)."""
    from oracle import dense, network
    inst = W.random_small(seed, n=3 + seed, n_gates=14, n_noises=3, two_qubit_noise=True)
    rng = np.random.default_rng(seed)
    tensors, loops = network.alg2_network(inst)
    labels = sorted({x for _, ls in tensors for x in ls})
    full = network.contract(tensors, loops, order="greedy")[0]
    assert abs(full.real - dense.fidelity(inst)["S"]) <= 1e-10
    for s in (1, 2, 4):
        cut = [int(x) for x in rng.choice(labels, s, replace=False)]
        assert abs(_sliced_sum(tensors, loops, cut) - full) <= 1e-12 * abs(full)
    choice = [int(rng.integers(len(nz.kraus))) for nz in inst.noises]
    tensors, loops = network.alg1_network(inst, choice)
    labels = sorted({x for _, ls in tensors for x in ls})
    t = network.contract(tensors, loops, order="greedy")[0]
    cut = [int(x) for x in rng.choice(labels, 3, replace=False)]
    assert abs(_sliced_sum(tensors, loops, cut) - t) <= 1e-12 * max(1.0, abs(t))


# --------------------------------------------------------------------------- GPU


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _run(inst, alg, precision="f64", use_graph=False, evals=1, **kw):
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, inst)
        info = ajf.ajf_plan(c.handle, alg, trials=4, precision=precision, use_graph=use_graph, **kw)
        rs = [ajf.ajf_fidelity(c.handle) for _ in range(evals)]
        t = ajf.ajf_alg1_traces(c.handle, inst.n_combinations()) if alg == 1 else None
    return rs, t, info


@pytest.mark.gpu
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("s", [1, 2, 3])
def test_sliced_matches_oracle(gpu, seed, s):
    """Random small instances (Haar gates, mixed and 2-qubit noises): F_J, 1 - F_J and every
    trace of the sliced plans against the dense definition, to the FP64 tolerance."""
    from oracle import dense
    inst = W.random_small(seed, n=3 + seed % 3, n_gates=14, n_noises=2 + seed % 3,
                          two_qubit_noise=(seed % 2 == 0))
    ref = dense.fidelity(inst)
    for alg in (1, 2):
        (r,), t, info = _run(inst, alg, slice_bonds=s)
        assert info["n_sliced_bonds"] == s
        assert abs(r["F"] - ref["F"]) <= 1e-12
        assert abs(r["one_minus_F"] - ref["one_minus_F"]) <= 1e-12
        if alg == 1:
            np.testing.assert_allclose(t, ref["traces"], atol=1e-12 * 2 ** inst.n)
            assert r["traces_done"] == inst.n_combinations()


@pytest.mark.gpu
def test_example3_sliced(gpu):
    """Example 3's traces (4p, 0, 0, 0) and F_J = p^2; Example 4's S = 16 p^2, sliced."""
    p = 0.95
    inst = W.qft2_noisy(p)
    (r,), t, _ = _run(inst, 1, slice_bonds=2)
    np.testing.assert_allclose(t, [4 * p, 0, 0, 0], atol=1e-13)
    assert r["F"] == pytest.approx(p * p, abs=1e-13)
    (r,), _, _ = _run(inst, 2, slice_bonds=3)
    assert r["S"] == pytest.approx(16 * p * p, abs=1e-12)


@pytest.fixture(scope="module")
def mid0():
    from oracle import network
    inst = W.mid(0)
    return inst, network.alg2_fidelity(inst, order="minfill")


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("bf16x6", 1e-6)])
def test_mid_auto_slicing_under_a_tight_budget(gpu, mid0, precision, tol):
    """mid instance, Alg. II, with a budget one fifth of the unsliced arena: AJF_SLICE_AUTO
    slices, the arena fits, and F_J matches the oracle (tensor-core GEMMs in bf16x6)."""
    inst, ref = mid0
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, inst)
        base = ajf.ajf_plan(c.handle, 2, trials=4, precision=precision)
    budget = base["arena_bytes"] / 5
    (r, r2), _, info = _run(inst, 2, precision, use_graph=True, evals=2, slice_bonds="auto",
                            mem_budget_bytes=budget)
    assert info["n_sliced_bonds"] >= 1 and info["arena_bytes"] <= budget
    assert abs(r["F"] - ref["F"]) <= tol
    assert abs(r2["F"] - r["F"]) <= 1e-14  # graph replay, new slice values between runs
    if precision == "bf16x6":
        assert info["n_tc_gemms"] > 0


@pytest.mark.gpu
def test_single_run_paths_reject_sliced_plans(gpu):
    inst = W.tiny(2)
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, inst)
        ajf.ajf_plan(c.handle, 2, trials=2, slice_bonds=1)
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_fidelity_noalloc(c.handle, 2)
        assert e.value.status == ajf.AJF_E_STATE
        ajf.ajf_upload(c.handle)
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_launch(c.handle, 0)
        assert e.value.status == ajf.AJF_E_STATE and "sliced" in str(e.value)
        r = ajf.ajf_fidelity_alg2(c.handle)
    from oracle import dense
    assert abs(r["F"] - dense.fidelity(inst)["F"]) <= 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("alg", [1, 2])
def test_batch_of_sliced_and_unsliced_contexts(gpu, alg):
    """ajf_fidelity_batch over contexts on their own streams: bond-sliced ones (1-3 labels) enqueue
    all their runs at once next to unsliced ones; every F_J (and Alg. I trace) against the oracle."""
    import torch
    from oracle import dense
    insts = [W.random_small(s, n=3 + s % 3, n_gates=14, n_noises=2 + s % 2, two_qubit_noise=(s % 2 == 0))
             for s in range(4)]
    streams = [torch.cuda.Stream() for _ in insts]
    ctxs = [ajf.Context(0, st.cuda_stream) for st in streams]
    try:
        for k, (c, inst) in enumerate(zip(ctxs, insts)):
            ajf.load_instance(c.handle, inst)
            ajf.ajf_plan(c.handle, alg, trials=4, slice_bonds=k % 4)
        for _ in range(2):  # the second call replays graphs and reuses the staging buffers
            rs = ajf.ajf_fidelity_batch([c.handle for c in ctxs], alg)
            for r, inst, c in zip(rs, insts, ctxs):
                ref = dense.fidelity(inst)
                assert abs(r["F"] - ref["F"]) <= 1e-12
                assert abs(r["one_minus_F"] - ref["one_minus_F"]) <= 1e-12
                if alg == 1:
                    t = ajf.ajf_alg1_traces(c.handle, inst.n_combinations())
                    np.testing.assert_allclose(t, ref["traces"], atol=1e-12 * 2 ** inst.n)
    finally:
        for c in ctxs:
            c.close()
