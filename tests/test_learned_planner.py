"""The learned merge scorer (AJF_PLANNER_LEARNED): dataset, training, planning and F_J parity.

A planner only chooses the order of pairwise contractions, so whatever path the learned scorer
proposes, F_J must equal the oracle's to the FP64 tolerance. CPU tests cover the dataset builder
and host-side scoring; GPU tests train the MLP with the library's CUDA kernels and check F_J.
"""
import math

import numpy as np
import pytest

from paper_2103_11595_gb300 import ajf
from paper_2103_11595_gb300 import workloads as W


def _dataset(seeds, trials=1, negatives=4):
    chunks = []
    with ajf.Context(-1) as c:
        for s in seeds:
            ajf.load_instance(c.handle, W.random_pairs_circuit(s))
            chunks.append(ajf.ajf_learned_dataset(c.handle, 2, trials=trials, seed=s, negatives=negatives))
    return np.concatenate(chunks)


def _random_model(seed=0):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(ajf.ajf_learned_param_count()) * 0.05).astype(np.float32)


def test_param_count():
    # 16 features -> 224 -> 192 -> 1, biases included
    assert ajf.ajf_learned_param_count() == 16 * 224 + 224 + 224 * 192 + 192 + 192 + 1


def test_dataset_shape_and_content():
    d = _dataset([3])
    assert d.ndim == 3 and d.shape[1:] == (2, 16) and d.shape[0] > 0
    assert np.isfinite(d).all()
    # the chosen and the other candidate differ in at least one feature for most pairs
    assert np.mean(np.any(d[:, 0, :] != d[:, 1, :], axis=1)) > 0.5


def test_learned_without_model_is_greedy():
    inst = W.mid(1)
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, inst)
        g = ajf.ajf_plan(c.handle, 2, planner="greedy", trials=1)
        l = ajf.ajf_plan(c.handle, 2, planner="learned", trials=1)
    assert l["cmacs"] == g["cmacs"] and l["width"] == g["width"]


def test_host_learned_plan_is_valid_and_judged():
    """Host scoring with a model: the greedy planner judges, so the kept path is never worse in
    estimated time than the one-pass greedy path; the plan cache keys on the model version."""
    inst = W.random_pairs_circuit(10001)
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, inst)
        ajf.ajf_set_learned_model(c.handle, _random_model())

        def plan(planner):
            try:
                return ajf.ajf_plan(c.handle, 2, planner=planner, trials=1, mem_budget_bytes=1e18)
            except ajf.AjfError as e:
                assert e.status == ajf.AJF_E_BUDGET
                return e.info

        g = plan("greedy")
        l1 = plan("learned")
        assert l1["cmacs"] > 0 and math.isfinite(l1["cmacs"])
        assert l1["planner_used"] in (ajf.AJF_PLANNER_GREEDY, ajf.AJF_PLANNER_LEARNED)
        if l1["planner_used"] == ajf.AJF_PLANNER_GREEDY:
            assert l1["cmacs"] == g["cmacs"]
        ajf.ajf_set_learned_model(c.handle, _random_model(1))
        l2 = plan("learned")
        assert l2["plan_cached"] == 0


def test_set_model_rejects_wrong_size():
    with ajf.Context(-1) as c:
        with pytest.raises(ajf.AjfError):
            ajf.ajf_set_learned_model(c.handle, np.zeros(10, np.float32))


# --------------------------------------------------------------------------- GPU


@pytest.fixture(scope="module")
def gpu_built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def trained(gpu_built):
    data = _dataset(range(6))
    w1, loss1 = ajf.ajf_learned_train(0, data, epochs=1, batch=256, lr=1e-3, seed=0)
    w8, loss8 = ajf.ajf_learned_train(0, data, epochs=8, batch=256, lr=1e-3, seed=0)
    return data, (w1, loss1), (w8, loss8)


@pytest.mark.gpu
def test_training_reduces_ranking_loss(trained):
    data, (w1, loss1), (w8, loss8) = trained
    assert w8.shape == (ajf.ajf_learned_param_count(),) and np.isfinite(w8).all()
    assert math.isfinite(loss1) and math.isfinite(loss8)
    # softplus ranking loss of an uninformed scorer is log 2
    assert loss8 < loss1 and loss8 < math.log(2.0)


@pytest.mark.gpu
@pytest.mark.parametrize("alg", [1, 2])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_learned_plan_fidelity_tiny(trained, alg, seed):
    from oracle import dense
    inst = W.tiny(seed)
    ref = dense.fidelity(inst)
    _, _, (w8, _) = trained
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, inst)
        ajf.ajf_set_learned_model(c.handle, w8)
        ajf.ajf_plan(c.handle, alg, planner="learned", trials=2, precision="f64")
        r = ajf.ajf_fidelity_alg1(c.handle) if alg == 1 else ajf.ajf_fidelity_alg2(c.handle)
    assert abs(r["F"] - ref["F"]) <= 1e-12


@pytest.mark.gpu
def test_learned_plan_fidelity_mid(trained):
    """n = 16, 200 gates, 10 noises: the learned path (device scoring) gives the oracle's F_J."""
    from oracle import network
    inst = W.mid(0)
    ref = network.alg2_fidelity(inst, order="minfill")
    _, _, (w8, _) = trained
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, inst)
        ajf.ajf_set_learned_model(c.handle, w8)
        info = ajf.ajf_plan(c.handle, 2, planner="learned", trials=1, precision="f64")
        r = ajf.ajf_fidelity_alg2(c.handle)
    assert info["planner_used"] in (ajf.AJF_PLANNER_GREEDY, ajf.AJF_PLANNER_LEARNED)
    assert abs(r["F"] - ref["F"]) <= 1e-12
