"""The persistent step interpreter (ajf_launch_queue / ajf_fidelity_batch_queue): one launch runs the
default-lowered programs of many contexts as one task queue, tensor-core GEMM tiles included.

It runs the same device code as the per-context path (the same bodies, the same GEMM work items,
the same fixed summation orders), so its results must equal that path's bit for bit; against the
CPU oracle the path's own tolerance applies (FP64: 1e-12; bf16x6: 1e-6). Its bounded-wait failure
path is tested without any fault: a task that waits for a phase that can never complete.
"""
import numpy as np
import pytest

from oracle import dense, network
from paper_2103_11595_gb300 import ajf
from paper_2103_11595_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def contexts(jobs, precision="bf16x6", trials=4):
    """One context per (instance, alg), planned with the default lowering."""
    ctxs, infos = [], []
    for inst, alg in jobs:
        c = ajf.Context(0)
        ajf.load_instance(c.handle, inst)
        infos.append(ajf.ajf_plan(c.handle, alg, precision=precision, trials=trials))
        ctxs.append(c)
    return ctxs, infos


def close(ctxs):
    for c in ctxs:
        c.close()


def per_context(ctxs, jobs):
    return [ajf.ajf_fidelity_alg1(c.handle) if alg == 1 else ajf.ajf_fidelity_alg2(c.handle)
            for c, (_, alg) in zip(ctxs, jobs)]


def mixed_jobs():
    return [(W.random_small(21, n=7, n_gates=50, n_noises=3, two_qubit_noise=True), 2),
            (W.mid(3, n=10, n_gates=120, n_noises=6), 2),
            (W.batching_circuit(6), 1),
            (W.batching_circuit(9), 1),
            (W.random_small(22, n=8, n_gates=60, n_noises=2), 2)]


def test_timeout_is_reported_and_the_device_stays_usable():
    """A task whose predecessor phase can never complete: its wait expires after 50 ms, the kernel
    records code 21, every block returns, and a real interpreter launch then still works."""
    st, code = ajf.ajf_selftest_queue_timeout(0, 50.0)
    assert st == ajf.AJF_E_TIMEOUT and code == 21
    jobs = [(W.random_small(23, n=6, n_gates=40, n_noises=2), 2)]
    ctxs, _ = contexts(jobs)
    try:
        ref = per_context(ctxs, jobs)
        r = ajf.ajf_fidelity_batch_queue([c.handle for c in ctxs], 2)
        assert r[0]["F"] == ref[0]["F"]
    finally:
        close(ctxs)


def test_one_launch_equals_the_per_context_path_bit_for_bit():
    """Mixed instances (Alg. I and Alg. II, 7-16 qubits, tensor-core GEMMs, K splits): the
    interpreter's F, S and 1 - F equal each context's own run exactly, launch after launch."""
    jobs = mixed_jobs()
    ctxs, infos = contexts(jobs)
    try:
        assert sum(i["n_tc_gemms"] for i in infos) > 0
        ref = per_context(ctxs, jobs)
        for alg in (1, 2):
            idx = [i for i, (_, a) in enumerate(jobs) if a == alg]
            handles = [ctxs[i].handle for i in idx]
            for _ in range(3):  # the first launch builds the tables and the graph; later ones replay it
                got = ajf.ajf_fidelity_batch_queue(handles, alg)
                for k, i in enumerate(idx):
                    assert got[k]["F"] == ref[i]["F"], (i, got[k]["F"], ref[i]["F"])
                    assert got[k]["S"] == ref[i]["S"] and got[k]["one_minus_F"] == ref[i]["one_minus_F"]
    finally:
        close(ctxs)


def test_alg1_traces_after_a_launch():
    """Alg. I contexts run by the interpreter keep their traces: ajf_alg1_traces matches the oracle."""
    inst = W.random_small(24, n=5, n_gates=30, n_noises=3, two_qubit_noise=True)
    ctxs, _ = contexts([(inst, 1)], precision="f64")
    try:
        ajf.ajf_fidelity_batch_queue([ctxs[0].handle], 1)
        t = ajf.ajf_alg1_traces(ctxs[0].handle, inst.n_combinations())
        ref = dense.fidelity(inst)
        assert np.max(np.abs(t - ref["traces"])) <= 1e-12 * 2 ** inst.n
    finally:
        close(ctxs)


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("bf16x6", 1e-6)])
def test_against_the_oracle(precision, tol):
    """Small networks in FP64 (no GEMM-class steps) and mid-size ones in bf16x6 against the dense
    oracle (n <= 8) or the oracle's network contraction."""
    if precision == "f64":
        jobs = [(W.tiny(s), 1 + s % 2) for s in range(12)]
    else:
        jobs = [(W.random_small(25, n=8, n_gates=60, n_noises=3), 2), (W.batching_circuit(6), 1),
                (W.batching_circuit(13), 1)]
    ctxs, _ = contexts(jobs, precision=precision)
    try:
        for alg in (1, 2):
            idx = [i for i, (_, a) in enumerate(jobs) if a == alg]
            if not idx:
                continue
            got = ajf.ajf_fidelity_batch_queue([ctxs[i].handle for i in idx], alg)
            for k, i in enumerate(idx):
                inst = jobs[i][0]
                F = dense.fidelity(inst)["F"] if inst.n <= 6 else network.alg2_fidelity(inst, order="minfill")["F"]
                assert abs(got[k]["F"] - F) <= tol, (i, got[k]["F"], F)
    finally:
        close(ctxs)


def test_batching_workload_in_one_launch():
    """The batching workload at full size (64 circuits, n = 8..20, 6 depolarising noises, 4096 traces
    each; Alg. I, bf16x6) in ONE interpreter launch: every F_J equals the per-context path's, and
    the circuits up to 10 qubits equal the oracle's within 1e-6."""
    jobs = [(W.batching_circuit(s), 1) for s in range(64)]
    ctxs, infos = contexts(jobs, trials=8)
    try:
        handles = [c.handle for c in ctxs]
        got = ajf.ajf_fidelity_batch_queue(handles, 1)
        ref = ajf.ajf_fidelity_batch(handles, 1)
        for g, r in zip(got, ref):
            assert g["F"] == r["F"]
        for (inst, _), g in zip(jobs, got):
            if inst.n <= 10:
                assert abs(g["F"] - network.alg2_fidelity(inst, order="minfill")["F"]) <= 1e-6
    finally:
        close(ctxs)


def test_autotuner_keeps_results():
    """The autotuner times the candidate task shapes and keeps one of them; results are unchanged."""
    jobs = mixed_jobs()[:3]
    ctxs, _ = contexts(jobs)
    try:
        ref = per_context(ctxs, jobs)
        idx = [i for i, (_, a) in enumerate(jobs) if a == 2]
        handles = [ctxs[i].handle for i in idx]
        gi, bt = ajf.ajf_autotune_queue(handles, reps=2)
        assert gi in (1, 2, 4) and bt in (152, 304, 608)
        got = ajf.ajf_fidelity_batch_queue(handles, 2)
        for k, i in enumerate(idx):
            assert got[k]["F"] == ref[i]["F"]
    finally:
        close(ctxs)


def test_rejected_plans():
    """Persistent-lowered and sliced plans, and FP64 plans with GEMM-class steps, are refused."""
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, W.tiny(1))
        ajf.ajf_plan(c.handle, 1, trials=2, lowering="persistent")
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_fidelity_batch_queue([c.handle], 1)
        assert e.value.status == ajf.AJF_E_STATE
        ajf.ajf_plan(c.handle, 2, trials=2, slice_bonds=2)
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_fidelity_batch_queue([c.handle], 2)
        assert e.value.status == ajf.AJF_E_STATE
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, W.mid(3, n=10, n_gates=120, n_noises=6))
        info = ajf.ajf_plan(c.handle, 2, precision="f64", trials=4)
        assert info["n_gemm_steps"] > 0
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_fidelity_batch_queue([c.handle], 2)
        assert e.value.status == ajf.AJF_E_UNSUPPORTED
