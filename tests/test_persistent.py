"""Persistent execution: many small networks in one kernel launch, one thread block per network.

The persistent lowering turns every pairwise step into a CUDA-core gather or reduction step in
FP64, so the results must match the oracle to the FP64 tolerance (|dF| <= 1e-12) like the
default FP64 path. CPU tests cover the lowering and option checks; GPU tests compare with the
oracle on the tiny config, Examples 3/4, random small instances (2-qubit noise, different
implementation skeleton), networks whose tensors stay in the arena instead of shared memory, a
batch mixing persistent and default plans, and the asynchronous device-result entry point.
"""
import numpy as np
import pytest

from paper_2103_11595_gb300 import ajf
from paper_2103_11595_gb300 import workloads as W


def _plan_host(inst, alg, **kw):
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, inst)
        info = ajf.ajf_plan(c.handle, alg, **kw)
        launches = ajf.ajf_plan_launches(c.handle)
    return info, launches


@pytest.mark.parametrize("alg", [1, 2])
def test_persistent_lowering_has_no_gemm(alg):
    info, launches = _plan_host(W.batching_circuit(24), alg, lowering="persistent", trials=2)
    assert info["n_gemm_steps"] == 0
    assert {l["kind"] for l in launches} <= {"leaves", "small", "splitk", "final"}
    d_info, d_launches = _plan_host(W.batching_circuit(24), alg, trials=2)
    assert d_info["n_gemm_steps"] > 0  # the default lowering does use GEMMs on this circuit
    assert info["cmacs"] == d_info["cmacs"]  # same path: lowering does not change the plan


def test_persistent_lowering_requires_f64():
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, W.tiny(0))
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_plan(c.handle, 2, precision="bf16x6", lowering="persistent")
        assert e.value.status == ajf.AJF_E_ARG
        with pytest.raises(ajf.AjfError):
            ajf.ajf_plan(c.handle, 2, lowering=7)


def test_launch_persistent_needs_persistent_plan_and_device():
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, W.tiny(0))
        ajf.ajf_plan(c.handle, 2, lowering="persistent")
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_launch_persistent([c.handle])
        assert e.value.status == ajf.AJF_E_ARG  # host-only context


# --------------------------------------------------------------------------- GPU


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _contexts(insts, alg, lowering="persistent", stream=None):
    ctxs = []
    for inst in insts:
        c = ajf.Context(0, stream) if stream else ajf.Context(0)
        ajf.load_instance(c.handle, inst)
        ajf.ajf_plan(c.handle, alg, trials=4, lowering=lowering)
        ctxs.append(c)
    return ctxs


def _close(ctxs):
    for c in ctxs:
        c.close()


@pytest.mark.gpu
@pytest.mark.parametrize("alg", [1, 2])
def test_tiny_config_one_launch(gpu, alg):
    """Tiny config, seeds 0-99 in one persistent launch: F_J and (Alg. I) traces vs the oracle."""
    from oracle import dense
    insts = [W.tiny(s) for s in range(100)]
    refs = [dense.fidelity(i) for i in insts]
    ctxs = _contexts(insts, alg)
    try:
        res, n_p = ajf.ajf_fidelity_batch_persistent([c.handle for c in ctxs], alg)
        assert n_p == len(insts)
        for r, ref in zip(res, refs):
            assert abs(r["F"] - ref["F"]) <= 1e-12
            assert abs(r["one_minus_F"] - ref["one_minus_F"]) <= 1e-12
        if alg == 1:
            for c, inst, ref in list(zip(ctxs, insts, refs))[:10]:
                t = ajf.ajf_alg1_traces(c.handle, inst.n_combinations())
                np.testing.assert_allclose(t, ref["traces"], atol=1e-12 * 2 ** inst.n)
    finally:
        _close(ctxs)


@pytest.mark.gpu
@pytest.mark.parametrize("p", [0.3, 0.999])
def test_examples_3_and_4(gpu, p):
    """Example 3: traces (4p, 0, 0, 0) and F = p^2; Example 4: Alg. II value 16 p^2."""
    inst = W.qft2_noisy(p)
    for alg in (1, 2):
        ctxs = _contexts([inst], alg)
        try:
            (r,), _ = ajf.ajf_fidelity_batch_persistent([ctxs[0].handle], alg)
            assert r["F"] == pytest.approx(p * p, abs=1e-13)
            if alg == 1:
                np.testing.assert_allclose(ajf.ajf_alg1_traces(ctxs[0].handle, 4), [4 * p, 0, 0, 0], atol=1e-12)
            else:
                assert r["S"] == pytest.approx(16 * p * p, abs=1e-12)
        finally:
            _close(ctxs)


@pytest.mark.gpu
def test_random_small_instances(gpu):
    """Haar gates, mixed and 2-qubit noises, a different implementation skeleton; both algorithms."""
    from oracle import dense
    insts = []
    for seed in range(12):
        inst = W.random_small(seed, n=3 + seed % 4, n_gates=16, n_noises=2 + seed % 3,
                              two_qubit_noise=(seed % 2 == 0))
        if seed % 3 == 1:
            rng = np.random.default_rng(seed)
            impl = list(inst.ideal)
            impl[1] = W.Gate(impl[1].qubits, W.haar_unitary(rng, 2 ** impl[1].arity))
            inst.impl = impl
        insts.append(inst)
    refs = [dense.fidelity(i)["F"] for i in insts]
    for alg in (1, 2):
        ctxs = _contexts(insts, alg)
        try:
            res, _ = ajf.ajf_fidelity_batch_persistent([c.handle for c in ctxs], alg)
            for r, ref in zip(res, refs):
                assert abs(r["F"] - ref) <= 1e-12
        finally:
            _close(ctxs)


@pytest.mark.gpu
def test_arena_resident_networks_and_mixed_batch(gpu):
    """Batching-config circuits: the larger persistent plans keep their tensors in the arena
    (work region above the shared-memory limit); a batch mixes persistent and default plans and
    every result equals the default FP64 path's."""
    seeds = [0, 8, 40, 48]  # small batching-config circuits (n = 10..20)
    insts = [W.batching_circuit(s) for s in seeds]
    ref = []
    for inst in insts:
        with ajf.Context(0) as c:
            ajf.load_instance(c.handle, inst)
            ajf.ajf_plan(c.handle, 1, trials=4)
            ref.append(ajf.ajf_fidelity_alg1(c.handle)["F"])
    lows = ["persistent", "persistent", "default", "persistent"]
    widths = [_plan_host(i, 1, trials=4, lowering="persistent")[0]["width"] for i, l in zip(insts, lows)
              if l == "persistent"]
    assert max(widths) >= 13  # a 2^13-element complex FP64 tensor alone exceeds the 96 KiB of shared memory
    ctxs = []
    try:
        for inst, low in zip(insts, lows):
            ctxs += _contexts([inst], 1, lowering=low)
        res, n_p = ajf.ajf_fidelity_batch_persistent([c.handle for c in ctxs], 1)
        assert n_p == 3
        for r, f in zip(res, ref):
            assert abs(r["F"] - f) <= 1e-12
    finally:
        _close(ctxs)


@pytest.mark.gpu
def test_launch_persistent_device_results_repeat(gpu):
    """The asynchronous entry point writes {S, F, 1-F} per network to device memory; repeated
    launches (cached job table) and contexts on different streams give the same values."""
    import torch
    from oracle import dense
    insts = [W.tiny(s, n=4, n_gates=24) for s in range(16)]
    refs = [dense.fidelity(i)["F"] for i in insts]
    streams = [torch.cuda.Stream() for _ in range(4)]
    ctxs = []
    try:
        for k, inst in enumerate(insts):
            ctxs += _contexts([inst], 2, stream=streams[k % 4].cuda_stream)
        out = torch.zeros(len(insts), 3, dtype=torch.float64, device="cuda")
        for rep in range(3):
            out.zero_()
            torch.cuda.synchronize()
            ajf.ajf_launch_persistent([c.handle for c in ctxs], out.data_ptr())
            torch.cuda.synchronize()
            F = out[:, 1].cpu().numpy()
            np.testing.assert_allclose(F, refs, atol=1e-12, rtol=0)
        # the regular launch path runs a persistent-lowered plan too
        r = ajf.ajf_fidelity_alg2(ctxs[0].handle)
        assert abs(r["F"] - refs[0]) <= 1e-12
    finally:
        _close(ctxs)


def test_autotune_needs_device_batch():
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, W.tiny(0))
        ajf.ajf_plan(c.handle, 2, lowering="persistent")
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_autotune_persistent([c.handle])
        assert e.value.status == ajf.AJF_E_ARG  # host-only context


@pytest.mark.gpu
@pytest.mark.parametrize("alg", [1, 2])
def test_autotuned_block_size_keeps_results(gpu, alg):
    """The autotuner times the batch at 256, 128 and 64 threads per block; the chosen size is
    used by later launches of the same batch, and every size gives the oracle's F_J."""
    from oracle import dense
    insts = [W.tiny(s) for s in range(40)]
    refs = [dense.fidelity(i)["F"] for i in insts]
    ctxs = _contexts(insts, alg)
    try:
        with pytest.raises(ajf.AjfError):
            ajf.ajf_autotune_persistent([c.handle for c in ctxs], reps=0)
        t = ajf.ajf_autotune_persistent([c.handle for c in ctxs], reps=3)
        assert t in (64, 128, 256)
        res, n_p = ajf.ajf_fidelity_batch_persistent([c.handle for c in ctxs], alg)
        assert n_p == len(insts)
        for r, ref in zip(res, refs):
            assert abs(r["F"] - ref) <= 1e-12
        # a new batch of the same structures (fresh contexts) runs at the remembered size
        again = _contexts(insts, alg)
        try:
            res2, _ = ajf.ajf_fidelity_batch_persistent([c.handle for c in again], alg)
            for r, ref in zip(res2, refs):
                assert abs(r["F"] - ref) <= 1e-12
        finally:
            _close(again)
    finally:
        _close(ctxs)
