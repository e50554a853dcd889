"""ajf_fidelity_noalloc: evaluation in the library's fixed 64 MiB device arena, for callers that
cannot allocate device memory (memory reserved by another allocator, hard memory caps, paths that
must not enter the allocator). It must give the same results as the allocating entry points,
call after call, and refuse plans that do not fit the fixed arena.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

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


# (name, instance, precision, tolerance against the allocating path, tolerance against the
# oracle): the same program on the same device gives the same bits in any arena; against the
# CPU oracle the path's own tolerance applies (FP64: 1e-12; FP32-accumulated bf16x6: 1e-6)
CASES = [("tiny", lambda: W.tiny(4), "f64", 1e-12, 1e-12),
         ("small5", lambda: W.random_small(11, n=5, n_gates=40, n_noises=3, two_qubit_noise=True), "f64", 1e-12,
          1e-12),
         ("line10", lambda: W.mid(3, n=10, n_gates=120, n_noises=6), "bf16x6", 1e-12, 1e-6)]


def _oracle_F(inst):
    from oracle import dense, network
    return dense.fidelity(inst)["F"] if inst.n <= 6 else network.alg2_fidelity(inst, order="minfill")["F"]


@pytest.mark.parametrize("alg", [1, 2])
@pytest.mark.parametrize("name,make,precision,tol,tol_oracle", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_allocating_entry_point(name, make, precision, tol, tol_oracle, alg):
    inst = make()
    F_oracle = _oracle_F(inst)
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, inst)
        info = ajf.ajf_plan(c.handle, alg, precision=precision, trials=8)
        if precision != "f64":  # the tensor-core GEMM path runs in the fixed arena too
            assert info["n_tc_gemms"] > 0, info
        assert ajf.ajf_workspace_size(c.handle) <= 64 << 20
        ref = ajf.ajf_fidelity_alg1(c.handle) if alg == 1 else ajf.ajf_fidelity_alg2(c.handle)
        for _ in range(2):  # two calls in a row share (and overwrite) the fixed arena
            r = ajf.ajf_fidelity_noalloc(c.handle, alg)
            assert abs(r["F"] - ref["F"]) <= tol
            assert abs(r["S"] - ref["S"]) <= tol * max(1.0, abs(ref["S"]))
            assert r["traces_done"] == ref["traces_done"]
            assert abs(r["F"] - F_oracle) <= tol_oracle, (r["F"], F_oracle)
        # the allocating path still works after the fixed-arena calls (its own prepared launches)
        again = ajf.ajf_fidelity_alg1(c.handle) if alg == 1 else ajf.ajf_fidelity_alg2(c.handle)
        assert again["F"] == ref["F"]
        if alg == 1:  # the allocating path's trace buffer is untouched
            t = ajf.ajf_alg1_traces(c.handle, inst.n_combinations())
            assert np.isclose(np.sum(np.abs(t) ** 2) / 4 ** inst.n, ref["F"], atol=1e-12)


def test_noalloc_alternating_contexts():
    """Two contexts used one after the other leave no state in the shared arena that matters."""
    a, b = W.tiny(5), W.random_small(12, n=4, n_gates=20, n_noises=2)
    with ajf.Context(0) as ca, ajf.Context(0) as cb:
        for c, inst in ((ca, a), (cb, b)):
            ajf.load_instance(c.handle, inst)
            ajf.ajf_plan(c.handle, 2, trials=4)
        ra, rb = ajf.ajf_fidelity_alg2(ca.handle), ajf.ajf_fidelity_alg2(cb.handle)
        for _ in range(2):
            assert abs(ajf.ajf_fidelity_noalloc(ca.handle, 2)["F"] - ra["F"]) <= 1e-12
            assert abs(ajf.ajf_fidelity_noalloc(cb.handle, 2)["F"] - rb["F"]) <= 1e-12


def test_noalloc_rejects_plans_larger_than_the_fixed_arena():
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, W.mid(0))
        ajf.ajf_plan(c.handle, 2, precision="bf16x3", trials=4)
        assert ajf.ajf_workspace_size(c.handle) > 64 << 20
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_fidelity_noalloc(c.handle, 2)
        assert e.value.status == ajf.AJF_E_NOMEM
        assert "64" in str(e.value) or "67108864" in str(e.value)
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_fidelity_noalloc(c.handle, 1)
        assert e.value.status == ajf.AJF_E_STATE
