"""The batching workload at its full size, in the launch configuration the bench times.

64 circuits (n ~ U{8..20}, 50-300 gates of U3 + nearest-neighbour CX, 6 depolarising noises:
4096 Kraus combinations each), Alg. I (Sec. IV-A):
  - networks of at most 2e6 planned flops get the persistent lowering (FP64) and run together in
    one persistent-kernel launch;
  - the others run their bf16x6 tensor-core programs on streams of their own, at the same time.
Every result is compared with the FP64 default path, and the eight 8-qubit circuits also with the
oracle's own Alg. II network contraction (one evaluation takes it about 1-2 s here). FP64 results
must agree to 1e-12, bf16x6 results to 1e-6.
"""
import numpy as np
import pytest

from paper_2103_11595_gb300 import ajf
from paper_2103_11595_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PERSISTENT_FLOPS_MAX = 2e6  # bench.py's default split between the persistent and default paths


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_batching_config_full_size():
    import torch
    from oracle import network
    insts = [W.batching_circuit(s) for s in range(64)]
    ctxs, streams, persistent = [], [], []
    try:
        for inst in insts:
            with ajf.Context(-1) as probe:
                ajf.load_instance(probe.handle, inst)
                small = ajf.ajf_plan(probe.handle, 1, trials=8, lowering="persistent")["flops"] <= PERSISTENT_FLOPS_MAX
            s = torch.cuda.Stream()
            c = ajf.Context(0, s.cuda_stream)
            ajf.load_instance(c.handle, inst)
            if small:
                ajf.ajf_plan(c.handle, 1, trials=8, lowering="persistent")
            else:
                info = ajf.ajf_plan(c.handle, 1, trials=8, precision="bf16x6", use_graph=True)
                assert info["n_tc_gemms"] > 0 or info["n_gemm_steps"] == 0
            ctxs.append(c)
            streams.append(s)
            persistent.append(small)
        res, n_p = ajf.ajf_fidelity_batch_persistent([c.handle for c in ctxs], 1)
        assert n_p == sum(persistent) and 0 < n_p < 64
        res2, _ = ajf.ajf_fidelity_batch_persistent([c.handle for c in ctxs], 1)  # graph replay
    finally:
        for c in ctxs:
            c.close()
    F = np.array([r["F"] for r in res])
    assert np.max(np.abs(F - np.array([r["F"] for r in res2]))) <= 1e-13
    assert np.all((F > 0) & (F <= 1))

    # the FP64 default path, one context at a time
    F64 = []
    for inst in insts:
        with ajf.Context(0) as c:
            ajf.load_instance(c.handle, inst)
            ajf.ajf_plan(c.handle, 1, trials=8)
            F64.append(ajf.ajf_fidelity_alg1(c.handle)["F"])
    F64 = np.array(F64)
    for i in range(64):
        tol = 1e-12 if persistent[i] else 1e-6
        assert abs(F[i] - F64[i]) <= tol, (i, F[i], F64[i])

    # the oracle on the 8-qubit circuits
    small_n = [i for i, inst in enumerate(insts) if inst.n == 8]
    assert len(small_n) == 8
    for i in small_n:
        ref = network.alg2_fidelity(insts[i], order="minfill")
        assert abs(F64[i] - ref["F"]) <= 1e-12
        assert abs(F[i] - ref["F"]) <= (1e-12 if persistent[i] else 1e-6)
