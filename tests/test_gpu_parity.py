"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the same seeded inputs.

Tolerances (stated for the whole path):
  FP64 contraction (AJF_PREC_F64):        |dF| <= 1e-12, traces |dt| <= 1e-12 * d
  FP32-accumulated contractions:          |dF| <= 1e-6, relative error of 1 - F <= 1e-3
The FP64 end of the path (trace, sum |t|^2, F, 1 - F) is FP64 in every mode.
"""
import math

import numpy as np
import pytest

from oracle import dense, network
from paper_2103_11595_gb300 import ajf
from paper_2103_11595_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-6, "bf16x6": 1e-6}
# bounded modes: the two-term splits keep a floating leading term whose TMEM accumulation truncates
# once per promoted K block, a small systematic shrink of every GEMM result (F comes out low); the
# scaled fp16 split carries ~22 bits of each row block's largest entry, within 1e-6 on the line and
# grid workloads but up to ~1.4e-5 on Alg. I networks whose rows span many Kraus-weight scales
BOUND = {"tf32x3": 5e-6, "bf16x3": 5e-6, "f16x3": 3e-5}


def check_bounded(r, ref, precision):
    """A bounded mode: |dF| within its measured bound (the truncating modes err low)."""
    err = r["F"] - ref["F"]
    print(f"{precision}: dF = {err:.3e}")
    assert abs(err) <= BOUND[precision]
    if precision != "f16x3":
        assert err <= 1e-7


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def run(inst, alg, precision="f64", planner="auto", trials=8, use_graph=False, seed=0):
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, inst)
        info = ajf.ajf_plan(c.handle, alg, precision=precision, planner=planner, trials=trials,
                            use_graph=use_graph, seed=seed)
        r = ajf.ajf_fidelity_alg1(c.handle) if alg == 1 else ajf.ajf_fidelity_alg2(c.handle)
        t = ajf.ajf_alg1_traces(c.handle, inst.n_combinations()) if alg == 1 else None
    return r, t, info


def check(r, ref, tol, rel_inf=1e-3):
    assert abs(r["F"] - ref["F"]) <= tol, (r["F"], ref["F"])
    assert abs(r["S"] / 4 ** 0 - ref["S"]) <= tol * max(1.0, abs(ref["S"])), (r["S"], ref["S"])
    if ref["one_minus_F"] > 1e-9 and tol > 1e-10:
        assert abs(r["one_minus_F"] - ref["one_minus_F"]) <= rel_inf * ref["one_minus_F"]


# --------------------------------------------------------------------------- worked examples


@pytest.mark.parametrize("p", [0.3, 0.95, 0.999])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_example3_and_4(p, precision):
    """Example 3: traces (4p,0,0,0), F = p^2; Example 4: Alg. II value 16 p^2."""
    inst = W.qft2_noisy(p)
    tol = TOL[precision]
    r1, t, _ = run(inst, 1, precision)
    np.testing.assert_allclose(t, [4 * p, 0, 0, 0], atol=4 * tol)
    assert r1["F"] == pytest.approx(p * p, abs=tol)
    r2, _, _ = run(inst, 2, precision)
    assert r2["S"] == pytest.approx(16 * p * p, abs=16 * tol)
    assert r2["F"] == pytest.approx(p * p, abs=tol)


def test_early_exit_decision():
    """Remark after Example 3: p = 0.95 is 0.1-equivalent (F = 0.9025 > 0.9), not 0.09-equivalent."""
    inst = W.qft2_noisy(0.95)
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, inst)
        ajf.ajf_plan(c.handle, 1, trials=2)
        assert ajf.ajf_fidelity_alg1(c.handle, eps=0.1)["equivalent"] == 1
        assert ajf.ajf_fidelity_alg1(c.handle, eps=0.09)["equivalent"] == 0
        assert ajf.ajf_fidelity_alg1(c.handle)["equivalent"] == -1


# --------------------------------------------------------------------------- tiny config


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_tiny_config(seed, precision):
    inst = W.tiny(seed)
    ref = dense.fidelity(inst)
    tol = TOL[precision]
    r1, t, _ = run(inst, 1, precision)
    check(r1, ref, tol)
    np.testing.assert_allclose(t, ref["traces"], atol=8 * tol * 2 ** inst.n)
    r2, _, _ = run(inst, 2, precision)
    check(r2, ref, tol)


@pytest.mark.parametrize("seed", range(8))
def test_random_small_instances(seed):
    """Haar gates, mixed noises, a 2-qubit noise, implementation skeleton != ideal."""
    inst = W.random_small(seed, n=3 + seed % 3, n_gates=14, n_noises=2 + seed % 3,
                          two_qubit_noise=(seed % 2 == 0))
    if seed % 3 == 1:
        rng = np.random.default_rng(seed)
        impl = list(inst.ideal)
        impl[1] = W.Gate(impl[1].qubits, W.haar_unitary(rng, 2 ** impl[1].arity))
        inst.impl = impl
    ref = dense.fidelity(inst)
    for alg in (1, 2):
        r, t, _ = run(inst, alg, "f64", planner=["greedy", "minfill", "auto"][seed % 3])
        check(r, ref, 1e-12)
        if alg == 1:
            np.testing.assert_allclose(t, ref["traces"], atol=1e-12 * 2 ** inst.n)


@pytest.mark.parametrize("planner", ["greedy", "minfill"])
@pytest.mark.parametrize("seed", range(3))
def test_order_invariance_on_device(planner, seed):
    """Different contraction orders (planner, seed) give the same F_J."""
    inst = W.random_small(20 + seed, n=5, n_gates=30, n_noises=3)
    ref = dense.fidelity(inst)["F"]
    for s in range(3):
        r, _, _ = run(inst, 2, "f64", planner=planner, trials=1, seed=s)
        assert r["F"] == pytest.approx(ref, abs=1e-12)


# --------------------------------------------------------------------------- edge cases


def test_noiseless_and_idle_wires():
    """No noise: F = 1; qubits no gate touches close into loops (factor 2 per wire)."""
    inst = W.Instance(4, [W.Gate((1,), W.H), W.Gate((1, 2), W.CX)], [])
    for alg in (1, 2):
        r, _, _ = run(inst, alg)
        assert r["F"] == pytest.approx(1.0, abs=1e-13)
    inst = W.Instance(4, [W.Gate((1,), W.H)], [W.Noise(0, (1,), W.depolarising(0.2))])
    for alg in (1, 2):
        r, _, _ = run(inst, alg)
        assert r["F"] == pytest.approx(0.85, abs=1e-13)


def test_single_op_wire_closure():
    """An implementation without a gate the ideal circuit has on one wire (one op on that wire)."""
    ideal = [W.Gate((0,), W.H), W.Gate((1,), W.T)]
    impl = [W.Gate((0,), W.H), W.Gate((0,), W.I2)]
    inst = W.Instance(2, ideal, [W.Noise(0, (0,), W.amplitude_damping(0.3))], impl=impl)
    ref = dense.fidelity(inst)
    for alg in (1, 2):
        r, _, _ = run(inst, alg)
        check(r, ref, 1e-12)


def test_padded_kraus_count():
    """A 3-operator Kraus set (padded to 4 with a zero operator) and a 16-operator 2-qubit set."""
    k3 = np.stack([np.sqrt(0.5) * W.I2, np.sqrt(0.3) * W.X, np.sqrt(0.2) * W.Z])
    inst = W.random_small(3, n=3, n_gates=8, n_noises=0)
    inst.noises = [W.Noise(2, (1,), k3), W.Noise(5, (0, 2), W.two_qubit_depolarising(0.1))]
    ref = dense.fidelity(inst)
    r, t, _ = run(inst, 1)
    check(r, ref, 1e-12)
    np.testing.assert_allclose(t, ref["traces"], atol=1e-12 * 8)


def test_cuda_graph_replay_matches():
    inst = W.tiny(2)
    ref = dense.fidelity(inst)
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, inst)
        ajf.ajf_plan(c.handle, 2, trials=4, use_graph=True)
        for _ in range(3):
            assert ajf.ajf_fidelity_alg2(c.handle)["F"] == pytest.approx(ref["F"], abs=1e-12)


def test_borrowed_workspace_and_stream():
    import torch
    inst = W.random_small(1, n=4, n_gates=16, n_noises=2)
    ref = dense.fidelity(inst)
    stream = torch.cuda.Stream()
    with ajf.Context(0, stream.cuda_stream) as c:
        ajf.load_instance(c.handle, inst)
        ajf.ajf_plan(c.handle, 2, trials=4)
        nbytes = ajf.ajf_workspace_size(c.handle)
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        ajf.ajf_set_workspace(c.handle, ws.data_ptr(), nbytes)
        assert ajf.ajf_fidelity_alg2(c.handle)["F"] == pytest.approx(ref["F"], abs=1e-12)
        small = torch.empty(256, dtype=torch.uint8, device="cuda")
        ajf.ajf_set_workspace(c.handle, small.data_ptr(), 256)
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_fidelity_alg2(c.handle)
        assert e.value.status == ajf.AJF_E_NOMEM


def test_launch_async_device_result():
    import torch
    inst = W.tiny(3)
    ref = dense.fidelity(inst)
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, inst)
        ajf.ajf_plan(c.handle, 2, trials=2, use_graph=True)
        ajf.ajf_upload(c.handle)
        out = torch.zeros(3, dtype=torch.float64, device="cuda")
        ajf.ajf_launch(c.handle, out.data_ptr())
        torch.cuda.synchronize()
        assert out[1].item() == pytest.approx(ref["F"], abs=1e-12)


def test_batch_of_contexts():
    insts = [W.random_small(40 + s, n=3 + s % 2, n_gates=12, n_noises=2) for s in range(4)]
    ctxs = [ajf.Context(0) for _ in insts]
    try:
        for c, inst in zip(ctxs, insts):
            ajf.load_instance(c.handle, inst)
            ajf.ajf_plan(c.handle, 1, trials=2)
        res = ajf.ajf_fidelity_alg1_batch([c.handle for c in ctxs])
        for r, inst in zip(res, insts):
            assert r["F"] == pytest.approx(dense.fidelity(inst)["F"], abs=1e-12)
    finally:
        for c in ctxs:
            c.close()


# --------------------------------------------------------------------------- full-size (n = 16) cases


def test_mid_noiseless_and_single_noise_closed_forms():
    """n=16, 200 gates: no noise gives F = 1; one noise anywhere gives sum |tr K|^2 / 4."""
    inst = W.mid(0)
    noises = inst.noises
    inst.noises = []
    for prec in ("f64", "f32"):
        r, _, _ = run(inst, 2, prec, trials=8)
        assert r["F"] == pytest.approx(1.0, abs=TOL[prec])
    inst.noises = [noises[3]]
    expect = sum(abs(np.trace(K)) ** 2 for K in noises[3].kraus) / 4
    for alg in (1, 2):
        r, _, _ = run(inst, alg, "f64", trials=8)
        assert r["F"] == pytest.approx(expect, abs=1e-12)


@pytest.fixture(scope="module")
def mid0_oracle():
    inst = W.mid(0)
    return inst, network.alg2_fidelity(inst, order="minfill")


@pytest.mark.parametrize("precision", ["f64", "f32", "tf32x3", "bf16x6", "f16x3"])
def test_mid_config_alg2(mid0_oracle, precision):
    """n=16 line, 200 gates, 10 mixed noises: Alg. II on the GPU vs the oracle's own network."""
    inst, ref = mid0_oracle
    r, _, info = run(inst, 2, precision, trials=16)
    assert info["width"] <= 28
    if precision in ("tf32x3", "bf16x6", "f16x3"):
        assert info["n_tc_gemms"] > 0
    if precision in BOUND and precision != "f16x3":
        check_bounded(r, ref, precision)
    else:  # f16x3 is bounded, but within 1e-6 on this workload (every bench seed is checked too)
        check(r, ref, TOL.get(precision, 1e-6))


@pytest.mark.parametrize("precision,bound", [("tf32", 1e-3), ("bf16x3", 5e-6)])
def test_mid_config_low_precision_error_is_bounded(mid0_oracle, precision, bound):
    """One-pass TF32 (11 significant bits) and the two-term bf16 split (16 bits) are not FP32-class
    operand precisions; their errors are measured and bounded (bf16x3 reached 1.2e-6 .. 3.9e-6 on
    validation circuits)."""
    inst, ref = mid0_oracle
    r, _, info = run(inst, 2, precision, trials=16)
    assert info["n_tc_gemms"] > 0
    err = abs(r["F"] - ref["F"])
    print(f"{precision}: |dF| = {err:.3e}")
    assert err <= bound


@pytest.fixture(scope="module")
def precision_oracle():
    inst = W.precision(0, depth=4)
    return inst, network.alg2_fidelity(inst, order="minfill")


@pytest.mark.parametrize("precision", ["f64", "tf32x3", "bf16x6", "f16x3"])
def test_precision_config_alg2(precision_oracle, precision):
    """4x5 grid, depth-4 brickwork of Haar SU(4), depolarising on both qubits of every gate
    (62 noises): Alg. II against the oracle; bf16x6 within 1e-6, tf32x3 within its bound."""
    inst, ref = precision_oracle
    r, _, info = run(inst, 2, precision, trials=16)
    if precision != "f64":
        assert info["n_tc_gemms"] > 0
    if precision in BOUND:
        check_bounded(r, ref, precision)
    else:
        check(r, ref, TOL[precision])


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x6", "f16x3"])
def test_batching_circuit_alg1(precision):
    """A circuit of the batching workload (n=14, 296 gates, 6 depolarising noises, 4096 traces):
    Alg. I on tensor cores against Alg. I and Alg. II in FP64; two traces against the oracle."""
    inst = W.batching_circuit(1)
    r64, t64, _ = run(inst, 1, "f64", trials=8)
    r2, _, _ = run(inst, 2, "f64", trials=8)
    assert abs(r64["F"] - r2["F"]) <= 1e-12
    r, t, info = run(inst, 1, precision, trials=8)
    assert info["n_tc_gemms"] > 0
    if precision in BOUND:
        check_bounded(r, r64, precision)
    else:
        err = abs(r["F"] - r64["F"])
        print(f"{precision}: |dF| = {err:.3e}")
        assert err <= TOL[precision]
    for choice in ([0] * 6, [1, 0, 2, 0, 0, 3]):
        idx = 0
        for c in choice:
            idx = idx * 4 + c
        val = network.alg1_trace(inst, choice, order="minfill", rng=None)
        assert abs(t64[idx] - val) <= 1e-12 * 2 ** inst.n


def test_mid_config_alg1_vs_alg2(mid0_oracle):
    """Alg. I (open Kraus indices) and Alg. II agree at full size; sampled traces match the
    oracle's single-network Alg. I contraction one by one."""
    inst, ref = mid0_oracle
    r1, t, _ = run(inst, 1, "f64", trials=16)
    check(r1, ref, 1e-12)
    rng = np.random.default_rng(0)
    dims = [nz.n_kraus for nz in inst.noises]
    for _ in range(3):
        choice = [int(rng.integers(d)) for d in dims]
        idx = 0
        for j, d in enumerate(dims):
            idx = idx * d + choice[j]
        val = network.alg1_trace(inst, choice, order="minfill")
        assert abs(t[idx] - val) <= 1e-12 * 2 ** inst.n


@pytest.mark.parametrize("use_graph", [False, True])
def test_replan_same_structure_new_values(use_graph):
    """A re-plan of the same circuit structure with new gate and noise values reuses the lowered
    program (and its CUDA graph) and uploads only the new values: F_J follows the new values."""
    base = W.random_small(5, n=6, n_gates=40, n_noises=3)
    rng = np.random.default_rng(11)
    def same_kind(nz, k):  # new values, same number of Kraus operators
        kr = W.depolarising(0.05 * (k + 1)) if nz.n_kraus == 4 else W.amplitude_damping(0.1 * (k + 1))
        assert kr.shape == nz.kraus.shape
        return W.Noise(nz.after_gate, nz.qubits, kr)
    other = W.Instance(base.n, [W.Gate(g.qubits, W.haar_unitary(rng, 2 ** len(g.qubits))) for g in base.ideal],
                       [same_kind(nz, k) for k, nz in enumerate(base.noises)])
    with ajf.Context(0) as c:
        for k, inst in enumerate([base, other, base]):
            ajf.load_instance(c.handle, inst)
            info = ajf.ajf_plan(c.handle, 2, precision="f64", trials=4, use_graph=use_graph)
            assert info["plan_cached"] == (1 if k > 0 else 0)
            r = ajf.ajf_fidelity_alg2(c.handle)
            assert abs(r["F"] - dense.fidelity(inst)["F"]) <= 1e-12


# --------------------------------------------------------------------------- reduced precision vs the oracle

_ORACLE_F = {}


def _oracle_alg2(key, make):
    """The oracle's F_J and 1 - F_J (doubled network, min-fill order, complex128), once per input."""
    if key not in _ORACLE_F:
        _ORACLE_F[key] = network.alg2_fidelity(make(), order="minfill")
    return _ORACLE_F[key]


@pytest.mark.parametrize("precision", ["bf16x6", "f16x3", "tf32x3"])
@pytest.mark.parametrize("seed", [4, 10, 29, 36])
def test_batching_alg1_tensor_cores_vs_oracle(seed, precision):
    """Batching workload circuits with n <= 16 (6 depolarising noises, 4096 traces): Alg. I on the
    tensor cores against the oracle's F_J directly (Sec. III: F_J = sum |tr|^2 / d^2): bf16x6 within
    the FP32-accumulated tolerance (1 - F_J to 1e-3 relative), tf32x3 within its bound."""
    inst = W.batching_circuit(seed)
    assert inst.n <= 16
    ref = _oracle_alg2(("batch", seed), lambda: W.batching_circuit(seed))
    r, _, info = run(inst, 1, precision, trials=8)
    assert info["n_tc_gemms"] > 0
    print(f"seed {seed} {precision}: |dF| = {abs(r['F'] - ref['F']):.3e}")
    if precision in BOUND:
        check_bounded(r, ref, precision)
    else:
        check(r, ref, TOL[precision])


@pytest.mark.parametrize("precision", ["bf16x6", "f16x3"])
@pytest.mark.parametrize("seed", range(10))
def test_mid_bench_seeds_vs_oracle(seed, precision):
    """Every instance the bench times (mid workload, seeds 0-9, Alg. II, the bench's 32 planner
    restarts) against the oracle's own network contraction: bf16x6 within the FP32-accumulated
    tolerance; the scaled fp16 split within 1e-6 here too (measured), though it is a bounded mode."""
    ref = _oracle_alg2(("mid", seed), lambda: W.mid(seed))
    r, _, info = run(W.mid(seed), 2, precision, trials=32)
    assert info["n_tc_gemms"] > 0
    print(f"mid seed {seed} {precision}: |dF| = {abs(r['F'] - ref['F']):.3e}")
    check(r, ref, 1e-6)
