"""Host-side replay of the device programs (ajf_check_plan): no device needed.

A device memory checker is not available to this library, so every lowered program is replayed
on the host instead. Every address a kernel can form is a base offset plus distinct powers of
two from the step's index maps, so the largest is known. The replay checks:
  - every access lies inside its buffer and arena region, and every operand bit is addressed
    (else elements would be skipped);
  - every read finds the launch that wrote it;
  - no launch writes over a buffer that it, or a later launch, still reads;
  - no two writes of one launch overlap.
These tests run it over the plans of every workload, precision, lowering and slicing option,
and check that planted mistakes of each kind are reported.
"""
import pytest

from paper_2103_11595_gb300 import ajf
from paper_2103_11595_gb300 import workloads as W

ALL_MODES = ["f64", "f32", "tf32", "tf32x3", "bf16x3", "bf16x6"]


def _check(inst, alg, trials=4, **kw):
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, inst)
        info = ajf.ajf_plan(c.handle, alg, trials=trials, **kw)
        ajf.ajf_check_plan(c.handle)
        return info


@pytest.mark.parametrize("precision", ALL_MODES)
def test_tiny_and_small_plans(precision):
    for seed in range(10):
        for alg in (1, 2):
            _check(W.tiny(seed), alg, precision=precision)
            _check(W.random_small(seed, n=3 + seed % 3, n_gates=14, n_noises=2 + seed % 3,
                                  two_qubit_noise=(seed % 2 == 0)), alg, precision=precision)


@pytest.mark.parametrize("precision", ["f64", "bf16x6", "tf32x3", "f32"])
def test_mid_plans(precision):
    """The bench's workload (mid seeds 0-9, Alg. II) and Alg. I on three seeds."""
    for seed in range(10):
        info = _check(W.mid(seed), 2, precision=precision)
        assert info["n_gemm_steps"] > 0
    for seed in range(3):
        _check(W.mid(seed), 1, precision=precision)


def test_precision_and_batching_plans():
    for seed in range(5):
        for precision in ALL_MODES:
            _check(W.precision(seed, depth=4), 2, precision=precision)
    for seed in range(64):
        _check(W.batching_circuit(seed), 1, precision="bf16x6")


def test_persistent_sliced_and_simplified_plans():
    for seed in range(20):
        for alg in (1, 2):
            _check(W.tiny(seed), alg, lowering="persistent")
    for seed in range(4):
        _check(W.batching_circuit(seed), 1, lowering="persistent")
        _check(W.mid(seed), 2, precision="bf16x6", slice_bonds=2 + seed)
        _check(W.mid(seed), 1, slice_bonds=1 + seed)
        _check(W.mid(seed), 1, alg1_slices=1 + seed)
        _check(W.mid(seed), 2, precision="bf16x6", simplify="all")
    _check(W.mid(0), 2, planner="learned")


RULES = {1: "outside the work region", 2: "addresses repeat or overflow", 3: "over its own input",
         4: "that no earlier launch wrote", 5: "writes overlapping buffers", 6: "before unit",
         7: "bit is not addressed", 8: "GEMM shape differs from its gathers"}


@pytest.mark.parametrize("mutation", sorted(RULES))
def test_planted_mistakes_are_reported(mutation):
    """Each mistake is planted in a copy of the program; the check must report it, by the rule
    meant for it (3, 5 and 6 move their buffer's readers along, so that only the overlap is wrong)."""
    cases = ((W.tiny(0), 2, "f64"), (W.tiny(3), 1, "f64"), (W.mid(0), 2, "bf16x6"), (W.batching_circuit(2), 1, "bf16x6"))
    if mutation == 8:  # needs a GEMM: the networks with tensor-core steps
        cases = ((W.mid(0), 2, "bf16x6"), (W.mid(1), 2, "f64"), (W.mid(2), 1, "tf32x3"))
    for inst, alg, precision in cases:
        with ajf.Context(-1) as c:
            ajf.load_instance(c.handle, inst)
            ajf.ajf_plan(c.handle, alg, trials=4, precision=precision)
            report = ajf.ajf_selftest_check_plan(c.handle, mutation)
            assert RULES[mutation] in report, report
            ajf.ajf_check_plan(c.handle)  # the context's own program is unchanged


def test_check_needs_a_plan():
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, W.tiny(0))
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_check_plan(c.handle)
        assert e.value.status == ajf.AJF_E_STATE
        ajf.ajf_plan(c.handle, 2, trials=2)
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_selftest_check_plan(c.handle, 99)
        assert e.value.status == ajf.AJF_E_ARG
