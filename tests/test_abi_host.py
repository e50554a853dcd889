"""CPU tests of the C-ABI library: it loads, exports every declared symbol, and its host-side logic
(validation, planning, error codes) behaves as include/ajf.h states. No kernel runs here."""
import os
import re

import numpy as np
import pytest

from paper_2103_11595_gb300 import ajf
from paper_2103_11595_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ajf_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert "ajf_fidelity_alg2" in names and "ajf_load_circuit" in names and "ajf_plan" in names
    L = ajf.lib()
    for n in names:
        assert hasattr(L, n), n


def test_version_string():
    assert "sm_103a" in ajf.ajf_version()


def host_ctx():
    return ajf.Context(-1)


def test_rejects_non_unitary_gate():
    with host_ctx() as c:
        bad = W.Gate((0,), np.array([[1, 0], [0, 0.5]], dtype=np.complex128))
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_load_circuit(c.handle, ajf.AJF_IDEAL, 1, *ajf.pack_gates([bad]))
        assert e.value.status == ajf.AJF_E_NOT_UNITARY


def test_rejects_non_trace_preserving_noise():
    with host_ctx() as c:
        ajf.load_instance(c.handle, W.identity_with_noises(1, []))
        kr = W.depolarising(0.1) * 1.01
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_add_noise(c.handle, 0, (0,), kr)
        assert e.value.status == ajf.AJF_E_NOT_TP


@pytest.mark.parametrize("case", ["qubit", "repeat", "after", "arity"])
def test_rejects_bad_indices(case):
    with host_ctx() as c:
        if case == "qubit":
            with pytest.raises(ajf.AjfError) as e:
                ajf.ajf_load_circuit(c.handle, ajf.AJF_IDEAL, 2, *ajf.pack_gates([W.Gate((2,), W.H)]))
        elif case == "repeat":
            with pytest.raises(ajf.AjfError) as e:
                ajf.ajf_load_circuit(c.handle, ajf.AJF_IDEAL, 2, *ajf.pack_gates([W.Gate((1, 1), W.CX)]))
        elif case == "after":
            ajf.load_instance(c.handle, W.identity_with_noises(2, []))
            with pytest.raises(ajf.AjfError) as e:
                ajf.ajf_add_noise(c.handle, 5, (0,), W.depolarising(0.1))
        else:
            ajf.load_instance(c.handle, W.identity_with_noises(2, []))
            with pytest.raises(ajf.AjfError) as e:
                ajf.ajf_add_noise(c.handle, 0, (0, 1, 0, 1), W.depolarising(0.1))
        assert e.value.status == ajf.AJF_E_ARG


def test_call_order_errors():
    with host_ctx() as c:
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_add_noise(c.handle, 0, (0,), W.depolarising(0.1))
        assert e.value.status == ajf.AJF_E_STATE
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_plan(c.handle, 2)
        assert e.value.status == ajf.AJF_E_STATE
        ajf.load_instance(c.handle, W.tiny(0))
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_fidelity_alg2(c.handle)
        assert e.value.status == ajf.AJF_E_STATE
        with pytest.raises(ajf.AjfError):
            ajf.ajf_plan(c.handle, 3)


@pytest.mark.parametrize("alg", [1, 2])
@pytest.mark.parametrize("planner", ["greedy", "minfill", "auto", "learned"])
def test_planning_tiny(alg, planner):
    with host_ctx() as c:
        inst = W.tiny(1)
        ajf.load_instance(c.handle, inst)
        info = ajf.ajf_plan(c.handle, alg, planner=planner, trials=4)
        n_leaves = 2 * len(inst.ideal) + len(inst.noises)
        if alg == 2:
            n_leaves = 2 * n_leaves - len(inst.noises)
        assert info["n_leaves"] >= n_leaves
        assert info["n_steps"] == info["n_leaves"] - 1 - (0 if alg == 1 else 0) or info["n_steps"] > 0
        assert info["n_open_bits"] == (4 if alg == 1 else 0)
        assert info["width"] >= 2 and info["cmacs"] > 0
        assert info["flops"] == pytest.approx(8 * info["cmacs"], rel=1e-12)


def test_plan_is_deterministic():
    with host_ctx() as c:
        ajf.load_instance(c.handle, W.mid(0))
        a = ajf.ajf_plan(c.handle, 2, trials=3, seed=5)
        b = ajf.ajf_plan(c.handle, 2, trials=3, seed=5)
        assert a["cmacs"] == b["cmacs"] and a["width"] == b["width"]


def test_budget_error_reports_plan():
    with host_ctx() as c:
        ajf.load_instance(c.handle, W.mid(0))
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_plan(c.handle, 2, trials=2, mem_budget_bytes=1e6)
        assert e.value.status == ajf.AJF_E_BUDGET
        assert e.value.info["width"] >= 16


def test_alg1_too_many_open_bits_is_budget_error():
    """4x5 grid with a noise on both qubits of every gate: 124 open Kraus bits for Alg. I."""
    with host_ctx() as c:
        ajf.load_instance(c.handle, W.precision(0, depth=4))
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_plan(c.handle, 1, trials=1)
        assert e.value.status == ajf.AJF_E_BUDGET


def test_host_context_cannot_run():
    with host_ctx() as c:
        ajf.load_instance(c.handle, W.tiny(0))
        ajf.ajf_plan(c.handle, 2, trials=1)
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_fidelity_alg2(c.handle)
        assert e.value.status == ajf.AJF_E_STATE


def test_precision_config_as_written_is_over_budget():
    """The 4x5 grid at depth 12 (the precision config as written) plans to a width near 2^80
    elements for Alg. II: the call reports AJF_E_BUDGET with that width and cost. Depth 6 needs
    arenas of about 2^32 elements and more (over a 50 GB budget); depth 4 (2^22-2^24) fits."""
    with host_ctx() as c:
        ajf.load_instance(c.handle, W.precision(0, depth=12))
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_plan(c.handle, 2, trials=2)
        assert e.value.status == ajf.AJF_E_BUDGET
        assert e.value.info["width"] >= 64 and e.value.info["cmacs"] > 1e25
        ajf.load_instance(c.handle, W.precision(0, depth=6))
        with pytest.raises(ajf.AjfError) as e:
            ajf.ajf_plan(c.handle, 2, trials=2, mem_budget_bytes=50e9)
        assert e.value.status == ajf.AJF_E_BUDGET
        ajf.load_instance(c.handle, W.precision(0, depth=4))
        info = ajf.ajf_plan(c.handle, 2, trials=2, mem_budget_bytes=280e9)
        assert info["width"] <= 26


def test_load_packed_matches_load_instance():
    """The flat-array loader (the C-ABI calls alone) gives the same plan as load_instance."""
    inst = W.random_small(5, n=4, n_gates=20, n_noises=3, two_qubit_noise=True)
    inst.impl = list(inst.ideal)
    infos = []
    for loader in (lambda c: ajf.load_instance(c, inst), lambda c: ajf.load_packed(c, ajf.pack_instance(inst))):
        with host_ctx() as c:
            loader(c.handle)
            infos.append(ajf.ajf_plan(c.handle, 2, trials=2))
    for k in ("cmacs", "width", "n_leaves", "upload_bytes"):
        assert infos[0][k] == infos[1][k]
