"""Planner regression guard on the host: the AUTO planner's plans of the ten mid instances (the
benchmark's step) pass the host-side plan check and keep their planned work at or below the level
the lowering-aware time model reaches (1.074e12 flops per step with 32 restarts; 1.55e12 with the
flop-count model it replaced). No GPU: host-only contexts plan and check."""
from paper_2103_11595_gb300 import ajf
from paper_2103_11595_gb300 import workloads as W


def test_mid_plans_checked_and_within_budget():
    total = 0.0
    for s in range(10):
        with ajf.Context(-1) as c:
            ajf.load_instance(c.handle, W.mid(s))
            info = ajf.ajf_plan(c.handle, 2, precision="bf16x6", trials=32)
            ajf.ajf_check_plan(c.handle)
            launches = ajf.ajf_plan_launches(c.handle)
            assert sum(1 for l in launches if l["kind"] == "gemm_tc") == info["n_tc_gemms"]
            total += info["flops"]
    assert total <= 1.10e12, total
