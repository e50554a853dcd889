"""One F_J evaluation sharded over ranks: the independent runs of a sliced plan (bond slices for
Alg. II, Kraus-index slices for Alg. I) split into contiguous blocks, one FP64 all-reduce of the
partial S. The CPU tests cover the range arithmetic and the all-reduce with two gloo ranks
(127.0.0.1); the GPU tests run every rank's block in one process, one after another (their
kernels never wait on one another), and check F_J against the oracle.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2103_11595_gb300 import ajf, sharded
from paper_2103_11595_gb300 import workloads as W


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_shard_ranges_partition_the_units(world):
    for n in range(0, 23):
        ranges = [sharded.shard_range(n, r, world) for r in range(world)]
        covered = [i for first, count in ranges for i in range(first, first + count)]
        assert covered == list(range(n))
        sizes = [count for _, count in ranges]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharded.shard_range(4, 2, 2)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_units, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # stand-in for the device runs: unit i contributes 1 + i / 8 (exact in binary)
    sharded.partial_S = lambda handle, r, w: sum(1 + i / 8 for i in range(*_span(sharded.shard_range(n_units, r, w))))
    res = sharded.sharded_fidelity(None, 1, rank, world)
    out.put((rank, res))
    dist.destroy_process_group()


def _span(fc):
    return fc[0], fc[0] + fc[1]


def test_two_gloo_ranks_all_reduce_the_partial_sums():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    n_units = 13
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, n_units, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total = sum(1 + i / 8 for i in range(n_units))
    for _, r in res:
        assert r["S"] == total
        assert r["F"] == total / 4 and r["one_minus_F"] == (4 - total) / 4


def test_slice_counts_of_plans():
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, W.tiny(0))      # 2 depolarising noises, 4 Kraus operators each
        with pytest.raises(ajf.AjfError) as e:           # no plan yet
            ajf.ajf_slice_count(c.handle)
        assert e.value.status == ajf.AJF_E_STATE
        ajf.ajf_plan(c.handle, 1, trials=2)
        with pytest.raises(ajf.AjfError) as e:           # an Alg. I plan has no Alg. II slices
            ajf.ajf_alg2_slice_range(c.handle, 0, 1)
        assert e.value.status == ajf.AJF_E_STATE and "Alg. II" in str(e.value)
        ajf.ajf_plan(c.handle, 2, trials=2)
        assert ajf.ajf_slice_count(c.handle) == 1
        ajf.ajf_plan(c.handle, 2, trials=2, slice_bonds=3)
        assert ajf.ajf_slice_count(c.handle) == 8
        ajf.ajf_plan(c.handle, 1, trials=2, alg1_slices=2)
        assert ajf.ajf_slice_count(c.handle) == 16
        ajf.ajf_plan(c.handle, 2, trials=2, slice_bonds=1)
        with pytest.raises(ajf.AjfError) as e:           # host-only contexts run nothing
            ajf.ajf_alg2_slice_range(c.handle, 0, 1)
        assert e.value.status == ajf.AJF_E_STATE


def test_shard_units_of_plans():
    """ajf_shard_units: Kraus slices for a sliced Alg. I plan, bond slices for Alg. II, and the
    whole evaluation as one unit for an Alg. I plan without Kraus slices (bond sliced or not)."""
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, W.tiny(0))
        ajf.ajf_plan(c.handle, 1, trials=2)
        assert ajf.ajf_shard_units(c.handle) == (ajf.AJF_UNITS_WHOLE, 1)
        ajf.ajf_plan(c.handle, 1, trials=2, slice_bonds=2)
        assert ajf.ajf_shard_units(c.handle) == (ajf.AJF_UNITS_WHOLE, 1)
        ajf.ajf_plan(c.handle, 1, trials=2, alg1_slices=2)
        assert ajf.ajf_shard_units(c.handle) == (ajf.AJF_UNITS_KRAUS_SLICES, 16)
        ajf.ajf_plan(c.handle, 2, trials=2, slice_bonds=3)
        assert ajf.ajf_shard_units(c.handle) == (ajf.AJF_UNITS_BOND_SLICES, 8)
        ajf.ajf_plan(c.handle, 2, trials=2)
        assert ajf.ajf_shard_units(c.handle) == (ajf.AJF_UNITS_BOND_SLICES, 1)
        # every rank derives the same split: the whole Alg. I evaluation lands on rank 0 alone
        ajf.ajf_plan(c.handle, 1, trials=2, slice_bonds=2)
        assert [sharded.rank_work(c.handle, r, 3) for r in range(3)] == [(0, 0, 1), (0, 1, 0), (0, 1, 0)]


def test_fidelity_from_sum():
    """F = S / 4^n and 1 - F = (4^n - S) / 4^n in FP64, Definition 1's decision, argument checks."""
    r = ajf.ajf_fidelity_from_sum(2, 15.5, eps=0.05, traces_done=7)
    assert r["F"] == 15.5 / 16 and r["one_minus_F"] == 0.5 / 16 and r["S"] == 15.5
    assert r["equivalent"] == 1 and r["traces_done"] == 7
    assert ajf.ajf_fidelity_from_sum(2, 15.0, eps=0.05)["equivalent"] == 0
    assert ajf.ajf_fidelity_from_sum(2, 15.0)["equivalent"] == -1
    # 1 - F keeps the digits that S / 4^n rounds away near F = 1
    n = 20
    S = 4.0 ** n - 3.0
    assert ajf.ajf_fidelity_from_sum(n, S)["one_minus_F"] == 3.0 / 4.0 ** n
    for bad in ((0, 1.0), (63, 1.0), (2, -1.0), (2, float("nan")), (2, float("inf"))):
        with pytest.raises(ajf.AjfError):
            ajf.ajf_fidelity_from_sum(*bad)
    with pytest.raises(ajf.AjfError):
        ajf.ajf_fidelity_from_sum(2, 1.0, eps=1.5)


def _whole_unit_rank(rank, world, port, out):
    """A rank holding an Alg. I plan without Kraus slices (host-only context): it must reach the
    all-reduce whatever its block is, with the device run replaced by an exact stand-in S."""
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    with ajf.Context(-1) as c:
        ajf.load_instance(c.handle, W.tiny(0))
        ajf.ajf_plan(c.handle, 1, trials=2)
        kind, first, count = sharded.rank_work(c.handle, rank, world)
        ajf.ajf_fidelity = lambda h, eps=-1.0: {"S": 60.0}   # stand-in for the device evaluation
        res = sharded.sharded_fidelity(c.handle, 3, rank, world)
    out.put((rank, (kind, first, count), res))
    dist.destroy_process_group()


def test_unsliced_alg1_plan_over_two_gloo_ranks():
    """An Alg. I plan without Kraus slices is one unit: rank 0 runs it, rank 1 contributes 0, and
    both ranks return the same F (no rank stops short of the all-reduce)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_whole_unit_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == (ajf.AJF_UNITS_WHOLE, 0, 1) and res[1][1] == (ajf.AJF_UNITS_WHOLE, 1, 0)
    for _, _, r in res:
        assert r["S"] == 60.0 and r["F"] == 60.0 / 64 and r["one_minus_F"] == 4.0 / 64


# --------------------------------------------------------------------------- GPU


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _sharded(inst, alg, world, precision="f64", **plan):
    """Every rank's block in its own context, one after another; the all-reduce is their sum."""
    parts = []
    for r in range(world):
        with ajf.Context(0) as c:
            ajf.load_instance(c.handle, inst)
            ajf.ajf_plan(c.handle, alg, trials=4, precision=precision, **plan)
            parts.append(sharded.partial_S(c.handle, r, world))
    return ajf.ajf_fidelity_from_sum(inst.n, sum(parts))


@pytest.mark.gpu
@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("world", [1, 2, 3])
def test_alg2_bond_slices_sharded(gpu, seed, world):
    from oracle import dense
    inst = W.random_small(seed, n=3 + seed, n_gates=14, n_noises=3, two_qubit_noise=(seed % 2 == 0))
    ref = dense.fidelity(inst)
    r = _sharded(inst, 2, world, slice_bonds=3)
    assert abs(r["F"] - ref["F"]) <= 1e-12
    assert abs(r["one_minus_F"] - ref["one_minus_F"]) <= 1e-12


@pytest.mark.gpu
def test_alg2_unsliced_plan_is_one_unit(gpu):
    """Without bond slicing the plan is one unit: the second rank's block is empty."""
    from oracle import dense
    inst = W.tiny(4)
    r = _sharded(inst, 2, 2)
    assert abs(r["F"] - dense.fidelity(inst)["F"]) <= 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("world", [2, 5])
def test_alg1_kraus_slices_sharded(gpu, world):
    """Alg. I sharded by Kraus-index slices (checkpoint state moved to each rank's first slice)."""
    from oracle import dense
    inst = W.random_small(7, n=4, n_gates=14, n_noises=3, two_qubit_noise=True)
    ref = dense.fidelity(inst)
    r = _sharded(inst, 1, world, alg1_slices=2)
    assert abs(r["F"] - ref["F"]) <= 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("slice_bonds", [0, 2])
def test_alg1_whole_unit_sharded(gpu, slice_bonds):
    """An Alg. I plan without Kraus slices (unsliced, or bond sliced) over two ranks: rank 0 runs
    the whole evaluation, rank 1 contributes 0, and F_J equals the oracle's."""
    from oracle import dense
    inst = W.random_small(8, n=4, n_gates=14, n_noises=3)
    ref = dense.fidelity(inst)
    r = _sharded(inst, 1, 2, slice_bonds=slice_bonds)
    assert abs(r["F"] - ref["F"]) <= 1e-12
    assert abs(r["one_minus_F"] - ref["one_minus_F"]) <= 1e-12


@pytest.mark.gpu
def test_mid_instance_sharded_over_four_ranks(gpu):
    """mid instance (n = 16), Alg. II with 4 bond slices in bf16x6 over 4 ranks, against the
    oracle's own network contraction (FP32-accumulated tolerance)."""
    from oracle import network
    inst = W.mid(0)
    ref = network.alg2_fidelity(inst, order="minfill")
    r = _sharded(inst, 2, 4, precision="bf16x6", slice_bonds=4)
    assert abs(r["F"] - ref["F"]) <= 1e-6


@pytest.mark.gpu
def test_slice_range_checks(gpu):
    with ajf.Context(0) as c:
        ajf.load_instance(c.handle, W.tiny(5))
        ajf.ajf_plan(c.handle, 2, trials=2, slice_bonds=2)
        for first, count in ((-1, 1), (0, 5), (4, 1), (2, -1)):
            with pytest.raises(ajf.AjfError) as e:
                ajf.ajf_alg2_slice_range(c.handle, first, count)
            assert e.value.status == ajf.AJF_E_ARG
        assert ajf.ajf_alg2_slice_range(c.handle, 4, 0) == 0.0
        whole = ajf.ajf_alg2_slice_range(c.handle, 0, 4)
        parts = sum(ajf.ajf_alg2_slice_range(c.handle, i, 1) for i in range(4))
        assert abs(whole - parts) <= 1e-12 * abs(whole)
        assert abs(whole - ajf.ajf_fidelity_alg2(c.handle)["S"]) <= 1e-12 * abs(whole)
