"""One F_J evaluation sharded over ranks (one process per GPU).

The units are the independent runs of one evaluation, as the library reports them
(ajf_shard_units): the Kraus-index slices of a sliced Alg. I plan (every trace lies in exactly
one slice, so the slices' sums of |t_i|^2 add up to S), the bond slices of an Alg. II plan (their
scalars add up to S, since slicing splits the contraction's sum over label values), or, for an
Alg. I plan without Kraus slices, the whole evaluation as one unit (its bond slices add traces,
not |t|^2, so they do not split S). Each rank runs a contiguous block of the units through the C
ABI; one FP64 all-reduce of the partial S completes the evaluation, and ajf_fidelity_from_sum
forms F_J = S / 4^n and 1 - F_J (Sec. III). Every rank derives the same split from the same plan,
so all ranks reach the all-reduce. Evaluations of different circuits need no collective at all:
bench.py shards those (weak scaling).

Argument marshalling and the range arithmetic only: every contraction runs in libajf's kernels.
"""
from typing import Callable, Tuple

from . import ajf


def shard_range(n_units: int, rank: int, world: int) -> Tuple[int, int]:
    """(first, count) of rank's contiguous block; the first n_units % world ranks get one more."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("bad rank, world size or unit count")
    base, extra = divmod(n_units, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def rank_work(handle, rank: int, world: int) -> Tuple[int, int, int]:
    """(unit kind, first, count) of rank's block for the context's current plan."""
    kind, n = ajf.ajf_shard_units(handle)
    first, count = shard_range(n, rank, world)
    return kind, first, count


def partial_S(handle, rank: int, world: int) -> float:
    """This rank's part of S for the context's current plan."""
    kind, first, count = rank_work(handle, rank, world)
    if count == 0:
        return 0.0
    if kind == ajf.AJF_UNITS_BOND_SLICES:
        return ajf.ajf_alg2_slice_range(handle, first, count)
    if kind == ajf.AJF_UNITS_KRAUS_SLICES:
        state = ajf.ajf_alg1_checkpoint(handle)
        state.update(next_slice=first, S=0.0, traces_done=0)
        ajf.ajf_alg1_restore(handle, state)
        return ajf.ajf_alg1_continue(handle, -1.0, max_slices=count)["S"]
    return ajf.ajf_fidelity(handle)["S"]


def torch_all_reduce_sum(x: float) -> float:
    """FP64 sum over the ranks of the default torch.distributed group (gloo: host tensor; nccl:
    a tensor on the current CUDA device)."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t)
    return float(t.item())


def sharded_fidelity(handle, n_qubits: int, rank: int, world: int,
                     all_reduce: Callable[[float], float] = torch_all_reduce_sum) -> dict:
    """F_J of the context's plan with the work split over `world` ranks; every rank returns the
    same S, F and 1 - F (formed in the library from the reduced S)."""
    S = all_reduce(partial_S(handle, rank, world))
    return ajf.ajf_fidelity_from_sum(n_qubits, S)
