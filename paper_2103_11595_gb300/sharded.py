"""One F_J evaluation sharded over ranks (one process per GPU).

The independent runs of a sliced plan are the units: the Kraus-index slices of a sliced Alg. I
plan (every trace lies in exactly one slice, so the slices' sums of |t_i|^2 add up to S) or the
bond slices of an Alg. II plan (their scalars add up to S, since slicing splits the contraction's
sum over label values). Each rank runs a contiguous block of the units through the C ABI; one
FP64 all-reduce of the partial S completes the evaluation, F_J = S / 4^n (Sec. III). Evaluations
of different circuits need no collective at all: bench.py shards those (weak scaling).

Argument marshalling and the range arithmetic only: every contraction runs in libajf's kernels.
"""
import math
from typing import Callable, Tuple

from . import ajf


def shard_range(n_units: int, rank: int, world: int) -> Tuple[int, int]:
    """(first, count) of rank's contiguous block; the first n_units % world ranks get one more."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("bad rank, world size or unit count")
    base, extra = divmod(n_units, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def partial_S(handle, rank: int, world: int) -> float:
    """This rank's part of S for the context's current plan (Alg. II: bond slices; Alg. I: the
    Kraus-index slices of an alg1_slices plan)."""
    alg = ajf.ajf_planned_alg(handle)
    first, count = shard_range(ajf.ajf_slice_count(handle), rank, world)
    if alg == 2:
        return ajf.ajf_alg2_slice_range(handle, first, count)
    if count == 0:
        return 0.0
    state = ajf.ajf_alg1_checkpoint(handle)
    state.update(next_slice=first, S=0.0, traces_done=0)
    ajf.ajf_alg1_restore(handle, state)
    return ajf.ajf_alg1_continue(handle, -1.0, max_slices=count)["S"]


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
    same S, F and 1 - F (computed as (4^n - S) / 4^n in FP64)."""
    S = all_reduce(partial_S(handle, rank, world))
    d2 = math.ldexp(1.0, 2 * n_qubits)
    return {"S": S, "F": S / d2, "one_minus_F": (d2 - S) / d2}
