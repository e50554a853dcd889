"""Thin ctypes binding of libajf (include/ajf.h), with the same function names.

Argument marshalling only: every step of the computation runs inside the library's CUDA
kernels. Importing this module does not load the library; the first call does, and raises if
``libajf.so`` has not been built (``__graft_entry__.build()``) -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libajf.so")

AJF_OK, AJF_E_ARG, AJF_E_NOT_UNITARY, AJF_E_NOT_TP, AJF_E_STATE = 0, 1, 2, 3, 4
AJF_E_BUDGET, AJF_E_NOMEM, AJF_E_CUDA, AJF_E_TIMEOUT, AJF_E_UNSUPPORTED = 5, 6, 7, 8, 9
AJF_IDEAL, AJF_IMPL = 0, 1
AJF_UNITS_WHOLE, AJF_UNITS_KRAUS_SLICES, AJF_UNITS_BOND_SLICES = 0, 1, 2
AJF_PLANNER_AUTO, AJF_PLANNER_GREEDY, AJF_PLANNER_MINFILL, AJF_PLANNER_LEARNED = 0, 1, 2, 3
AJF_PREC_F64, AJF_PREC_F32, AJF_PREC_TF32, AJF_PREC_TF32X3, AJF_PREC_BF16X3, AJF_PREC_BF16X6 = 0, 1, 2, 3, 4, 5
AJF_PREC_F16X3 = 6
PRECISIONS = {"f64": AJF_PREC_F64, "f32": AJF_PREC_F32, "tf32": AJF_PREC_TF32, "tf32x3": AJF_PREC_TF32X3,
              "bf16x3": AJF_PREC_BF16X3, "bf16x6": AJF_PREC_BF16X6, "f16x3": AJF_PREC_F16X3}
PLANNERS = {"auto": AJF_PLANNER_AUTO, "greedy": AJF_PLANNER_GREEDY, "minfill": AJF_PLANNER_MINFILL,
            "learned": AJF_PLANNER_LEARNED}


class PlanOpts(ctypes.Structure):
    _fields_ = [("planner", ctypes.c_int32), ("precision", ctypes.c_int32), ("trials", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("seed", ctypes.c_uint64), ("mem_budget_bytes", ctypes.c_double),
                ("lowering", ctypes.c_int32), ("simplify", ctypes.c_int32), ("alg1_slices", ctypes.c_int32),
                ("slice_bonds", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("cmacs", ctypes.c_double), ("flops", ctypes.c_double), ("bytes", ctypes.c_double),
                ("gemm_flops", ctypes.c_double), ("gemm_bytes", ctypes.c_double), ("arena_bytes", ctypes.c_double),
                ("plan_seconds", ctypes.c_double), ("width", ctypes.c_int32), ("n_steps", ctypes.c_int32),
                ("n_gemm_steps", ctypes.c_int32), ("n_leaves", ctypes.c_int32), ("n_open_bits", ctypes.c_int32),
                ("planner_used", ctypes.c_int32), ("n_launches", ctypes.c_int32), ("n_tc_gemms", ctypes.c_int32),
                ("plan_cached", ctypes.c_int32), ("n_removed", ctypes.c_int32), ("upload_bytes", ctypes.c_double),
                ("n_sliced_bonds", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class KernelStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double)]


AJF_LOWER_DEFAULT, AJF_LOWER_PERSISTENT = 0, 1
AJF_ALG_AUTO = 0
AJF_SIMPLIFY_SWAP, AJF_SIMPLIFY_CANCEL = 1, 2
AJF_SLICE_AUTO, AJF_MAX_SLICE_BONDS = -1, 24
SIMPLIFY = {"none": 0, "swap": AJF_SIMPLIFY_SWAP, "cancel": AJF_SIMPLIFY_CANCEL,
            "all": AJF_SIMPLIFY_SWAP | AJF_SIMPLIFY_CANCEL}
LOWERINGS = {"default": AJF_LOWER_DEFAULT, "persistent": AJF_LOWER_PERSISTENT}
KERNEL_CLASSES = ["leaves", "small", "splitk", "gather", "gemm_simt", "gemm_tc", "final", "persistent"]


class LaunchInfo(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("terms", ctypes.c_int32), ("M", ctypes.c_int64), ("N", ctypes.c_int64),
                ("K", ctypes.c_int64), ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("F", ctypes.c_double), ("one_minus_F", ctypes.c_double), ("S", ctypes.c_double),
                ("traces_done", ctypes.c_int64), ("equivalent", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class Alg1State(ctypes.Structure):
    _fields_ = [("next_slice", ctypes.c_int64), ("n_slices", ctypes.c_int64), ("S", ctypes.c_double),
                ("traces_done", ctypes.c_int64), ("plan_sig", ctypes.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class AjfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"ajf status {status}: {message}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "ajf_create": (I32, [ctypes.POINTER(P), ctypes.c_int, P]),
            "ajf_destroy": (None, [P]),
            "ajf_last_error": (ctypes.c_char_p, [P]),
            "ajf_load_circuit": (I32, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P]),
            "ajf_add_noise": (I32, [P, I32, I32, P, I32, P]),
            "ajf_clear_noise": (I32, [P]),
            "ajf_plan": (I32, [P, ctypes.c_int, ctypes.POINTER(PlanOpts), ctypes.POINTER(PlanInfo)]),
            "ajf_set_workspace": (I32, [P, P, ctypes.c_size_t]),
            "ajf_workspace_size": (I32, [P, ctypes.POINTER(ctypes.c_size_t)]),
            "ajf_fidelity_alg1": (I32, [P, D, ctypes.POINTER(Result)]),
            "ajf_fidelity_alg2": (I32, [P, D, ctypes.POINTER(Result)]),
            "ajf_fidelity": (I32, [P, D, ctypes.POINTER(Result)]),
            "ajf_alg1_continue": (I32, [P, D, I64, ctypes.POINTER(Result)]),
            "ajf_alg1_checkpoint": (I32, [P, ctypes.POINTER(Alg1State)]),
            "ajf_alg1_restore": (I32, [P, ctypes.POINTER(Alg1State)]),
            "ajf_autotune_persistent": (I32, [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, ctypes.POINTER(I32)]),
            "ajf_planned_alg": (I32, [P, ctypes.POINTER(ctypes.c_int)]),
            "ajf_slice_count": (I32, [P, ctypes.POINTER(I64)]),
            "ajf_shard_units": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(I64)]),
            "ajf_fidelity_from_sum": (I32, [ctypes.c_int, D, D, I64, ctypes.POINTER(Result)]),
            "ajf_check_plan": (I32, [P]),
            "ajf_selftest_check_plan": (I32, [P, ctypes.c_int]),
            "ajf_alg2_slice_range": (I32, [P, I64, I64, ctypes.POINTER(D)]),
            "ajf_alg1_traces": (I32, [P, P, I64]),
            "ajf_launch": (I32, [P, P]),
            "ajf_upload": (I32, [P]),
            "ajf_fidelity_alg1_batch": (I32, [ctypes.POINTER(P), ctypes.c_int, D, ctypes.POINTER(Result)]),
            "ajf_fidelity_batch": (I32, [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, D, ctypes.POINTER(Result)]),
            "ajf_version": (ctypes.c_char_p, []),
            "ajf_selftest_gemm": (I32, [ctypes.c_int, ctypes.c_int, ctypes.c_int, I64, I64, I64, P, P, P]),
            "ajf_fidelity_noalloc": (I32, [P, ctypes.c_int, D, ctypes.POINTER(Result)]),
            "ajf_selftest_split_gemm": (I32, [ctypes.c_int, ctypes.c_int, I64, I64, I64, P, P, P]),
            "ajf_selftest_wait_timeout": (I32, [ctypes.c_int, D, ctypes.POINTER(I32)]),
            "ajf_learned_param_count": (I32, []),
            "ajf_set_learned_model": (I32, [P, P, I32]),
            "ajf_learned_dataset": (I32, [P, ctypes.c_int, I32, ctypes.c_uint64, I32, P, I64, ctypes.POINTER(I64)]),
            "ajf_learned_train": (I32, [ctypes.c_int, P, I64, I32, I32, ctypes.c_float, ctypes.c_uint64, P, I32,
                                        ctypes.POINTER(D)]),
            "ajf_plan_launches": (I32, [P, ctypes.POINTER(LaunchInfo), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
            "ajf_profile_enable": (I32, [P, ctypes.c_int]),
            "ajf_profile_read": (I32, [P, ctypes.POINTER(KernelStats), ctypes.c_int]),
            "ajf_launch_persistent": (I32, [ctypes.POINTER(P), ctypes.c_int, P]),
            "ajf_launch_queue": (I32, [ctypes.POINTER(P), ctypes.c_int, P]),
            "ajf_queue_profile": (I32, [P, P, ctypes.c_int, ctypes.c_int]),
            "ajf_selftest_queue_timeout": (I32, [ctypes.c_int, D, ctypes.POINTER(I32)]),
            "ajf_fidelity_batch_queue": (I32, [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, D,
                                               ctypes.POINTER(Result)]),
            "ajf_autotune_queue": (I32, [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, ctypes.POINTER(I32),
                                         ctypes.POINTER(I32)]),
            "ajf_fidelity_batch_persistent": (I32, [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, D,
                                                    ctypes.POINTER(Result), ctypes.POINTER(I32)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(ctx, status: int):
    if status != AJF_OK:
        msg = lib().ajf_last_error(ctx).decode() if ctx else ""
        raise AjfError(status, msg)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------- C-ABI mirrors


def ajf_version() -> str:
    return lib().ajf_version().decode()


def ajf_create(device: int = 0, stream: Optional[int] = None) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    st = lib().ajf_create(ctypes.byref(ctx), device, ctypes.c_void_p(stream) if stream else None)
    if st != AJF_OK:
        raise AjfError(st, f"ajf_create(device={device}) failed")
    return ctx


def ajf_destroy(ctx) -> None:
    lib().ajf_destroy(ctx)


def ajf_last_error(ctx) -> str:
    return lib().ajf_last_error(ctx).decode()


def ajf_load_circuit(ctx, role: int, n_qubits: int, arity: np.ndarray, qubits: np.ndarray, mats: np.ndarray) -> None:
    arity = np.ascontiguousarray(arity, dtype=np.int32)
    qubits = np.ascontiguousarray(qubits, dtype=np.int32)
    mats = np.ascontiguousarray(mats, dtype=np.complex128)
    _check(ctx, lib().ajf_load_circuit(ctx, role, n_qubits, int(arity.size), _ptr(arity), _ptr(qubits), _ptr(mats)))


def ajf_add_noise(ctx, after_gate: int, qubits: Sequence[int], kraus: np.ndarray) -> None:
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    k = np.ascontiguousarray(kraus, dtype=np.complex128)
    _check(ctx, lib().ajf_add_noise(ctx, int(after_gate), int(q.size), _ptr(q), int(k.shape[0]), _ptr(k)))


def ajf_clear_noise(ctx) -> None:
    _check(ctx, lib().ajf_clear_noise(ctx))


def ajf_plan(ctx, alg: int, planner="auto", precision="f64", trials: int = 0, use_graph: bool = False,
             seed: int = 0, mem_budget_bytes: float = 0.0, lowering="default", simplify="none",
             alg1_slices: int = 0, slice_bonds=0) -> dict:
    """alg: 1, 2 or AJF_ALG_AUTO (0). slice_bonds: a count of labels to slice, or "auto"
    (AJF_SLICE_AUTO: as many as the memory budget needs)."""
    o = PlanOpts()
    o.slice_bonds = AJF_SLICE_AUTO if slice_bonds == "auto" else int(slice_bonds)
    o.simplify = SIMPLIFY[simplify] if isinstance(simplify, str) else int(simplify)
    o.alg1_slices = int(alg1_slices)
    o.lowering = LOWERINGS[lowering] if isinstance(lowering, str) else int(lowering)
    o.planner = PLANNERS[planner] if isinstance(planner, str) else int(planner)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.trials = int(trials)
    o.use_graph = 1 if use_graph else 0
    o.seed = int(seed)
    o.mem_budget_bytes = float(mem_budget_bytes)
    info = PlanInfo()
    st = lib().ajf_plan(ctx, int(alg), ctypes.byref(o), ctypes.byref(info))
    if st != AJF_OK:
        err = AjfError(st, ajf_last_error(ctx))
        err.info = info.as_dict()
        raise err
    return info.as_dict()


def ajf_set_workspace(ctx, dev_ptr: int, nbytes: int) -> None:
    _check(ctx, lib().ajf_set_workspace(ctx, ctypes.c_void_p(dev_ptr) if dev_ptr else None, int(nbytes)))


def ajf_workspace_size(ctx) -> int:
    n = ctypes.c_size_t()
    _check(ctx, lib().ajf_workspace_size(ctx, ctypes.byref(n)))
    return int(n.value)


def ajf_upload(ctx) -> None:
    _check(ctx, lib().ajf_upload(ctx))


def ajf_fidelity_alg1(ctx, eps: float = -1.0) -> dict:
    r = Result()
    _check(ctx, lib().ajf_fidelity_alg1(ctx, float(eps), ctypes.byref(r)))
    return r.as_dict()


def ajf_fidelity(ctx, eps: float = -1.0) -> dict:
    """The planned algorithm (ajf_plan's choice under AJF_ALG_AUTO)."""
    r = Result()
    _check(ctx, lib().ajf_fidelity(ctx, float(eps), ctypes.byref(r)))
    return r.as_dict()


def ajf_alg1_continue(ctx, eps: float = -1.0, max_slices: int = 0) -> dict:
    """Run up to max_slices more slices of a sliced Alg. I plan (0: all that remain)."""
    r = Result()
    _check(ctx, lib().ajf_alg1_continue(ctx, float(eps), int(max_slices), ctypes.byref(r)))
    return r.as_dict()


def ajf_alg1_checkpoint(ctx) -> dict:
    st = Alg1State()
    _check(ctx, lib().ajf_alg1_checkpoint(ctx, ctypes.byref(st)))
    return st.as_dict()


def ajf_alg1_restore(ctx, state: dict) -> None:
    st = Alg1State(**state)
    _check(ctx, lib().ajf_alg1_restore(ctx, ctypes.byref(st)))


def ajf_planned_alg(ctx) -> int:
    a = ctypes.c_int()
    _check(ctx, lib().ajf_planned_alg(ctx, ctypes.byref(a)))
    return int(a.value)


def ajf_check_plan(ctx) -> None:
    """Host-side replay of the plan's address arithmetic and buffer lifetimes; raises on a violation."""
    _check(ctx, lib().ajf_check_plan(ctx))


def ajf_selftest_check_plan(ctx, mutation: int) -> str:
    """Plant mistake `mutation` in a copy of the plan; returns the check's report (raises if missed)."""
    _check(ctx, lib().ajf_selftest_check_plan(ctx, int(mutation)))
    return ajf_last_error(ctx)


def ajf_slice_count(ctx) -> int:
    n = ctypes.c_int64()
    _check(ctx, lib().ajf_slice_count(ctx, ctypes.byref(n)))
    return int(n.value)


def ajf_shard_units(ctx) -> tuple:
    """(kind, n_units): how one evaluation of the plan splits into independent units
    (AJF_UNITS_WHOLE, AJF_UNITS_KRAUS_SLICES or AJF_UNITS_BOND_SLICES)."""
    k, n = ctypes.c_int32(), ctypes.c_int64()
    _check(ctx, lib().ajf_shard_units(ctx, ctypes.byref(k), ctypes.byref(n)))
    return int(k.value), int(n.value)


def ajf_fidelity_from_sum(n_qubits: int, S: float, eps: float = -1.0, traces_done: int = 0) -> dict:
    """F, 1 - F and the decision from S = sum |tr|^2 (no context, no device)."""
    r = Result()
    st = lib().ajf_fidelity_from_sum(int(n_qubits), float(S), float(eps), int(traces_done), ctypes.byref(r))
    if st != AJF_OK:
        raise AjfError(st, "ajf_fidelity_from_sum: bad arguments")
    return r.as_dict()


def ajf_alg2_slice_range(ctx, first: int, count: int) -> float:
    """Sum of the scalars of bond slices [first, first + count) of an Alg. II plan (FP64)."""
    s = ctypes.c_double()
    _check(ctx, lib().ajf_alg2_slice_range(ctx, int(first), int(count), ctypes.byref(s)))
    return float(s.value)


def ajf_fidelity_alg2(ctx, eps: float = -1.0) -> dict:
    r = Result()
    _check(ctx, lib().ajf_fidelity_alg2(ctx, float(eps), ctypes.byref(r)))
    return r.as_dict()


def ajf_fidelity_noalloc(ctx, alg: int, eps: float = -1.0) -> dict:
    """Same evaluation as ajf_fidelity_alg1/alg2, in the library's fixed 64 MiB device arena,
    without any allocation (for callers that cannot allocate device memory)."""
    r = Result()
    _check(ctx, lib().ajf_fidelity_noalloc(ctx, int(alg), float(eps), ctypes.byref(r)))
    return r.as_dict()


def ajf_alg1_traces(ctx, count: int) -> np.ndarray:
    out = np.empty(int(count), dtype=np.complex128)
    _check(ctx, lib().ajf_alg1_traces(ctx, _ptr(out), int(count)))
    return out


def ajf_launch(ctx, dev_result_ptr: int) -> None:
    _check(ctx, lib().ajf_launch(ctx, ctypes.c_void_p(dev_result_ptr) if dev_result_ptr else None))


def ajf_fidelity_alg1_batch(ctxs: Sequence, eps: float = -1.0) -> list:
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    res = (Result * len(ctxs))()
    st = lib().ajf_fidelity_alg1_batch(arr, len(ctxs), float(eps), res)
    if st != AJF_OK:
        msgs = "; ".join(ajf_last_error(c) for c in ctxs if ajf_last_error(c))
        raise AjfError(st, msgs)
    return [r.as_dict() for r in res]


def ajf_selftest_gemm(device: int, kind: int, A: np.ndarray, B: np.ndarray, M: int, N: int, K: int) -> np.ndarray:
    """Tensor-core GEMM self-test: A (npass, M, K), B (npass, N, K) as float32 (kind 0) or bf16 bit
    patterns in uint16 (kind 1); returns sum_p A_p B_p^T as float64."""
    A = np.ascontiguousarray(A)
    B = np.ascontiguousarray(B)
    npass = A.shape[0]
    C = np.empty((M, N), dtype=np.float64)
    st = lib().ajf_selftest_gemm(device, kind, npass, M, N, K, _ptr(A), _ptr(B), _ptr(C))
    if st != AJF_OK:
        raise AjfError(st, "ajf_selftest_gemm failed")
    return C


def ajf_selftest_split_gemm(device: int, precision: str, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A @ B.T (FP64 in, FP64 out) through the path's operand split and tensor-core GEMM."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    (M, K), (N, K2) = A.shape, B.shape
    assert K == K2
    C = np.empty((M, N), dtype=np.float64)
    st = lib().ajf_selftest_split_gemm(device, PRECISIONS[precision], M, N, K, _ptr(A), _ptr(B), _ptr(C))
    if st != AJF_OK:
        raise AjfError(st, "ajf_selftest_split_gemm failed")
    return C


def ajf_plan_launches(ctx) -> list:
    n = ctypes.c_int()
    _check(ctx, lib().ajf_plan_launches(ctx, None, 0, ctypes.byref(n)))
    arr = (LaunchInfo * max(1, n.value))()
    _check(ctx, lib().ajf_plan_launches(ctx, arr, n.value, ctypes.byref(n)))
    return [{"kind": KERNEL_CLASSES[a.kind], "terms": a.terms, "M": a.M, "N": a.N, "K": a.K, "flops": a.flops,
             "bytes": a.bytes} for a in arr[:n.value]]


def ajf_selftest_wait_timeout(device: int, wait_ms: float) -> tuple:
    """Returns (status, code): AJF_E_TIMEOUT and the expired wait's code when the bounded-wait
    failure path works."""
    code = ctypes.c_int32()
    st = lib().ajf_selftest_wait_timeout(device, float(wait_ms), ctypes.byref(code))
    return st, code.value


def ajf_learned_param_count() -> int:
    return int(lib().ajf_learned_param_count())


def default_learned_model() -> np.ndarray:
    """The merge scorer trained on the 2000 training circuits of the learned-planner workload
    (paper_2103_11595_gb300/data/merge_scorer.npy, written by learned_planner train)."""
    return np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "merge_scorer.npy"))


def ajf_set_learned_model(ctx, weights: Optional[np.ndarray]) -> None:
    if weights is None:
        _check(ctx, lib().ajf_set_learned_model(ctx, None, 0))
        return
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(ctx, lib().ajf_set_learned_model(ctx, _ptr(w), int(w.size)))


def ajf_learned_dataset(ctx, alg: int, trials: int = 8, seed: int = 0, negatives: int = 8) -> np.ndarray:
    """(n, 2, 16) float32 ranking pairs from the loaded circuit (taken merge, other candidate)."""
    n = ctypes.c_int64()
    _check(ctx, lib().ajf_learned_dataset(ctx, int(alg), int(trials), int(seed), int(negatives), None, 0,
                                          ctypes.byref(n)))
    out = np.empty((max(1, n.value), 2, 16), dtype=np.float32)
    _check(ctx, lib().ajf_learned_dataset(ctx, int(alg), int(trials), int(seed), int(negatives), _ptr(out), n.value,
                                          ctypes.byref(n)))
    return out[:n.value]


def ajf_learned_train(device: int, pairs: np.ndarray, epochs: int = 10, batch: int = 512, lr: float = 1e-3,
                      seed: int = 0) -> tuple:
    """Train the merge scorer on the GPU; returns (weights float32[47201], final mean loss)."""
    p = np.ascontiguousarray(pairs, dtype=np.float32)
    w = np.empty(ajf_learned_param_count(), dtype=np.float32)
    loss = ctypes.c_double()
    st = lib().ajf_learned_train(int(device), _ptr(p), int(p.shape[0]), int(epochs), int(batch), float(lr), int(seed),
                                 _ptr(w), int(w.size), ctypes.byref(loss))
    if st != AJF_OK:
        raise AjfError(st, "ajf_learned_train failed")
    return w, float(loss.value)


def ajf_profile_enable(ctx, on: bool = True) -> None:
    _check(ctx, lib().ajf_profile_enable(ctx, 1 if on else 0))


def ajf_profile_read(ctx) -> dict:
    arr = (KernelStats * len(KERNEL_CLASSES))()
    _check(ctx, lib().ajf_profile_read(ctx, arr, len(KERNEL_CLASSES)))
    return {name: {"launches": s.launches, "ms": s.ms, "flops": s.flops, "bytes": s.bytes}
            for name, s in zip(KERNEL_CLASSES, arr)}


def ajf_fidelity_batch(ctxs: Sequence, alg: int, eps: float = -1.0) -> list:
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    res = (Result * len(ctxs))()
    st = lib().ajf_fidelity_batch(arr, len(ctxs), int(alg), float(eps), res)
    if st != AJF_OK:
        msgs = "; ".join(ajf_last_error(c) for c in ctxs if ajf_last_error(c))
        raise AjfError(st, msgs)
    return [r.as_dict() for r in res]


def ajf_launch_persistent(ctxs: Sequence, dev_results: int = 0) -> None:
    """One persistent-kernel launch over `ctxs` (all planned with lowering="persistent"); results
    as 3 doubles per context to the device pointer `dev_results` (0: none). Does not wait."""
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    st = lib().ajf_launch_persistent(arr, len(ctxs), ctypes.c_void_p(dev_results) if dev_results else None)
    if st != AJF_OK:
        raise AjfError(st, "; ".join(ajf_last_error(c) for c in ctxs if ajf_last_error(c)))


def ajf_launch_queue(ctxs: Sequence, dev_results: int = 0) -> None:
    """One step-interpreter launch over the contexts (enqueued on the first context's stream)."""
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    st = lib().ajf_launch_queue(arr, len(ctxs), ctypes.c_void_p(dev_results) if dev_results else None)
    if st != AJF_OK:
        raise AjfError(st, ajf_last_error(ctxs[0]))


def ajf_selftest_queue_timeout(device: int, wait_ms: float) -> tuple:
    """(status, code): AJF_E_TIMEOUT and code 21 when the interpreter's bounded wait works."""
    code = ctypes.c_int32()
    st = lib().ajf_selftest_queue_timeout(int(device), float(wait_ms), ctypes.byref(code))
    return int(st), int(code.value)


QUEUE_TASK_KINDS = ["leaves", "small", "splitk", "splitk_done", "dot", "gather", "gemm_tc", "split_sum", "open",
                    "final"]


def ajf_queue_profile(ctx, reset: bool = True) -> dict:
    """Per kind of interpreter task: busy seconds, seconds waiting for the previous launch, tasks."""
    out = np.zeros(3 * len(QUEUE_TASK_KINDS))
    _check(ctx, lib().ajf_queue_profile(ctx, _ptr(out), out.size, 1 if reset else 0))
    return {k: {"busy_s": out[3 * i], "wait_s": out[3 * i + 1], "tasks": int(out[3 * i + 2])}
            for i, k in enumerate(QUEUE_TASK_KINDS)}


def ajf_fidelity_batch_queue(ctxs: Sequence, alg: int, eps: float = -1.0) -> list:
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    res = (Result * len(ctxs))()
    st = lib().ajf_fidelity_batch_queue(arr, len(ctxs), int(alg), float(eps), res)
    if st != AJF_OK:
        raise AjfError(st, ajf_last_error(ctxs[0]))
    return [r.as_dict() for r in res]


def ajf_autotune_queue(ctxs: Sequence, reps: int = 3) -> tuple:
    """(GEMM work items per task, tasks per CUDA-core launch) chosen for this batch."""
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    gi, bt = ctypes.c_int32(), ctypes.c_int32()
    st = lib().ajf_autotune_queue(arr, len(ctxs), int(reps), ctypes.byref(gi), ctypes.byref(bt))
    if st != AJF_OK:
        raise AjfError(st, ajf_last_error(ctxs[0]))
    return int(gi.value), int(bt.value)


def ajf_autotune_persistent(ctxs: Sequence, reps: int = 5) -> int:
    """Measure the persistent launch of this batch at 256, 128 and 64 threads per block and keep
    the fastest for batches of the same signature; returns the block size."""
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    t = ctypes.c_int32()
    st = lib().ajf_autotune_persistent(arr, len(ctxs), int(reps), ctypes.byref(t))
    if st != AJF_OK:
        raise AjfError(st, "; ".join(ajf_last_error(c) for c in ctxs if ajf_last_error(c)))
    return int(t.value)


def ajf_fidelity_batch_persistent(ctxs: Sequence, alg: int, eps: float = -1.0) -> tuple:
    """(results, n_persistent): persistent-lowered contexts in one launch, the others on their streams."""
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    res = (Result * len(ctxs))()
    n = ctypes.c_int32()
    st = lib().ajf_fidelity_batch_persistent(arr, len(ctxs), int(alg), float(eps), res, ctypes.byref(n))
    if st != AJF_OK:
        raise AjfError(st, "; ".join(ajf_last_error(c) for c in ctxs if ajf_last_error(c)))
    return [r.as_dict() for r in res], int(n.value)


# ----------------------------------------------------------------------------- marshalling helpers


def pack_gates(gates) -> tuple:
    """(arity, qubits, mats) arrays for ajf_load_circuit from objects with .qubits and .mat."""
    arity = np.array([len(g.qubits) for g in gates], dtype=np.int32)
    qubits = np.array([q for g in gates for q in g.qubits], dtype=np.int32)
    mats = (np.concatenate([np.asarray(g.mat, dtype=np.complex128).reshape(-1) for g in gates])
            if gates else np.zeros(0, dtype=np.complex128))
    return arity, qubits, np.ascontiguousarray(mats)


def load_instance(ctx, inst) -> None:
    """Load an instance (ideal circuit, optional implementation skeleton, noises) into a context."""
    ajf_load_circuit(ctx, AJF_IDEAL, inst.n, *pack_gates(inst.ideal))
    if getattr(inst, "impl", None) is not None:
        ajf_load_circuit(ctx, AJF_IMPL, inst.n, *pack_gates(inst.impl))
    for nz in inst.noises:
        ajf_add_noise(ctx, nz.after_gate, nz.qubits, nz.kraus)


def pack_instance(inst) -> tuple:
    """The flat C-ABI arrays of an instance, made once: (n, ideal arrays, implementation arrays or
    None, [(after_gate, qubits, kraus)]), each array contiguous in the ABI's dtype."""
    impl = getattr(inst, "impl", None)
    noises = [(int(nz.after_gate), np.ascontiguousarray(nz.qubits, dtype=np.int32),
               np.ascontiguousarray(nz.kraus, dtype=np.complex128)) for nz in inst.noises]
    return (int(inst.n), pack_gates(inst.ideal), pack_gates(impl) if impl is not None else None, noises)


def load_packed(ctx, packed) -> None:
    """load_instance from pack_instance's arrays: the C-ABI calls only."""
    n, ideal, impl, noises = packed
    L = lib()
    a, q, m = ideal
    _check(ctx, L.ajf_load_circuit(ctx, AJF_IDEAL, n, int(a.size), _ptr(a), _ptr(q), _ptr(m)))
    if impl is not None:
        a, q, m = impl
        _check(ctx, L.ajf_load_circuit(ctx, AJF_IMPL, n, int(a.size), _ptr(a), _ptr(q), _ptr(m)))
    for after, qq, k in noises:
        _check(ctx, L.ajf_add_noise(ctx, after, int(qq.size), _ptr(qq), int(k.shape[0]), _ptr(k)))


class Context:
    """Owning wrapper around an ajf_ctx handle."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        self.handle = ajf_create(device, stream)

    def close(self):
        if self.handle:
            ajf_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
