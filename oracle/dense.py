"""O1: the Jamiolkowski fidelity by its trace formula, with dense matrices (test infrastructure).

Sec. III ("Ease of calculation"): for an ideal unitary U and a noisy implementation E = {E_i},
    F_J(E, U) = (1/d^2) * sum_i |tr(U^dagger E_i)|^2,   d = 2^n.
Sec. IV-A (Alg. I): each choice (j_1..j_m) of one Kraus operator per noisy gate gives one Kraus
operator E_i of the whole circuit, obtained by putting N^k_{j_k} in place of noisy gate k; there
are prod_k n_k choices.

Combinations are enumerated lexicographically over the noise list, the last noise varying
fastest. Plain FP64; only practical for n <= ~10.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def apply_op(M: np.ndarray, n: int, qubits, G: np.ndarray) -> np.ndarray:
    """Return (G acting on `qubits`, identity elsewhere) @ M for a 2^n x c matrix M."""
    a = len(qubits)
    T = M.reshape((2,) * n + (-1,))
    Gt = np.asarray(G, dtype=np.complex128).reshape((2,) * (2 * a))
    R = np.tensordot(Gt, T, axes=(list(range(a, 2 * a)), list(qubits)))
    R = np.moveaxis(R, list(range(a)), list(qubits))
    return R.reshape(2 ** n, -1)


def circuit_matrix(n: int, gates) -> np.ndarray:
    """Product g_L ... g_1 of a gate list (the first gate acts first, Sec. II-A)."""
    M = np.eye(2 ** n, dtype=np.complex128)
    for g in gates:
        M = apply_op(M, n, g.qubits, g.mat)
    return M


def timeline(inst):
    """Operations of the noisy implementation in time order: ('gate', g) and ('noise', j).
    Noises with after_gate = -1 come first; a noise follows the gate it is placed after; noises
    after the same gate keep their list order (Fig. 2)."""
    ops = [("noise", j) for j, nz in enumerate(inst.noises) if nz.after_gate < 0]
    for gi, _ in enumerate(inst.skeleton):
        ops.append(("gate", gi))
        ops.extend(("noise", j) for j, nz in enumerate(inst.noises) if nz.after_gate == gi)
    return ops


def combinations(inst):
    """All Kraus choices (j_1, ..., j_m), lexicographic, last noise fastest (Sec. IV-A)."""
    return itertools.product(*[range(nz.kraus.shape[0]) for nz in inst.noises])


def kraus_of_circuit(inst, choice) -> np.ndarray:
    """E_i: the implementation with noisy gate k replaced by its Kraus operator N^k_{j_k}."""
    n = inst.n
    M = np.eye(2 ** n, dtype=np.complex128)
    for kind, idx in timeline(inst):
        if kind == "gate":
            g = inst.skeleton[idx]
            M = apply_op(M, n, g.qubits, g.mat)
        else:
            nz = inst.noises[idx]
            M = apply_op(M, n, nz.qubits, nz.kraus[choice[idx]])
    return M


def traces(inst) -> np.ndarray:
    """t_i = tr(U^dagger E_i) for every combination i, in enumeration order."""
    U = circuit_matrix(inst.n, inst.ideal)
    out = []
    for choice in combinations(inst):
        E = kraus_of_circuit(inst, choice)
        out.append(np.sum(np.conj(U) * E))  # tr(U^dagger E) = sum_ab conj(U_ab) E_ab
    return np.array(out, dtype=np.complex128)


def fidelity(inst) -> dict:
    """F_J = sum_i |t_i|^2 / d^2, with S = sum_i |t_i|^2 and 1 - F_J = (d^2 - S) / d^2."""
    t = traces(inst)
    d2 = float(4 ** inst.n)
    S = math.fsum(float(abs(x) ** 2) for x in t)
    return {"F": S / d2, "one_minus_F": (d2 - S) / d2, "S": S, "traces": t}
