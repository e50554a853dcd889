"""Brute-force forms for tiny circuits (test infrastructure).

1. Sec. IV-B: sum_i |tr(U^dagger E_i)|^2 = tr((U^dagger (x) U^T) M_E), with the matrix
   representation M_E = sum_i E_i (x) E_i^*. M_E is built as Alg. II's steps describe: every
   unitary gate V becomes V (x) V^* on (q, q'), every noisy gate {N_k} becomes
   M_N = sum_k N_k (x) N_k^* on (q, q'), all multiplied in time order; the ideal side likewise
   gives U (x) U^*, whose adjoint is U^dagger (x) U^T. Dense 4^n x 4^n: n <= 5.
2. Sec. III: F_J(E, U) is the state fidelity F(rho_E, rho_U) = (tr sqrt(sqrt(rho) sigma
   sqrt(rho)))^2 between the Jamiolkowski states rho_E = (I (x) E)(|Psi><Psi|), with
   |Psi> = d^{-1/2} sum_i |ii>. Computed from that definition with PSD square roots, without the
   trace formula. Dense 4^n x 4^n: n <= 3.
"""
from __future__ import annotations

import numpy as np

from .dense import apply_op, combinations, kraus_of_circuit, timeline


def doubled_matrix(inst, gates, with_noise: bool) -> np.ndarray:
    """Product over time of V (x) V^* (and M_N for noisy gates) on 2n qubits (q then q')."""
    n = inst.n
    M = np.eye(4 ** n, dtype=np.complex128)
    if not with_noise:
        for g in gates:
            V = np.kron(g.mat, np.conj(g.mat))
            M = apply_op(M, 2 * n, list(g.qubits) + [q + n for q in g.qubits], V)
        return M
    for kind, idx in timeline(inst):
        if kind == "gate":
            g = inst.skeleton[idx]
            V = np.kron(g.mat, np.conj(g.mat))
            qs = list(g.qubits) + [q + n for q in g.qubits]
        else:
            nz = inst.noises[idx]
            V = sum(np.kron(K, np.conj(K)) for K in nz.kraus)
            qs = list(nz.qubits) + [q + n for q in nz.qubits]
        M = apply_op(M, 2 * n, qs, V)
    return M


def alg2_sum(inst) -> float:
    """S = tr((U^dagger (x) U^T) M_E); real up to rounding."""
    ME = doubled_matrix(inst, inst.skeleton, True)
    UE = doubled_matrix(inst, inst.ideal, False)
    val = np.sum(np.conj(UE) * ME)  # tr(UE^dagger ME)
    return complex(val)


def _psd_sqrt(A: np.ndarray) -> np.ndarray:
    A = 0.5 * (A + A.conj().T)
    w, V = np.linalg.eigh(A)
    w = np.clip(w, 0.0, None)
    return (V * np.sqrt(w)) @ V.conj().T


def choi_state(inst, kraus_list) -> np.ndarray:
    """rho = sum_i (I (x) E_i)|Psi><Psi|(I (x) E_i)^dagger as a d^2 x d^2 density matrix."""
    d = 2 ** inst.n
    rho = np.zeros((d * d, d * d), dtype=np.complex128)
    for E in kraus_list:
        # (I (x) E) d^{-1/2} sum_i |i>|i>  =  d^{-1/2} sum_i |i> (x) E|i>; row i holds E[:, i].
        v = (E.T / np.sqrt(d)).reshape(-1)
        rho += np.outer(v, np.conj(v))
    return rho


def jamiolkowski_fidelity(inst) -> float:
    """F(rho_U, rho_E) by the mixed-state fidelity formula of Sec. III."""
    from .dense import circuit_matrix
    U = circuit_matrix(inst.n, inst.ideal)
    rho_u = choi_state(inst, [U])
    rho_e = choi_state(inst, [kraus_of_circuit(inst, c) for c in combinations(inst)])
    s = _psd_sqrt(rho_u)
    inner = _psd_sqrt(s @ rho_e @ s)
    return float(np.real(np.trace(inner)) ** 2)
