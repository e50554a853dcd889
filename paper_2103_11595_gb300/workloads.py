"""Seeded synthetic workloads: ideal circuits, noisy implementations, noise Kraus sets.

This module only *draws inputs*. It computes no fidelity, no trace and no contraction, so both
the CUDA path and the CPU oracle can consume its output without sharing any of the method's
arithmetic.

Conventions (fixed here, used by every consumer):
  * A circuit is a list of gates applied left to right (the first gate acts first).
  * Qubit 0 is the most significant tensor factor; within a gate matrix the first listed qubit is
    the most significant factor of that gate.
  * Every matrix is complex128, row-major, ``2^a x 2^a`` for an ``a``-qubit gate.
  * A noise ``after_gate = g`` is applied right after implementation gate ``g``; ``-1`` means
    before the first gate (Sec. II-B, Fig. 2: noisy gates interleaved with unitary ones).
  * Kraus sets satisfy ``sum_k K_k^dagger K_k = I`` (Sec. II-B).

Gate and noise readings where the paper is silent (the paper defines only X, Y, Z, H, S, the
controlled-S and SWAP in Sec. II-A, and bit/phase/bit-phase flip and depolarisation in Example 2):
  T = diag(1, e^{i pi/4});  Rz(t) = diag(e^{-it/2}, e^{it/2});
  U3(t,f,l) = [[cos t/2, -e^{il} sin t/2], [e^{if} sin t/2, e^{i(f+l)} cos t/2]];
  CX: control = first listed qubit;  CZ = diag(1,1,1,-1);
  Haar SU(4): QR of a complex Ginibre matrix, phases of R's diagonal divided out (Mezzadri 2007),
  scaled by det^{-1/4}.
  Depolarising with error probability p: sqrt(1-3p/4) I, sqrt(p/4) X, Y, Z (so the paper's
  "probability of no error" is 1-3p/4; ``paper_depolarising`` takes the paper's p directly).
  Amplitude damping: K0 = [[1,0],[0,sqrt(1-g)]], K1 = [[0,sqrt(g)],[0,0]].
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# ----------------------------------------------------------------------------- data model


@dataclass
class Gate:
    qubits: Tuple[int, ...]
    mat: np.ndarray  # (2^a, 2^a) complex128
    name: str = ""

    @property
    def arity(self) -> int:
        return len(self.qubits)


@dataclass
class Noise:
    after_gate: int
    qubits: Tuple[int, ...]
    kraus: np.ndarray  # (n_kraus, 2^a, 2^a) complex128
    name: str = ""

    @property
    def arity(self) -> int:
        return len(self.qubits)

    @property
    def n_kraus(self) -> int:
        return int(self.kraus.shape[0])


@dataclass
class Instance:
    """An ideal circuit U, a noisy implementation (skeleton gates + noises) and a name."""
    n: int
    ideal: List[Gate]
    noises: List[Noise] = field(default_factory=list)
    impl: Optional[List[Gate]] = None  # None: the implementation skeleton is the ideal circuit
    name: str = ""

    @property
    def skeleton(self) -> List[Gate]:
        return self.ideal if self.impl is None else self.impl

    def n_combinations(self) -> int:
        c = 1
        for nz in self.noises:
            c *= nz.n_kraus
        return c


# ----------------------------------------------------------------------------- gate matrices

_SQ2 = np.sqrt(2.0)
I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / _SQ2
S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
T = np.array([[1, 0], [0, np.exp(1j * np.pi / 4)]], dtype=np.complex128)
CX = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)
CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
CS = np.diag([1, 1, 1, 1j]).astype(np.complex128)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def rz(theta: float) -> np.ndarray:
    return np.diag([np.exp(-0.5j * theta), np.exp(0.5j * theta)]).astype(np.complex128)


def u3(theta: float, phi: float, lam: float) -> np.ndarray:
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    return np.array([[c, -np.exp(1j * lam) * s],
                     [np.exp(1j * phi) * s, np.exp(1j * (phi + lam)) * c]], dtype=np.complex128)


def haar_unitary(rng: np.random.Generator, dim: int) -> np.ndarray:
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / _SQ2
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return (q * (d / np.abs(d))).astype(np.complex128)


def haar_su(rng: np.random.Generator, dim: int) -> np.ndarray:
    u = haar_unitary(rng, dim)
    det = np.linalg.det(u)
    return (u * det ** (-1.0 / dim)).astype(np.complex128)


# ----------------------------------------------------------------------------- noise Kraus sets


def depolarising(p: float) -> np.ndarray:
    """Error probability p: rho -> (1-p) rho + p I/2."""
    return np.stack([np.sqrt(1 - 0.75 * p) * I2, np.sqrt(p / 4) * X,
                     np.sqrt(p / 4) * Y, np.sqrt(p / 4) * Z]).astype(np.complex128)


def paper_depolarising(p: float) -> np.ndarray:
    """Example 2's parametrisation: p is the probability of no error."""
    q = (1 - p) / 3
    return np.stack([np.sqrt(p) * I2, np.sqrt(q) * X, np.sqrt(q) * Y,
                     np.sqrt(q) * Z]).astype(np.complex128)


def bit_flip(p: float) -> np.ndarray:
    """Example 2: flips with probability 1-p."""
    return np.stack([np.sqrt(p) * I2, np.sqrt(1 - p) * X]).astype(np.complex128)


def phase_flip(p: float) -> np.ndarray:
    return np.stack([np.sqrt(p) * I2, np.sqrt(1 - p) * Z]).astype(np.complex128)


def bitphase_flip(p: float) -> np.ndarray:
    return np.stack([np.sqrt(p) * I2, np.sqrt(1 - p) * Y]).astype(np.complex128)


def amplitude_damping(gamma: float) -> np.ndarray:
    k0 = np.array([[1, 0], [0, np.sqrt(1 - gamma)]], dtype=np.complex128)
    k1 = np.array([[0, np.sqrt(gamma)], [0, 0]], dtype=np.complex128)
    return np.stack([k0, k1])


def two_qubit_depolarising(p: float) -> np.ndarray:
    """rho -> (1-p) rho + p I/4 on two qubits: 16 Pauli-product Kraus operators."""
    paulis = [I2, X, Y, Z]
    ops = []
    for a in range(4):
        for b in range(4):
            w = 1 - 15 * p / 16 if (a == 0 and b == 0) else p / 16
            ops.append(np.sqrt(w) * np.kron(paulis[a], paulis[b]))
    return np.stack(ops).astype(np.complex128)


# ----------------------------------------------------------------------------- fixed examples


def qft2_noisy(p: float) -> Instance:
    """Fig. 1 / Fig. 2: QFT_2 = H(q1); CS(q2 controls S on q1); H(q2); SWAP, with a bit flip N on
    q2 in the first column and a phase flip N' on q1 right after the controlled-S (Example 3)."""
    gates = [Gate((0,), H, "H"), Gate((1, 0), CS, "CS"), Gate((1,), H, "H"),
             Gate((0, 1), SWAP, "SWAP")]
    noises = [Noise(-1, (1,), bit_flip(p), "bf"), Noise(1, (0,), phase_flip(p), "pf")]
    return Instance(2, gates, noises, name=f"qft2_noisy(p={p})")


# ----------------------------------------------------------------------------- random circuits


def _noises_after_random_gates(rng, gates: Sequence[Gate], k: int, make_kraus) -> List[Noise]:
    k = min(k, len(gates))
    picks = sorted(rng.choice(len(gates), size=k, replace=False).tolist())
    out = []
    for g in picks:
        qs = gates[g].qubits
        q = qs[int(rng.integers(len(qs)))]
        kr, nm = make_kraus(rng)
        out.append(Noise(int(g), (int(q),), kr, nm))
    return out


def tiny(seed: int, n: int = 3, n_gates: int = 20, n_noises: int = 2, p: float = 0.01) -> Instance:
    """n=3, 20 gates uniform over {H, T, S, CX on a random ordered pair, Rz(theta)}, two
    depolarising noises p=0.01 after distinct random gates."""
    rng = np.random.default_rng(seed)
    gates: List[Gate] = []
    for _ in range(n_gates):
        kind = int(rng.integers(5))
        if kind == 3:
            a, b = rng.choice(n, size=2, replace=False)
            gates.append(Gate((int(a), int(b)), CX, "CX"))
        else:
            q = int(rng.integers(n))
            if kind == 0:
                gates.append(Gate((q,), H, "H"))
            elif kind == 1:
                gates.append(Gate((q,), T, "T"))
            elif kind == 2:
                gates.append(Gate((q,), S, "S"))
            else:
                gates.append(Gate((q,), rz(rng.uniform(0, 2 * np.pi)), "Rz"))
    noises = _noises_after_random_gates(rng, gates, n_noises, lambda r: (depolarising(p), "dep"))
    return Instance(n, gates, noises, name=f"tiny(seed={seed})")


def line_u3_cx(rng, n: int, n_gates: int) -> List[Gate]:
    """Alternating layers: U3 on every qubit (angles ~U[0,2pi)), then a nearest-neighbour CX brick
    on pairs (0,1),(2,3),... then (1,2),(3,4),... alternately (control = lower index); truncated
    at n_gates."""
    gates: List[Gate] = []
    layer = 0
    while len(gates) < n_gates:
        if layer % 2 == 0:
            for q in range(n):
                th, ph, la = rng.uniform(0, 2 * np.pi, size=3)
                gates.append(Gate((q,), u3(th, ph, la), "U3"))
        else:
            start = 0 if (layer // 2) % 2 == 0 else 1
            for q in range(start, n - 1, 2):
                gates.append(Gate((q, q + 1), CX, "CX"))
        layer += 1
    return gates[:n_gates]


def _mixed_noise(rng, lo=1e-4, hi=1e-2):
    if rng.random() < 0.5:
        p = float(rng.uniform(lo, hi))
        return depolarising(p), "dep"
    g = float(rng.uniform(lo, hi))
    return amplitude_damping(g), "ad"


def mid(seed: int, n: int = 16, n_gates: int = 200, n_noises: int = 10) -> Instance:
    """n=16 line, 200 gates of U3 layers and NN-CX bricks, 10 noises after distinct random gates,
    each depolarising (p~U[1e-4,1e-2]) or amplitude damping (gamma~U[1e-4,1e-2]) w.p. 1/2."""
    rng = np.random.default_rng(1_000_000 + seed)
    gates = line_u3_cx(rng, n, n_gates)
    noises = _noises_after_random_gates(rng, gates, n_noises, _mixed_noise)
    return Instance(n, gates, noises, name=f"mid(seed={seed},n={n},g={n_gates},k={n_noises})")


def grid_bonds(rows: int, cols: int):
    """Four colour classes of the grid's bonds: horizontal even/odd, vertical even/odd."""
    idx = lambda r, c: r * cols + c
    hor_e = [(idx(r, c), idx(r, c + 1)) for r in range(rows) for c in range(0, cols - 1, 2)]
    hor_o = [(idx(r, c), idx(r, c + 1)) for r in range(rows) for c in range(1, cols - 1, 2)]
    ver_e = [(idx(r, c), idx(r + 1, c)) for r in range(0, rows - 1, 2) for c in range(cols)]
    ver_o = [(idx(r, c), idx(r + 1, c)) for r in range(1, rows - 1, 2) for c in range(cols)]
    return [hor_e, hor_o, ver_e, ver_o]


def precision(seed: int, depth: int = 4, rows: int = 4, cols: int = 5) -> Instance:
    """4x5 grid, `depth` layers of a 4-colour brickwork of Haar SU(4) gates; after every two-qubit
    gate a single-qubit depolarising noise on each of its two qubits, p~U[1e-4,1e-3]."""
    rng = np.random.default_rng(2_000_000 + seed)
    colours = grid_bonds(rows, cols)
    gates: List[Gate] = []
    noises: List[Noise] = []
    for d in range(depth):
        for (a, b) in colours[d % 4]:
            gates.append(Gate((a, b), haar_su(rng, 4), "SU4"))
            g = len(gates) - 1
            for q in (a, b):
                noises.append(Noise(g, (q,), depolarising(float(rng.uniform(1e-4, 1e-3))), "dep"))
    return Instance(rows * cols, gates, noises, name=f"precision(seed={seed},depth={depth})")


def batching_circuit(seed: int, n_noises: int = 6) -> Instance:
    """n~U{8..20}, gates~U{50..300}: U3 layers + NN-CX bricks on a line; 6 depolarising noises
    p~U[1e-4,1e-2] after distinct random gates (4^6 = 4096 Kraus combinations)."""
    rng = np.random.default_rng(3_000_000 + seed)
    n = int(rng.integers(8, 21))
    g = int(rng.integers(50, 301))
    gates = line_u3_cx(rng, n, g)
    noises = _noises_after_random_gates(
        rng, gates, n_noises, lambda r: (depolarising(float(r.uniform(1e-4, 1e-2))), "dep"))
    return Instance(n, gates, noises, name=f"batch(seed={seed},n={n},g={g})")


def random_pairs_circuit(seed: int, n_range=(10, 24), g_range=(100, 400),
                         k_range=(5, 40)) -> Instance:
    """n~U{10..24}, gates~U{100..400}: U3 w.p. 1/2, else CX or CZ (1/4 each) on a uniformly random
    ordered pair; 5..40 noises, depolarising or amplitude damping."""
    rng = np.random.default_rng(4_000_000 + seed)
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    ng = int(rng.integers(g_range[0], g_range[1] + 1))
    gates: List[Gate] = []
    for _ in range(ng):
        u = rng.random()
        if u < 0.5:
            q = int(rng.integers(n))
            th, ph, la = rng.uniform(0, 2 * np.pi, size=3)
            gates.append(Gate((q,), u3(th, ph, la), "U3"))
        else:
            a, b = rng.choice(n, size=2, replace=False)
            gates.append(Gate((int(a), int(b)), CX if u < 0.75 else CZ, "CX" if u < 0.75 else "CZ"))
    k = int(rng.integers(k_range[0], k_range[1] + 1))
    noises = _noises_after_random_gates(rng, gates, k, _mixed_noise)
    return Instance(n, gates, noises, name=f"learned(seed={seed},n={n},g={ng},k={k})")


def random_small(seed: int, n: int, n_gates: int, n_noises: int, two_qubit_noise: bool = False,
                 haar: bool = True) -> Instance:
    """Small random instances for parity tests: Haar 1q/2q gates on random qubits, mixed noises
    (depolarising, amplitude damping, flips, optionally a 2-qubit depolarising)."""
    rng = np.random.default_rng(5_000_000 + seed)
    gates: List[Gate] = []
    for _ in range(n_gates):
        if n >= 2 and rng.random() < 0.4:
            a, b = rng.choice(n, size=2, replace=False)
            gates.append(Gate((int(a), int(b)), haar_unitary(rng, 4) if haar else CX, "G2"))
        else:
            q = int(rng.integers(n))
            gates.append(Gate((q,), haar_unitary(rng, 2), "G1"))
    kinds = [lambda r: (depolarising(float(r.uniform(0.01, 0.3))), "dep"),
             lambda r: (amplitude_damping(float(r.uniform(0.01, 0.3))), "ad"),
             lambda r: (bit_flip(float(r.uniform(0.7, 0.99))), "bf"),
             lambda r: (phase_flip(float(r.uniform(0.7, 0.99))), "pf")]
    noises = _noises_after_random_gates(rng, gates, n_noises,
                                        lambda r: kinds[int(r.integers(len(kinds)))](r))
    if two_qubit_noise and n >= 2 and gates:
        g = int(rng.integers(len(gates)))
        a, b = rng.choice(n, size=2, replace=False)
        noises.append(Noise(g, (int(a), int(b)), two_qubit_depolarising(float(rng.uniform(0.01, 0.2))), "dep2"))
        noises.sort(key=lambda z: z.after_gate)
    return Instance(n, gates, noises, name=f"small(seed={seed},n={n},g={n_gates},k={n_noises})")


def identity_with_noises(n: int, noises: List[Noise]) -> Instance:
    """The identity circuit on n qubits, written as one identity gate per qubit so noises have
    gates to follow."""
    gates = [Gate((q,), I2.copy(), "I") for q in range(n)]
    return Instance(n, gates, noises, name=f"identity(n={n})")


CONFIG_MAKERS = {
    "tiny": tiny,
    "mid": mid,
    "precision": precision,
    "batching": batching_circuit,
    "learned": random_pairs_circuit,
}
