"""CPU oracle for the Jamiolkowski fidelity F_J(E, U) -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 (complex128) code written from the paper, used to check the CUDA path.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may
import it. The product path (the C-ABI library and its Python binding) never imports, calls or
links anything here, and this package imports nothing from the product.

Modules:
  dense    -- O1: the definition F_J = (1/d^2) sum_i |tr(U^dagger E_i)|^2 (Sec. III, "Ease of
              calculation") with dense 2^n x 2^n matrices, one Kraus combination at a time
              (the enumeration of Alg. I, Sec. IV-A).
  superop  -- the matrix representation M_E = sum_i E_i (x) E_i^* and tr((U^dagger (x) U^T) M_E)
              (Sec. IV-B), and F_J as the fidelity of the two Jamiolkowski states (Sec. III),
              for brute force on <= 4 qubits.
  network  -- O2: Alg. I and Alg. II miter networks built step by step as Sec. IV-A/IV-B state
              them, wires closed into a trace (Fig. 3), contracted pairwise with numpy.tensordot
              along a simple smallest-result-first order of its own.

Every function takes an instance object with attributes ``n``, ``ideal`` (list of gates with
``qubits`` and ``mat``), ``skeleton`` (implementation gates) and ``noises`` (``after_gate``,
``qubits``, ``kraus``); qubit 0 is the most significant factor.

Parity pins: every function here is pinned by tests in ``tests/test_oracle_pins.py`` (worked
Examples 3 and 4, closed forms, the Choi-state definition, the average-fidelity relation,
stability, chaining, cross-agreement). None is "parity unpinned".
"""
