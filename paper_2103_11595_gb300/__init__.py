"""GB300-native Jamiolkowski-fidelity equivalence checking of noisy quantum circuits.

Importing the package loads nothing heavy. ``paper_2103_11595_gb300.ajf`` is the thin ctypes
binding of the C-ABI library ``libajf``; ``paper_2103_11595_gb300.workloads`` draws the seeded
synthetic inputs.
"""
