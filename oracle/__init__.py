"""FP64 CPU oracle for the parareal all-at-once partially explicit splitting
scheme (Wang, Yang, Leung, arXiv:2411.09244).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / reference
arm of `bench.py` may import, call or execute it.  It shares no code with the
CUDA path; the only common module is the seeded input generator
(`paper_2411_09244_gb300.inputs`), which holds none of the method's
arithmetic.

Every function follows the paper's definitions step by step in plain
NumPy/SciPy FP64 (dense or sparse direct solves, no blocking or fusion):

    fem.py       Q1 fine discretisation (Section 2, eq. (2.2)-(2.3))
    spaces.py    CEM-GMsFEM auxiliary eigenproblems and oversampled bases,
                 the split V_H1 / V_H2 (Section 3, eqs. (3.1)-(3.7))
    reduced.py   Galerkin matrices (eq. (3.8)), gamma (eq. (4.15)),
                 time-step condition (Section 3.2), initial projection
    scheme.py    coarse propagator G, sequential fine scheme, WR fine
                 propagator with alpha-circulant diagonalisation
                 (eqs. (2.4)-(2.5), (4.1)-(4.13))
    parareal.py  Algorithm 1 with update (2.7) and stopping rule (2.8)
    adjoint.py   transposed (adjoint) sweeps for the observation misfit

Readings of passages where the paper is silent or garbled are listed in the
docstrings where they are used.  Parity status: the pieces with a pin in
`tests/test_oracle_*.py` are pinned; the multiscale space split (the
canonical complement basis inside each block's auxiliary space) has no
external value to pin against and is "parity unpinned" beyond its structural
invariants (constraints, direct sum, gamma < 1).
"""
