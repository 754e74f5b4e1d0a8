"""Oracle: plain serial FP64 CPU statement of the high-order kinetic relaxation
Poisson solver.  TEST INFRASTRUCTURE ONLY -- imported by tests, by
``__graft_entry__.smoke()`` and by the benchmark's CPU-baseline leg, never by
the product library.

Parity status: every function here is pinned by ``-m "not gpu"`` tests
(``tests/test_oracle_*.py``) against closed forms, exact quadrature moments,
the paper's printed weights and Table 2 errors, brute-force dense solves and
invariants.  Unpinned: the amplitude a_N of the paper's error fit (Table 1)
and the exact error measure of its Figs. 1-6, which the text leaves garbled;
the tests pin the per-node errors of Table 2 and the convergence orders
instead.
"""
from .lattice import LATTICES, MAX_ORDER, Lattice, lattice  # noqa: F401
from .oracle import (Result, build, density, grid3, solve, source, step,  # noqa: F401
                     tau_from_knudsen, threads)
