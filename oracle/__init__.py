"""Plain, slow FP64 CPU oracle of the IB-LBM time step (arXiv 2102.01305, Sec. 2).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code with
the CUDA path (``paper_2102_01305_gb300``); the only common module is the
seeded input generator ``workloads``, which holds none of the method's
arithmetic.

Every function follows the paper's equations in the paper's order, in numpy
float64, with no blocking, fusion or reordering beyond what an equation
states; numpy/scipy primitives (sparse products, dense LU) serve as single
steps.  Readings of garbled or silent passages are listed in each docstring.

Modules
-------
lattice     D2Q9 (Eq. 5) and D3Q19 velocity sets and weights.
lbm         equilibrium (Eq. 4), Guo forcing (Eq. 8), moments (Eqs. 9, 11),
            BGK collision (Eq. 7), streaming with periodic / halfway
            bounce-back / Zou-He faces (Sec. 2.1, Sec. 3.1).
ib          4-point cosine delta (Eq. 14), interpolation (Eq. 17), spreading
            (Eq. 15), the implicit system A X = B (Eqs. 18-19) and its dense
            direct solve, marker forces (Eq. 26, Sec. 3.7).
kinematics  wave forms (Eqs. 20, 21, 23) and rigid marker motion (Sec. 3.3).
sim         the whole step in the paper's order (Sec. 2.2).

Parity status
-------------
Every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against closed forms, exact invariants, brute
force on tiny inputs or a published solution.  The physical outputs of the
paper's wing and cylinder cases (its Figs. 2, 6, 10, 11) are printed only as
figures: the whole-run force histories are therefore parity unpinned against
the paper itself; they are pinned only through their parts.
"""
from . import lattice, lbm, ib, kinematics, sim  # noqa: F401
