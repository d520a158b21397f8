"""CPU FP64 oracle of the Fast Kernel Transform.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import, call, link or execute
anything in this package.  The product library (``paper_2106_04487_gb300``)
never imports it and shares no code with it.

Contents:
  tables.py      exact rational expansion tables (Sec. A.2, Theorem 3.1)
  fkt_oracle.c   FP64 dense MVM and step-by-step FKT (Algorithm 1)
  oracle.py      build + ctypes wrapper, zonal harmonic point selection

Parity status: every function is pinned by a ``-m "not gpu"`` test against
values the paper prints (Table 4), closed forms, library special functions
(scipy Gegenbauer / Hermite / Legendre, sympy derivatives), the Cartesian
Taylor polynomial computed by a Cauchy integral, and brute-force invariants.
"""
