"""CPU oracle for the multi-level power-series EFIE H-Matrix solve
(arxiv 2307.03968) — TEST INFRASTRUCTURE ONLY.

Plain, slow, complex128 code that follows the paper step by step.  Only the
tests, the smoke check and the benchmark's CPU-baseline leg may import it; the
product path (``paper_2307_03968_gb300``) never does, and this package never
imports the product path.  It shares no code with the CUDA library: the only
common inputs come from ``synth`` (meshes and incidence directions).

Modules
  efie.c     RWG Galerkin EFIE entries, RHS, far field, ACA   (§II eqs. 1-5, §III)
  rwg.py     RWG basis enumeration and the ctypes wrapper of efie.c
  hmatrix.py cluster tree, admissibility, block partition, near fill,
             ACA + recompression, half storage                (§III eqs. 6-7)
  series.py  leaf inverse and the multi-level power series    (§IV eqs. 8-22)
  rcs.py     bistatic / monostatic RCS from the current       (§V, Figs. 2-4)
  mie.py     Mie series of a PEC sphere (textbook closed form, not in the paper)

Parity status
  Every function above is pinned by tests under ``tests/test_oracle_*.py``.
  The paper prints no values of the nested multi-level series at finite K; it
  is pinned by brute force instead: on an operator with far blocks on three
  levels, at 1, 2 and 3 levels and K = 1, 2 (plain and refined), it equals the
  same operators formed as dense matrix products with explicit matrix powers,
  and it reaches the closed form A_m^{-1} b as K grows.
"""
