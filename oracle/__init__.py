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
  The nested multi-level series at finite K has no printed values in the
  paper; beyond the brute-force dense recursion it is "parity unpinned".
"""
