"""GB300 (sm_103a) multi-level power-series solver for EFIE H-Matrices
(arxiv 2307.03968).  The compute path is the CUDA library ``_lib/libhmps.so``
behind the C ABI of ``include/hmps.h``; ``hm`` is its Python binding."""

from .hm import HMatrix, HmError, load, version  # noqa: F401
