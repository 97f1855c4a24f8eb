"""Test helpers: hand an oracle H-Matrix to the CUDA library through
hm_build_from_blocks, so both sides solve the same operator.  Test
infrastructure only (imports the oracle and the product binding)."""

import numpy as np


def export_oracle(H):
    """(perm, leaf_off, self_blocks, near, far) in the argument form of
    paper_2307_03968_gb300.hm.HMatrix.from_blocks for an oracle HMatrix."""
    leaf_off = [0] + [o + n for (o, n) in H.leaves]
    near = [(io, jo, B) for (io, m, jo, n, B) in H.near]
    far = []
    for lev, lst in sorted(H.far.items()):
        for (io, m, jo, n, U, V) in lst:
            far.append((lev, io, jo, U, V))
    return H.perm, leaf_off, H.D, near, far


def gpu_operator(H, keep_fp64=False):
    from paper_2307_03968_gb300.hm import HMatrix
    perm, leaf_off, D, near, far = export_oracle(H)
    A = HMatrix.from_blocks(perm, leaf_off, D, near, far, keep_fp64=keep_fp64)
    A.factor_leaf()
    return A


def rel_err(x, ref):
    """max over columns of |x - ref|_2 / |ref|_2 (columns = right-hand sides)."""
    x = np.atleast_2d(x)
    ref = np.atleast_2d(ref)
    return max(np.linalg.norm(x[i] - ref[i]) / np.linalg.norm(ref[i]) for i in range(ref.shape[0]))
