"""Values the paper prints, as fixtures under tests/golden/ (each file cites its
passage).  arxiv 2307.03968 §IV-A: the 15-wavelength PEC plate has 67,200
unknown edges; the synthetic plate mesh and the oracle's RWG edge count must give
exactly that number, and the paper's binary tree to level 6 then has leaves of
about 1,050 unknowns."""

import os

import synth
from oracle.rwg import rwg_edges

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fixture(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v) if "." in v else int(v)
    return vals


def test_paper_plate_unknown_count():
    g = _fixture("paper_plate_unknowns.txt")
    n, size = g["squares_per_side"], g["size_lambda"]
    xyz, tri = synth.plate((size, size), (n, n))
    assert len(tri) == 2 * n * n
    ev, _, _ = rwg_edges(tri)
    assert len(ev) == g["unknowns"] == 3 * n * n - 2 * n
    # the binary tree to the paper's level: 2^level leaves of about 1,050 unknowns
    leaves = 2 ** g["tree_level"]
    assert leaves == 64 and 1000 < g["unknowns"] / leaves < 1100
