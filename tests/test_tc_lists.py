"""Host logic of the block products' work lists (csrc/hm_lists.h), compiled with the
host compiler and checked on random small-block sets: every block gives its two
directed products (eq. 6 and eq. 8 with the half storage of §III); the owner-computes
residual takes each once, by output cluster; the tensor-core product's stage-1 batches
stack each low-rank product's W rows in order, over its own input cluster, into T
chunks that are each written once, and its second launch holds exactly the directed
products, in units of at most TC_UNIT_CHUNKS K chunks.  The snake order in which the
persistent product and residual kernels take their blocks holds each block once, with
the round-robin warps' cost sums within the largest cost of one another.  Three damaged
list sets must fail the same checks."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2307_03968_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("tc_lists") / "tc_lists_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Wextra", "-Werror", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "tc_lists_check.cpp")], check=True)
    return exe


def run(exe, seed, mode):
    p = subprocess.run([exe, str(seed), str(mode)], capture_output=True, text=True)
    return p.returncode, p.stdout.strip()


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_lists_hold_the_kernels_invariants(checker, seed, mode):
    rc, out = run(checker, seed, mode)
    assert rc == 0 and out.startswith("ok"), out


@pytest.mark.parametrize("mode", [5, 6, 7])
def test_damaged_lists_fail(checker, mode):
    rc, out = run(checker, 1, mode)
    assert rc == 1 and out.startswith("FAIL"), out
