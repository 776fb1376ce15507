"""Host logic of the tensor-core contraction: the planner that cuts the pair rows into 128-row tiles with windows of
singles, lays out tensor memory and shared memory, and writes the gather index of every output.

tests/tc_planner_check.cu is compiled from the kernel source (host code only is run) and checked on every shape the
tensor-core path accepts (all pairs of ng maps, ng (ng + 1) / 2 <= 512, against nh <= 32 singles), on the closed
triplets of 2..32 bins and on random triplet subsets: budgets (tensor memory <= 512 columns with at least two A
stages, shared memory <= 227 KB), window and accumulator alignment, and that every output lands exactly once at
the (unit, column, row) that holds its pair and single.  CPU only: no CUDA call is made.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    from paper_2404_07249_gb300 import build
    try:
        nvcc = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path_factory.mktemp("planner") / "tc_planner_check")
    cmd = [nvcc, *build.ARCH, "-std=c++17", "-O1", "--expt-relaxed-constexpr",
           "-I", os.path.join(ROOT, "include"), "-I", build.CSRC,
           os.path.join(ROOT, "tests", "tc_planner_check.cu"), "-o", exe,
           "-L", libdir, "-lpolybin", "-Xlinker", "-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


def test_planner_invariants(checker):
    r = subprocess.run([checker], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-1000:]
    assert r.stdout.strip().endswith("0 failures"), r.stdout[-500:]
