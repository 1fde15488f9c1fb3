"""The BVH builder's output, checked on the host (no GPU).

`tests/bvh_check.cpp` is compiled with the host compiler against the
library's builder (`csrc/bvh_build.cpp`) and walks the emitted node array:
the triangle order is a permutation, leaves cover it exactly once with at
most two triangles each, every vertex lies inside every box above its leaf
(quantised BVH4 boxes decoded from their node's 8-bit grid in binary64), and
unused BVH4 slots reference the sentinel leaf past the triangles with an
inverted box (which no slab test accepts).  Cases: random
small triangles, triangles with one shared centroid (the builder splits by
count), long slivers, and a tiny scene; BVH4 with binary32 and with
quantised bounds, and BVH2.

`tests/bvh_walk_check.cpp` checks the reference traversal the bench measures
the kernel's traversal work against (`csrc/bvh_walk.cpp`): through the
built BVH it finds the same closest hits as a loop over every triangle.
"""
import os
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
CSRC = ROOT / "paper_2402_08273_gb300" / "csrc"
CUDA_INC = Path(os.environ.get("CUDA_HOME", "/usr/local/cuda")) / "include"
LEAF_MAX = 2


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not (CUDA_INC / "cuda_runtime.h").exists():
        pytest.skip("needs a host C++ compiler and the CUDA headers")
    exe = tmp_path_factory.mktemp("bvh") / "bvh_check"
    subprocess.run([cxx, "-O2", "-std=c++17", f"-I{CUDA_INC}", f"-I{ROOT / 'include'}", f"-I{CSRC}",
                    str(ROOT / "tests" / "bvh_check.cpp"), str(CSRC / "bvh_build.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    return exe


@pytest.mark.parametrize("layout", ["4", "4q", "2"])
@pytest.mark.parametrize("n_tris,mode,seed", [(20_000, 0, 1), (300, 1, 2), (5_000, 2, 3), (5, 0, 4), (777, 0, 5)])
def test_bvh_structure(checker, layout, n_tris, mode, seed):
    r = subprocess.run([str(checker), layout, str(n_tris), str(mode), str(seed), str(LEAF_MAX)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok ")


@pytest.fixture(scope="module")
def walker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not (CUDA_INC / "cuda_runtime.h").exists():
        pytest.skip("needs a host C++ compiler and the CUDA headers")
    exe = tmp_path_factory.mktemp("walk") / "bvh_walk_check"
    subprocess.run([cxx, "-O2", "-std=c++17", f"-I{CUDA_INC}", f"-I{ROOT / 'include'}", f"-I{CSRC}",
                    str(ROOT / "tests" / "bvh_walk_check.cpp"), str(CSRC / "bvh_build.cpp"),
                    str(CSRC / "bvh_walk.cpp"), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    return exe


@pytest.mark.parametrize("layout", ["4", "4q", "2"])
@pytest.mark.parametrize("n_tris,seed", [(3000, 1), (40, 2)])
def test_reference_traversal_matches_brute_force(walker, layout, n_tris, seed):
    r = subprocess.run([str(walker), layout, str(n_tris), str(seed)], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok ") and int(r.stdout.split()[1]) > (100 if n_tris > 1000 else 0)
