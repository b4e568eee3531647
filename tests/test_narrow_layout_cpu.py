"""Host logic of the narrow-column layout (no GPU): groups of consecutive narrow columns touch
pairwise disjoint subjects and fit half the shared buffers, and each segment's mark names the
one earlier step that can change its subject (the GPU re-gathers a segment exactly when that
step was not zero).  The check compiles the library's host source into a small C++ program and
compares every mark with a brute-force search over the columns."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "narrow_layout_check.cpp")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = os.environ.get("NVCC") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc")
                                      else shutil.which("nvcc"))
    if not nvcc:
        pytest.skip("nvcc not available")
    import __graft_entry__
    lib = __graft_entry__._build_module().build()
    exe = str(tmp_path_factory.mktemp("narrow") / "narrow_layout_check")
    # the host source is compiled in; the kernels' launchers it names come from the built
    # library and are never called, so the program needs no GPU
    cmd = [nvcc, "-std=c++17", "-O2", "-I" + os.path.join(ROOT, "include"), SRC, lib,
           "-Xlinker", "-rpath=" + os.path.dirname(lib), "-o", exe, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


@pytest.mark.parametrize("nsub,J,seed,S,gmax", [(20000, 400, 1, 8, 8), (20000, 400, 2, 8, 8), (5000, 300, 3, 4, 8),
                                                 (20000, 400, 4, 8, 1), (8000, 250, 5, 16, 3)])
def test_narrow_groups_and_marks(checker, nsub, J, seed, S, gmax):
    r = subprocess.run([checker, str(nsub), str(J), str(seed), str(S), str(gmax)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    words = r.stdout.split()
    stats = dict(zip(words[0::2], words[1::2]))
    assert int(stats["mismatches"]) == 0
    assert int(stats["segments"]) > 1000 and int(stats["runs"]) > 5
    assert int(stats["after_wide"]) > 0
    if gmax > 1:
        assert int(stats["after_prev"]) > 0 and int(stats["multi"]) > 0
