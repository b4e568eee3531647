"""The data layout sccs_create builds on the device, against its definitions.  Two small C++
programs link the library, make a handle, copy its layout back through the layout diagnostic
(sccs_debug_layout) and compare it with a brute-force construction: the whole layout (kept
subjects and rows, each column's kept rows, Y'X_j and event pairs, every slice's segments,
diagonal-major rows and group bases, the cluster columns and their groups), and the narrow
columns (groups of consecutive narrow columns touch pairwise disjoint subjects and fit half the
shared buffers; each segment's mark names the one earlier step that can change its subject, so
the GPU re-gathers a segment exactly when that step was not zero)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

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


SLICE_SRC = os.path.join(ROOT, "tests", "native", "slice_layout_check.cpp")


@pytest.fixture(scope="module")
def slice_checker(tmp_path_factory):
    nvcc = os.environ.get("NVCC") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc")
                                      else shutil.which("nvcc"))
    if not nvcc:
        pytest.skip("nvcc not available")
    import __graft_entry__
    lib = __graft_entry__._build_module().build()
    exe = str(tmp_path_factory.mktemp("slices") / "slice_layout_check")
    cmd = [nvcc, "-std=c++17", "-O2", "-I" + os.path.join(ROOT, "include"), SLICE_SRC, lib,
           "-Xlinker", "-rpath=" + os.path.dirname(lib), "-o", exe, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


@pytest.mark.parametrize("nsub,J,seed,S,messy,C,cmax", [(8000, 120, 5, 7, 1, 0, 0), (8000, 120, 6, 7, 0, 0, 0),
                                                         (3000, 60, 7, 1, 1, 0, 0), (20000, 90, 8, 33, 1, 0, 0),
                                                         (500, 40, 9, 4, 0, 0, 0), (8000, 120, 10, 32, 1, 16, 300),
                                                         (20000, 90, 11, 24, 0, 8, 100000),
                                                         (6000, 50, 12, 8, 1, 4, 5000), (3000, 30, 13, 8, 1, 8, 10**9)])
def test_slice_layout_against_brute_force(slice_checker, nsub, J, seed, S, messy, C, cmax):
    """The whole layout -- kept subjects and rows, per-column kept rows, Y'X_j and event
    pairs, every (shard, column) slice's segments, diagonal-major rows and group bases -- against
    a brute-force construction, with dropped subjects and shuffled columns (messy) or without; with
    C > 0 also the cluster columns (at most cmax nonzeros and every slice over the C cluster shards
    within the staging caps), their slices over those shards, and the next-grid-column map."""
    r = subprocess.run([slice_checker, str(nsub), str(J), str(seed), str(S), str(messy), str(C), str(cmax)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
    if C:
        words = r.stdout.split()
        ncl = int(words[words.index("cluster_columns") + 1])
        assert 0 < ncl <= J, r.stdout
        if cmax < 10**6:
            assert ncl < J, r.stdout   # both kinds of column occur
