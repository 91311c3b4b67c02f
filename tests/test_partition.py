"""Work partition of the tiled phases (host code, sgml_tasks.h), checked on the CPU.

Every (problem, tile, plane) of every level that holds an unknown is covered by exactly one task,
the task count stays within the bound the library allocates for, and the CTAs receive equal shares
of level 0 -- for the contiguous cut and the slab cut, both tile shapes, 2-D and 3-D, single
problems and batches of mixed sizes.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1703_07206_gb300", "csrc")


def _cuda_include():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            return os.path.join(cand, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    inc = _cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("part") / "partition_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", inc, "-o", exe,
                           os.path.join(HERE, "native", "partition_check.cpp")])
    out = subprocess.check_output([exe], text=True)
    rows = []
    for line in out.strip().splitlines():
        dim, ns, G, tx, slab, ok, share, maxnz0 = line.split()
        rows.append(dict(dim=int(dim), ns=ns, G=int(G), tx=int(tx), slab=int(slab), ok=int(ok), share=float(share),
                         maxnz0=int(maxnz0)))
    return rows


def test_every_plane_covered_once(results):
    assert len(results) == 54
    bad = [r for r in results if not r["ok"]]
    assert not bad, bad


def test_level0_shares_are_balanced(results):
    for r in results:
        if r["ns"] in ("8", "7,7,7,7,7,7,7,7,7,7,7,7,7,7,7,7") or (r["dim"] == 2 and r["ns"] == "10"):
            # large levels: within one slab (or one tile-plane) of the mean
            assert r["share"] <= 1.12, r


def test_slab_cut_reaches_level0_where_the_parity_tests_need_it(results):
    """129^3 on 304 CTAs: a slab height of 4 puts level 0 on the slab cut (pieces of at most
    3/2 x 4 planes, dealt in turn), the contiguous cut gives runs of ~13.6 planes.  The GPU parity
    tests of the headline recipe rely on this to compare the slab path with the oracle."""
    for tx in (32, 64):
        slab = [r for r in results if r["dim"] == 3 and r["ns"] == "7" and r["tx"] == tx and r["slab"] == 4][0]
        runs = [r for r in results if r["dim"] == 3 and r["ns"] == "7" and r["tx"] == tx and r["slab"] == 0][0]
        assert slab["maxnz0"] <= 6 < runs["maxnz0"], (slab, runs)
