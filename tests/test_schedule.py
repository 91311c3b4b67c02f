"""The cycle's phase table and the coarse tail's placement (host code, sgml_schedule.h), checked on the
CPU.

* The sweeps of one cycle on 33^2 follow the visit sequence of Algorithm 3 pinned in
  tests/golden/alg3_schedule_33x33.txt (the library merges tooth 0's two level-0 visits with the
  final one: consecutive runs at one level are compared as one run).
* Marking the coarse tail changes no phase (operation, level, tooth, sweep, flags, interpolation
  tooth); exactly one phase starts it, the restriction into level n - 3; every phase inside it
  touches only the three coarsest levels and the first phase after it touches a finer one; with
  n_r = 2 it spans the 23 phases of the restrictions into those levels, teeth n - 1 and n - 2 and
  the start of tooth n - 3.
* The CTA picked to run the tail has no tiles on levels n - 5 .. n - 1 and is the last such CTA.
"""
import os
import shutil
import subprocess

import pytest

from tests.test_partition import CSRC, HERE, _cuda_include


@pytest.fixture(scope="module")
def out(tmp_path_factory):
    inc = _cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("sched") / "schedule_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", inc, "-o", exe,
                           os.path.join(HERE, "native", "schedule_check.cpp")])
    return subprocess.check_output([exe], text=True).strip().splitlines()


def _golden_runs():
    runs = []
    with open(os.path.join(HERE, "golden", "alg3_schedule_33x33.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            level, sweeps = (int(v) for v in line.split())
            if runs and runs[-1][0] == level:
                runs[-1][1] += sweeps
            else:
                runs.append([level, sweeps])
    return runs


def test_visit_sequence_matches_algorithm_3_golden(out):
    line = [l for l in out if l.startswith("visits")][0]
    got = [[int(a), int(b)] for a, b in (tok.split(":") for tok in line.split()[1:])]
    assert got == _golden_runs()


def test_coarse_tail_marks_only_the_three_coarsest_levels(out):
    rows = [list(map(int, l.split()[1:])) for l in out if l.startswith("phases")]
    assert len(rows) == 11 * 3 * 2 * 2
    for n, n_r, pair, eq10, same, starts, op, level, span, inner, boundary in rows:
        assert same == 1, (n, n_r, pair, eq10)
        if n < 4:
            assert starts == 0
            continue
        assert starts == 1 and op == 0 and level == n - 3, (n, n_r)
        assert inner == 1 and boundary == 1, (n, n_r, pair, eq10)
        if n_r == 2 and pair == 0:
            assert span == 23, (n, span)


def test_tail_cta_is_the_last_idle_one(out):
    rows = [list(map(int, l.split()[1:])) for l in out if l.startswith("tailcta")]
    assert len(rows) == 6 * 2 * 3
    for dim, n, G, tx, cta, idle, last in rows:
        assert 0 <= cta < G and idle == 1 and last == 1, (n, G, tx, cta)
