"""Batched uneven 2-D Helmholtz problems (row A8): the full 256-problem workload (sides 65..1025,
k^2 in [0, 10], mixed Dirichlet/Neumann sides) solved in one persistent launch, checked per problem
with the oracle's residual (a property that holds at any size) and, for the small ones, against the
oracle's converged solution; CUDA-graph capture of run_cycle; the launch-shape autotuner."""
import numpy as np
import pytest

from oracle.oracle import Problem
from paper_1703_07206_gb300 import autotune, inputs, sgml
from tests.gpu_helpers import gpu_grid, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch256():
    return inputs.helmholtz_batch_2d(count=256, seed=4000)


def test_full_batch_converges_and_oracle_residuals_agree(batch256):
    g = gpu_grid(batch256, sgml.MIXED, max_cycles=200)
    st, cyc, rel = g.solve_to_tol(1e-10)
    assert st == sgml.OK and np.all(rel <= 1e-10)
    rng = np.random.default_rng(1)
    for b in sorted(rng.choice(len(batch256), size=24, replace=False)):
        d = batch256[b]
        u = g.get_solution(int(b))
        p = oracle_problem(d)
        assert p.rel_residual(u, d["f"]) <= 1.2e-10, b
        if d["n"] <= 7:  # small problems: the oracle's own converged solution
            u_ref, c_ref, _ = p.solve(d["f"], tol=1e-12, max_cycles=200)
            g1 = gpu_grid([d], sgml.MIXED, max_cycles=200)
            g1.solve_to_tol(1e-12)
            assert rel_l2(g1.get_solution(0), u_ref) <= 1e-10


def test_cuda_graph_capture_of_run_cycle():
    import torch
    probs = [inputs.random_problem(2, n, seed=600 + n) for n in (5, 6, 4)]
    for mode in (0, 1):
        g = gpu_grid(probs, sgml.MIXED)
        ref = gpu_grid(probs, sgml.MIXED)
        stream = torch.cuda.Stream()
        g2 = sgml.Grid(2, [d["n"] for d in probs], precision=sgml.MIXED, stream=stream)
        for b, d in enumerate(probs):
            sgml.problem_into_grid(g2, b, d)
        g2.set_launch(0, 1, mode, 64, 32)
        with torch.cuda.stream(stream):
            g2.run_cycle(2)  # warm-up: builds every table outside the capture
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            g2.run_cycle(2)
        graph.replay()
        graph.replay()
        torch.cuda.synchronize()
        ref.set_launch(0, 1, mode, 64, 32)
        ref.run_cycle(2)
        ref.run_cycle(2)
        ref.run_cycle(2)
        for b in range(len(probs)):
            assert np.array_equal(g2.get_solution(b), ref.get_solution(b)), (mode, b)


def test_autotuner_picks_a_candidate_and_caches(tmp_path):
    d = inputs.dielectric_spheres_3d(n=6, seed=2000)
    g = gpu_grid([d], sgml.MIXED)
    cache = str(tmp_path / "tune.json")
    r1 = autotune.tune(g, cycles=2, cache_path=cache)
    assert not r1["cached"] and r1["choice"] in autotune.DEFAULT_CANDIDATES
    r2 = autotune.tune(g, cycles=2, cache_path=cache)
    assert r2["cached"] and r2["choice"] == r1["choice"]
    st, cyc, rel = g.solve_to_tol(1e-10)
    assert st == sgml.OK
    ref = gpu_grid([d], sgml.MIXED)
    ref.solve_to_tol(1e-10)
    assert np.array_equal(g.get_solution(0), ref.get_solution(0))


def test_batch_beyond_the_cached_stop_flags_matches_single_solves():
    """300 problems: the kernels keep the first 256 problems' stop flags in shared memory and read
    the rest from global memory, and problem 0's descriptor from shared memory.  Problems stop at
    different cycles; each one's solution must equal, bit for bit, its solve alone (the arithmetic
    of a node does not depend on the batch or the work partition)."""
    probs = [inputs.random_problem(2, 3 + (b % 3), seed=5000 + b, flux=(b % 7 == 0)) for b in range(300)]
    g = gpu_grid(probs, sgml.MIXED, max_cycles=300)
    st, cyc, rel = g.solve_to_tol(1e-10)
    assert st == sgml.OK and np.all(rel <= 1e-10)
    assert len(set(int(c) for c in np.asarray(cyc).ravel())) > 1  # the problems stop at different cycles
    for b in (0, 1, 255, 256, 257, 298, 299):
        d = probs[b]
        g1 = gpu_grid([d], sgml.MIXED, max_cycles=300)
        st1, cyc1, _ = g1.solve_to_tol(1e-10)
        assert st1 == sgml.OK and int(np.asarray(cyc1).ravel()[0]) == int(np.asarray(cyc).ravel()[b]), b
        assert np.array_equal(g.get_solution(b), g1.get_solution(0)), b
        assert oracle_problem(d).rel_residual(g.get_solution(b), d["f"]) <= 1.2e-10, b
