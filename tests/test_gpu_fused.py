"""Fused sweep pairs and four-row sweeps (3-D, mixed form) against the FP64 oracle.

With fusion the k sweeps of a visit (Algorithm 2) run two at a time: the first sweep is evaluated on
each tile widened by one cell and kept on chip for the second.  It is the same Jacobi iteration, so
after a fixed number of cycles the solution must match the oracle within the mixed-form bound of
the unfused path (relative L2 <= 2e-5, FP32 cycle), and fused and unfused runs may differ only by
FP32 rounding (<= 1e-5).  Cases cover homogeneous and heterogeneous sigma, Neumann faces with
prescribed flux (the ring cells outside the domain are mirror images), odd sweep counts (a pair plus
a single sweep), fusion on every level, both tile shapes with ragged edge tiles, and a batch whose
problems run different sweep counts in the same visit.
"""
import numpy as np
import pytest

from paper_1703_07206_gb300 import inputs, sgml
from tests.gpu_helpers import gpu_grid, oracle_cycles, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

CASES = [
    ("hetero_flux_n4", lambda: inputs.random_problem(3, 4, seed=601, flux=True)),
    ("hetero_n5", lambda: inputs.random_problem(3, 5, seed=602)),
    ("poisson_n4", lambda: inputs.random_problem(3, 4, seed=603, hetero=False, helmholtz=False, mixed_bc=False)),
    ("neumann_flux_n5", lambda: inputs.random_problem(3, 5, seed=604, flux=True, helmholtz=True)),
]


def mixed_grid(problems, pair_levels, tile_x=64, **params):
    g = gpu_grid(problems, sgml.MIXED, **params)
    g.set_fusion(pair_levels)
    g.set_launch(0, 1, 0, tile_x, 16)
    return g


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("pair_levels", [1, 2, 13])
@pytest.mark.parametrize("n_r", [1, 2, 3])
def test_fused_cycles_match_oracle(name, make, pair_levels, n_r):
    d = make()
    p = oracle_problem(d, n_r=n_r)
    u_ref = oracle_cycles(p, d["f"], 2)
    g = mixed_grid([d], pair_levels, n_r=n_r)
    g.run_cycle(2)
    u = g.get_solution(0)
    assert rel_l2(u, u_ref) <= 2e-5, rel_l2(u, u_ref)
    g0 = mixed_grid([d], 0, n_r=n_r)
    g0.run_cycle(2)
    assert rel_l2(u, g0.get_solution(0)) <= 1e-5


@pytest.mark.parametrize("tile_x", [32, 64])
@pytest.mark.parametrize("flux", [False, True])
def test_fused_ragged_tiles_65cubed(tile_x, flux):
    """65^3: edge tiles one node wide (x0 = 64) and, with Neumann faces, kept in the partition."""
    d = inputs.random_problem(3, 6, seed=610 + int(flux), flux=flux)
    p = oracle_problem(d)
    u_ref = oracle_cycles(p, d["f"], 1)
    g = mixed_grid([d], 1, tile_x=tile_x)
    g.run_cycle(1)
    assert rel_l2(g.get_solution(0), u_ref) <= 2e-5


def test_fused_batch_with_uneven_sweep_counts():
    """n_r = 4: a visit of tooth n_b - 1 does 2 sweeps in the small problems and 4 in the large one;
    the pair phases must serve each problem its own count."""
    probs = [inputs.random_problem(3, n, seed=620 + n, flux=(n == 4)) for n in (5, 3, 4)]
    g = mixed_grid(probs, 13, n_r=4)
    g.run_cycle(2)
    for b, d in enumerate(probs):
        u_ref = oracle_cycles(oracle_problem(d, n_r=4), d["f"], 2)
        assert rel_l2(g.get_solution(b), u_ref) <= 2e-5, b


def test_fused_solve_converges_to_oracle_solution():
    d = inputs.random_problem(3, 5, seed=630, flux=True)
    u_ref, c_ref, _ = oracle_problem(d).solve(d["f"], tol=1e-12, max_cycles=400)
    g = mixed_grid([d], 1, max_cycles=400)
    st, cyc, rel = g.solve_to_tol(1e-12)
    assert st == sgml.OK
    assert rel_l2(g.get_solution(0), u_ref) <= 1e-10


def test_phase_table_pairs_sweeps_on_fused_levels():
    d = inputs.random_problem(3, 5, seed=640)
    for pair_levels, n_r in ((0, 2), (1, 2), (2, 3), (13, 1)):
        g = mixed_grid([d], pair_levels, n_r=n_r)
        ph = g.get_phases()
        sweeps = [q for q in ph if q[0] == 1]
        # every sweep index of every visit is performed exactly once
        total = sum(q[3] for q in sweeps)
        g0 = mixed_grid([d], 0, n_r=n_r)
        assert total == len([q for q in g0.get_phases() if q[0] == 1])
        for op, level, first, count in sweeps:
            assert count == 1 or (count == 2 and level < pair_levels and first % 2 == 0)
            if level >= pair_levels:
                assert count == 1
    # 2-D and FP64 grids never pair
    g2 = gpu_grid([inputs.random_problem(2, 5, seed=641)], sgml.MIXED)
    g2.set_fusion(13)
    assert all(q[3] <= 1 for q in g2.get_phases())
    g3 = gpu_grid([d], sgml.FP64)
    g3.set_fusion(13)
    assert all(q[3] <= 1 for q in g3.get_phases())


# --- four-row sweeps (tiles of 64 x 16 / 32 x 32 columns, four nodes per thread) ---------------

def quad_grid(problems, quad_levels, tile_x=64, **params):
    g = gpu_grid(problems, sgml.MIXED, **params)
    g.set_fusion(0)
    g.set_quad(quad_levels)
    g.set_launch(0, 1, 0, tile_x, 32)
    return g


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("quad_levels", [1, 13])
@pytest.mark.parametrize("n_r", [1, 2, 3])
def test_four_row_sweeps_match_oracle(name, make, quad_levels, n_r):
    d = make()
    p = oracle_problem(d, n_r=n_r)
    u_ref = oracle_cycles(p, d["f"], 2)
    g = quad_grid([d], quad_levels, n_r=n_r)
    g.run_cycle(2)
    u = g.get_solution(0)
    assert rel_l2(u, u_ref) <= 2e-5, rel_l2(u, u_ref)
    g0 = quad_grid([d], 0, n_r=n_r)
    g0.run_cycle(2)
    assert rel_l2(u, g0.get_solution(0)) <= 1e-5


@pytest.mark.parametrize("flux", [False, True])
def test_four_row_sweeps_ragged_65cubed_and_tile_shapes(flux):
    """65^3 with edge tiles one node wide; 64 x 16 and 32 x 32 tiles give identical results."""
    d = inputs.random_problem(3, 6, seed=650 + int(flux), flux=flux)
    u_ref = oracle_cycles(oracle_problem(d), d["f"], 1)
    sols = []
    for tile_x in (64, 32):
        g = quad_grid([d], 13, tile_x=tile_x)
        g.run_cycle(1)
        sols.append(g.get_solution(0))
        assert rel_l2(sols[-1], u_ref) <= 2e-5
    assert np.array_equal(sols[0], sols[1])


def test_four_row_sweeps_batch_with_uneven_sweep_counts():
    probs = [inputs.random_problem(3, n, seed=660 + n, flux=(n == 4)) for n in (5, 3, 4)]
    g = quad_grid(probs, 13, n_r=4)
    g.run_cycle(2)
    for b, d in enumerate(probs):
        u_ref = oracle_cycles(oracle_problem(d, n_r=4), d["f"], 2)
        assert rel_l2(g.get_solution(b), u_ref) <= 2e-5, b
