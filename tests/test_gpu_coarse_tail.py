"""Coarse tail (3-D mixed form, one problem, `sgml_set_coarse_tail`): CTA 0 runs the phases that touch
only the three coarsest levels in shared memory instead of as grid phases.  The same operations in
the same order: solutions, cycle counts and residual histories must be bit-identical with it on and
off -- for odd and even sweep counts per visit (n_r = 1, 2, 3: the visit results end in either
ping-pong buffer), Neumann faces with fluxes, constant and heterogeneous coefficients, the smallest
grid it applies to (17^3, where the tail starts at level 1), and short launches, which are also
checked against the oracle."""
import numpy as np
import pytest

from paper_1703_07206_gb300 import inputs, sgml
from tests.gpu_helpers import gpu_grid, oracle_cycles, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu

CASES = {
    "dielectric_65cubed": lambda: inputs.dielectric_spheres_3d(n=6, seed=2000),
    "dielectric_129cubed": lambda: inputs.dielectric_spheres_3d(n=7, seed=2001),
    "neumann_flux_33cubed": lambda: inputs.random_problem(3, 5, seed=320, flux=True),
    "mixed_faces_17cubed": lambda: inputs.random_problem(3, 4, seed=321, flux=True),
    "poisson_65cubed": lambda: inputs.random_problem(3, 6, seed=322, hetero=False, helmholtz=False, mixed_bc=False),
    "capacitor_33cubed": lambda: inputs.capacitor_3d(n=5),
}


def _run(d, tail, n_r=2, cycles=None):
    g = gpu_grid([d], sgml.MIXED, n_r=n_r, max_cycles=400)
    g.set_coarse_tail(tail)
    if cycles is None:
        st, cyc, rel = g.solve_to_tol(1e-10)
        assert st == sgml.OK, (st, cyc, rel)
        out = (g.get_solution(0), int(cyc[0]), g.get_history(0))
    else:
        g.run_cycle(cycles)
        out = (g.get_solution(0), cycles, None)
    g.close()
    return out


@pytest.mark.parametrize("n_r", [2, 1, 3])
@pytest.mark.parametrize("name", list(CASES))
def test_coarse_tail_solves_bit_identically(name, n_r):
    if n_r != 2 and name == "dielectric_129cubed":
        pytest.skip("n_r variants run on the smaller grids")
    d = CASES[name]()
    u_on, c_on, h_on = _run(d, True, n_r)
    u_off, c_off, h_off = _run(d, False, n_r)
    assert c_on == c_off
    assert np.array_equal(h_on, h_off)
    assert np.array_equal(u_on, u_off)


@pytest.mark.parametrize("k", [1, 3])
def test_coarse_tail_short_launches_match_oracle(k):
    d = CASES["neumann_flux_33cubed"]()
    u_on, _, _ = _run(d, True, cycles=k)
    u_off, _, _ = _run(d, False, cycles=k)
    assert np.array_equal(u_on, u_off)
    u_ref = oracle_cycles(oracle_problem(d), d["f"], k)
    assert rel_l2(u_on, u_ref) <= 2e-5 * k, rel_l2(u_on, u_ref)
