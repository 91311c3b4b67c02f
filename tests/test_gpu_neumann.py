"""All-Neumann problems with a >= 0 (Sec. 3.2, Eq. 10) on the GPU against the oracle.

L u = f - <f> with zero normal derivatives everywhere, for the zero-mean u: the paper's force
potential (a = 0.1, a finite delta source along a circle, 65^2) and a = 0 (pure Neumann Poisson,
singular without the projection), 2-D and 3-D, heterogeneous sigma.  Both sides subtract the source
mean and project the constant mode out of u after every cycle; the FP64 form matches the oracle
cycle by cycle, and converged solutions of both forms match the oracle's.
"""
import numpy as np
import pytest

from paper_1703_07206_gb300 import inputs, sgml
from tests.gpu_helpers import gpu_grid, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


def neumann_problem(dim, n, a, seed, hetero=True):
    rng = np.random.default_rng(seed)
    N = 2 ** n + 1
    shape = (N,) * dim
    f = rng.standard_normal(shape)
    sigma = np.exp(0.4 * rng.standard_normal(shape)) if hetero else None
    return dict(dim=dim, n=n, f=f, sigma=sigma, a=None, a_scalar=float(a),
                faces=[inputs.NEUMANN] * (2 * dim), values=[0.0] * (2 * dim))


CASES = [
    ("circle65_a0.1", lambda: inputs.neumann_helmholtz_2d(6, a=0.1)),
    ("rand33_a0", lambda: neumann_problem(2, 5, 0.0, 801)),
    ("rand17cubed_a0.1", lambda: neumann_problem(3, 4, 0.1, 802)),
    ("rand17cubed_a0_const", lambda: neumann_problem(3, 4, 0.0, 803, hetero=False)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [sgml.FP64, sgml.MIXED])
def test_eq10_converged_solution_matches_oracle(name, make, precision):
    d = make()
    p = oracle_problem(d)
    assert p.projects_mean()
    u_ref, c_ref, _ = p.solve(d["f"], tol=1e-12, max_cycles=400)
    assert c_ref >= 0
    g = gpu_grid([d], precision, max_cycles=400)
    st, cyc, rel = g.solve_to_tol(1e-12 if precision == sgml.FP64 else 1e-10)
    assert st == sgml.OK, (st, cyc, rel)
    u = g.get_solution(0)
    assert rel_l2(u, u_ref) <= (1e-11 if precision == sgml.FP64 else 1e-8)
    assert abs(p.mean(u)) <= 1e-12 * np.abs(u).max()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_eq10_fp64_cycles_match_oracle(name, make):
    d = make()
    p = oracle_problem(d)
    fp = d["f"] - p.mean(d["f"])
    u_ref = p.lift()
    for _ in range(3):
        u_ref = u_ref + p.cycle(p.residual(u_ref, fp))
        u_ref = u_ref - p.mean(u_ref)
    g = gpu_grid([d], sgml.FP64)
    g.run_cycle(3)
    assert rel_l2(g.get_solution(0), u_ref) <= 1e-12


def test_eq10_in_a_batch_and_back_to_dirichlet():
    probs = [inputs.neumann_helmholtz_2d(5, a=0.1), inputs.random_problem(2, 5, seed=810),
             neumann_problem(2, 4, 0.0, 811)]
    g = gpu_grid(probs, sgml.MIXED, max_cycles=400)
    st, cyc, rel = g.solve_to_tol(1e-10)
    assert st == sgml.OK
    for b, d in enumerate(probs):
        u_ref, _, _ = oracle_problem(d).solve(d["f"], tol=1e-12, max_cycles=400)
        assert rel_l2(g.get_solution(b), u_ref) <= 1e-9, b
    # the first problem gets Dirichlet faces: its source is restored to the one given
    faces = [inputs.DIRICHLET] * 4
    g.set_bc(0, faces, [0.0] * 4)
    st, cyc, rel = g.solve_to_tol(1e-10)
    assert st == sgml.OK
    d = dict(probs[0], faces=faces)
    u_ref, _, _ = oracle_problem(d).solve(d["f"], tol=1e-12, max_cycles=400)
    assert rel_l2(g.get_solution(0), u_ref) <= 1e-9


def test_eq10_needs_zero_derivatives():
    d = inputs.neumann_helmholtz_2d(4, a=0.1)
    g = gpu_grid([d], sgml.MIXED)
    g.set_bc(0, [inputs.NEUMANN] * 4, [0.0, 0.5, 0.0, 0.0])
    with pytest.raises(sgml.SGMLError):
        g.solve_to_tol(1e-10)


@pytest.mark.parametrize("dim", [2, 3])
def test_boundary_change_on_an_existing_grid_matches_a_fresh_grid(dim):
    """Nodes that become fixed keep no stale correction or residual from the previous solve."""
    d = inputs.random_problem(dim, 5 if dim == 2 else 4, seed=820 + dim, mixed_bc=False, helmholtz=True)
    neu = dict(d, faces=[inputs.NEUMANN] * (2 * dim), values=[0.0] * (2 * dim), a=None, a_scalar=-1.0)
    g = gpu_grid([neu], sgml.MIXED, max_cycles=400)
    assert g.solve_to_tol(1e-10)[0] == sgml.OK
    dirf = dict(neu, faces=[inputs.DIRICHLET] * (2 * dim))
    g.set_bc(0, dirf["faces"], dirf["values"])
    assert g.solve_to_tol(1e-10)[0] == sgml.OK
    fresh = gpu_grid([dirf], sgml.MIXED, max_cycles=400)
    assert fresh.solve_to_tol(1e-10)[0] == sgml.OK
    assert np.array_equal(g.get_solution(0), fresh.get_solution(0))
