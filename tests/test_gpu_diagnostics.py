"""Diagnostic pseudo-residual per level (Sec. 3.1) on the GPU against the oracle.

The largest |delta L_l e - r_l| met by each level's sweeps during one cycle: the FP64 form equals
the oracle's to rounding (the GPU forms it as |e_new - e| / delta tau); the mixed form to FP32
accuracy.  Recording it changes no result.
"""
import numpy as np
import pytest

from paper_1703_07206_gb300 import inputs, sgml
from tests.gpu_helpers import gpu_grid, oracle_problem

pytestmark = pytest.mark.gpu

CASES = [
    ("rand2d_n5_flux", lambda: inputs.random_problem(2, 5, seed=701, flux=True)),
    ("rand3d_n4", lambda: inputs.random_problem(3, 4, seed=702)),
    ("rand3d_n5_flux", lambda: inputs.random_problem(3, 5, seed=703, flux=True)),
    ("poisson3d_n4", lambda: inputs.random_problem(3, 4, seed=704, hetero=False, helmholtz=False, mixed_bc=False)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision,tol", [(sgml.FP64, 1e-9), (sgml.MIXED, 2e-3)])
def test_pseudo_residual_matches_oracle(name, make, precision, tol):
    d = make()
    p = oracle_problem(d)
    r0 = p.residual(p.lift(), d["f"])
    _, ref = p.cycle_diag(r0)
    g = gpu_grid([d], precision)
    g.set_diagnostics(4)
    g.run_cycle(1)
    got = g.get_diagnostics(0)[0, : d["n"]]
    assert np.all(ref > 0)
    assert np.all(np.abs(got - ref) <= tol * ref), (got, ref)


def test_recording_changes_no_result():
    d = inputs.random_problem(3, 5, seed=705, flux=True)
    sols = []
    for cycles in (0, 8):
        g = gpu_grid([d], sgml.MIXED)
        if cycles:
            g.set_diagnostics(cycles)
        g.run_cycle(3)
        sols.append(g.get_solution(0))
        if cycles:
            diag = g.get_diagnostics(0)
            assert diag.shape == (8, 13)
            # cycles 0..2 recorded (all levels active), nothing beyond the levels of the problem
            assert np.all(diag[:3, :5] > 0) and np.all(diag[:, 5:] == 0)
    assert np.array_equal(sols[0], sols[1])
