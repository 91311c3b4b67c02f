"""The heterogeneous capacitor of Sec. 3.4 (Eqs. 15-16) on the GPU.

div(sigma grad u) = 0 on the unit cube, sigma = 0.55 +- 0.45 tanh((r - 0.2) / 0.1) (r: distance to
the centre; both signs: a conducting or an insulating ball), u = -1 on the bottom face and +1 on the
top face, zero normal derivative on the four lateral faces.  It exercises the non-zero Dirichlet
lift, 3-D mixed boundary conditions, a zero source (the residual is normalised by the initial one)
and a smooth coefficient contrast of 10.

* 33^3: the converged GPU solution (both forms) equals the oracle's converged solution.
* 129^3 (the paper's size): the oracle's residual of the GPU solution is at the tolerance, the
  solution obeys the maximum principle (|u| <= 1), and it is odd under z -> 1 - z (sigma is even
  about the centre and the boundary values are odd), which no part of the solver imposes.
"""
import numpy as np
import pytest

from paper_1703_07206_gb300 import inputs, sgml
from tests.gpu_helpers import gpu_grid, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("precision", [sgml.MIXED, sgml.FP64])
def test_capacitor_33_matches_oracle(sign, precision):
    d = inputs.capacitor_3d(n=5, sign=sign)
    u_ref, c_ref, _ = oracle_problem(d).solve(d["f"], tol=1e-12, max_cycles=400)
    assert c_ref >= 0
    g = gpu_grid([d], precision, max_cycles=400)
    st, cyc, rel = g.solve_to_tol(1e-12)
    assert st == sgml.OK
    assert rel_l2(g.get_solution(0), u_ref) <= 1e-10


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_capacitor_129_residual_and_symmetry(sign):
    d = inputs.capacitor_3d(n=7, sign=sign)
    g = gpu_grid([d], sgml.MIXED, max_cycles=400)
    st, cyc, rel = g.solve_to_tol(1e-10)
    assert st == sgml.OK and rel[0] <= 1e-10
    u = g.get_solution(0)
    p = oracle_problem(d)
    # relative to the initial residual (f = 0): r0 = -delta L (lifted boundary values)
    r0 = np.abs(p.residual(p.lift(), d["f"])[p.unknown_mask()]).max()
    r = np.abs(p.residual(u, d["f"])[p.unknown_mask()]).max()
    assert r <= 1.2e-10 * r0
    assert np.abs(u).max() <= 1.0 + 1e-12
    # odd symmetry in z (array axis 0 is z)
    assert np.abs(u + u[::-1, :, :]).max() <= 1e-8
    # and the mirror symmetries of the lateral directions
    assert np.abs(u - u[:, ::-1, :]).max() <= 1e-8
    assert np.abs(u - u[:, :, ::-1]).max() <= 1e-8
