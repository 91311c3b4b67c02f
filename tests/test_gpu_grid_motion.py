"""Grid motion of the grid-deformation application (Sec. 3.2, Eq. 11) on the GPU against the oracle.

* Random smooth potentials and positive sources, 2-D and 3-D, start points inside and outside the
  domain: the GPU positions equal the oracle's to rounding after every step count tried.
* Fig. 5's circle: the force potential solved by the library (all-Neumann Helmholtz, a = 0.1,
  65^2, mixed form), then the grid moved on the GPU and by the oracle from the same potential.
* Argument errors: a source whose denominator could vanish, t1 < t0, negative step counts.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle
from paper_1703_07206_gb300 import inputs, sgml
from tests.gpu_helpers import gpu_grid

pytestmark = pytest.mark.gpu


def smooth_field(dim, n, seed, modes=5):
    rng = np.random.default_rng(seed)
    X = oracle.grid_nodes(dim, 2 ** n + 1)
    u = np.zeros(X.shape[1:])
    for _ in range(modes):
        k = rng.integers(0, 4, size=dim)
        ph = rng.uniform(0, 2 * np.pi, size=dim)
        term = rng.standard_normal() / (1 + k.sum())
        for a in range(dim):
            term = term * np.cos(np.pi * k[a] * X[a] + ph[a])
        u += term
    return u


@pytest.mark.parametrize("dim,n,steps", [(2, 5, 60), (2, 6, 25), (3, 4, 40), (3, 6, 12)])
def test_motion_matches_oracle(dim, n, steps):
    u = smooth_field(dim, n, 1000 + 10 * dim + n)
    f = 0.3 + np.abs(smooth_field(dim, n, 2000 + 10 * dim + n))
    rng = np.random.default_rng(3000 + n)
    x0 = oracle.grid_nodes(dim, 2 ** n + 1) + rng.uniform(-0.4, 0.4, size=(dim,) + u.shape) / 2 ** n
    x0.reshape(dim, -1)[:, :7] = rng.uniform(-0.2, 1.2, size=(dim, 7))  # some start outside: clamped
    want = oracle.grid_motion(u, f, steps, 0.0, 1.0, x0)
    got = sgml.grid_motion(torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda(), steps, 0.0, 1.0,
                           torch.from_numpy(x0).cuda()).cpu().numpy()
    assert np.all((got >= 0) & (got <= 1))
    assert np.abs(got - want).max() <= 1e-12
    assert np.abs(want - x0).max() > 1e-3  # something moved


def test_motion_in_pieces_equals_one_run():
    """t in [0, 0.5] then [0.5, 1] with half the steps each is the same Euler sequence."""
    u = smooth_field(2, 5, 11)
    f = 0.5 + np.abs(smooth_field(2, 5, 12))
    ug, fg = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
    whole = sgml.grid_motion(ug, fg, 40)
    half = sgml.grid_motion(ug, fg, 20, 0.0, 0.5)
    both = sgml.grid_motion(ug, fg, 20, 0.5, 1.0, half)
    assert torch.abs(whole - both).max().item() <= 1e-14
    assert torch.equal(sgml.grid_motion(ug, fg, 0), sgml.grid_motion(ug, fg, 0, 0.3, 0.7))


def test_circle_force_potential_motion():
    d = inputs.neumann_helmholtz_2d(6, a=0.1)
    g = gpu_grid([d], sgml.MIXED, max_cycles=400)
    st, cyc, rel = g.solve_to_tol(1e-10)
    assert st == sgml.OK
    N = 65
    u = torch.empty((N, N), dtype=torch.float64, device="cuda")
    g.get_solution(0, u)
    f = torch.from_numpy(d["f"]).cuda()
    x = sgml.grid_motion(u, f, 100).cpu().numpy()
    want = oracle.grid_motion(u.cpu().numpy(), d["f"], 100)
    assert np.abs(x - want).max() <= 1e-12
    assert np.all(x[0][:, 0] == 0.0) and np.all(x[0][:, -1] == 1.0)
    assert np.all(x[1][0, :] == 0.0) and np.all(x[1][-1, :] == 1.0)
    r0 = np.hypot(*(oracle.grid_nodes(2, N) - 0.5))
    r1 = np.hypot(*(x - 0.5))
    assert np.count_nonzero(np.abs(r1 - 0.25) < 0.01) > 5 * np.count_nonzero(np.abs(r0 - 0.25) < 0.01)


def test_motion_argument_errors():
    u = torch.zeros((17, 17), dtype=torch.float64, device="cuda")
    f = torch.full((17, 17), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(sgml.SGMLError):
        sgml.grid_motion(u, f, 10)  # int f < 0
    f2 = torch.ones((17, 17), dtype=torch.float64, device="cuda")
    f2[8, 8] = -200.0  # int f > 0 but t f + int f < 0 near the node at t = 1
    with pytest.raises(sgml.SGMLError):
        sgml.grid_motion(u, f2, 10)
    sgml.grid_motion(u, f2, 10, 0.0, 0.001)  # fine while t stays small
    lib = sgml.load()
    x = torch.zeros((2, 17, 17), dtype=torch.float64, device="cuda")
    for args in ((2, 4, 0.5, 0.2, 10), (2, 4, 0.0, 1.0, -1), (4, 4, 0.0, 1.0, 1), (2, 0, 0.0, 1.0, 1)):
        dim, n, t0, t1, k = args
        st = lib.sgml_grid_motion(dim, n, u.data_ptr(), f2.data_ptr(), t0, t1, k, x.data_ptr(), None)
        assert st == sgml.ERR_ARG, args
    host = np.zeros((2, 17, 17))
    st = lib.sgml_grid_motion(2, 4, u.data_ptr(), f2.data_ptr(), 0.0, 1.0, 1,
                              host.ctypes.data_as(ctypes.c_void_p), None)
    assert st == sgml.ERR_ARG
    assert lib.sgml_grid_motion(2, 4, u.data_ptr(), f2.data_ptr(), 0.0, 1.0, 1, u.data_ptr(), None) == sgml.ERR_ARG
