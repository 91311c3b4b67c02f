"""Pins of the oracle's grid motion (Sec. 3.2, Eq. 11) to facts fixed outside the oracle.

* grad u: central differences are exact on quadratics inside, the Neumann images give a zero normal
  derivative on the faces, and the error on a smooth cosine field falls as h^2.
* int f dOmega: the trapezoid rule is exact on linear fields and has the known h^2 / 6 error on x^2.
* Motion: no motion under a constant potential; for a quadratic potential and a constant source the
  Euler product has a closed form; for a linear potential and a linear source the Euler positions
  converge at first order to a high-accuracy ODE solution (scipy), which fixes the t f term.
* The circle force potential of Fig. 5: face nodes slide along their faces, the grid keeps the
  square's symmetries, stays untangled and gathers nodes at the circle.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import oracle
from oracle.oracle import Problem
from paper_1703_07206_gb300 import inputs


def coords(dim, n):
    x = oracle.grid_nodes(dim, 2 ** n + 1)
    return [x[a] for a in range(dim)]


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_exact_on_quadratics_inside_and_zero_normal_on_faces(dim):
    n = 4
    N = 2 ** n + 1
    X = coords(dim, n)
    coef = [1.0, -3.0, 0.5][:dim]
    lin = [0.2, 0.7, -1.1][:dim]
    u = sum(coef[a] * X[a] ** 2 + lin[a] * X[a] for a in range(dim)) + 0.3 * X[0] * X[1]
    g = oracle.neumann_gradient(u)
    for a in range(dim):
        want = 2 * coef[a] * X[a] + lin[a] + 0.3 * (X[1] if a == 0 else (X[0] if a == 1 else 0.0))
        ax = dim - 1 - a  # array axis of coordinate a
        inside = [slice(None)] * dim
        inside[ax] = slice(1, N - 1)
        assert np.abs(g[a][tuple(inside)] - want[tuple(inside)]).max() <= 1e-12
        for face in (0, N - 1):
            sl = [slice(None)] * dim
            sl[ax] = face
            assert np.all(g[a][tuple(sl)] == 0.0)


def test_gradient_second_order_on_a_neumann_cosine():
    errs = []
    for n in (4, 5, 6):
        X, Y = coords(2, n)
        u = np.cos(np.pi * X) * np.cos(2 * np.pi * Y)
        g = oracle.neumann_gradient(u)
        gx = -np.pi * np.sin(np.pi * X) * np.cos(2 * np.pi * Y)
        gy = -2 * np.pi * np.cos(np.pi * X) * np.sin(2 * np.pi * Y)
        errs.append(max(np.abs(g[0] - gx).max(), np.abs(g[1] - gy).max()))
    assert 3.7 < errs[0] / errs[1] < 4.3 and 3.7 < errs[1] / errs[2] < 4.3


@pytest.mark.parametrize("dim", [2, 3])
def test_trapezoid_integral(dim):
    n = 3
    h = 1.0 / 2 ** n
    X = coords(dim, n)
    lin = 1.0 + sum((a + 2.0) * X[a] for a in range(dim))
    assert abs(oracle.trapezoid(lin) - (1.0 + sum((a + 2.0) / 2 for a in range(dim)))) <= 1e-14
    assert abs(oracle.trapezoid(X[dim - 1] ** 2) - (1.0 / 3.0 + h * h / 6.0)) <= 1e-14


def test_constant_potential_moves_nothing():
    N = 17
    rng = np.random.default_rng(3)
    f = rng.uniform(0.5, 2.0, size=(N, N))
    x = oracle.grid_motion(np.full((N, N), 2.5), f, 40)
    assert np.array_equal(x, oracle.grid_nodes(2, N))


@pytest.mark.parametrize("dim", [2, 3])
def test_contraction_closed_form(dim):
    """u = -(alpha/2) |x - c|^2, f = c0: inside, v = alpha (x - c) / (c0 (1 + t)), so every Euler step
    scales x - c by 1 + dt alpha / (c0 (1 + t_k))."""
    n = 4
    N = 2 ** n + 1
    X = coords(dim, n)
    c0, alpha, K = 1.7, -0.6 * 1.7, 50
    u = -0.5 * alpha * sum((X[a] - 0.5) ** 2 for a in range(dim))
    f = np.full(u.shape, c0)
    x = oracle.grid_motion(u, f, K)
    dt = 1.0 / K
    scale = np.prod([1.0 + dt * alpha / (c0 * (1.0 + k * dt)) for k in range(K)])
    inner = tuple([slice(1, N - 1)] * dim)
    for a in range(dim):
        want = 0.5 + (X[a] - 0.5) * scale
        assert np.abs(x[a][inner] - want[inner]).max() <= 1e-13


def test_source_term_first_order_convergence_to_the_ode():
    """u = -g x (grad u = -g inside), f = c0 + beta x: dx/dt = g / (t (c0 + beta x) + c0 + beta / 2)."""
    N = 33
    X, Y = coords(2, 5)
    gval, c0, beta = 0.35, 0.6, 2.0
    u = -gval * X
    f = c0 + beta * X + 0.0 * Y
    F = c0 + beta / 2
    x_start = np.array([0.25, 0.3125, 0.40625])

    def rhs(t, x):
        return gval / (t * (c0 + beta * x) + F)

    exact = [solve_ivp(rhs, (0.0, 1.0), [s], rtol=1e-12, atol=1e-14).y[0, -1] for s in x_start]
    assert max(exact) < 1.0 - 2.0 / (N - 1) and min(e - s for e, s in zip(exact, x_start)) > 0.1
    cols = np.rint(x_start * (N - 1)).astype(int)
    errs = []
    for K in (100, 200, 400):
        xm = oracle.grid_motion(u, f, K)
        errs.append(np.abs(xm[0][N // 2, cols] - exact).max())
        assert np.all(xm[1] == oracle.grid_nodes(2, N)[1])  # no y motion
    assert errs[2] < 2e-3
    assert 1.85 < errs[0] / errs[1] < 2.15 and 1.85 < errs[1] / errs[2] < 2.15


@pytest.fixture(scope="module")
def circle_motion():
    """The circle source of Fig. 5 summed over the square's eight symmetries (the sampled circle
    itself is symmetric only to the sampling), its force potential and the moved grid."""
    d = inputs.neumann_helmholtz_2d(6, a=0.1)
    f = d["f"] + d["f"][:, ::-1]
    f = f + f[::-1, :]
    f = 0.125 * (f + f.T)
    p = Problem(2, 6, faces=d["faces"], values=d["values"], a_scalar=d["a_scalar"])
    u, cycles, _ = p.solve(f, tol=1e-12, max_cycles=400)
    assert cycles >= 0
    return f, u, oracle.grid_motion(u, f, 100)


def test_circle_faces_slide_along_their_faces(circle_motion):
    _, _, x = circle_motion
    assert np.all(x[0][:, 0] == 0.0) and np.all(x[0][:, -1] == 1.0)
    assert np.all(x[1][0, :] == 0.0) and np.all(x[1][-1, :] == 1.0)
    assert np.all((x >= 0.0) & (x <= 1.0))
    # the face nodes do slide: tangential motion on the faces
    assert np.abs(x[1][:, 0] - oracle.grid_nodes(2, x.shape[1])[1][:, 0]).max() > 1e-3


def test_circle_motion_keeps_the_square_symmetries(circle_motion):
    _, u, x = circle_motion
    # mirror x -> 1 - x and the diagonal swap x <-> y
    assert np.abs(x[0] - (1.0 - x[0][:, ::-1])).max() <= 1e-9
    assert np.abs(x[0] - x[1].T).max() <= 1e-9


def test_circle_motion_gathers_nodes_at_the_circle_without_crossing_it(circle_motion):
    """Inside the ring -grad u points outwards, outside it inwards: nodes crowd into the ring's
    band from both sides and none crosses it; grid rows and columns keep their order."""
    f, _, x = circle_motion
    X, Y = x[0], x[1]
    N = X.shape[0]
    h = 1.0 / (N - 1)
    g0 = oracle.grid_nodes(2, N)
    r0 = np.hypot(g0[0] - 0.5, g0[1] - 0.5)
    r1 = np.hypot(X - 0.5, Y - 0.5)
    before = np.count_nonzero(np.abs(r0 - 0.25) < 0.01)
    after = np.count_nonzero(np.abs(r1 - 0.25) < 0.01)
    assert after > 5 * before
    assert not np.any((r0 < 0.25 - h) & (r1 > 0.25 + h))
    assert not np.any((r0 > 0.25 + h) & (r1 < 0.25 - h))
    assert np.all(np.diff(X, axis=1) > 0) and np.all(np.diff(Y, axis=0) > 0)
    assert np.all(Y[N // 2] == 0.5)  # the symmetry line y = 1/2 is invariant
