"""Pins of the FP64 CPU oracle to facts that do not come from the oracle itself.

Each test checks one part of the oracle against something the paper or the mathematics fixes: a
closed form, an exact property, a brute-force computation written independently here, or a number
printed in the paper (tests/golden/).  Together they are chosen so that a dropped term, a wrong sign
or index, or a transposed operand anywhere in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy.fft import dstn, idstn

from oracle import oracle
from oracle.oracle import DIRICHLET, NEUMANN, Problem
from paper_1703_07206_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_facts():
    out = {}
    with open(os.path.join(GOLDEN, "paper_facts.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


def grid(dim, n):
    N = 2 ** n + 1
    x = np.linspace(0.0, 1.0, N)
    if dim == 2:
        Y, X = np.meshgrid(x, x, indexing="ij")
        return X, Y, np.zeros_like(X)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def level_mask(shape, nu):
    s = 2 ** nu
    m = np.ones(shape, dtype=bool)
    for ax in range(len(shape)):
        idx = np.arange(shape[ax]) % s == 0
        sh = [1] * len(shape)
        sh[ax] = shape[ax]
        m &= idx.reshape(sh)
    return m


# --------------------------------------------------------------------------------------------
# Restriction (Algorithm 1, Eqs. 3-4): closed-form tent convolution of the even extension
# --------------------------------------------------------------------------------------------

def tent_restriction(f, nu):
    """Direct (non-recursive) convolution with the separable tent of half-width 2^nu,
    weights (2^nu - |j|) / 4^nu per axis, applied to the even (mirror) extension of f."""
    s = 2 ** nu
    g = np.pad(f, s, mode="reflect")
    w = np.array([(s - abs(j)) / s ** 2 for j in range(-s + 1, s)])
    for ax in range(f.ndim):
        g = np.apply_along_axis(lambda v: np.convolve(v, w, mode="same"), ax, g)
    sl = tuple(slice(s, s + f.shape[ax]) for ax in range(f.ndim))
    return g[sl]


@pytest.mark.parametrize("dim,n", [(2, 5), (3, 3)])
def test_restriction_is_tent_convolution(dim, n):
    rng = np.random.default_rng(1)
    p = Problem(dim, n, faces=[NEUMANN] * (2 * dim), a_scalar=-1.0)
    f = rng.standard_normal(p.shape)
    for nu in range(0, n):
        g = p.restriction(f, nu)
        ref = tent_restriction(f, nu)
        m = level_mask(p.shape, nu)
        assert np.abs(g - ref)[m].max() < 1e-13, nu


def test_restriction_preserves_constants_and_linears():
    p = Problem(2, 5)
    X, Y, _ = grid(2, 5)
    for nu in range(1, 5):
        m = level_mask(p.shape, nu)
        assert np.abs(p.restriction(np.full(p.shape, 3.5), nu) - 3.5)[m].max() < 1e-14
        s = 2 ** nu
        interior = m.copy()
        interior[:s, :] = interior[-s:, :] = interior[:, :s] = interior[:, -s:] = False
        lin = 2.0 * X - 0.5 * Y + 1.0
        assert np.abs(p.restriction(lin, nu) - lin)[interior].max() < 1e-13


# --------------------------------------------------------------------------------------------
# Radial stencil (Eq. 5) with the consistent constant: exactness, eigenvalues, literal ratio
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n", [(2, 4), (3, 3)])
def test_stencil_exact_linear_sigma_quadratic_u(dim, n):
    """div(sigma grad u) for sigma linear and u quadratic is reproduced exactly at every level."""
    X, Y, Z = grid(dim, n)
    sig = 1.0 + 0.3 * X + 0.2 * Y + 0.1 * Z
    if dim == 2:
        u = X ** 2 + Y ** 2 + X * Y
        ex = 4 * sig + 0.3 * (2 * X + Y) + 0.2 * (2 * Y + X)
    else:
        u = X ** 2 + Y ** 2 + Z ** 2 + X * Y + Y * Z
        ex = 6 * sig + 0.3 * (2 * X + Y) + 0.2 * (2 * Y + X + Z) + 0.1 * (2 * Z + Y)
    p = Problem(dim, n, sigma=sig, a_scalar=-0.7)
    m = p.unknown_mask()
    for nu in range(0, n - 1):
        sig_nu = p.restriction(sig, nu)
        a_nu = np.full(p.shape, -0.7)
        Lu = p.apply_op(u, nu=nu, sig=sig if nu == 0 else sig_nu, a=a_nu)
        mm = m & level_mask(p.shape, nu)
        # the restriction of a linear sigma is exact at nodes whose tent support stays inside the
        # domain, so compare where every stencil neighbour is such a node
        s = 2 ** nu
        inner = np.zeros_like(mm)
        inner[(slice(2 * s, -2 * s),) * dim] = True
        ref = ex - 0.7 * u
        if nu == 0:
            assert np.abs(Lu - ref)[mm].max() < 1e-12
        else:
            assert np.abs(Lu - ref)[mm & inner].max() < 1e-11


@pytest.mark.parametrize("dim", [2, 3])
def test_neumann_images_with_flux_exact(dim):
    """On Neumann faces the image u_mirror + 2 k h g reproduces (x + c)^2 exactly when g is its
    outward derivative, so delta L of it is 2 at every unknown, boundary nodes included."""
    n = 4 if dim == 2 else 3
    X, Y, Z = grid(dim, n)
    c = 0.37
    u = (X + c) ** 2
    faces = [NEUMANN, NEUMANN] + [DIRICHLET] * (2 * dim - 2)
    values = [-2 * c, 2 * (1 + c)] + [0.0] * (2 * dim - 2)
    p = Problem(dim, n, faces=faces, values=values)
    Lu = p.apply_op(u, with_flux=True)
    m = p.unknown_mask()
    assert np.abs(Lu - 2.0)[m].max() < 1e-10
    # without the flux term the boundary values are wrong: the images matter
    Lu0 = p.apply_op(u, with_flux=False)
    assert np.abs(Lu0 - 2.0)[m].max() > 1.0


def stencil_eigenvalue(dim, h, ks, kappa):
    """Closed-form symbol of the constant-coefficient radial stencil on the sine mode ks."""
    cs = [math.cos(math.pi * k * h) for k in ks] + [1.0] * (3 - dim)
    lam = 0.0
    for oz in ((-1, 0, 1) if dim == 3 else (0,)):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                o = (ox, oy, oz)
                nz = sum(1 for v in o if v)
                if nz == 0:
                    continue
                w = 1 / math.sqrt(nz)
                prod = 1.0
                for d in range(3):
                    if o[d]:
                        prod *= cs[d]
                lam += w * (prod - 1.0)
    return kappa * lam / h ** 2


def consistent_kappa(dim):
    return math.sqrt(2) - 1 if dim == 2 else 2.0 / (2 + 8 / math.sqrt(2) + 8 / math.sqrt(3))


@pytest.mark.parametrize("dim,n", [(2, 4), (3, 3)])
def test_stencil_sine_modes_are_eigenvectors(dim, n):
    p = Problem(dim, n)
    X, Y, Z = grid(dim, n)
    rng = np.random.default_rng(3)
    for _ in range(4):
        ks = rng.integers(1, p.N - 1, size=dim)
        u = np.sin(np.pi * ks[0] * X) * np.sin(np.pi * ks[1] * Y)
        if dim == 3:
            u = u * np.sin(np.pi * ks[2] * Z)
        lam = stencil_eigenvalue(dim, p.h, ks, consistent_kappa(dim))
        Lu = p.apply_op(u)
        m = p.unknown_mask()
        assert np.abs(Lu - lam * u)[m].max() < 1e-9 * abs(lam)


@pytest.mark.parametrize("dim", [2, 3])
def test_symbol_maximum_matches_stability_bound(dim):
    """The largest |symbol| of the consistent stencil is exactly 4/h^2 (the (pi, 0, ..) mode), so
    the explicit step is stable for delta tau < h^2 / 2 as stated in Sec. 2."""
    facts = golden_facts()
    h = 1.0
    best = 0.0
    for c in [(a, b, d) for a in (-1, 1) for b in (-1, 1) for d in ((-1, 1) if dim == 3 else (1,))]:
        # cos(pi k h) = +-1 corners of the symbol; pass ks with the right cosines
        ks = [0 if v == 1 else 1 for v in c][:dim]
        best = max(best, abs(stencil_eigenvalue(dim, h, ks, consistent_kappa(dim))))
    assert abs(best - 4.0) < 1e-12
    assert abs(2.0 / best - facts["stability_factor"]) < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_literal_constant_is_uniform_scale(dim):
    """The printed 3/(13h) of Eq. 5 (and its 2-D analogue 1/(2h)) scales the consistent stencil by
    one constant factor."""
    facts = golden_facts()
    literal = facts["eq5_literal_constant_3d"] if dim == 3 else 0.5
    n = 3
    X, Y, Z = grid(dim, n)
    u = np.cos(2 * X + Y) + Z
    p_c = Problem(dim, n)
    p_l = Problem(dim, n, stencil=1)
    m = p_c.unknown_mask()
    r = p_l.apply_op(u)[m] / p_c.apply_op(u)[m]
    assert np.allclose(r, literal / consistent_kappa(dim), rtol=1e-12)


def test_golden_distance_factors():
    facts = golden_facts()
    assert facts["eq5_l_edge"] == pytest.approx(math.sqrt(2), rel=1e-15)
    assert facts["eq5_l_corner"] == pytest.approx(math.sqrt(3), rel=1e-15)
    # the face/edge/corner weights 1/l enter delta L: check them through a single-neighbour probe
    p = Problem(3, 2)
    for off, l in (((1, 0, 0), facts["eq5_l_face"]), ((1, 1, 0), facts["eq5_l_edge"]),
                   ((1, 1, 1), facts["eq5_l_corner"])):
        u = np.zeros(p.shape)
        u[2 + off[2], 2 + off[1], 2 + off[0]] = 1.0
        Lu = p.apply_op(u)
        expect = consistent_kappa(3) / p.h ** 2 / l
        assert Lu[2, 2, 2] == pytest.approx(expect, rel=1e-13)


# --------------------------------------------------------------------------------------------
# Pseudo-time step (Sec. 2 bound, Sec. 3.4 local step)
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_local_step_equals_theta_times_bound(dim):
    facts = golden_facts()
    n = 4 if dim == 2 else 3
    theta = 0.7
    p = Problem(dim, n, theta=theta)
    for nu in range(0, n - 1):
        H = 2 ** nu * p.h
        dt = p.local_step(nu)
        m = p.unknown_mask() & level_mask(p.shape, nu)
        assert np.abs(dt[m] - theta * facts["stability_factor"] * H * H).max() < 1e-15
    # node-local option of Sec. 3.4: theta * H^2 / (2 sigma_i)
    rng = np.random.default_rng(5)
    sig = np.exp(rng.standard_normal(p.shape))
    q = Problem(dim, n, sigma=sig, theta=theta, dt_mode=1)
    dt = q.local_step(0)
    m = q.unknown_mask()
    assert np.allclose(dt[m], theta * p.h ** 2 / (2 * sig[m]), rtol=1e-14)


def level_operator_diagonal(p, nu, sig_nu, a_nu):
    """Diagonal of the level-nu operator delta L_nu on the level-nu unknowns, read off the operator
    itself (apply_op, pinned above by exactness and eigenvalue tests): the column of node i is
    delta L_nu applied to the unit vector at i.  Columns of nodes that are three or more level-nu
    cells apart in every coordinate have disjoint supports (the stencil and its even images reach
    one level-nu cell), so one probe vector per colour class (index mod 3 per axis) gives every
    diagonal entry exactly."""
    s = 2 ** nu
    idx = [np.arange(p.N) for _ in range(p.dim)]
    coarse = [np.where(i % s == 0, i // s, -1) for i in idx]
    diag = np.zeros(p.shape)
    m = p.unknown_mask() & level_mask(p.shape, nu)
    for colour in np.ndindex(*([3] * p.dim)):
        e = np.ones(p.shape, dtype=bool)
        for ax in range(p.dim):  # array axis ax holds coordinate dim - 1 - ax
            c = coarse[ax]
            sel = (c >= 0) & (c % 3 == colour[ax])
            sh = [1] * p.dim
            sh[ax] = p.N
            e &= sel.reshape(sh)
        probe = e.astype(float)
        col = p.apply_op(probe, nu=nu, sig=sig_nu, a=a_nu)
        diag[e & m] = col[e & m]
    return diag, m


def brute_force_diagonal(p, nu, sig_nu, a_nu):
    """The same diagonal, one unit column at a time (small grids only)."""
    diag = np.zeros(p.shape)
    m = p.unknown_mask() & level_mask(p.shape, nu)
    for flat in np.flatnonzero(m):
        e = np.zeros(p.shape)
        e.ravel()[flat] = 1.0
        diag.ravel()[flat] = p.apply_op(e, nu=nu, sig=sig_nu, a=a_nu).ravel()[flat]
    return diag


@pytest.mark.parametrize("dim,n,seed", [(2, 5, 41), (2, 4, 42), (3, 3, 43), (3, 4, 44)])
def test_local_step_is_jacobi_scaled_by_assembled_diagonal(dim, n, seed):
    """Sec. 2 stability bound and Sec. 3.4 local step, Jacobi-scaled reading: at every level nu the
    oracle's pseudo-time step is theta (kappa_d S_d / 2) / D_i with D_i = -(delta L_nu)_ii, the
    operator built with the level-nu (tent-restricted) sigma and a.  Heterogeneous sigma, per-node
    a <= 0 and mixed Dirichlet / Neumann faces: a dropped or flipped -a, a wrong sigma average or a
    sigma taken from the wrong level changes D_i and fails here."""
    facts = golden_facts()
    d = inputs.random_problem(dim, n, seed, hetero=True, helmholtz=True, mixed_bc=True)
    faces = list(d["faces"])
    if NEUMANN not in faces:
        faces[1] = NEUMANN
    if DIRICHLET not in faces:
        faces[0] = DIRICHLET
    theta = 0.7
    p = Problem(dim, n, faces=faces, sigma=d["sigma"], a=d["a"], theta=theta)
    w = [1.0 / facts["eq5_l_face"], 1.0 / facts["eq5_l_edge"], 1.0 / facts["eq5_l_corner"]]
    counts = [4, 4, 0] if dim == 2 else [6, 12, 8]  # face, edge, corner neighbours
    S = sum(c * wk for c, wk in zip(counts, w))
    gain = consistent_kappa(dim) * S / 2.0  # sqrt(2) in 2-D
    if dim == 2:
        assert abs(gain - math.sqrt(2)) < 1e-15  # (sqrt 2 - 1)(4 + 2 sqrt 2) / 2 = sqrt 2
    for nu in range(0, n):
        sig_nu = tent_restriction(d["sigma"], nu)
        a_nu = tent_restriction(d["a"], nu)
        diag, m = level_operator_diagonal(p, nu, sig_nu, a_nu)
        if m.sum() <= 64:
            assert np.array_equal(diag[m], brute_force_diagonal(p, nu, sig_nu, a_nu)[m])
        D = -diag[m]
        assert np.all(D > 0)
        dt = p.local_step(nu)
        np.testing.assert_allclose(dt[m], theta * gain / D, rtol=1e-12, atol=0)
        assert np.all(dt[~m] == 0.0)


def test_local_step_pin_fails_on_planted_mistakes():
    """The pin above is sharp: a step built from a flipped -a, from sigma_i alone instead of the
    link average, or from level-0 coefficients at a coarse level departs from the oracle's step by
    far more than its tolerance."""
    d = inputs.random_problem(3, 3, 45, hetero=True, helmholtz=True, mixed_bc=True)
    p = Problem(3, 3, faces=d["faces"], sigma=d["sigma"], a=d["a"])
    gain = consistent_kappa(3) * (6 + 12 / math.sqrt(2) + 8 / math.sqrt(3)) / 2.0
    for nu in (0, 1):
        sig_nu, a_nu = tent_restriction(d["sigma"], nu), tent_restriction(d["a"], nu)
        diag, m = level_operator_diagonal(p, nu, sig_nu, a_nu)
        dt = p.local_step(nu)[m]
        good = 0.7 * gain / -diag[m]
        assert np.abs(dt / good - 1).max() < 1e-12
        plus_a = 0.7 * gain / (-diag[m] + 2 * a_nu[m])   # -a flipped to +a
        assert np.abs(dt / plus_a - 1).max() > 1e-3
        H = 2 ** nu * p.h
        k = consistent_kappa(3)
        sigma_i = 0.7 * gain / (k / H ** 2 * sig_nu[m] * (6 + 12 / math.sqrt(2) + 8 / math.sqrt(3)) - a_nu[m])
        assert np.abs(dt / sigma_i - 1).max() > 1e-3
        if nu == 1:
            diag0, _ = level_operator_diagonal(p, nu, d["sigma"], d["a"])  # level-0 coefficients
            wrong_level = 0.7 * gain / -diag0[m]
            assert np.abs(dt / wrong_level - 1).max() > 1e-3


# --------------------------------------------------------------------------------------------
# Interpolation (Sec. 2, Algorithm 2): multilinear reproduction and nesting
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n", [(2, 5), (3, 3)])
def test_interpolation_reproduces_multilinear(dim, n):
    p = Problem(dim, n)
    X, Y, Z = grid(dim, n)
    ml = 1.0 + 2 * X - 3 * Y + 0.5 * X * Y
    if dim == 3:
        ml = ml + Z - 2 * X * Z + 0.25 * X * Y * Z
    for nu in range(1, n):
        m = level_mask(p.shape, nu)
        delta = np.where(m, ml, 0.0)
        e = np.where(m, 7.0, 0.0)
        out = p.interpolate_add(delta, e, nu)
        assert np.abs(out[~m] - ml[~m]).max() < 1e-13
        assert np.all(out[m] == 7.0)


def test_interpolation_is_nested():
    p = Problem(2, 5)
    rng = np.random.default_rng(9)
    m2, m1 = level_mask(p.shape, 2), level_mask(p.shape, 1)
    d2 = np.where(m2, rng.standard_normal(p.shape), 0.0)
    direct = p.interpolate_add(d2, d2.copy(), 2)
    step1 = p.interpolate_add(d2, d2.copy(), 2)
    step1 = np.where(m1, step1, 0.0)  # values on the level-1 subset only
    twostep = p.interpolate_add(step1, step1.copy(), 1)
    assert np.abs(direct - twostep).max() < 1e-14


# --------------------------------------------------------------------------------------------
# Algorithm 3 schedule
# --------------------------------------------------------------------------------------------

def test_schedule_matches_golden_33x33():
    rows = []
    with open(os.path.join(GOLDEN, "alg3_schedule_33x33.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                a, b = line.split()
                rows.append((int(a), int(b)))
    assert Problem(2, 5, n_r=2).schedule() == rows


# --------------------------------------------------------------------------------------------
# Cycle and outer recurrence
# --------------------------------------------------------------------------------------------

def test_cycle_linear_and_zero():
    d = inputs.random_problem(2, 4, seed=11)
    p = Problem(2, 4, faces=d["faces"], sigma=d["sigma"], a=d["a"])
    rng = np.random.default_rng(12)
    r1, r2 = rng.standard_normal(p.shape), rng.standard_normal(p.shape)
    m = p.unknown_mask()
    r1[~m] = r2[~m] = 0.0
    e1, e2 = p.cycle(r1), p.cycle(r2)
    e12 = p.cycle(2.5 * r1 - 0.75 * r2)
    assert np.abs(e12 - (2.5 * e1 - 0.75 * e2)).max() < 1e-12 * np.abs(e12).max()
    assert np.all(p.cycle(np.zeros(p.shape)) == 0.0)


def assemble(p):
    """Dense matrix of delta L_0 on the unknowns, built column by column from unit vectors, and the
    affine part b = delta L_0(lift) (Dirichlet values and Neumann fluxes)."""
    m = p.unknown_mask().ravel()
    idx = np.flatnonzero(m)
    A = np.zeros((idx.size, idx.size))
    for j, col in enumerate(idx):
        e = np.zeros(p.shape)
        e.ravel()[col] = 1.0
        A[:, j] = p.apply_op(e).ravel()[idx]
    b = p.apply_op(p.lift(), with_flux=True).ravel()[idx]
    return A, b, idx


@pytest.mark.parametrize("dim,n,seed", [(2, 3, 21), (2, 4, 22), (3, 2, 23), (3, 3, 24)])
def test_converged_solution_equals_dense_solve(dim, n, seed):
    d = inputs.random_problem(dim, n, seed, flux=True)
    vals = list(d["values"])
    for k in range(2 * dim):  # non-zero Dirichlet values too
        if d["faces"][k] == DIRICHLET:
            vals[k] = 0.5 * (k + 1)
    p = Problem(dim, n, faces=d["faces"], values=vals, sigma=d["sigma"], a=d["a"])
    A, b, idx = assemble(p)
    u_ref = p.lift().ravel()
    u_ref[idx] = np.linalg.solve(A, d["f"].ravel()[idx] - b)
    u, cycles, hist = p.solve(d["f"], tol=1e-13, max_cycles=300)
    assert cycles > 0
    err = np.linalg.norm(u.ravel() - u_ref) / np.linalg.norm(u_ref)
    assert err < 1e-11


def test_dirichlet_operator_symmetric():
    d = inputs.random_problem(3, 2, seed=31, mixed_bc=False)
    p = Problem(3, 2, sigma=d["sigma"], a=d["a"])
    A, _, _ = assemble(p)
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 4)])
def test_converged_solution_equals_dst_solve(dim, n):
    """Constant coefficients, Dirichlet 0: the discrete solution from the DST-I diagonalisation with
    the closed-form eigenvalues."""
    p = Problem(dim, n, a_scalar=-2.0)
    rng = np.random.default_rng(41)
    f = rng.standard_normal(p.shape)
    inner = (slice(1, -1),) * dim
    N = p.N
    ks = np.arange(1, N - 1)
    kap = consistent_kappa(dim)
    grids = np.meshgrid(*([ks] * dim), indexing="ij")
    lam = np.zeros_like(grids[0], dtype=float)
    for idx in np.ndindex(lam.shape):
        lam[idx] = stencil_eigenvalue(dim, p.h, [ks[i] for i in idx[::-1]], kap) - 2.0
    u_ref = np.zeros(p.shape)
    u_ref[inner] = idstn(dstn(f[inner], type=1) / lam, type=1)
    u, cycles, _ = p.solve(f, tol=1e-13, max_cycles=200)
    assert cycles > 0
    assert np.abs(u - u_ref).max() < 1e-11 * np.abs(u_ref).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_single_unknown_closed_form(dim):
    """N = 3 with Dirichlet faces: one unknown, delta L u = (a - kappa S / h^2) u."""
    p = Problem(dim, 1, a_scalar=-1.5)
    f = np.zeros(p.shape)
    c = (1,) * dim
    f[c] = 3.0
    S = 4 + 4 / math.sqrt(2) if dim == 2 else 6 + 12 / math.sqrt(2) + 8 / math.sqrt(3)
    u, cycles, _ = p.solve(f, tol=1e-14, max_cycles=100)
    assert cycles > 0
    assert u[c] == pytest.approx(3.0 / (-1.5 - consistent_kappa(dim) * S / p.h ** 2), rel=1e-13)


def test_manufactured_sine_second_order():
    errs = []
    for n in (4, 5, 6):
        d = inputs.poisson_sine_2d(n)
        u, c, _ = Problem(2, n).solve(d["f"], tol=1e-12)
        assert c > 0
        errs.append(np.abs(u - d["exact"]).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.8 < r1 < 4.2 and 3.8 < r2 < 4.2


def test_paper_polynomial_l1_error_second_order():
    """Sec. 3.1, Eqs. 7-9: the normalised L1 error of the converged solution falls by ~4 per
    halving of h."""
    errs = []
    for n in (5, 6, 7):
        d = inputs.poisson_polynomial_2d(n)
        u, c, _ = Problem(2, n).solve(d["f"], tol=1e-12)
        assert c > 0
        errs.append(np.abs(u - d["exact"]).sum() / np.abs(d["exact"]).sum())
    assert 3.8 < errs[0] / errs[1] < 4.2 and 3.8 < errs[1] / errs[2] < 4.2


def test_per_cycle_reduction_and_machine_precision():
    """Sec. 3.1: with n_r = 2 each cycle reduces the error by a little less than 10^-2, and the
    recurrence converges to machine precision."""
    facts = golden_facts()
    d = inputs.poisson_polynomial_2d(7)
    p = Problem(2, 7)
    u, c, hist = p.solve(d["f"], tol=1e-13, max_cycles=20)
    assert c > 0 and hist[-1] <= 1e-13
    rates = hist[1:5] / hist[0:4]
    assert np.all(rates < 3 * facts["per_cycle_reduction"])
    assert np.all(rates > facts["per_cycle_reduction"] / 10)


def test_stability_limit_theta_above_one_diverges():
    """Beyond the maximum stable step (theta > 1) the (pi, 0) mode is amplified every sweep and
    the recurrence does not converge."""
    d = inputs.poisson_sine_2d(5)
    rng = np.random.default_rng(2)
    f = d["f"] + rng.standard_normal(d["f"].shape)
    _, c_ok, _ = Problem(2, 5, theta=0.7).solve(f, tol=1e-10, max_cycles=40)
    _, c_bad, hist = Problem(2, 5, theta=1.5).solve(f, tol=1e-10, max_cycles=20)
    assert c_ok > 0 and c_bad == -1 and hist[-1] > 1.0


# --------------------------------------------------------------------------------------------
# Adjoint gradient: central finite differences of J
# --------------------------------------------------------------------------------------------

def test_sigma_and_source_gradient_match_finite_differences():
    dim, n = 3, 2
    rng = np.random.default_rng(51)
    d = inputs.random_problem(dim, n, seed=52, helmholtz=False, mixed_bc=False)
    sig, f = d["sigma"], d["f"]
    u_t = rng.standard_normal(sig.shape)

    def J(s, ff):
        u, c, _ = Problem(dim, n, sigma=s).solve(ff, tol=1e-15, max_cycles=400)
        return 0.5 * np.sum((u - u_t)[Problem(dim, n).unknown_mask()] ** 2), u

    J0, u = J(sig, f)
    p = Problem(dim, n, sigma=sig)
    m = p.unknown_mask()
    g = np.where(m, u - u_t, 0.0)
    lam, c, _ = p.solve(g, tol=1e-15, max_cycles=400)
    gs = p.sigma_gradient(lam, u)
    nodes = [tuple(rng.integers(0, p.N, size=dim)) for _ in range(8)] + [(2, 2, 2), (0, 2, 2)]
    for node in nodes:
        step = 3e-4 * sig[node]
        sp, sm = sig.copy(), sig.copy()
        sp[node] += step
        sm[node] -= step
        fd = (J(sp, f)[0] - J(sm, f)[0]) / (2 * step)
        assert abs(fd - gs[node]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gs).max()), node
    for node in [tuple(rng.integers(1, p.N - 1, size=dim)) for _ in range(4)]:
        step = 1e-4
        fp, fm = f.copy(), f.copy()
        fp[node] += step
        fm[node] -= step
        fd = (J(sig, fp)[0] - J(sig, fm)[0]) / (2 * step)
        assert abs(fd - lam[node]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(lam).max())


def test_sampled_residual_equals_full_residual():
    d = inputs.random_problem(3, 3, seed=61, flux=True)
    p = Problem(3, 3, faces=d["faces"], values=d["values"], sigma=d["sigma"], a=d["a"])
    u = np.random.default_rng(62).standard_normal(p.shape)
    full = p.residual(u, d["f"]).ravel()
    idx = np.random.default_rng(63).choice(full.size, size=50, replace=False)
    assert np.array_equal(p.residual_at(u, d["f"], idx), full[idx])


# --- post-processing of Sec. 3.3: v = curl psi (Eq. 14) and streamlines --------------------------

def _axes3(n):
    N = 2 ** n + 1
    x = np.linspace(0.0, 1.0, N)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def test_curl_exact_on_quadratic_potentials():
    """Second-order differences (central inside, one-sided on faces) are exact on quadratics."""
    X, Y, Z = _axes3(3)
    psi = np.stack([Y ** 2 + 0.3 * X * Z, Z ** 2 - 0.7 * X * Y, X ** 2 + Y * Z])
    v = oracle.curl(psi)
    # curl = (d psi_z/dy - d psi_y/dz, d psi_x/dz - d psi_z/dx, d psi_y/dx - d psi_x/dy)
    want = np.stack([Z - 2 * Z, 0.3 * X - 2 * X, -0.7 * Y - 2 * Y])
    assert np.abs(v - want).max() <= 1e-11


def test_curl_agrees_with_numpy_gradient():
    rng = np.random.default_rng(7)
    N = 17
    psi = rng.standard_normal((3, N, N, N))
    h = 1.0 / (N - 1)
    d = [[np.gradient(psi[c], h, axis=ax, edge_order=2) for ax in range(3)] for c in range(3)]  # axis 0 = z
    want = np.stack([d[2][1] - d[1][0], d[0][0] - d[2][2], d[1][2] - d[0][1]])
    assert np.abs(oracle.curl(psi) - want).max() <= 1e-10 * np.abs(want).max()


def test_curl_is_divergence_free_inside():
    rng = np.random.default_rng(8)
    N = 17
    psi = rng.standard_normal((3, N, N, N))
    v = oracle.curl(psi)
    h = 1.0 / (N - 1)
    div = sum(np.gradient(v[c], h, axis=2 - c) for c in range(3))
    assert np.abs(div[2:-2, 2:-2, 2:-2]).max() <= 1e-9 * np.abs(v).max() / h


def test_streamline_of_constant_field_is_straight():
    N = 9
    c = np.array([0.11, -0.05, 0.07])
    v = np.stack([np.full((N, N, N), c[k]) for k in range(3)])
    seeds = np.array([[0.2, 0.5, 0.3], [0.9, 0.1, 0.95]])
    paths, lengths = oracle.streamlines(v, seeds, dt=0.1, nsteps=40)
    for s in range(2):
        L = lengths[s]
        t = 0.1 * np.arange(L)[:, None]
        assert np.abs(paths[s, :L] - (seeds[s] + t * c)).max() <= 1e-13
        # stopped exactly when the next position would leave the cube
        nxt = seeds[s] + 0.1 * L * c
        assert L == 41 or not np.all((nxt >= 0) & (nxt <= 1))


def test_streamline_of_rigid_rotation_closes():
    """v = (-(y - 1/2), x - 1/2, 0): trilinear interpolation is exact for linear fields, and RK4
    closes one revolution (T = 2 pi) to its fourth-order error."""
    X, Y, Z = _axes3(3)
    v = np.stack([-(Y - 0.5), X - 0.5, 0.0 * Z])
    steps = 1000
    dt = 2 * np.pi / steps
    seed = np.array([[0.8, 0.5, 0.4]])
    paths, lengths = oracle.streamlines(v, seed, dt=dt, nsteps=steps)
    assert lengths[0] == steps + 1
    r = np.hypot(paths[0, :, 0] - 0.5, paths[0, :, 1] - 0.5)
    assert np.abs(r - 0.3).max() <= 1e-10
    assert np.abs(paths[0, -1] - seed[0]).max() <= 1e-9
    assert np.abs(paths[0, :, 2] - 0.4).max() == 0.0


# --- diagnostic pseudo-residual of Sec. 3.1 -----------------------------------------------------

def test_diagnostic_pseudo_residual_on_a_single_level_is_the_residual():
    """With one level the cycle starts its level-0 sweeps from e = 0: the largest pseudo-residual
    |delta L e - r| is max |r| ("for the full mesh, both residuals are the same")."""
    for dim, seed in ((2, 11), (3, 12)):
        d = inputs.random_problem(dim, 1, seed=seed, mixed_bc=False)
        p = Problem(dim, 1, faces=d["faces"], values=d["values"], sigma=d.get("sigma"), a=d.get("a"),
                    a_scalar=d.get("a_scalar", 0.0))
        r = p.residual(p.lift(), d["f"])
        _, diag = p.cycle_diag(r)
        assert diag[0] == pytest.approx(np.abs(r[p.unknown_mask()]).max(), rel=1e-15)


def test_diagnostic_pseudo_residual_is_homogeneous_and_matches_the_cycle():
    d = inputs.random_problem(3, 3, seed=13)
    p = Problem(3, 3, faces=d["faces"], values=d["values"], sigma=d.get("sigma"), a=d.get("a"),
                a_scalar=d.get("a_scalar", 0.0))
    r = p.residual(p.lift(), d["f"])
    e1, d1 = p.cycle_diag(r)
    e2, d2 = p.cycle_diag(-2.5 * r)
    assert np.all(d1 > 0)
    assert np.allclose(d2, 2.5 * d1, rtol=1e-12)
    assert np.array_equal(e1, p.cycle(r))


# --- pure-Neumann problems (Sec. 3.2, Eq. 10) ----------------------------------------------------

def trapezoid_weights(p):
    w = np.ones(p.shape)
    for ax in range(p.dim):
        sl = [slice(None)] * p.dim
        sl[ax] = 0
        w[tuple(sl)] *= 0.5
        sl[ax] = -1
        w[tuple(sl)] *= 0.5
    return w


@pytest.mark.parametrize("dim,n,a,hetero", [(2, 4, 0.1, False), (2, 3, 0.0, True), (3, 2, 0.1, True), (3, 3, 0.0, False)])
def test_pure_neumann_solve_equals_projected_dense_solve(dim, n, a, hetero):
    """L u = f - <f>, zero normal derivative everywhere: the oracle's converged solution equals the
    dense solve (a != 0) or the dense least-squares solve with the zero-mean constraint (a = 0),
    and has zero trapezoid mean."""
    rng = np.random.default_rng(40 + n)
    N = 2 ** n + 1
    shape = (N,) * dim
    f = rng.standard_normal(shape)
    sigma = np.exp(0.4 * rng.standard_normal(shape)) if hetero else None
    p = Problem(dim, n, faces=[NEUMANN] * (2 * dim), values=[0.0] * (2 * dim), sigma=sigma, a_scalar=a)
    assert p.projects_mean()
    A, b, idx = assemble(p)
    assert idx.size == f.size and np.abs(b).max() == 0.0
    w = trapezoid_weights(p).ravel()
    rhs = f.ravel() - np.dot(w, f.ravel()) / w.sum()
    if a != 0.0:
        u_ref = np.linalg.solve(A, rhs)
    else:
        K = np.vstack([A, w[None, :]])
        u_ref = np.linalg.lstsq(K, np.concatenate([rhs, [0.0]]), rcond=None)[0]
    u, cycles, hist = p.solve(f, tol=1e-13, max_cycles=400)
    assert cycles > 0
    assert np.linalg.norm(u.ravel() - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
    assert abs(p.mean(u)) <= 1e-13 * np.abs(u).max()


def test_circle_source_has_the_circle_length_as_integral():
    f = inputs.circle_source_2d(6, radius=0.25)
    h = 1.0 / 64
    assert np.sum(f) * h * h == pytest.approx(2 * np.pi * 0.25, rel=1e-12)
