"""Seeded synthetic inputs for the SGML solver (host side, NumPy).

This module builds problem data only -- sources, coefficients and boundary types -- and holds none of
the solver's arithmetic.  Tests feed the same arrays to the CUDA library and to the CPU oracle.

Sign convention: every generator returns the source in the paper's form L u = f with
L = div(sigma grad) + a (Sec. 3).  A problem stated as -div(eps grad u) + k^2 u = f therefore comes
back as f_paper = -f and a = -k^2.

Arrays are float64, shape (N, N) indexed [y, x] in 2-D and (N, N, N) indexed [z, y, x] in 3-D, with
N = 2**n + 1 and x_i = i / (N - 1) on the unit square / cube.  Seeds follow 1000 * workload + problem.
"""
from __future__ import annotations

import math
import numpy as np

DIRICHLET = 0
NEUMANN = 1


def _axes(n, dim):
    N = 2 ** n + 1
    x = np.linspace(0.0, 1.0, N)
    if dim == 2:
        Y, X = np.meshgrid(x, x, indexing="ij")
        return (X, Y)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return (X, Y, Z)


def _problem(dim, n, f, sigma=None, a=None, a_scalar=0.0, faces=None, values=None, **extra):
    d = dict(dim=dim, n=n, f=f, sigma=sigma, a=a, a_scalar=float(a_scalar),
             faces=list(faces) if faces is not None else [DIRICHLET] * (2 * dim),
             values=list(values) if values is not None else [0.0] * (2 * dim))
    d.update(extra)
    return d


def poisson_sine_2d(n=7):
    """-Lap u = 2 pi^2 sin(pi x) sin(pi y) on the unit square, u = 0 on the boundary (exact
    u = sin(pi x) sin(pi y)).  129 x 129 nodes at n = 7."""
    X, Y = _axes(n, 2)
    exact = np.sin(np.pi * X) * np.sin(np.pi * Y)
    return _problem(2, n, -2.0 * np.pi ** 2 * exact, exact=exact)


def poisson_polynomial_2d(n=7):
    """Sec. 3.1: Lap u = f with u = -x^2 y^2 (1 - x^2)(1 - y^2) (Eq. 7) and f of Eq. 8, u = 0 on the
    boundary of the unit square."""
    X, Y = _axes(n, 2)
    exact = -X ** 2 * Y ** 2 * (1 - X ** 2) * (1 - Y ** 2)
    f = -2.0 * (Y ** 2 * (1 - 6 * X ** 2) * (1 - Y ** 2) + X ** 2 * (1 - 6 * Y ** 2) * (1 - X ** 2))
    return _problem(2, n, f, exact=exact)


def gaussian_charges(n, rng, count, width_nodes=2.0, lo=0.15, hi=0.85):
    """Sum of `count` normalised 3-D Gaussians of std width_nodes*h with random sign, centres
    uniform in [lo, hi]^3."""
    X, Y, Z = _axes(n, 3)
    h = 1.0 / 2 ** n
    s = width_nodes * h
    f = np.zeros_like(X)
    norm = (2.0 * np.pi * s * s) ** -1.5
    for _ in range(count):
        c = rng.uniform(lo, hi, size=3)
        q = 1.0 if rng.uniform() < 0.5 else -1.0
        f += q * norm * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * s * s))
    return f


def dielectric_spheres_3d(n=8, seed=2000, spheres=32, charges=8, eps_in=80.0):
    """div(eps grad u) = f on the unit cube, u = 0 on the boundary.  eps = 1 with `spheres` random
    balls (centres U[0.12, 0.88]^3, radii U[0.03, 0.12]) where nodes inside get eps_in; f is a sum of
    `charges` unit Gaussian charges of std 2h, random sign, centres U[0.15, 0.85]^3.  257^3 at n = 8."""
    rng = np.random.default_rng(seed)
    X, Y, Z = _axes(n, 3)
    eps = np.ones_like(X)
    for _ in range(spheres):
        c = rng.uniform(0.12, 0.88, size=3)
        r = rng.uniform(0.03, 0.12)
        inside = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2 <= r * r
        eps[inside] = eps_in
    f = gaussian_charges(n, rng, charges)
    return _problem(3, n, f, sigma=eps)


def trefoil_vorticity_3d(n=9, width_nodes=3.0, circulation=1.0, cutoff=6.0):
    """Sec. 3.3 (Eqs. 12-13): vorticity of a thin tube of Gaussian cross-section (std width_nodes*h,
    circulation 1) along the trefoil (sin t + 2 sin 2t, cos t - 2 cos 2t, -sin 3t), scaled by 0.4/3
    and centred in the unit cube.  Returns three problems Lap psi_i = -omega_i, psi = 0 on the
    boundary (513^3 at n = 9)."""
    N = 2 ** n + 1
    h = 1.0 / (N - 1)
    s = width_nodes * h
    scale = 0.4 / 3.0

    def curve(t):
        return scale * np.array([np.sin(t) + 2 * np.sin(2 * t), np.cos(t) - 2 * np.cos(2 * t),
                                 -np.sin(3 * t)]) + 0.5

    def tangent(t):
        return scale * np.array([np.cos(t) + 4 * np.cos(2 * t), -np.sin(t) + 4 * np.sin(2 * t),
                                 -3 * np.cos(3 * t)])

    tt = np.linspace(0, 2 * np.pi, 4097)
    vmax = np.max(np.linalg.norm(tangent(tt), axis=0))
    samples = int(math.ceil(2 * np.pi / (h / (2 * vmax))))
    dt = 2 * np.pi / samples
    omega = np.zeros((3, N, N, N))
    norm = (2.0 * np.pi * s * s) ** -1.5
    rad = int(math.ceil(cutoff * s / h))
    x = np.linspace(0.0, 1.0, N)
    for j in range(samples):
        t = j * dt
        c = curve(t)
        w = circulation * tangent(t) * dt
        i0 = np.clip(np.round(c / h).astype(int) - rad, 0, N - 1)
        i1 = np.clip(np.round(c / h).astype(int) + rad + 1, 0, N)
        xs, ys, zs = x[i0[0]:i1[0]], x[i0[1]:i1[1]], x[i0[2]:i1[2]]
        g = norm * np.exp(-((zs[:, None, None] - c[2]) ** 2 + (ys[None, :, None] - c[1]) ** 2
                            + (xs[None, None, :] - c[0]) ** 2) / (2 * s * s))
        for k in range(3):
            omega[k, i0[2]:i1[2], i0[1]:i1[1], i0[0]:i1[0]] += w[k] * g
    return [_problem(3, n, -omega[k]) for k in range(3)]


def helmholtz_batch_2d(count=256, seed=4000, exponents=(6, 7, 8, 9, 10)):
    """`count` independent problems -Lap u + k^2 u = f on the unit square with side 2^n + 1, n
    uniform in `exponents`; k^2 ~ U[0, 10]; f = sum of 16 modes a sin(pi p x + phi) sin(pi q y + psi)
    with a ~ N(0, 1), p, q in 1..8, phases U[0, 2 pi); each side Dirichlet or Neumann with
    probability 1/2 and homogeneous values.  When all four sides are Neumann and k^2 < 0.1 the -x
    side is made Dirichlet (so that the operator is non-singular)."""
    probs = []
    for b in range(count):
        rng = np.random.default_rng(seed + b)
        n = int(rng.choice(np.asarray(exponents)))
        k2 = float(rng.uniform(0.0, 10.0))
        x = np.linspace(0.0, 1.0, 2 ** n + 1)
        f = np.zeros((x.size, x.size))
        for _ in range(16):
            amp = rng.normal()
            p_, q_ = rng.integers(1, 9, size=2)
            phi, psi = rng.uniform(0, 2 * np.pi, size=2)
            # separable mode, same products in the same order as amp * sin(.. X ..) * sin(.. Y ..)
            f += (amp * np.sin(np.pi * p_ * x + phi))[None, :] * np.sin(np.pi * q_ * x + psi)[:, None]
        faces = [DIRICHLET if rng.uniform() < 0.5 else NEUMANN for _ in range(4)]
        if all(t == NEUMANN for t in faces) and k2 < 0.1:
            faces[0] = DIRICHLET
        probs.append(_problem(2, n, -f, a_scalar=-k2, faces=faces, k2=k2))
    return probs


def smoothed_field(n, rng, width_nodes=4.0):
    """White N(0, 1) noise on the grid, Gaussian-filtered with std width_nodes (in nodes, reflecting
    edges) and rescaled to zero mean and unit standard deviation."""
    from scipy.ndimage import gaussian_filter
    N = 2 ** n + 1
    g = gaussian_filter(rng.standard_normal((N, N, N)), width_nodes, mode="reflect")
    g -= g.mean()
    return g / g.std()


def lognormal_dielectric_batch_3d(count=16, n=7, seed=5000, charges=4, perturb=0.1):
    """`count` problems div(eps grad u) = f on the unit cube, u = 0 on the boundary, with
    ln eps a smoothed unit-variance Gaussian field (std 4h) and f four Gaussian charges (std 2h).
    Each problem also carries eps_target = eps * exp(perturb * g'), g' a second smoothed field: the
    solution with eps_target is the target u_t of J = 1/2 ||u - u_t||^2.  129^3 at n = 7."""
    probs = []
    for b in range(count):
        rng = np.random.default_rng(seed + b)
        eps = np.exp(smoothed_field(n, rng))
        f = gaussian_charges(n, rng, charges)
        eps_t = eps * np.exp(perturb * smoothed_field(n, rng))
        probs.append(_problem(3, n, f, sigma=eps, eps_target=eps_t))
    return probs


def capacitor_3d(n=7, sign=+1.0):
    """Sec. 3.4 (Eqs. 15-16): div(sigma grad u) = 0 on the unit cube with
    sigma = 0.55 +- 0.45 tanh((r - 0.2) / 0.1), r the distance to the centre; u = -1 on the bottom
    (z = 0) and u = 1 on the top (z = 1); zero normal derivative on the lateral faces."""
    X, Y, Z = _axes(n, 3)
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    sigma = 0.55 + sign * 0.45 * np.tanh((r - 0.2) / 0.1)
    faces = [NEUMANN, NEUMANN, NEUMANN, NEUMANN, DIRICHLET, DIRICHLET]
    values = [0.0, 0.0, 0.0, 0.0, -1.0, 1.0]
    return _problem(3, n, np.zeros_like(X), sigma=sigma, faces=faces, values=values)


def circle_source_2d(n=6, radius=0.25, centre=(0.5, 0.5)):
    """Sec. 3.2: a finite delta function along a circle -- the curve resampled at equidistant points
    a mesh spacing apart, each depositing its arc length times a tensor product of hat functions
    (bilinear, support 2h x 2h) of unit integral."""
    N = 2 ** n + 1
    h = 1.0 / (N - 1)
    count = int(math.ceil(2 * np.pi * radius / h))
    ds = 2 * np.pi * radius / count
    f = np.zeros((N, N))
    for j in range(count):
        t = 2 * np.pi * j / count
        px, py = centre[0] + radius * np.cos(t), centre[1] + radius * np.sin(t)
        i0, j0 = int(np.floor(px / h)), int(np.floor(py / h))
        tx, ty = px / h - i0, py / h - j0
        for dj, wy in ((0, 1 - ty), (1, ty)):
            for di, wx in ((0, 1 - tx), (1, tx)):
                f[j0 + dj, i0 + di] += ds * wx * wy / (h * h)
    return f


def neumann_helmholtz_2d(n=6, a=0.1, radius=0.25):
    """Sec. 3.2, Eq. 10: Lap u + a u = f - <f> with zero normal derivative on every side (the
    force potential of the grid deformation), f the circle source of `circle_source_2d`; a = 0.1 as
    in the paper's Fig. 5.  The solver subtracts the mean <f> itself and returns the zero-mean u."""
    f = circle_source_2d(n, radius)
    return _problem(2, n, f, a_scalar=a, faces=[NEUMANN] * 4, values=[0.0] * 4)


def random_problem(dim, n, seed, hetero=True, helmholtz=True, mixed_bc=True, flux=False):
    """Small random problem for parity tests: smooth random source, optional log-normal-ish sigma,
    optional per-node a <= 0, random Dirichlet/Neumann faces (at least one Dirichlet unless a < 0
    everywhere), optional non-zero Dirichlet values and Neumann fluxes."""
    rng = np.random.default_rng(seed)
    N = 2 ** n + 1
    shape = (N,) * dim
    f = rng.standard_normal(shape)
    sigma = np.exp(0.5 * rng.standard_normal(shape)) if hetero else None
    a = -rng.uniform(0.0, 5.0, size=shape) if helmholtz else None
    faces = [DIRICHLET] * (2 * dim)
    if mixed_bc:
        faces = [DIRICHLET if rng.uniform() < 0.5 else NEUMANN for _ in range(2 * dim)]
        if not helmholtz and all(t == NEUMANN for t in faces):
            faces[0] = DIRICHLET
    values = [0.0] * (2 * dim)
    if flux:
        values = [float(rng.uniform(-1, 1)) for _ in range(2 * dim)]
    return _problem(dim, n, f, sigma=sigma, a=a, faces=faces, values=values)
