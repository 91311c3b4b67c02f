"""FP64 CPU oracle of the SGML method (arXiv 1703.07206), Python side.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline leg of the benchmark
load this module.  The CUDA library never calls it and shares no code with it.

The arithmetic is in ``sgml_oracle.c`` (plain C, FP64, no fast-math).  This module compiles it with
gcc on first use (or via :func:`build`), declares the ctypes signatures and converts NumPy arrays.
Every field is a full single-grid array of shape ``(N, N)`` (2-D, indexed ``[y, x]``) or
``(N, N, N)`` (3-D, ``[z, y, x]``) with ``N = 2**n + 1``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgml_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

DIRICHLET = 0
NEUMANN = 1


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int),
        ("face_type", ctypes.c_int * 6),
        ("face_value", ctypes.c_double * 6),
        ("sigma", ctypes.POINTER(ctypes.c_double)),
        ("a", ctypes.POINTER(ctypes.c_double)),
        ("a_scalar", ctypes.c_double),
        ("n_r", ctypes.c_int),
        ("theta", ctypes.c_double),
        ("stencil", ctypes.c_int),
        ("dt_mode", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (plain -O2, no fast-math, no FMA
    contraction), with OpenMP for its per-node loops when the compiler offers it (results do not
    depend on the thread count), else serial."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.check_call(base + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def default_threads() -> int:
    """Host threads the oracle uses unless told otherwise: ORACLE_THREADS, else every core in this
    process's affinity mask."""
    env = os.environ.get("ORACLE_THREADS")
    if env:
        return max(1, int(env))
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def set_threads(n: int) -> int:
    """Use n host threads in the oracle's per-node loops (1 if it was built without OpenMP);
    returns the count now in effect."""
    return int(_load().orc_set_threads(int(n)))


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.c_int
        lib.orc_apply_op.argtypes = [P, I, D, D, D, I, D]
        lib.orc_restriction.argtypes = [P, I, D, D]
        lib.orc_local_step.argtypes = [P, I, D, D, D]
        lib.orc_interpolate_add.argtypes = [P, I, D, D]
        lib.orc_visit.argtypes = [P, I, I, D, D, D, D, D]
        lib.orc_cycle_diag.argtypes = [P, D, D, D]
        lib.orc_projects_mean.argtypes = [P]
        lib.orc_projects_mean.restype = I
        lib.orc_mean.argtypes = [P, D]
        lib.orc_mean.restype = ctypes.c_double
        lib.orc_cycle.argtypes = [P, D, D]
        lib.orc_schedule.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I), I]
        lib.orc_schedule.restype = I
        lib.orc_lift.argtypes = [P, D]
        lib.orc_residual.argtypes = [P, D, D, D]
        lib.orc_residual_at.argtypes = [P, D, D, ctypes.POINTER(ctypes.c_long), ctypes.c_long, D]
        lib.orc_max_norm.argtypes = [P, D]
        lib.orc_max_norm.restype = ctypes.c_double
        lib.orc_solve.argtypes = [P, D, ctypes.c_double, I, D, D]
        lib.orc_solve.restype = I
        lib.orc_sigma_gradient.argtypes = [P, D, D, D]
        lib.orc_curl.argtypes = [I, D, D]
        lib.orc_streamlines.argtypes = [I, D, D, I, ctypes.c_double, I, D, ctypes.POINTER(I)]
        lib.orc_trapezoid.argtypes = [I, I, D]
        lib.orc_trapezoid.restype = ctypes.c_double
        lib.orc_neumann_gradient.argtypes = [I, I, D, D]
        lib.orc_grid_motion.argtypes = [I, I, D, D, ctypes.c_double, ctypes.c_double, I, D]
        lib.orc_set_threads.argtypes = [I]
        lib.orc_set_threads.restype = I
        lib.orc_set_threads(default_threads())
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f64(a, shape):
    if a is None:
        return None
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if out.shape != shape:
        raise ValueError(f"expected shape {shape}, got {out.shape}")
    return out


class Problem:
    """One boundary value problem L u = f with L = div(sigma grad) + a on the unit square/cube.

    ``faces``: 2*dim face types in the order -x,+x,-y,+y(,-z,+z) (DIRICHLET or NEUMANN);
    ``values``: per face Dirichlet value or outward normal derivative.
    """

    def __init__(self, dim, n, faces=None, values=None, sigma=None, a=None, a_scalar=0.0,
                 n_r=2, theta=0.7, stencil=0, dt_mode=0):
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.dim, self.n = dim, n
        self.N = 2 ** n + 1
        self.shape = (self.N,) * dim
        faces = list(faces) if faces is not None else [DIRICHLET] * (2 * dim)
        values = list(values) if values is not None else [0.0] * (2 * dim)
        self.faces = faces + [DIRICHLET] * (6 - len(faces))
        self.values = [float(v) for v in values] + [0.0] * (6 - len(values))
        self.sigma = _f64(sigma, self.shape)
        self.a = _f64(a, self.shape)
        self.a_scalar = float(a_scalar)
        self.n_r, self.theta, self.stencil, self.dt_mode = n_r, float(theta), stencil, dt_mode
        self._c = _Problem()
        self._c.dim, self._c.n = dim, n
        for k in range(6):
            self._c.face_type[k] = self.faces[k]
            self._c.face_value[k] = self.values[k]
        self._c.sigma = _ptr(self.sigma)
        self._c.a = _ptr(self.a)
        self._c.a_scalar = self.a_scalar
        self._c.n_r, self._c.theta = n_r, self.theta
        self._c.stencil, self._c.dt_mode = stencil, dt_mode

    @property
    def h(self):
        return 1.0 / (self.N - 1)

    def _arr(self, a):
        return _f64(a, self.shape)

    def _new(self):
        return np.zeros(self.shape)

    # --- operators ------------------------------------------------------------------------
    def apply_op(self, u, nu=0, sig=None, a=None, with_flux=False):
        """delta L_nu u at level-nu unknowns (Eq. 5 + a u), zero elsewhere."""
        lib = _load()
        u = self._arr(u)
        sig = self._arr(sig) if sig is not None else self.sigma if nu == 0 else None
        a = self._arr(a) if a is not None else self.a if nu == 0 else None
        out = self._new()
        lib.orc_apply_op(ctypes.byref(self._c), nu, _ptr(sig), _ptr(a), _ptr(u), int(with_flux), _ptr(out))
        return out

    def restriction(self, f, nu):
        """restriction(nu) of Algorithm 1; valid at level-nu nodes."""
        lib = _load()
        f = self._arr(f)
        g = self._new()
        lib.orc_restriction(ctypes.byref(self._c), nu, _ptr(f), _ptr(g))
        return g

    def restricted_coeffs(self, nu):
        sig = self.restriction(self.sigma, nu) if self.sigma is not None else None
        a = self.restriction(self.a, nu) if self.a is not None else None
        return sig, a

    def local_step(self, nu):
        lib = _load()
        sig, a = self.restricted_coeffs(nu)
        out = self._new()
        lib.orc_local_step(ctypes.byref(self._c), nu, _ptr(sig), _ptr(a), _ptr(out))
        return out

    def interpolate_add(self, delta, e, nu):
        """e + I_nu(delta) on the nodes outside the level-nu subset."""
        lib = _load()
        delta = self._arr(delta)
        e = self._arr(e).copy()
        lib.orc_interpolate_add(ctypes.byref(self._c), nu, _ptr(delta), _ptr(e))
        return e

    def visit(self, e, r, nu, k):
        lib = _load()
        e = self._arr(e).copy()
        r_nu = self.restriction(r, nu)
        sig, a = self.restricted_coeffs(nu)
        lib.orc_visit(ctypes.byref(self._c), nu, k, _ptr(r_nu), _ptr(sig), _ptr(a), _ptr(e), None)
        return e

    def cycle(self, r):
        lib = _load()
        r = self._arr(r)
        e = self._new()
        lib.orc_cycle(ctypes.byref(self._c), _ptr(r), _ptr(e))
        return e

    def cycle_diag(self, r):
        """The cycle and its diagnostic pseudo-residuals: (e, d) with d[nu] the largest
        |delta L_nu e - r_nu| met by the level-nu sweeps of the cycle (Sec. 3.1)."""
        lib = _load()
        r = self._arr(r)
        e = self._new()
        d = np.zeros(self.n)
        lib.orc_cycle_diag(ctypes.byref(self._c), _ptr(r), _ptr(e), _ptr(d))
        return e, d

    def schedule(self):
        lib = _load()
        cap = 4 * self.n + 8
        lv = (ctypes.c_int * cap)()
        sw = (ctypes.c_int * cap)()
        m = lib.orc_schedule(ctypes.byref(self._c), lv, sw, cap)
        return [(lv[i], sw[i]) for i in range(m)]

    def lift(self):
        lib = _load()
        u = self._new()
        lib.orc_lift(ctypes.byref(self._c), _ptr(u))
        return u

    def residual(self, u, f):
        lib = _load()
        u, f = self._arr(u), self._arr(f)
        r = self._new()
        lib.orc_residual(ctypes.byref(self._c), _ptr(u), _ptr(f), _ptr(r))
        return r

    def residual_at(self, u, f, flat_idx):
        """f - delta L u at the given flat node indices (0 at fixed nodes)."""
        lib = _load()
        u, f = self._arr(u), self._arr(f)
        idx = np.ascontiguousarray(np.asarray(flat_idx, dtype=np.int64))
        out = np.zeros(idx.size)
        lib.orc_residual_at(ctypes.byref(self._c), _ptr(u), _ptr(f), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                            idx.size, _ptr(out))
        return out

    def max_norm(self, v):
        return _load().orc_max_norm(ctypes.byref(self._c), _ptr(self._arr(v)))

    def rel_residual(self, u, f):
        """||f - delta L u||_inf / ||f||_inf over unknowns (Sec. 3.1)."""
        fn = self.max_norm(f)
        rn = self.max_norm(self.residual(u, f))
        if fn == 0.0:
            fn = self.max_norm(self.residual(self.lift(), f))
        return rn / fn if fn > 0 else 0.0

    def projects_mean(self):
        """All faces Neumann and a >= 0 constant: the solve works on L u = f - <f> (Eq. 10) for the
        zero-mean u."""
        return bool(_load().orc_projects_mean(ctypes.byref(self._c)))

    def mean(self, v):
        """Trapezoid-rule mean over the unit square / cube."""
        return _load().orc_mean(ctypes.byref(self._c), _ptr(self._arr(v)))

    def solve(self, f, tol=1e-12, max_cycles=200):
        """Outer recurrence; returns (u, cycles or -1, history of relative residuals)."""
        lib = _load()
        f = self._arr(f)
        u = self._new()
        hist = np.zeros(max_cycles + 1)
        c = lib.orc_solve(ctypes.byref(self._c), _ptr(f), float(tol), int(max_cycles), _ptr(u), _ptr(hist))
        nh = (c if c >= 0 else max_cycles) + 1
        return u, c, hist[:nh]

    def sigma_gradient(self, lam, u):
        lib = _load()
        g = self._new()
        lib.orc_sigma_gradient(ctypes.byref(self._c), _ptr(self._arr(lam)), _ptr(self._arr(u)), _ptr(g))
        return g

    def unknown_mask(self):
        """Boolean mask of unknowns (nodes not on a Dirichlet face)."""
        m = np.ones(self.shape, dtype=bool)
        for k in range(self.dim):
            ax = self.dim - 1 - k  # x is the last array axis
            lo = [slice(None)] * self.dim
            hi = [slice(None)] * self.dim
            lo[ax], hi[ax] = 0, self.N - 1
            if self.faces[2 * k] == DIRICHLET:
                m[tuple(lo)] = False
            if self.faces[2 * k + 1] == DIRICHLET:
                m[tuple(hi)] = False
        return m


# --- post-processing of Sec. 3.3 (velocity from the stream vector potential, streamlines) ------
def curl(psi):
    """v = curl psi (Eq. 14) on the unit cube: psi of shape (3, N, N, N) (components x, y, z; each
    indexed [z, y, x]); second-order central differences inside, one-sided on the faces."""
    psi = np.ascontiguousarray(np.asarray(psi, dtype=np.float64))
    if psi.ndim != 4 or psi.shape[0] != 3 or psi.shape[1] != psi.shape[2] or psi.shape[2] != psi.shape[3]:
        raise ValueError("psi must have shape (3, N, N, N)")
    N = psi.shape[1]
    n = int(round(np.log2(N - 1)))
    if 2 ** n + 1 != N:
        raise ValueError("N must be 2^n + 1")
    v = np.empty_like(psi)
    _load().orc_curl(n, _ptr(psi), _ptr(v))
    return v


def streamlines(v, seeds, dt, nsteps):
    """RK4 streamlines of the node field v (3, N, N, N), trilinear between nodes, from seeds (S, 3)
    (x, y, z); returns (paths (S, nsteps + 1, 3), lengths (S,)): positions until the path leaves
    the unit cube or nsteps steps are done."""
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    N = v.shape[1]
    n = int(round(np.log2(N - 1)))
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.float64).reshape(-1, 3))
    S = seeds.shape[0]
    paths = np.full((S, nsteps + 1, 3), np.nan)
    lengths = (ctypes.c_int * S)()
    _load().orc_streamlines(n, _ptr(v), _ptr(seeds), S, float(dt), int(nsteps), _ptr(paths), lengths)
    return paths, np.array(lengths[:], dtype=np.int64)


# --- grid motion of Sec. 3.2 (Eq. 11) ------------------------------------------------------------
def _square_field(v, name):
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    dim = v.ndim
    N = v.shape[0]
    n = int(round(np.log2(N - 1))) if N > 2 else 0
    if dim not in (2, 3) or any(s != N for s in v.shape) or n < 1 or 2 ** n + 1 != N:
        raise ValueError(f"{name} must be an N^2 or N^3 array with N = 2^n + 1")
    return v, dim, n


def grid_nodes(dim, N):
    """Node positions of the unit grid: array (dim, N, ..., N), component a = coordinate x_a."""
    x = np.linspace(0.0, 1.0, N)
    mesh = np.meshgrid(*([x] * dim), indexing="ij")  # mesh[k] varies along array axis k
    return np.stack([mesh[dim - 1 - a] for a in range(dim)])


def trapezoid(f):
    """Trapezoid-rule integral of the node field f over the unit square / cube."""
    f, dim, n = _square_field(f, "f")
    return _load().orc_trapezoid(dim, n, _ptr(f))


def neumann_gradient(u):
    """grad u at the nodes (dim, N, ...), central differences with the Neumann images."""
    u, dim, n = _square_field(u, "u")
    g = np.empty((dim,) + u.shape)
    _load().orc_neumann_gradient(dim, n, _ptr(u), _ptr(g))
    return g


def grid_motion(u, f, nsteps, t0=0.0, t1=1.0, x=None):
    """Node positions after nsteps forward-Euler steps of dx/dt = -grad u / (t f + int f) (Eq. 11)
    from pseudo-time t0 to t1, starting from x (default: the grid nodes); array (dim, N, ..., N)."""
    u, dim, n = _square_field(u, "u")
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    if f.shape != u.shape:
        raise ValueError("f and u must have the same shape")
    x = grid_nodes(dim, u.shape[0]) if x is None else np.array(x, dtype=np.float64, copy=True)
    x = np.ascontiguousarray(x)
    if x.shape != (dim,) + u.shape:
        raise ValueError("x must have shape (dim,) + u.shape")
    _load().orc_grid_motion(dim, n, _ptr(u), _ptr(f), float(t0), float(t1), int(nsteps), _ptr(x))
    return x
