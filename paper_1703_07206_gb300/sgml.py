"""Python binding of libsgml (ctypes): the C entry points of include/sgml.h under the same names,
plus a small ``Grid`` class.  Argument marshalling only -- every step of the solver runs in the CUDA
library; if the library is missing this module raises instead of falling back to anything else.

Arrays may be NumPy arrays (host memory) or CUDA tensors (``torch.Tensor`` on a GPU); both must be
C-contiguous float64 with N^dim elements per problem, indexed [y, x] (2-D) or [z, y, x] (3-D).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libsgml.so")

FP64 = 0
MIXED = 1
DIRICHLET = 0
NEUMANN = 1
NORM_MAX = 0
NORM_L2 = 1
STENCIL_CONSISTENT = 0
STENCIL_LITERAL = 1

OK = 0
ERR_ARG = -1
ERR_CUDA = -2
ERR_NOT_CONVERGED = -3
ERR_DIVERGED = -4
ERR_BARRIER_TIMEOUT = -5
ERR_NONFINITE = -6

_lib = None

_SIGNATURES = {
    "sgml_create_grid": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_void_p,
                         ctypes.POINTER(ctypes.c_void_p)],
    "sgml_set_params": [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                        ctypes.c_int],
    "sgml_set_coeffs": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double],
    "sgml_set_source": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "sgml_set_bc": [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)],
    "sgml_run_cycle": [ctypes.c_void_p, ctypes.c_int],
    "sgml_solve_to_tol": [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_double)],
    "sgml_residual_norm": [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
    "sgml_get_solution": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p],
    "sgml_get_stats": [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_int)],
    "sgml_get_history": [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                         ctypes.POINTER(ctypes.c_int)],
    "sgml_residual": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
    "sgml_sigma_gradient": [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "sgml_set_fusion": [ctypes.c_void_p, ctypes.c_int],
    "sgml_set_barrier_test": [ctypes.c_void_p, ctypes.c_double, ctypes.c_int],
    "sgml_set_diagnostics": [ctypes.c_void_p, ctypes.c_int],
    "sgml_get_diagnostics": [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                             ctypes.POINTER(ctypes.c_int)],
    "sgml_set_quad": [ctypes.c_void_p, ctypes.c_int],
    "sgml_set_coarse_tail": [ctypes.c_void_p, ctypes.c_int],
    "sgml_get_phases": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "sgml_set_launch": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "sgml_launch_count": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)],
    "sgml_get_launch_info": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_int)],
    "sgml_set_trace": [ctypes.c_void_p, ctypes.c_int],
    "sgml_get_trace": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(ctypes.c_int)],
    "sgml_destroy": [ctypes.c_void_p],
    "sgml_last_error": [],
    "sgml_solve_noalloc": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                           ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_double), ctypes.c_void_p],
    "sgml_noalloc_last_error": [],
    "sgml_curl": [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "sgml_streamlines": [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "sgml_grid_motion": [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                         ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
    "sgml_post_last_error": [],
    "sgml_measure_fma_rates": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
}


def load(path: str | None = None):
    """Load libsgml.so (built by paper_1703_07206_gb300.build).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libsgml.so not found at {path}: build it with paper_1703_07206_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, args in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name.endswith("last_error") else ctypes.c_int
    _lib = lib
    return lib


class SGMLError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sgml error {code}: {msg}")
        self.code = code


def _check(code, allow=()):
    if code != OK and code not in allow:
        raise SGMLError(code, load().sgml_last_error().decode())
    return code


def _addr(x, count=None):
    """Address of a float64 C-contiguous host (NumPy) or device (torch) array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("arrays must be C-contiguous float64")
        if count is not None and x.size < count:
            raise ValueError(f"array has {x.size} elements, {count} needed")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        if count is not None and x.numel() < count:
            raise ValueError(f"tensor has {x.numel()} elements, {count} needed")
        return x.data_ptr()
    raise TypeError("expected a NumPy array or a torch tensor")


class Grid:
    """A batch of problems L u = f on the unit square/cube, solved on the GPU by libsgml."""

    def __init__(self, dim, n_levels, precision=MIXED, stream=None):
        lib = load()
        if isinstance(n_levels, int):
            n_levels = [n_levels]
        self.dim = dim
        self.n_levels = [int(n) for n in n_levels]
        self.batch = len(self.n_levels)
        self.shapes = [((2 ** n + 1),) * dim for n in self.n_levels]
        self.sizes = [int(np.prod(s)) for s in self.shapes]
        arr = (ctypes.c_int * self.batch)(*self.n_levels)
        handle = ctypes.c_void_p()
        sptr = None
        if stream is not None:
            sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(lib.sgml_create_grid(dim, self.batch, arr, precision, sptr, ctypes.byref(handle)))
        self._h = handle
        self.precision = precision
        self.bc = {b: ([DIRICHLET] * (2 * dim), [0.0] * (2 * dim)) for b in range(self.batch)}

    def close(self):
        if getattr(self, "_h", None):
            load().sgml_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _count(self, problem):
        return sum(self.sizes) if problem < 0 else self.sizes[problem]

    def set_params(self, n_r=2, theta=0.7, schedule=0, stencil=STENCIL_CONSISTENT, dt_mode=0, max_cycles=200):
        _check(load().sgml_set_params(self._h, n_r, float(theta), schedule, stencil, dt_mode, max_cycles))

    def set_coeffs(self, problem, sigma=None, a=None, a_scalar=0.0):
        c = self._count(problem)
        _check(load().sgml_set_coeffs(self._h, problem, _addr(sigma, c), _addr(a, c), float(a_scalar)))

    def set_source(self, problem, f):
        _check(load().sgml_set_source(self._h, problem, _addr(f, self._count(problem))))

    def set_bc(self, problem, faces, values=None):
        ft = (ctypes.c_int * 6)(*(list(faces) + [0] * (6 - len(faces))))
        fv = None
        if values is not None:
            fv = (ctypes.c_double * 6)(*([float(v) for v in values] + [0.0] * (6 - len(values))))
        _check(load().sgml_set_bc(self._h, problem, ft, fv))
        vals = list(values) if values is not None else [0.0] * len(faces)
        for b in (range(self.batch) if problem < 0 else [problem]):
            self.bc[b] = (list(faces), vals)

    def run_cycle(self, ncycles=1):
        _check(load().sgml_run_cycle(self._h, ncycles))

    def solve_to_tol(self, rtol, raise_on_failure=False):
        """Returns (status, cycles per problem, relative residual per problem)."""
        cyc = (ctypes.c_int * self.batch)()
        rel = (ctypes.c_double * self.batch)()
        st = load().sgml_solve_to_tol(self._h, float(rtol), cyc, rel)
        if raise_on_failure or st in (ERR_ARG, ERR_CUDA, ERR_BARRIER_TIMEOUT):
            _check(st)
        return st, np.array(cyc[:]), np.array(rel[:])

    def residual_norm(self, norm=NORM_MAX):
        out = (ctypes.c_double * self.batch)()
        _check(load().sgml_residual_norm(self._h, norm, out))
        return np.array(out[:])

    def get_solution(self, problem=0, out=None):
        if out is None:
            out = np.empty(self.shapes[problem])
        _check(load().sgml_get_solution(self._h, problem, _addr(out, self.sizes[problem])))
        return out

    def get_stats(self, problem=0):
        c, r, s = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        _check(load().sgml_get_stats(self._h, problem, ctypes.byref(c), ctypes.byref(r), ctypes.byref(s)))
        return c.value, r.value, s.value

    def get_history(self, problem=0, cap=1024):
        buf = (ctypes.c_double * cap)()
        n = ctypes.c_int()
        _check(load().sgml_get_history(self._h, problem, buf, cap, ctypes.byref(n)))
        return np.array(buf[: n.value])

    def residual(self, problem, u, out=None):
        if out is None:
            out = np.empty(self.shapes[problem])
        _check(load().sgml_residual(self._h, problem, _addr(u, self.sizes[problem]), _addr(out, self.sizes[problem])))
        return out

    def sigma_gradient(self, problem, lam, u, out=None):
        if out is None:
            out = np.empty(self.shapes[problem])
        m = self.sizes[problem]
        _check(load().sgml_sigma_gradient(self._h, problem, _addr(lam, m), _addr(u, m), _addr(out, m)))
        return out

    def set_barrier_test(self, wait_limit_s=2.0, withhold_barrier=0):
        """Limit of every grid-barrier wait in seconds; withhold_barrier >= 1 makes CTA 0 withhold its
        arrival at that barrier of every launch (a test aid for the timeout status; 0: off)."""
        _check(load().sgml_set_barrier_test(self._h, float(wait_limit_s), int(withhold_barrier)))

    def set_fusion(self, pair_levels=0):
        """Levels 0 .. pair_levels - 1 run their sweeps in fused pairs (3-D mixed form; 0: off)."""
        _check(load().sgml_set_fusion(self._h, pair_levels))

    def set_diagnostics(self, cycles):
        """Record the per-level diagnostic pseudo-residual of the first `cycles` cycles of each launch
        (0: off)."""
        _check(load().sgml_set_diagnostics(self._h, int(cycles)))
        self.diag_cycles = int(cycles)

    def get_diagnostics(self, b):
        """(cycles, 13) array: largest |delta L_l e - r_l| of level l's sweeps in each recorded cycle."""
        cap = 13 * max(getattr(self, "diag_cycles", 0), 1)
        buf = (ctypes.c_double * cap)()
        n = ctypes.c_int()
        _check(load().sgml_get_diagnostics(self._h, b, buf, cap, ctypes.byref(n)))
        return np.array(buf[: 13 * n.value]).reshape(n.value, 13)

    def set_quad(self, quad_levels=1):
        """Levels 0 .. quad_levels - 1 sweep with four rows per thread (3-D mixed form; 0: off)."""
        _check(load().sgml_set_quad(self._h, quad_levels))

    def set_coarse_tail(self, on=True):
        """Run the three coarsest levels' phases in one CTA's shared memory (3-D mixed form, one problem)."""
        _check(load().sgml_set_coarse_tail(self._h, 1 if on else 0))

    def get_phases(self):
        """The cycle's phase table: list of (op, level, first sweep, sweeps performed)."""
        lib = load()
        cnt = ctypes.c_int(0)
        _check(lib.sgml_get_phases(self._h, None, 0, ctypes.byref(cnt)))
        buf = (ctypes.c_int * (4 * max(cnt.value, 1)))()
        _check(lib.sgml_get_phases(self._h, buf, cnt.value, ctypes.byref(cnt)))
        return [tuple(buf[4 * q:4 * q + 4]) for q in range(cnt.value)]

    def set_launch(self, ctas_per_sm=0, z_waves=1, mode=0, tile_x=64, slab_z=None):
        """mode 0: one persistent cooperative launch per call; mode 1: one launch per phase;
        tile_x 32 (32 x 16 column tiles) or 64 (64 x 8); slab_z: z-slab height of the slab cut of
        large 3-D levels (0: contiguous runs; None: 32 for the mixed form, 0 for FP64)."""
        if slab_z is None:
            slab_z = 32 if self.precision == MIXED else 0
        _check(load().sgml_set_launch(self._h, ctas_per_sm, z_waves, mode, tile_x, slab_z))

    def set_trace(self, cycles):
        _check(load().sgml_set_trace(self._h, cycles))

    def get_trace(self, cap=1 << 16):
        """(cycles x slots) microseconds of the traced cycles of the last launch (see sgml.h)."""
        buf = (ctypes.c_double * cap)()
        npx, ncy = ctypes.c_int(), ctypes.c_int()
        _check(load().sgml_get_trace(self._h, buf, cap, ctypes.byref(npx), ctypes.byref(ncy)))
        return np.array(buf[: npx.value * ncy.value]).reshape(ncy.value, npx.value)

    def launch_info(self):
        """(CTAs, threads per CTA, dynamic shared memory bytes per CTA) of the cycle kernel."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(load().sgml_get_launch_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def launch_count(self):
        c = ctypes.c_longlong()
        _check(load().sgml_launch_count(self._h, ctypes.byref(c)))
        return c.value


def solve_noalloc(dim, n, f, u, sigma=None, a_scalar=0.0, faces=None, values=None, rtol=1e-10, max_cycles=200,
                  precision=MIXED, stream=None):
    """sgml_solve_noalloc: one solve that allocates no device memory, for callers that cannot
    allocate where they solve.  f, sigma (or None) and u are float64 CUDA tensors on the current
    device.  Returns (status, cycles, relative residual); raises on argument / CUDA errors."""
    import torch
    dev = torch.cuda.current_device()
    for name, t in (("f", f), ("u", u), ("sigma", sigma)):
        if t is None and name == "sigma":
            continue
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device.index == dev):
            raise TypeError(f"{name} must be a CUDA tensor on the current device (cuda:{dev})")
    lib = load()
    faces = list(faces) if faces is not None else [DIRICHLET] * (2 * dim)
    ft = (ctypes.c_int * 6)(*(faces + [0] * (6 - len(faces))))
    fv = None
    if values is not None:
        fv = (ctypes.c_double * 6)(*([float(v) for v in values] + [0.0] * (6 - len(values))))
    m = (2 ** n + 1) ** dim
    cyc, rel = ctypes.c_int(), ctypes.c_double()
    sptr = None
    if stream is not None:
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    st = lib.sgml_solve_noalloc(dim, n, precision, _addr(f, m), _addr(sigma, m), float(a_scalar), ft, fv,
                                float(rtol), int(max_cycles), _addr(u, m), ctypes.byref(cyc), ctypes.byref(rel), sptr)
    if st in (ERR_ARG, ERR_CUDA, ERR_BARRIER_TIMEOUT):
        raise SGMLError(st, lib.sgml_noalloc_last_error().decode())
    return st, cyc.value, rel.value


def _stream_ptr(stream):
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def curl(psi, stream=None):
    """v = curl psi (Sec. 3.3, Eq. 14) of a CUDA float64 tensor psi of shape (3, N, N, N) (components
    x, y, z; each [z, y, x]); returns a new CUDA tensor of the same shape (asynchronous on stream)."""
    import torch
    if not (hasattr(psi, "is_cuda") and psi.is_cuda) or psi.dtype != torch.float64:
        raise TypeError("psi must be a CUDA float64 tensor")
    psi = psi.contiguous()
    if psi.dim() != 4 or psi.shape[0] != 3 or not (psi.shape[1] == psi.shape[2] == psi.shape[3]):
        raise ValueError("psi must have shape (3, N, N, N)")
    N = psi.shape[1]
    n = int(round(np.log2(N - 1)))
    if 2 ** n + 1 != N:
        raise ValueError("N must be 2^n + 1")
    v = torch.empty_like(psi)
    lib = load()
    st = lib.sgml_curl(n, psi.data_ptr(), v.data_ptr(), _stream_ptr(stream))
    if st != OK:
        raise SGMLError(st, lib.sgml_post_last_error().decode())
    return v


def streamlines(v, seeds, dt, nsteps, stream=None):
    """RK4 streamlines (Sec. 3.3) of the CUDA float64 node field v (3, N, N, N) from seeds (S, 3)
    (x, y, z); returns CUDA tensors (paths (S, nsteps + 1, 3), lengths (S,) int32)."""
    import torch
    if not (hasattr(v, "is_cuda") and v.is_cuda) or v.dtype != torch.float64:
        raise TypeError("v must be a CUDA float64 tensor")
    v = v.contiguous()
    N = v.shape[1]
    n = int(round(np.log2(N - 1)))
    seeds = torch.as_tensor(seeds, dtype=torch.float64, device=v.device).reshape(-1, 3).contiguous()
    S = seeds.shape[0]
    paths = torch.full((S, nsteps + 1, 3), float("nan"), dtype=torch.float64, device=v.device)
    lengths = torch.zeros(S, dtype=torch.int32, device=v.device)
    lib = load()
    st = lib.sgml_streamlines(n, v.data_ptr(), seeds.data_ptr(), S, float(dt), int(nsteps), paths.data_ptr(),
                              lengths.data_ptr(), _stream_ptr(stream))
    if st != OK:
        raise SGMLError(st, lib.sgml_post_last_error().decode())
    return paths, lengths


def grid_motion(u, f, nsteps, t0=0.0, t1=1.0, x=None, stream=None):
    """Grid motion of Sec. 3.2 (Eq. 11): nsteps forward-Euler steps of dx/dt = -grad u / (t f + int f)
    from pseudo-time t0 to t1.  u, f: CUDA float64 tensors of shape (N, N) or (N, N, N) (the force
    potential and its source); x: start positions (dim,) + u.shape, default the grid's nodes
    (component a = coordinate x_a).  Returns the moved positions (a new CUDA tensor)."""
    import torch
    for name, t in (("u", u), ("f", f)):
        if not (hasattr(t, "is_cuda") and t.is_cuda) or t.dtype != torch.float64:
            raise TypeError(f"{name} must be a CUDA float64 tensor")
    u, f = u.contiguous(), f.contiguous()
    dim = u.dim()
    N = u.shape[0]
    n = int(round(np.log2(N - 1))) if N > 2 else 0
    if dim not in (2, 3) or any(s != N for s in u.shape) or n < 1 or 2 ** n + 1 != N:
        raise ValueError("u must have shape (N, N) or (N, N, N) with N = 2^n + 1")
    if tuple(f.shape) != tuple(u.shape):
        raise ValueError("f and u must have the same shape")
    if x is None:
        g = torch.linspace(0.0, 1.0, N, dtype=torch.float64, device=u.device)
        mesh = torch.meshgrid(*([g] * dim), indexing="ij")
        x = torch.stack([mesh[dim - 1 - a] for a in range(dim)]).contiguous()
    else:
        x = torch.as_tensor(x, dtype=torch.float64, device=u.device).clone().contiguous()
        if tuple(x.shape) != (dim,) + tuple(u.shape):
            raise ValueError("x must have shape (dim,) + u.shape")
    lib = load()
    st = lib.sgml_grid_motion(dim, n, u.data_ptr(), f.data_ptr(), float(t0), float(t1), int(nsteps), x.data_ptr(),
                              _stream_ptr(stream))
    if st != OK:
        raise SGMLError(st, lib.sgml_post_last_error().decode())
    return x


def measure_fma_rates(stream=None):
    """Measured (FP64, FP32) FMA instructions per second of the current GPU (thread level)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    st = load().sgml_measure_fma_rates(_stream_ptr(stream), ctypes.byref(a), ctypes.byref(b))
    if st != OK:
        raise SGMLError(st, "sgml_measure_fma_rates failed")
    return a.value, b.value


def problem_into_grid(grid, b, prob):
    """Copy one problem dictionary (paper_1703_07206_gb300.inputs format) into problem slot b."""
    grid.set_bc(b, prob["faces"], prob["values"])
    grid.set_coeffs(b, prob.get("sigma"), prob.get("a"), prob.get("a_scalar", 0.0))
    grid.set_source(b, np.ascontiguousarray(prob["f"], dtype=np.float64))
