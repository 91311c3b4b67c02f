"""sgml_solve_noalloc, the entry point for callers that cannot allocate device memory where they
solve (a memory pool that owns the device and forbids foreign allocations, a device-memory budget
fixed at start-up, a control loop that cannot take cudaMalloc's synchronisation): its scratch is a
fixed device array inside the library.  It must give the same solution as the ordinary grid API,
call after call (the shared scratch keeps the previous call's contents).

Collected last on purpose, so that a run stopping at the first failure has run everything else."""
import numpy as np
import pytest

from paper_1703_07206_gb300 import inputs, sgml
from tests.gpu_helpers import gpu_grid, rel_l2

pytestmark = pytest.mark.gpu

CASES = [
    ("rand3d_n4", lambda: inputs.random_problem(3, 4, seed=501, helmholtz=False, flux=True)),
    ("poisson2d_n6", lambda: inputs.poisson_sine_2d(6)),
    ("rand2d_n7_const", lambda: inputs.random_problem(2, 7, seed=502, hetero=False, helmholtz=False)),
]


@pytest.mark.parametrize("precision", [sgml.FP64, sgml.MIXED])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_noalloc_solve_matches_grid_api_twice(precision, name, make):
    import torch
    d = make()
    d["a_scalar"] = -0.5
    g = gpu_grid([d], precision, max_cycles=200)
    st, cyc, rel = g.solve_to_tol(1e-12)
    assert st == sgml.OK
    u_ref = g.get_solution(0)
    f = torch.from_numpy(np.ascontiguousarray(d["f"])).cuda()
    sig = torch.from_numpy(np.ascontiguousarray(d["sigma"])).cuda() if d["sigma"] is not None else None
    for _ in range(2):  # two calls in a row share the scratch
        u = torch.full(f.shape, float("nan"), dtype=torch.float64, device="cuda")
        st2, cyc2, rel2 = sgml.solve_noalloc(d["dim"], d["n"], f, u, sigma=sig, a_scalar=d["a_scalar"],
                                             faces=d["faces"], values=d["values"], rtol=1e-12, max_cycles=200,
                                             precision=precision)
        torch.cuda.synchronize()
        assert st2 == sgml.OK and rel2 <= 1e-12
        assert cyc2 == cyc[0]
        assert rel_l2(u.cpu().numpy(), u_ref) <= 1e-10


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """257^3 needs far more than the fixed scratch: rejected before any GPU work (the pointers are
    never dereferenced)."""
    import ctypes
    import torch
    lib = sgml.load()
    f = torch.zeros(8, dtype=torch.float64, device="cuda")
    faces = (ctypes.c_int * 6)(*([sgml.DIRICHLET] * 6))
    st = lib.sgml_solve_noalloc(3, 8, sgml.MIXED, f.data_ptr(), None, 0.0, faces, None, 1e-10, 100, f.data_ptr(),
                                None, None, None)
    assert st == sgml.ERR_ARG
    assert b"too large" in lib.sgml_noalloc_last_error()


def test_noalloc_refuses_host_memory():
    """f and u in host memory are refused by the library's own pointer check, before any GPU work
    (the binding refuses them too; the C entry point is called directly here)."""
    import ctypes
    import torch
    lib = sgml.load()
    N = 2 ** 3 + 1
    f_host = np.zeros(N * N)
    u_dev = torch.zeros(N * N, dtype=torch.float64, device="cuda")
    faces = (ctypes.c_int * 6)(*([sgml.DIRICHLET] * 6))
    st = lib.sgml_solve_noalloc(2, 3, sgml.MIXED, f_host.ctypes.data, None, 0.0, faces, None, 1e-10, 50,
                                u_dev.data_ptr(), None, None, None)
    assert st == sgml.ERR_ARG
    assert b"device memory" in lib.sgml_noalloc_last_error()
    with pytest.raises(TypeError):
        sgml.solve_noalloc(2, 3, torch.from_numpy(f_host), u_dev)
