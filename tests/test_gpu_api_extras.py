"""Entry points around the solve: the FP64 residual and the adjoint sigma gradient with host and
device arrays (device arrays are used in place, host arrays staged through a buffer the grid
allocates once), and the arithmetic-rate measurement used as the FP64 form's roofline denominator."""
import numpy as np
import pytest

from paper_1703_07206_gb300 import inputs, sgml
from tests.gpu_helpers import gpu_grid, oracle_problem

pytestmark = pytest.mark.gpu


def test_fma_rates_are_measured():
    fp64, fp32 = sgml.measure_fma_rates()
    assert fp64 > 1e10 and fp32 > fp64  # FMA instructions per second, thread level


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 4)])
def test_residual_host_and_device_arrays_agree_with_oracle(dim, n):
    import torch
    d = inputs.random_problem(dim, n, seed=701, flux=True)
    g = gpu_grid([d], sgml.FP64)
    rng = np.random.default_rng(702)
    u = rng.standard_normal(d["f"].shape)
    r_host = g.residual(0, u)
    u_dev = torch.from_numpy(u).cuda()
    r_dev = torch.empty_like(u_dev)
    g.residual(0, u_dev, r_dev)
    assert np.array_equal(r_host, r_dev.cpu().numpy())
    r_ref = oracle_problem(d).residual(u, d["f"])
    assert np.abs(r_host - r_ref).max() <= 1e-12 * np.abs(r_ref).max()
    with pytest.raises(sgml.SGMLError):
        g.residual(0, u_dev, u_dev)  # r must not alias u
    g.close()


def test_sigma_gradient_allocates_nothing_per_call():
    """The 16-problem adjoint backward calls the gradient once per problem: after the first call
    the grid's staging buffer (host arrays) is reused and device arrays need none."""
    import torch
    probs = inputs.lognormal_dielectric_batch_3d(count=2, n=5, seed=5000)
    g = gpu_grid(probs, sgml.FP64)
    rng = np.random.default_rng(703)
    lam = rng.standard_normal(probs[0]["f"].shape)
    u = rng.standard_normal(probs[0]["f"].shape)
    ref = oracle_problem(probs[0]).sigma_gradient(lam, u)
    out = g.sigma_gradient(0, lam, u)  # host arrays: the staging buffer is allocated here
    assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    lam_d, u_d = torch.from_numpy(lam).cuda(), torch.from_numpy(u).cuda()
    out_d = torch.empty_like(lam_d)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    for b in range(2):
        for _ in range(5):
            g.sigma_gradient(b, lam, u)
            g.sigma_gradient(b, lam_d, u_d, out_d)
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 == free1  # no allocation by the library in the loop
    assert free0 - free1 < 64 << 20  # (the three test tensors only)
    assert np.array_equal(out_d.cpu().numpy(), g.sigma_gradient(1, lam, u))
    g.close()
