"""Post-processing of the vortex application (Sec. 3.3) on the GPU against the oracle.

* v = curl psi (Eq. 14): the GPU's differences equal the oracle's (same second-order formulas) to
  rounding; exact on quadratic potentials.
* RK4 streamlines in the trilinearly interpolated field: same paths and lengths as the oracle.
* The trefoil vortex at 129^3: the three stream-potential components solved by the library (mixed
  form, one batch), the velocity, and streamlines near and far from the knot as in Fig. 6.
"""
import numpy as np
import pytest
import torch

from oracle import oracle
from paper_1703_07206_gb300 import inputs, sgml
from tests.gpu_helpers import gpu_grid

pytestmark = pytest.mark.gpu


def smooth_potential(n, seed, modes=4):
    rng = np.random.default_rng(seed)
    N = 2 ** n + 1
    x = np.linspace(0.0, 1.0, N)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    psi = np.zeros((3, N, N, N))
    for c in range(3):
        for _ in range(modes):
            p, q, r = rng.integers(1, 4, size=3)
            ph = rng.uniform(0, 2 * np.pi, size=3)
            psi[c] += rng.standard_normal() * np.sin(np.pi * p * X + ph[0]) * np.sin(np.pi * q * Y + ph[1]) \
                * np.sin(np.pi * r * Z + ph[2]) / (p + q + r)
    return psi


@pytest.mark.parametrize("n", [4, 5, 7])  # 129^3: z-chunks of three planes
def test_curl_matches_oracle(n):
    rng = np.random.default_rng(900 + n)
    N = 2 ** n + 1
    psi = rng.standard_normal((3, N, N, N))
    v = sgml.curl(torch.from_numpy(psi).cuda()).cpu().numpy()
    ref = oracle.curl(psi)
    assert np.abs(v - ref).max() <= 1e-13 * np.abs(ref).max()


def test_curl_exact_on_quadratic_potentials():
    N = 9
    x = np.linspace(0.0, 1.0, N)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    psi = np.stack([Y ** 2 + 0.3 * X * Z, Z ** 2 - 0.7 * X * Y, X ** 2 + Y * Z])
    v = sgml.curl(torch.from_numpy(psi).cuda()).cpu().numpy()
    want = np.stack([Z - 2 * Z, 0.3 * X - 2 * X, -0.7 * Y - 2 * Y])
    assert np.abs(v - want).max() <= 1e-11


def test_streamlines_match_oracle():
    psi = smooth_potential(5, 910)
    v = oracle.curl(psi)
    rng = np.random.default_rng(911)
    seeds = rng.uniform(0.2, 0.8, size=(64, 3))
    seeds[0] = [1.2, 0.5, 0.5]  # outside: empty path
    dt, steps = 2e-3, 200
    p_ref, l_ref = oracle.streamlines(v, seeds, dt, steps)
    p, l = sgml.streamlines(torch.from_numpy(v).cuda(), seeds, dt, steps)
    p, l = p.cpu().numpy(), l.cpu().numpy()
    assert np.array_equal(l, l_ref) and l[0] == 0
    for s in range(1, len(seeds)):
        assert l[s] >= 1 and np.abs(p[s, :l[s]] - p_ref[s, :l[s]]).max() <= 1e-10, s


def test_trefoil_129_velocity_and_streamlines():
    n = 7
    probs = inputs.trefoil_vorticity_3d(n=n)
    g = gpu_grid(probs, sgml.MIXED, max_cycles=400)
    st, cyc, rel = g.solve_to_tol(1e-10)
    assert st == sgml.OK and np.all(rel <= 1e-10)
    N = 2 ** n + 1
    psi = torch.empty((3, N, N, N), dtype=torch.float64, device="cuda")
    for b in range(3):
        g.get_solution(b, psi[b])
    v = sgml.curl(psi)
    torch.cuda.synchronize()
    psi_h, v_h = psi.cpu().numpy(), v.cpu().numpy()
    ref = oracle.curl(psi_h)
    assert np.abs(v_h - ref).max() <= 1e-12 * np.abs(ref).max()
    # the velocity peaks at the knot: the fastest node lies within a few tube widths of the curve
    speed = np.linalg.norm(v_h, axis=0)
    k, j, i = np.unravel_index(np.argmax(speed), speed.shape)
    h = 1.0 / (N - 1)
    t = np.linspace(0, 2 * np.pi, 20001)
    curve = (0.4 / 3.0) * np.array([np.sin(t) + 2 * np.sin(2 * t), np.cos(t) - 2 * np.cos(2 * t), -np.sin(3 * t)]) + 0.5
    dist = np.min(np.linalg.norm(curve - np.array([i * h, j * h, k * h])[:, None], axis=0))
    assert dist <= 6 * h
    # two streamlines as in Fig. 6: one started next to the knot, one far from it
    c0 = curve[:, 0]
    seeds = np.array([c0 + np.array([2 * h, 2 * h, 0.0]), [0.5, 0.5, 0.93]])
    dt, steps = 5e-4, 300
    p, l = sgml.streamlines(v, seeds, dt, steps)
    p, l = p.cpu().numpy(), l.cpu().numpy()
    p_ref, l_ref = oracle.streamlines(v_h, seeds, dt, steps)
    assert np.array_equal(l, l_ref) and np.all(l > 1)
    for s in range(2):
        assert np.abs(p[s, :l[s]] - p_ref[s, :l[s]]).max() <= 1e-8, s
        assert np.all((p[s, :l[s]] >= 0) & (p[s, :l[s]] <= 1))
