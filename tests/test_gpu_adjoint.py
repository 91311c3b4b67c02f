"""Adjoint gradients through the autograd wrapper (row A9): dJ/dsigma and dJ/df of
J = 1/2 ||u - u_t||^2 for a batch of log-normal dielectric problems, against the CPU oracle's adjoint
(oracle solve of the adjoint + oracle gradient formula) and against fourth-order central finite
differences of J computed with GPU forward solves.  Tolerance 1e-6 relative to the component, or to
1 % of the gradient's max norm for components smaller than that (solves converged to 1e-13)."""
import numpy as np
import pytest

from oracle.oracle import Problem
from paper_1703_07206_gb300 import inputs, sgml

pytestmark = pytest.mark.gpu


def make_batch(count=3, n=4):
    return inputs.lognormal_dielectric_batch_3d(count=count, n=n, seed=5000)


@pytest.mark.parametrize("save_solution", [True, False])
def test_autograd_gradients_match_oracle_adjoint(save_solution):
    import torch
    from paper_1703_07206_gb300.autograd import SGMLSolve
    probs = make_batch()
    n = probs[0]["n"]
    f = torch.tensor(np.stack([d["f"] for d in probs]), device="cuda", requires_grad=True)
    sig = torch.tensor(np.stack([d["sigma"] for d in probs]), device="cuda", requires_grad=True)
    grid = sgml.Grid(3, [n] * len(probs), precision=sgml.FP64)
    grid.set_params(max_cycles=400)
    # targets: solutions with the perturbed coefficients (oracle, CPU)
    u_t = [Problem(3, n, sigma=d["eps_target"]).solve(d["f"], tol=1e-13, max_cycles=400)[0] for d in probs]
    ut = torch.tensor(np.stack(u_t), device="cuda")
    u = SGMLSolve.apply(f, sig, grid, 1e-13, save_solution)
    J = 0.5 * ((u - ut) ** 2).sum()
    J.backward()
    for b, d in enumerate(probs):
        p = Problem(3, n, sigma=d["sigma"])
        u_ref, c, _ = p.solve(d["f"], tol=1e-13, max_cycles=400)
        g = np.where(p.unknown_mask(), u_ref - u_t[b], 0.0)
        lam, c2, _ = p.solve(g, tol=1e-13, max_cycles=400)
        ds_ref = p.sigma_gradient(lam, u_ref)
        ds = sig.grad[b].cpu().numpy()
        df = f.grad[b].cpu().numpy()
        assert np.abs(ds - ds_ref).max() <= 1e-6 * np.abs(ds_ref).max()
        lam_in = np.where(p.unknown_mask(), lam, 0.0)
        assert np.abs(df - lam_in).max() <= 1e-6 * np.abs(lam).max()


def test_autograd_gradient_matches_finite_differences():
    import torch
    from paper_1703_07206_gb300.autograd import SGMLSolve
    d = make_batch(count=1)[0]
    n = d["n"]
    grid = sgml.Grid(3, [n], precision=sgml.FP64)
    grid.set_params(max_cycles=400)
    rng = np.random.default_rng(7)
    ut = torch.tensor(rng.standard_normal(d["f"].shape) * 1e-3, device="cuda")
    sig0 = torch.tensor(d["sigma"], device="cuda")
    f0 = torch.tensor(d["f"], device="cuda")

    def J(sig, f):
        return float(0.5 * ((SGMLSolve.apply(f, sig, grid, 1e-14, True) - ut) ** 2).sum())

    sig = sig0.clone().requires_grad_(True)
    f = f0.clone().requires_grad_(True)
    u = SGMLSolve.apply(f, sig, grid, 1e-14, True)
    (0.5 * ((u - ut) ** 2).sum()).backward()
    gs, gf = sig.grad.cpu().numpy(), f.grad.cpu().numpy()
    N = 2 ** n + 1
    def fd4(fun, base, node, h):
        """Fourth-order central difference of fun at base along `node`."""
        vals = []
        for k in (1, -1, 2, -2):
            x = base.clone()
            x[node] += k * h
            vals.append(fun(x))
        return (8 * (vals[0] - vals[1]) - (vals[2] - vals[3])) / (12 * h)

    for node in [(N // 2, N // 2, N // 2), (3, 5, 7), (1, 1, 1), (0, 4, 4)]:
        fd = fd4(lambda s: J(s, f0), sig0, node, 3e-4 * float(sig0[node]))
        assert abs(fd - gs[node]) <= 1e-6 * max(abs(fd), 1e-2 * np.abs(gs).max()), node
    for node in [(N // 2, N // 2, N // 2), (2, 6, 3)]:
        fd = fd4(lambda f: J(sig0, f), f0, node, 3e-3 * max(1.0, abs(float(f0[node]))))
        assert abs(fd - gf[node]) <= 1e-6 * max(abs(fd), 1e-2 * np.abs(gf).max()), node
