"""Element-wise parity with the FP64 oracle on the headline workload's recipe (3-D dielectric,
eps = 1 / 80 in 32 spheres, 8 Gaussian charges, Dirichlet 0) at 65^3 and 129^3 after one and two
cycles, and at the headline's 257^3 after one (Algorithm 3 plus the outer step of Sec. 2), in the
launch configuration the benchmark times: the default persistent launch (two CTAs per SM, 64 x 8
tiles, the library's default slab height), and with the slab cut of the work partition forced onto level 0 (at 257^3 the default
height takes it there; at 129^3 a height of 4 does), so that the slab pieces, many tiles per CTA and
every level of the pyramid are compared with the oracle node by node.

Tolerances (as in test_gpu_parity): FP64 form 1e-12 relative L2 (rounding order only); mixed form
2e-5 after two cycles (the cycle runs in FP32).
"""
import functools

import numpy as np
import pytest

from paper_1703_07206_gb300 import inputs, sgml
from tests.gpu_helpers import gpu_grid, oracle_problem, rel_l2

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def case(n, k=2):
    d = inputs.dielectric_spheres_3d(n=n, seed=2000)
    p = oracle_problem(d)
    u = p.lift()
    us = []
    for _ in range(k):
        u = u + p.cycle(p.residual(u, d["f"]))
        us.append(u)
    return d, us


def gpu_after(d, precision, cycles, slab):
    g = gpu_grid([d], precision, max_cycles=400)
    if slab is not None:
        g.set_launch(0, 1, 0, 64, slab)
    ctas, threads, smem = g.launch_info()
    g.run_cycle(cycles)
    u = g.get_solution(0)
    g.close()
    return u, ctas


SHAPES = [(6, None), (7, None), (7, 4)]  # (n, slab height; None: the library's default)


@pytest.mark.parametrize("n,slab", SHAPES, ids=[f"{2 ** n + 1}cubed-slab{s}" for n, s in SHAPES])
@pytest.mark.parametrize("cycles", [1, 2])
def test_fp64_form_matches_oracle_cycle_by_cycle(n, slab, cycles):
    d, us = case(n)
    u, ctas = gpu_after(d, sgml.FP64, cycles, slab)
    assert ctas >= 2 * 100  # the persistent launch at full occupancy (2 CTAs per SM)
    err = rel_l2(u, us[cycles - 1])
    assert err <= 1e-12, err


@pytest.mark.parametrize("n,slab", SHAPES, ids=[f"{2 ** n + 1}cubed-slab{s}" for n, s in SHAPES])
def test_mixed_form_close_to_oracle_after_two_cycles(n, slab):
    d, us = case(n)
    u, _ = gpu_after(d, sgml.MIXED, 2, slab)
    err = rel_l2(u, us[1])
    assert err <= 2e-5, err


def test_slab_cut_changes_no_bit_at_129_cubed():
    """The slab cut (height 4; the CPU partition tests show it reaches level 0 here) and the
    contiguous cut give the same result bit for bit: the work partition never changes a value."""
    d, _ = case(7)
    u_slab, _ = gpu_after(d, sgml.MIXED, 1, 4)
    u_runs, _ = gpu_after(d, sgml.MIXED, 1, 0)
    assert np.array_equal(u_slab, u_runs)


def test_both_forms_match_oracle_after_one_cycle_at_257_cubed():
    """The headline size itself, in the benchmark's launch shape (the default slab cut reaches
    level 0 here): the whole 257^3 iterate after one outer step and cycle, node by node, against the
    oracle's (about ten seconds of the oracle on the host's cores)."""
    d, us = case(8, 1)
    u, ctas = gpu_after(d, sgml.FP64, 1, None)
    assert ctas >= 2 * 100
    err = rel_l2(u, us[0])
    assert err <= 1e-12, err
    u, _ = gpu_after(d, sgml.MIXED, 1, None)
    err = rel_l2(u, us[0])
    assert err <= 2e-5, err
