"""Failure statuses of the solve (sgml.h): every one is driven by a test, and none of them faults,
traps or hangs the GPU.

- SGML_ERR_BARRIER_TIMEOUT: every grid-barrier wait of the persistent cycle kernel is bounded.  The
  test aid of sgml_set_barrier_test makes CTA 0 withhold its arrival at one barrier with a 1 ms wait
  limit; every CTA's wait runs out, the launch returns, and the status reaches the host.  The grid
  (and a fresh one) solves normally afterwards.
- SGML_ERR_DIVERGED: theta = 1.5 of the Sec. 2 stability bound (the (pi, 0) mode is amplified).
- SGML_ERR_NONFINITE: a NaN in the source.
- SGML_ERR_NOT_CONVERGED: max_cycles too small for the tolerance.
"""
import time

import numpy as np
import pytest

from paper_1703_07206_gb300 import inputs, sgml
from tests.gpu_helpers import gpu_grid

pytestmark = pytest.mark.gpu

FORMS = [sgml.FP64, sgml.MIXED]


@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("withhold", [1, 2, 7, 40])
def test_barrier_timeout_is_reported_and_the_grid_recovers(precision, withhold):
    d = inputs.random_problem(3, 5, seed=601, flux=True)
    g = gpu_grid([d], precision, max_cycles=100)
    g.set_barrier_test(1e-3, withhold)
    t0 = time.perf_counter()
    with pytest.raises(sgml.SGMLError) as ei:
        g.solve_to_tol(1e-10)
    assert ei.value.code == sgml.ERR_BARRIER_TIMEOUT
    assert time.perf_counter() - t0 < 1.0  # the bounded waits ended the launch
    # the same grid solves normally once the aid is off
    g.set_barrier_test(2.0, 0)
    st, cyc, rel = g.solve_to_tol(1e-10)
    assert st == sgml.OK and rel[0] <= 1e-10
    u_same = g.get_solution(0)
    g.close()
    # and a fresh grid gives the same solution bit for bit
    h = gpu_grid([d], precision, max_cycles=100)
    st2, cyc2, rel2 = h.solve_to_tol(1e-10)
    assert st2 == sgml.OK and cyc2[0] == cyc[0]
    assert np.array_equal(h.get_solution(0), u_same)
    h.close()


def test_withholding_past_the_last_barrier_changes_nothing():
    d = inputs.random_problem(2, 5, seed=602)
    g = gpu_grid([d], sgml.MIXED, max_cycles=100)
    st, cyc, rel = g.solve_to_tol(1e-10)
    u_ref = g.get_solution(0)
    g.set_barrier_test(2.0, 10 ** 8)  # no launch reaches that many barriers
    st2, cyc2, rel2 = g.solve_to_tol(1e-10)
    assert st == st2 == sgml.OK and cyc2[0] == cyc[0]
    assert np.array_equal(g.get_solution(0), u_ref)
    g.close()


@pytest.mark.parametrize("precision", FORMS)
def test_theta_beyond_the_stability_bound_diverges(precision):
    d = inputs.random_problem(2, 5, seed=603, hetero=False, helmholtz=False, mixed_bc=False)
    g = gpu_grid([d], precision, theta=1.5, max_cycles=100)
    st, cyc, rel = g.solve_to_tol(1e-10)
    assert st == sgml.ERR_DIVERGED
    assert 3 <= cyc[0] < 100 and rel[0] > 1.0
    c, r, s = g.get_stats(0)
    assert s == sgml.ERR_DIVERGED
    g.close()


@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("dim", [2, 3])
def test_nan_in_the_source_is_nonfinite(precision, dim):
    d = inputs.random_problem(dim, 4, seed=604)
    f = d["f"].copy()
    f[(4,) * dim] = np.nan
    d["f"] = f
    g = gpu_grid([d], precision, max_cycles=50)
    st, cyc, rel = g.solve_to_tol(1e-10)
    assert st == sgml.ERR_NONFINITE
    assert not np.isfinite(rel[0])
    g.close()


@pytest.mark.parametrize("precision", FORMS)
def test_too_few_cycles_is_not_converged(precision):
    d = inputs.random_problem(3, 4, seed=605)
    g = gpu_grid([d], precision, max_cycles=2)
    st, cyc, rel = g.solve_to_tol(1e-12)
    assert st == sgml.ERR_NOT_CONVERGED
    assert cyc[0] == 2 and rel[0] > 1e-12
    # run_cycle has no tolerance: the same budget is fine there
    g.run_cycle(2)
    c, r, s = g.get_stats(0)
    assert s == sgml.OK
    g.close()


def test_batch_reports_the_worst_status_per_problem():
    good = inputs.random_problem(2, 4, seed=606)
    bad = inputs.random_problem(2, 4, seed=607)
    f = bad["f"].copy()
    f[3, 3] = np.nan
    bad["f"] = f
    g = gpu_grid([good, bad], sgml.MIXED, max_cycles=100)
    st, cyc, rel = g.solve_to_tol(1e-10)
    assert st == sgml.ERR_NONFINITE
    assert rel[0] <= 1e-10 and not np.isfinite(rel[1])
    assert g.get_stats(0)[2] == sgml.OK and g.get_stats(1)[2] == sgml.ERR_NONFINITE
    g.close()
