"""Shared helpers of the GPU tests: build problems into a libsgml grid and into the oracle."""
import numpy as np

from oracle.oracle import Problem
from paper_1703_07206_gb300 import sgml


def oracle_problem(d, **kw):
    return Problem(d["dim"], d["n"], faces=d["faces"], values=d["values"], sigma=d.get("sigma"), a=d.get("a"),
                   a_scalar=d.get("a_scalar", 0.0), **kw)


def oracle_cycles(p, f, k):
    """u after k outer steps + cycles of the oracle, from the lifted boundary values."""
    u = p.lift()
    for _ in range(k):
        r = p.residual(u, f)
        u = u + p.cycle(r)
    return u


def gpu_grid(problems, precision, **params):
    dim = problems[0]["dim"]
    g = sgml.Grid(dim, [d["n"] for d in problems], precision=precision)
    if params:
        g.set_params(**params)
    for b, d in enumerate(problems):
        sgml.problem_into_grid(g, b, d)
    return g


def rel_l2(a, b):
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)
