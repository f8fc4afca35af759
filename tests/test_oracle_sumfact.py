"""The oracle's plain sum-factorised CPU apply (oracle/sumfact.c, the timed CPU baseline)
against the oracle's direct route (explicit L, O((p+1)^6) basis evaluation): the same
operator up to round-off, for every degree, boundary preset and both strategies, and
independent of the thread count."""
import os
import subprocess
import sys

import numpy as np
import pytest

import nhmf_inputs as inp
from oracle.fem import Operator
from oracle.mesh import Mesh
from oracle.sumfact import SumFactOperator


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n_el,p,bc", [(3, 1, 1), (3, 2, 2), (2, 3, 0), (2, 4, 1), (4, 2, 1), (3, 3, 2)])
def test_sumfact_equals_direct_route(n_el, p, bc):
    w = inp.small(inp.WORKLOADS["q2_64_clamp"], n_el, p)
    u, du = inp.draw_u(w), inp.draw_du(w)
    ref = Operator(Mesh(n_el, p), w.mu, w.lam, bc).apply(u, du)
    op = SumFactOperator(n_el, p, w.mu, w.lam, bc)
    assert rel(op.apply(u, du), ref) <= 1e-13
    op.set_cache(u)
    assert rel(op.apply(u, du, cached=True), ref) <= 1e-13


def test_sumfact_at_large_lambda_and_compression():
    w = inp.small(inp.WORKLOADS["q3_48_compress"], 3)
    u = inp.uniform_pm(4242, w.n_dofs, 0.01)
    du = inp.draw_vector(4343, w.n_dofs)
    ref = Operator(Mesh(w.n_el, w.degree), w.mu, w.lam, w.bc).apply(u, du)
    op = SumFactOperator(w.n_el, w.degree, w.mu, w.lam, w.bc)
    assert rel(op.apply(u, du), ref) <= 1e-13


def test_sumfact_result_independent_of_threads():
    code = ("import numpy as np, nhmf_inputs as inp\n"
            "from oracle.sumfact import SumFactOperator, threads\n"
            "w = inp.small(inp.WORKLOADS['q2_64_clamp'], 6)\n"
            "v = SumFactOperator(6, 2, w.mu, w.lam, w.bc).apply(inp.draw_u(w), inp.draw_du(w))\n"
            "print(threads(), v.tobytes().hex()[:4000], float(np.sum(v)))\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for nt in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=nt, PYTHONPATH=root)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=root, check=True)
        outs.append(r.stdout.split())
    assert outs[0][0] == "1" and outs[1][0] == "3"
    assert outs[0][1:] == outs[1][1:]


def test_sumfact_reports_nonpositive_jacobian():
    w = inp.small(inp.WORKLOADS["q2_64_clamp"], 2)
    u = np.zeros(w.n_dofs)
    M = w.n_nodes_1d
    u[M ** 3 + M * (M // 2) + M // 2] = 5.0       # u_y jumps by 5 over h/2: det F < 0 nearby
    op = SumFactOperator(2, 2, w.mu, w.lam, 0)
    with pytest.raises(ValueError, match="det F"):
        op.apply(u, np.ones(w.n_dofs))
