"""Geometric multigrid (Section 2.3): V-cycle-preconditioned flexible CG in FP64 and with an
FP32 V-cycle, against the oracle's operator; iteration counts stay small and nearly
independent of the mesh size (the defining property of multigrid)."""
import numpy as np
import pytest

import nhmf_inputs as inp
from oracle.fem import Operator
from oracle.mesh import Mesh
from oracle.solver import newton_load_steps
from tests.gpu_util import cuda, host, lib_or_fail, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nhmf():
    return lib_or_fail()


@pytest.mark.parametrize("solver", [4, 5])
@pytest.mark.parametrize("bc,p", [(1, 2), (2, 2), (2, 1), (1, 3)])
def test_gmg_linear_solve(nhmf, solver, bc, p):
    its = {}
    for n_el in (8, 16):
        # a mildly perturbed state: the tangent stays SPD (noisy states can make it indefinite)
        w = inp.Workload("g", n_el, p, 1.0, 1.5, bc, "scaled", 0.01, "normal", 1.0, 6100 + n_el, 6200 + n_el)
        u = inp.draw_u(w)
        b = inp.draw_vector(79, w.n_dofs)
        b[inp.dirichlet_mask(n_el, p, bc).reshape(-1)] = 0.0
        prob = nhmf.Problem.from_workload(w)
        prob.set_linearization(cuda(u), 3)
        x = cuda(np.zeros_like(u))
        it, inner, rel = prob.linear_solve(cuda(b), x, solver=solver, linear_rtol=1e-8)
        assert rel <= 1e-8
        if n_el == 8:
            op = Operator(Mesh(n_el, p), 1.0, 1.5, bc)
            true = np.linalg.norm(b - op.apply(u, host(x))) / np.linalg.norm(b)
            assert true <= 2e-8
        its[n_el] = it
    assert its[16] <= 40
    assert its[16] <= 2 * its[8] + 4


def test_gmg_newton_matches_oracle(nhmf):
    n_el, p, S, comp = 4, 2, 2, 0.08
    op = Operator(Mesh(n_el, p), 1.0, 1.5, bc=2)
    u_ref, _ = newton_load_steps(op, steps=S, compression=comp)
    for solver in (4, 5):
        prob = nhmf.Problem(n_el, p, 1.0, 1.5, 2)
        u = cuda(np.zeros(op.mesh.n_dofs))
        st = prob.solve(u, solver=solver, load_steps=S, compression=comp, linear_rtol=1e-10)
        assert all(r <= 1e-8 for r in st["rel_residual"])
        assert rel_l2(host(u), u_ref) <= 1e-7


def test_double_float_outer_applies(nhmf):
    """outer_apply = NHMF_DF64: the flexible solvers' outer Krylov applies in FP64-accurate
    double-float arithmetic.  The linear solve meets the same true FP64 residual (checked with
    the oracle), and Newton with mixed multigrid matches the oracle's Newton like the FP64 outer
    applies do."""
    w = inp.Workload("d", 8, 2, 1.0, 1.5, 2, "scaled", 0.01, "normal", 1.0, 6301, 6302)
    u = inp.draw_u(w)
    b = inp.draw_vector(81, w.n_dofs)
    b[inp.dirichlet_mask(8, 2, 2).reshape(-1)] = 0.0
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(u), nhmf.NHMF_CACHE_FP64 | nhmf.NHMF_CACHE_FP32 | nhmf.NHMF_CACHE_DF64)
    op = Operator(Mesh(8, 2), 1.0, 1.5, 2)
    for solver in (nhmf.NHMF_SOLVER_MIXED_FCG, nhmf.NHMF_SOLVER_MIXED_GMG):
        x = cuda(np.zeros_like(u))
        it, _, rel = prob.linear_solve(cuda(b), x, solver=solver, linear_rtol=1e-10, outer_apply=nhmf.NHMF_DF64)
        assert rel <= 1e-10, (solver, rel)
        assert np.linalg.norm(b - op.apply(u, host(x))) / np.linalg.norm(b) <= 2e-10
    n_el, p, S, comp = 4, 2, 2, 0.08
    op = Operator(Mesh(n_el, p), 1.0, 1.5, bc=2)
    u_ref, _ = newton_load_steps(op, steps=S, compression=comp)
    prob = nhmf.Problem(n_el, p, 1.0, 1.5, 2)
    uu = cuda(np.zeros(op.mesh.n_dofs))
    st = prob.solve(uu, solver=nhmf.NHMF_SOLVER_MIXED_GMG, load_steps=S, compression=comp, linear_rtol=1e-10,
                    outer_apply=nhmf.NHMF_DF64)
    assert all(r <= 1e-8 for r in st["rel_residual"])
    assert rel_l2(host(uu), u_ref) <= 1e-7
    with pytest.raises(nhmf.NhmfError):
        prob.solve(uu, solver=nhmf.NHMF_SOLVER_MIXED_GMG, strategy=nhmf.NHMF_ON_THE_FLY, load_steps=S,
                   compression=comp, outer_apply=nhmf.NHMF_DF64)
