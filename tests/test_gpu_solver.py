"""GPU solvers against the oracle (Sections 2.1-2.3): linear solves reach their tolerance on
the exact operator, Newton with load steps reaches the oracle's equilibrium, the mixed
(FP32-inner) solver reaches the same FP64 tolerance, and a split run resumes bit-exactly."""
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


@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("strategy", [0, 1])
def test_linear_solve_reaches_tolerance(nhmf, solver, strategy):
    w = inp.small(inp.WORKLOADS["q2_64_clamp"], 4)
    u = inp.draw_u(w)
    b = inp.draw_vector(77, w.n_dofs)
    op = Operator(Mesh(w.n_el, w.degree), w.mu, w.lam, w.bc)
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(u), 3)
    x = cuda(np.zeros_like(u))
    it, inner, rel = prob.linear_solve(cuda(b), x, solver=solver, strategy=strategy, linear_rtol=1e-8)
    assert rel <= 1e-8
    xs = host(x)
    true_rel = np.linalg.norm(b - op.apply(u, xs)) / np.linalg.norm(b)
    assert true_rel <= 2e-8, true_rel
    if solver == 1:
        assert inner > 0 and it < 40


@pytest.mark.parametrize("solver", [0, 1])
def test_newton_matches_oracle_equilibrium(nhmf, solver):
    n_el, p, S, comp = 3, 2, 3, 0.1
    op = Operator(Mesh(n_el, p), 1.0, 1.5, bc=2)
    u_ref, hist = newton_load_steps(op, steps=S, compression=comp)
    prob = nhmf.Problem(n_el, p, 1.0, 1.5, 2)
    u = cuda(np.zeros(op.mesh.n_dofs))
    stats = prob.solve(u, solver=solver, load_steps=S, compression=comp, linear_rtol=1e-10,
                       newton_rtol=1e-8)
    assert stats["steps_done"] == S
    assert all(r <= 1e-8 for r in stats["rel_residual"])
    ug = host(u)
    assert rel_l2(ug, u_ref) <= 1e-7
    # the oracle's FP64 residual of the GPU result (free rows) is at the tolerance level
    R = op.residual(ug)
    assert np.linalg.norm(R) <= 1e-7 * np.linalg.norm(op.apply(ug, ug))


def test_mixed_and_plain_agree_near_incompressible(nhmf):
    n_el, p, S, comp = 3, 3, 2, 0.05
    res = {}
    for solver in (0, 1):
        prob = nhmf.Problem(n_el, p, 1.0, 49.0, 2)
        u = cuda(np.zeros(3 * (p * n_el + 1) ** 3))
        stats = prob.solve(u, solver=solver, load_steps=S, compression=comp, linear_rtol=1e-8)
        res[solver] = (host(u), stats)
    assert rel_l2(res[1][0], res[0][0]) <= 1e-6
    assert res[1][1]["total_linear_iters"] < res[0][1]["total_linear_iters"]


def test_resume_is_bit_exact(nhmf):
    import torch
    n_el, p, S, comp = 3, 2, 3, 0.06
    prob = nhmf.Problem(n_el, p, 1.0, 1.5, 2)
    n = 3 * (p * n_el + 1) ** 3
    u_all = cuda(np.zeros(n))
    prob.solve(u_all, load_steps=S, compression=comp)
    u_part = cuda(np.zeros(n))
    prob.solve(u_part, load_steps=S, compression=comp, last_step=2)
    checkpoint = u_part.cpu().clone()            # host checkpoint after step 2
    prob2 = nhmf.Problem(n_el, p, 1.0, 1.5, 2)
    u_res = checkpoint.to("cuda:0")
    prob2.solve(u_res, load_steps=S, compression=comp, first_step=3)
    assert torch.equal(u_res, u_all)


def test_solver_argument_errors(nhmf):
    prob = nhmf.Problem(2, 1, 1.0, 1.5, 2)
    u = cuda(np.zeros(3 * 27))
    with pytest.raises(nhmf.NhmfError) as ei:
        prob.solve(u, load_steps=0)
    assert ei.value.status == 1
    with pytest.raises(nhmf.NhmfError) as ei:
        prob.solve(u, load_steps=2, first_step=3)
    assert ei.value.status == 1
    with pytest.raises(nhmf.NhmfError) as ei:
        prob.solve(u, load_steps=1, solver=2, compression=0.01)   # no trained network yet
    assert ei.value.status == 8
