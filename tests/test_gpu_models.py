"""The split neo-Hookean model (Eq. hypcomplex) and Algorithm 2 on the GPU against the oracle:
the same kernel skeleton with a second point code.  FP64 bar 1e-12, FP32 1e-5."""
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


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("bc", [1, 2])
def test_split_model_apply_residual_diagonal(nhmf, p, bc):
    n_el, mu, kappa = 3, 1.0, 20.0
    w = inp.Workload("split", n_el, p, mu, kappa, bc, "scaled", 0.05, "normal", 1.0, 5100 + p, 5200 + p)
    u, du = inp.draw_u(w), inp.draw_du(w)
    op = Operator(Mesh(n_el, p), mu, kappa, bc, model=1)
    prob = nhmf.Problem(n_el, p, mu, kappa, bc, model=nhmf.NHMF_MODEL_SPLIT)
    prob.set_linearization(cuda(u), nhmf.NHMF_CACHE_SPATIAL)
    ref = op.apply(u, du)
    for strat in (nhmf.NHMF_ON_THE_FLY, nhmf.NHMF_SPATIAL):
        v = cuda(np.zeros_like(u))
        prob.apply(cuda(du), v, nhmf.NHMF_FP64, strat)
        assert rel_l2(host(v), ref) <= 1e-12, strat
    v32 = cuda(np.zeros(u.size, dtype=np.float32))
    prob.apply(cuda(du.astype(np.float32)), v32, nhmf.NHMF_FP32, nhmf.NHMF_ON_THE_FLY)
    assert rel_l2(host(v32), ref) <= 1e-5
    r = cuda(np.zeros_like(u))
    prob.residual(cuda(u), r)
    assert rel_l2(host(r), op.residual(u)) <= 1e-12
    d = cuda(np.zeros_like(u))
    prob.diagonal(d)
    assert rel_l2(host(d), op.diagonal(u)) <= 1e-12
    with pytest.raises(nhmf.NhmfError):
        prob.apply(cuda(du), v, nhmf.NHMF_FP64, nhmf.NHMF_CACHED)


def test_split_model_newton_matches_oracle(nhmf):
    n_el, p, S, comp, mu, kappa = 3, 2, 2, 0.08, 1.0, 10.0
    op = Operator(Mesh(n_el, p), mu, kappa, bc=2, model=1)
    u_ref, _ = newton_load_steps(op, steps=S, compression=comp)
    for strat, solver in ((nhmf.NHMF_SPATIAL, nhmf.NHMF_SOLVER_JACOBI_CG), (nhmf.NHMF_ON_THE_FLY, nhmf.NHMF_SOLVER_MIXED_FCG)):
        prob = nhmf.Problem(n_el, p, mu, kappa, 2, model=nhmf.NHMF_MODEL_SPLIT)
        u = cuda(np.zeros(op.mesh.n_dofs))
        st = prob.solve(u, solver=solver, strategy=strat, load_steps=S, compression=comp, linear_rtol=1e-10)
        assert all(r <= 1e-8 for r in st["rel_residual"])
        assert rel_l2(host(u), u_ref) <= 1e-7


@pytest.mark.parametrize("p", [1, 2, 3])
def test_inclusions_every_operator(nhmf, p):
    import torch
    n_el = 8
    w = inp.Workload("inc", n_el, p, 1.0, 1.5, 1, "scaled", 0.03, "normal", 1.0, 5300 + p, 5400 + p)
    u, du = inp.draw_u(w), inp.draw_du(w)
    f = inp.inclusion_factors(n_el, 100.0)
    op = Operator(Mesh(n_el, p), 1.0, 1.5, 1, factors=f)
    prob = nhmf.Problem.from_workload(w)
    nhmf.nhmf_set_material_factors(prob.ctx, cuda(f))
    prob.set_linearization(cuda(u), nhmf.NHMF_CACHE_FP64 | nhmf.NHMF_CACHE_FP32 | nhmf.NHMF_CACHE_DF64 |
                           nhmf.NHMF_CACHE_SPATIAL)
    ref = op.apply(u, du)
    for prec, strat in ((0, 0), (0, 1), (0, 2), (2, 1)):
        v = cuda(np.zeros_like(u))
        prob.apply(cuda(du), v, prec, strat)
        assert rel_l2(host(v), ref) <= 1e-12, (prec, strat)
    for strat in (0, 1):
        v32 = cuda(np.zeros(u.size, dtype=np.float32))
        prob.apply(cuda(du.astype(np.float32)), v32, nhmf.NHMF_FP32, strat)
        assert rel_l2(host(v32), ref) <= 1e-5
    r = cuda(np.zeros_like(u))
    prob.residual(cuda(u), r)
    assert rel_l2(host(r), op.residual(u)) <= 1e-12
    d = cuda(np.zeros_like(u))
    prob.diagonal(d)
    assert rel_l2(host(d), op.diagonal(u)) <= 1e-12
    nhmf.nhmf_set_material_factors(prob.ctx, None)        # back to the homogeneous material
    v = cuda(np.zeros_like(u))
    prob.apply(cuda(du), v, 0, 1)
    assert rel_l2(host(v), Operator(Mesh(n_el, p), 1.0, 1.5, 1).apply(u, du)) <= 1e-12


def test_inclusions_newton_with_multigrid_matches_oracle(nhmf):
    n_el, p, S, comp = 8, 1, 2, 0.05
    f = inp.inclusion_factors(n_el, 100.0)
    op = Operator(Mesh(n_el, p), 1.0, 1.5, bc=2, factors=f)
    u_ref, _ = newton_load_steps(op, steps=S, compression=comp)
    for solver in (nhmf.NHMF_SOLVER_JACOBI_CG, nhmf.NHMF_SOLVER_MIXED_GMG):
        prob = nhmf.Problem(n_el, p, 1.0, 1.5, 2)
        nhmf.nhmf_set_material_factors(prob.ctx, cuda(f))
        u = cuda(np.zeros(op.mesh.n_dofs))
        st = prob.solve(u, solver=solver, load_steps=S, compression=comp, linear_rtol=1e-10)
        assert all(r <= 1e-8 for r in st["rel_residual"])
        assert rel_l2(host(u), u_ref) <= 1e-7, solver
