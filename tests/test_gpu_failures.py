"""Failure detection without a GPU fault: bad inputs made on the host surface as status codes
read from the device status word (no trap, no assert); the context stays usable afterwards."""
import numpy as np
import pytest

import nhmf_inputs as inp
from tests.gpu_util import cuda, host, lib_or_fail

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nhmf():
    return lib_or_fail()


def test_nan_in_state_is_reported_as_nonfinite(nhmf):
    w = inp.small(inp.WORKLOADS["q2_64_clamp"], 3)
    u = inp.draw_u(w)
    prob = nhmf.Problem.from_workload(w)
    bad = u.copy()
    bad[bad.size // 2] = np.nan
    r = cuda(np.zeros_like(u))
    with pytest.raises(nhmf.NhmfError) as ei:
        prob.residual(cuda(bad), r)
    assert ei.value.status in (4, 5)          # NaN makes det F or P non-finite
    prob.residual(cuda(u), r)                  # usable afterwards
    assert np.isfinite(host(r)).all()


def test_solver_reports_nonconvergence_within_its_budget(nhmf):
    w = inp.small(inp.WORKLOADS["q2_64_compress"], 4)
    prob = nhmf.Problem.from_workload(w)
    u = cuda(np.zeros(w.n_dofs))
    with pytest.raises(nhmf.NhmfError) as ei:
        prob.solve(u, load_steps=2, compression=0.05, newton_max_iter=1, linear_max_iter=3)
    assert ei.value.status == 7
    assert ei.value.stats["steps_done"] == 1


@pytest.mark.parametrize("n_el,p", [(1, 2), (3, 2), (5, 1), (2, 3)])
def test_multigrid_on_small_and_odd_meshes(nhmf, n_el, p):
    w = inp.Workload("g", n_el, p, 1.0, 1.5, 1, "scaled", 0.01, "normal", 1.0, 6500 + n_el, 6600 + n_el)
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(inp.draw_u(w)), 3)
    b = inp.draw_vector(81, w.n_dofs)
    b[inp.dirichlet_mask(n_el, p, 1).reshape(-1)] = 0.0
    x = cuda(np.zeros(w.n_dofs))
    for solver in (nhmf.NHMF_SOLVER_GMG, nhmf.NHMF_SOLVER_MIXED_GMG):
        it, inner, rel = prob.linear_solve(cuda(b), x, solver=solver, linear_rtol=1e-8)
        assert rel <= 1e-8
