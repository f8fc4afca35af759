"""The solvers' failure paths, made on the host (include/nhmf.h, "diagnostics"): a NaN in a
Newton update is reported as NHMF_ERR_NONFINITE and the context stays usable; a stalled
flexible Krylov solve and a learned solve whose network returns noise both end in the
Jacobi-CG fallback at the requested tolerance; the flags fire once; the JSONL metrics file
holds one object per Newton iteration, load step, linear solve and apply.  No device fault
is involved: every path runs on data and error codes."""
import json
import os

import numpy as np
import pytest

from tests.gpu_util import cuda, host, lib_or_fail, rel_l2
from tests.unet_cases import flat_params, he_params

pytestmark = pytest.mark.gpu

N_EL, P, S, COMP = 4, 2, 2, 0.08  # Q2 4^3, compression, lambda 1.5: M = 9 (a U-Net grid)


@pytest.fixture(scope="module")
def nhmf():
    return lib_or_fail()


def fresh(nhmf):
    prob = nhmf.Problem(N_EL, P, 1.0, 1.5, nhmf.NHMF_BC_COMPRESSION)
    return prob, cuda(np.zeros(prob.n_dofs))


def test_nan_in_update_is_reported_and_context_recovers(nhmf):
    prob, u = fresh(nhmf)
    nhmf.nhmf_set_inject(prob.ctx, nhmf.NHMF_INJECT_NAN_DU)
    with pytest.raises(nhmf.NhmfError) as e:
        prob.solve(u, load_steps=S, compression=COMP, linear_rtol=1e-10)
    assert e.value.status == 5  # NHMF_ERR_NONFINITE
    assert nhmf.nhmf_inject_pending(prob.ctx) == 0
    assert np.isfinite(host(u)).all()  # u kept its last accepted value
    u2 = cuda(np.zeros(prob.n_dofs))
    st = prob.solve(u2, load_steps=S, compression=COMP, linear_rtol=1e-10)
    assert all(r <= 1e-8 for r in st["rel_residual"])


@pytest.mark.parametrize("solver", ["MIXED_FCG", "MIXED_GMG"])
def test_stalled_flexible_solve_falls_back(nhmf, solver):
    sid = getattr(nhmf, "NHMF_SOLVER_" + solver)
    prob, u_ref = fresh(nhmf)
    prob.solve(u_ref, solver=sid, load_steps=S, compression=COMP, linear_rtol=1e-10)
    prob2, u = fresh(nhmf)
    nhmf.nhmf_set_inject(prob2.ctx, nhmf.NHMF_INJECT_CG_STALL)
    st = prob2.solve(u, solver=sid, load_steps=S, compression=COMP, linear_rtol=1e-10)
    assert nhmf.nhmf_inject_pending(prob2.ctx) == 0
    assert st["fallbacks"][0] >= 1
    assert all(r <= 1e-8 for r in st["rel_residual"])
    assert rel_l2(host(u), host(u_ref)) <= 1e-7


def test_stall_flag_waits_for_a_flexible_solve(nhmf):
    prob, u = fresh(nhmf)
    nhmf.nhmf_set_inject(prob.ctx, nhmf.NHMF_INJECT_CG_STALL)
    prob.solve(u, load_steps=1, compression=COMP, linear_rtol=1e-10)  # Jacobi-CG: not flexible
    assert nhmf.nhmf_inject_pending(prob.ctx) == nhmf.NHMF_INJECT_CG_STALL


def test_network_noise_falls_back_to_jacobi_cg(nhmf):
    prob, u = fresh(nhmf)
    nhmf.nhmf_unet_create(prob.ctx, 0)
    nhmf.nhmf_unet_set_params(prob.ctx, flat_params(he_params()))
    nhmf.nhmf_set_inject(prob.ctx, nhmf.NHMF_INJECT_UNET_GARBAGE)
    st = prob.solve(u, solver=nhmf.NHMF_SOLVER_LEARNED_FCG, load_steps=S, compression=COMP, linear_rtol=1e-10)
    assert nhmf.nhmf_inject_pending(prob.ctx) == 0
    assert st["fallbacks"][0] >= 1
    assert all(r <= 1e-8 for r in st["rel_residual"])
    prob2, u_ref = fresh(nhmf)
    prob2.solve(u_ref, load_steps=S, compression=COMP, linear_rtol=1e-10)
    assert rel_l2(host(u), host(u_ref)) <= 1e-7


def test_set_inject_rejects_unknown_flags(nhmf):
    prob, _ = fresh(nhmf)
    with pytest.raises(nhmf.NhmfError):
        nhmf.nhmf_set_inject(prob.ctx, 8)


def test_environment_sets_flags_at_create(nhmf, monkeypatch):
    monkeypatch.setenv("NHMF_INJECT", "cg_stall,unet_garbage")
    prob, _ = fresh(nhmf)
    assert nhmf.nhmf_inject_pending(prob.ctx) == nhmf.NHMF_INJECT_CG_STALL | nhmf.NHMF_INJECT_UNET_GARBAGE


def test_metrics_jsonl(nhmf, tmp_path):
    path = str(tmp_path / "metrics.jsonl")
    prob, u = fresh(nhmf)
    nhmf.nhmf_set_metrics_log(prob.ctx, path)
    st = prob.solve(u, solver=nhmf.NHMF_SOLVER_MIXED_GMG, load_steps=S, compression=COMP, linear_rtol=1e-10)
    prob.set_linearization(u, nhmf.NHMF_CACHE_FP64)
    v = cuda(np.zeros(prob.n_dofs))
    nhmf.nhmf_tangent_apply(prob.ctx, nhmf.NHMF_FP64, nhmf.NHMF_CACHED, u, v)
    b = cuda(np.ones(prob.n_dofs))
    x = cuda(np.zeros(prob.n_dofs))
    prob.linear_solve(b, x, linear_rtol=1e-8)
    nhmf.nhmf_set_metrics_log(prob.ctx, None)
    lines = [json.loads(l) for l in open(path).read().splitlines()]
    events = [l["event"] for l in lines]
    steps = [l for l in lines if l["event"] == "load_step"]
    iters = [l for l in lines if l["event"] == "newton_iteration"]
    assert len(steps) == S and [s["step"] for s in steps] == [1, 2]
    assert sum(s["newton_iters"] for s in steps) == sum(st["newton_iters"])
    assert len(iters) == sum(st["newton_iters"])
    assert all(s["converged"] for s in steps)
    assert [s["linear_iters"] for s in steps] == list(st["linear_iters"])
    assert all(i["rel_residual"] > 0 and i["seconds"] >= 0 for i in iters)
    for i in iters:  # the iteration's time splits into setup, linear solve and update
        assert min(i["setup_seconds"], i["linear_seconds"], i["update_seconds"]) >= 0
        # each of the four times is printed to 6 decimals: the sum may exceed by 4 x 0.5 us
        assert i["setup_seconds"] + i["linear_seconds"] + i["update_seconds"] <= i["seconds"] + 2.5e-6
    apply = [l for l in lines if l["event"] == "tangent_apply"]
    assert len(apply) == 1 and apply[0]["precision"] == "fp64" and apply[0]["strategy"] == "cached"
    assert apply[0]["ms"] > 0 and apply[0]["gdofs"] > 0 and apply[0]["dofs"] == prob.n_dofs
    lin = [l for l in lines if l["event"] == "linear_solve"]
    assert len(lin) == 1 and lin[0]["rel_residual"] <= 1e-8
    assert events[-1] == "linear_solve"
    size = os.path.getsize(path)
    nhmf.nhmf_tangent_apply(prob.ctx, nhmf.NHMF_FP64, nhmf.NHMF_CACHED, u, v)  # log closed
    assert os.path.getsize(path) == size
