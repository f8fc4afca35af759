"""The allocation-free Jacobi-CG entry point (nhmf_linear_solve_noalloc), for callers that
cannot allocate device memory once running (memory owned by a pool, loops that must avoid
cudaMalloc's implicit synchronisation, hosts that forbid allocation after start-up).

Called through the C ABI and checked against the allocating nhmf_linear_solve (Jacobi-CG)
on two calls in a row: the static scratch keeps the previous call's contents, so the second
call shows that the entry point clears what must start at zero.  This file sorts last so
that a stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest

import nhmf_inputs as inp
from tests.gpu_util import cuda, host, lib_or_fail, rel_l2

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def test_noalloc_solve_matches_allocating_solve_twice():
    nhmf = lib_or_fail()
    w = inp.small(inp.WORKLOADS["q2_64_clamp"], 8)          # Q2 8^3: 14,739 DoFs
    u = inp.draw_u(w)
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(u), nhmf.NHMF_CACHE_FP64)
    opts = nhmf.nhmf_solve_opts_default(solver=nhmf.NHMF_SOLVER_JACOBI_CG, linear_rtol=1e-10,
                                        linear_max_iter=5000, check_every=10)
    for call, (seed, strat) in enumerate([(91, nhmf.NHMF_CACHED), (92, nhmf.NHMF_ON_THE_FLY)]):
        b = cuda(inp.draw_vector(seed, w.n_dofs))
        opts.strategy = strat
        x_ref = cuda(np.zeros(w.n_dofs))
        it_ref, _, rel_ref = nhmf.nhmf_linear_solve(prob.ctx, opts, b, x_ref)
        x = cuda(np.full(w.n_dofs, np.nan))
        it, rel = nhmf.nhmf_linear_solve_noalloc(prob.ctx, strat, 1e-10, 5000, b, x)
        assert rel <= 2e-10, (call, rel)
        assert it == it_ref, (call, it, it_ref)
        assert rel_l2(host(x), host(x_ref)) <= FP64_TOL, call
        assert abs(rel - rel_ref) <= 1e-12


def test_noalloc_solve_allocates_no_device_memory():
    """Free device memory is unchanged across two calls on a context whose size no allocating
    solve has used (the allocating solve first runs on another size, so that every kernel the
    calls launch is already loaded), and an x that aliases b is rejected."""
    import torch
    nhmf = lib_or_fail()
    warm = inp.small(inp.WORKLOADS["q2_64_clamp"], 5)
    pw = nhmf.Problem.from_workload(warm)
    pw.set_linearization(cuda(inp.draw_u(warm)), nhmf.NHMF_CACHE_FP64)
    opts = nhmf.nhmf_solve_opts_default(solver=nhmf.NHMF_SOLVER_JACOBI_CG, linear_rtol=1e-8,
                                        linear_max_iter=2000, check_every=10)
    for strat in (nhmf.NHMF_CACHED, nhmf.NHMF_ON_THE_FLY):
        opts.strategy = strat
        nhmf.nhmf_linear_solve(pw.ctx, opts, cuda(inp.draw_vector(93, warm.n_dofs)), cuda(np.zeros(warm.n_dofs)))
    w = inp.small(inp.WORKLOADS["q2_64_clamp"], 7)          # Q2 7^3: 10,125 DoFs
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(inp.draw_u(w)), nhmf.NHMF_CACHE_FP64)
    b = cuda(inp.draw_vector(94, w.n_dofs))
    x = cuda(np.zeros(w.n_dofs))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for strat in (nhmf.NHMF_CACHED, nhmf.NHMF_ON_THE_FLY):
        it, rel = nhmf.nhmf_linear_solve_noalloc(prob.ctx, strat, 1e-8, 2000, b, x)
        assert rel <= 1e-8 and it > 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, strat
    with pytest.raises(nhmf.NhmfError) as ei:
        nhmf.nhmf_linear_solve_noalloc(prob.ctx, nhmf.NHMF_CACHED, 1e-8, 10, b, b)
    assert ei.value.status == 1


def test_noalloc_rejects_problems_beyond_the_scratch_limit():
    nhmf = lib_or_fail()
    w = inp.small(inp.WORKLOADS["q2_64_clamp"], 20)         # 206,763 DoFs > 131,072
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(inp.draw_u(w)), 0)
    b = cuda(np.ones(w.n_dofs))
    x = cuda(np.zeros(w.n_dofs))
    with pytest.raises(nhmf.NhmfError) as ei:
        nhmf.nhmf_linear_solve_noalloc(prob.ctx, nhmf.NHMF_ON_THE_FLY, 1e-8, 10, b, x)
    assert ei.value.status == 1 and "131072" in str(ei.value)
