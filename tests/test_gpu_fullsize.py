"""Parity at the full sizes of the benchmark workloads — Q2 64^3 and Q4 32^3 (6,440,067 DoFs
each), Q3 48^3 (9,145,875) and Q4 64^3 (50,923,779), the last two near-incompressible
(lambda 49) with the compression boundary conditions — in the launch configuration the
benchmark times, on sampled output rows the oracle computes one by one (its
apply_rows/residual_rows/diagonal_rows touch only the elements around each sampled DoF)."""
import numpy as np
import pytest

import nhmf_inputs as inp
from oracle.fem import Operator
from oracle.mesh import Mesh
from tests.gpu_util import cuda, host, lib_or_fail

pytestmark = pytest.mark.gpu


def sample_rows(w, count=400, seed=5):
    rng = np.random.default_rng(seed)
    m = w.n_nodes_1d
    rows = list(rng.choice(w.n_dofs, count, replace=False))
    # boundary and corner rows too: face x = 0 (Dirichlet), x = 1, the last DoF
    for c in range(3):
        rows += [c * m ** 3 + 0, c * m ** 3 + m - 1, c * m ** 3 + m ** 3 - 1, c * m ** 3 + (m // 2) * (1 + m + m * m)]
    return np.array(sorted(set(int(r) for r in rows)))


@pytest.mark.parametrize("name", ["q2_64_clamp", "q4_32_clamp", "q3_48_compress", "q4_64_compress"])
def test_fullsize_sampled_rows(name):
    import torch
    nhmf = lib_or_fail()
    w = inp.WORKLOADS[name]
    u, du = inp.draw_u(w), inp.draw_du(w)
    op = Operator(Mesh(w.n_el, w.degree), w.mu, w.lam, w.bc)
    rows = sample_rows(w)
    ref = op.apply_rows(u, du, rows)
    rref = op.residual_rows(u, rows)
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(u), nhmf.NHMF_CACHE_FP64 | nhmf.NHMF_CACHE_FP32 | nhmf.NHMF_CACHE_DF64 |
                           nhmf.NHMF_CACHE_SPATIAL)
    dut = cuda(du)
    idx = torch.from_numpy(rows).to("cuda:0")
    for strat in (nhmf.NHMF_ON_THE_FLY, nhmf.NHMF_CACHED):
        v = torch.empty_like(dut)
        prob.apply(dut, v, nhmf.NHMF_FP64, strat)
        got = host(v[idx])
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
        v32 = torch.empty(dut.shape, dtype=torch.float32, device="cuda:0")
        prob.apply(dut.float(), v32, nhmf.NHMF_FP32, strat)
        got32 = host(v32[idx])
        assert np.linalg.norm(got32 - ref) <= 1e-5 * np.linalg.norm(ref)
    vsp = torch.empty_like(dut)
    prob.apply(dut, vsp, nhmf.NHMF_FP64, nhmf.NHMF_SPATIAL)
    assert np.linalg.norm(host(vsp[idx]) - ref) <= 1e-12 * np.linalg.norm(ref)
    vdf = torch.empty_like(dut)
    prob.apply(dut, vdf, nhmf.NHMF_DF64, nhmf.NHMF_CACHED)
    assert np.linalg.norm(host(vdf[idx]) - ref) <= 1e-12 * np.linalg.norm(ref)
    r = torch.empty_like(dut)
    prob.residual(cuda(u), r)
    assert np.linalg.norm(host(r[idx]) - rref) <= 1e-12 * np.linalg.norm(rref)
    d = torch.empty_like(dut)
    prob.diagonal(d)
    assert torch.isfinite(d).all()
    dref = op.diagonal_rows(u, rows)
    assert np.linalg.norm(host(d[idx]) - dref) <= 1e-12 * np.linalg.norm(dref)
    prob.close()


def test_fullsize_newton_step_oracle_rows():
    """One load step of the Q2 64^3 compression problem (6,440,067 DoFs), solved to the 1e-8
    relative Newton tolerance by the mixed-precision multigrid solver and by plain FP64
    Jacobi-CG: the oracle's FP64 residual on sampled rows of each solved state is at the
    solver's tolerance, and both states agree."""
    import torch
    nhmf = lib_or_fail()
    w = inp.WORKLOADS["q2_64_compress"]
    op = Operator(Mesh(w.n_el, w.degree), w.mu, w.lam, w.bc)
    rows = sample_rows(w, count=64)
    prob = nhmf.Problem.from_workload(w)
    states = {}
    for name, sid in (("mixed_gmg", nhmf.NHMF_SOLVER_MIXED_GMG), ("plain", nhmf.NHMF_SOLVER_JACOBI_CG)):
        u = torch.zeros(w.n_dofs, dtype=torch.float64, device="cuda:0")
        st = prob.solve(u, solver=sid, load_steps=w.load_steps, compression=w.compression, first_step=1,
                        last_step=1, linear_rtol=1e-8)
        assert st["rel_residual"][0] <= 1e-8
        uu = host(u)
        R = op.residual_rows(uu, rows)
        scale = np.abs(op.apply_rows(uu, uu, rows)).max()
        assert np.abs(R).max() <= 1e-9 * scale, name
        states[name] = uu
    prob.close()
    a, b = states["mixed_gmg"], states["plain"]
    assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)
