"""Parity of the CUDA tangent application, residual and diagonal with the FP64 oracle
(Eq. F, Eq. DF, Algorithm 1, Section 2.3).  Bar: FP64 relative l2 <= 1e-12; FP32 results
report their error and must stay within 1e-5 (FP32 sum factorisation with FP32 accumulation
over at most (p+1)^3-term contractions and one conditioning factor of the operator)."""
import numpy as np
import pytest

import nhmf_inputs as inp
from oracle.fem import Operator
from oracle.mesh import Mesh
from tests.gpu_util import cuda, host, lib_or_fail, rel_l2

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


def case(n_el, p, bc, lam=1.5, seed=0, amp=0.05):
    w = inp.Workload(f"t{n_el}_{p}_{bc}", n_el, p, 1.0, lam, bc, "scaled", amp, "normal", 1.0,
                     3000 + seed + 10 * p + 100 * n_el, 4000 + seed + 10 * p + 100 * n_el)
    return w, inp.draw_u(w), inp.draw_du(w)


@pytest.fixture(scope="module")
def nhmf():
    return lib_or_fail()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("n_el", [1, 3, 5])
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_fp64_apply_both_strategies(nhmf, p, n_el, bc):
    w, u, du = case(n_el, p, bc)
    op = Operator(Mesh(n_el, p), w.mu, w.lam, bc)
    ref = op.apply(u, du)
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(u), nhmf.NHMF_CACHE_FP64 | nhmf.NHMF_CACHE_FP32 | nhmf.NHMF_CACHE_DF64 |
                           nhmf.NHMF_CACHE_SPATIAL)
    dut = cuda(du)
    for strat in (nhmf.NHMF_ON_THE_FLY, nhmf.NHMF_CACHED, nhmf.NHMF_SPATIAL):
        v = cuda(np.zeros_like(u))
        prob.apply(dut, v, nhmf.NHMF_FP64, strat)
        assert rel_l2(host(v), ref) <= FP64_TOL, (strat, rel_l2(host(v), ref))
    vdf = cuda(np.zeros_like(u))                  # double-float arithmetic: same FP64 bar
    prob.apply(dut, vdf, nhmf.NHMF_DF64, nhmf.NHMF_CACHED)
    assert rel_l2(host(vdf), ref) <= FP64_TOL, ("df64", rel_l2(host(vdf), ref))
    for strat in (nhmf.NHMF_ON_THE_FLY, nhmf.NHMF_CACHED):
        v32 = cuda(np.zeros(u.size, dtype=np.float32))
        prob.apply(cuda(du.astype(np.float32)), v32, nhmf.NHMF_FP32, strat)
        assert rel_l2(host(v32), ref) <= FP32_TOL, (strat, rel_l2(host(v32), ref))
    prob.close()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("model", [0, 1])
def test_apply_at_given_point(nhmf, p, model):
    """nhmf_tangent_apply_at (Algorithm 1 with u given): equals the oracle at that u without a
    stored linearisation point, leaves a stored one untouched, and is bitwise the same as
    setting u and applying on the fly."""
    w, u, du = case(3, p, 1)
    lam = w.lam if model == 0 else 5.0
    op = Operator(Mesh(3, p), w.mu, lam, 1, model=model)
    prob = nhmf.Problem(3, p, w.mu, lam, 1, model=model)
    ut, dut = cuda(u), cuda(du)
    v_at = cuda(np.zeros_like(u))
    prob.apply_at(ut, dut, v_at)                  # no set_linearization before
    assert rel_l2(host(v_at), op.apply(u, du)) <= FP64_TOL
    u2 = 0.5 * u
    prob.set_linearization(cuda(u2))
    v2 = cuda(np.zeros_like(u))
    prob.apply_at(ut, dut, v2)
    assert np.array_equal(host(v2), host(v_at))
    v_stored = cuda(np.zeros_like(u))
    prob.apply(dut, v_stored, nhmf.NHMF_FP64, nhmf.NHMF_ON_THE_FLY)   # still linearised at u2
    assert rel_l2(host(v_stored), op.apply(u2, du)) <= FP64_TOL
    prob.set_linearization(ut)
    v_set = cuda(np.zeros_like(u))
    prob.apply(dut, v_set, nhmf.NHMF_FP64, nhmf.NHMF_ON_THE_FLY)
    assert np.array_equal(host(v_set), host(v_at))
    with pytest.raises(nhmf.NhmfError):
        prob.apply_at(ut, dut, dut)                   # v aliasing du
    prob.close()


def test_q1_8_clamp_workload(nhmf):
    w = inp.WORKLOADS["q1_8_clamp"]
    u, du = inp.draw_u(w), inp.draw_du(w)
    ref = Operator(Mesh(w.n_el, w.degree), w.mu, w.lam, w.bc).apply(u, du)
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(u))
    v = cuda(np.zeros_like(u))
    prob.apply(cuda(du), v, nhmf.NHMF_FP64, nhmf.NHMF_ON_THE_FLY)
    assert rel_l2(host(v), ref) <= FP64_TOL


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("bc", [0, 1, 2])
def test_fp64_residual(nhmf, p, bc):
    w, u, _ = case(4, p, bc)
    ref = Operator(Mesh(4, p), w.mu, w.lam, bc).residual(u)
    prob = nhmf.Problem.from_workload(w)
    r = cuda(np.zeros_like(u))
    prob.residual(cuda(u), r)
    assert rel_l2(host(r), ref) <= FP64_TOL


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("bc", [0, 2])
def test_fp64_diagonal(nhmf, p, bc):
    w, u, _ = case(3, p, bc)
    ref = Operator(Mesh(3, p), w.mu, w.lam, bc).diagonal(u)
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(u))
    d = cuda(np.zeros_like(u))
    prob.diagonal(d)
    assert rel_l2(host(d), ref) <= FP64_TOL


@pytest.mark.parametrize("n_el,p", [(1, 1), (2, 1), (1, 2), (2, 2), (3, 1), (1, 3), (1, 4)])
def test_columns_match_assembled_matrix(nhmf, n_el, p):
    import torch
    w, u, _ = case(n_el, p, 1)
    op = Operator(Mesh(n_el, p), w.mu, w.lam, 1)
    K = op.assemble(u)
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(u), nhmf.NHMF_CACHE_FP64)
    n = u.size
    cols = np.arange(n) if n <= 400 else np.random.default_rng(1).choice(n, 400, replace=False)
    for strat in (nhmf.NHMF_ON_THE_FLY, nhmf.NHMF_CACHED):
        for j in cols:
            e = torch.zeros(n, dtype=torch.float64, device="cuda:0")
            e[j] = 1.0
            v = torch.empty_like(e)
            prob.apply(e, v, nhmf.NHMF_FP64, strat)
            col = host(v)
            assert np.abs(col - K[:, j]).max() <= 1e-12 * np.abs(K).max()


def test_bitwise_determinism(nhmf):
    import torch
    w, u, du = case(6, 2, 1)
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(u), nhmf.NHMF_CACHE_FP64 | nhmf.NHMF_CACHE_FP32 | nhmf.NHMF_CACHE_DF64)
    for prec, dt in ((nhmf.NHMF_FP64, np.float64), (nhmf.NHMF_FP32, np.float32)):
        for strat in (nhmf.NHMF_ON_THE_FLY, nhmf.NHMF_CACHED):
            dut = cuda(du.astype(dt))
            outs = []
            for _ in range(10):
                v = torch.empty_like(dut)
                prob.apply(dut, v, prec, strat)
                outs.append(v.clone())
            for o in outs[1:]:
                assert torch.equal(o, outs[0])


def test_bitwise_determinism_fp32_register_kernel(nhmf):
    """Q2 64^3: the one-thread-per-element FP32 kernel and the node gather, 10 applies each."""
    import torch
    w = inp.WORKLOADS["q2_64_clamp"]
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(inp.draw_u(w)), nhmf.NHMF_CACHE_FP32)
    dut = cuda(inp.draw_du(w).astype(np.float32))
    for strat in (nhmf.NHMF_ON_THE_FLY, nhmf.NHMF_CACHED):
        first = torch.empty_like(dut)
        prob.apply(dut, first, nhmf.NHMF_FP32, strat)
        for _ in range(9):
            v = torch.empty_like(dut)
            prob.apply(dut, v, nhmf.NHMF_FP32, strat)
            assert torch.equal(v, first)
    prob.close()


@pytest.mark.parametrize("p", [2, 3])
def test_fp32_error_near_incompressibility(nhmf, p):
    """lambda = 49 under 10 % compression (J ~ 0.9, so 2 lambda / mu ln J ~ -10): the FP32 on-the-fly
    apply forms J - 1 and ln J in FP32 from the FP32 displacement gradient, the cached one reads
    them computed in FP64.  Both stay within the FP32 bar; their errors are printed."""
    n_el = 6
    w = inp.Workload(f"c{p}", n_el, p, 1.0, 49.0, inp.BC_COMPRESSION, "scaled", 0.02, "normal", 1.0, 5100 + p, 5200 + p)
    m = Mesh(n_el, p)
    X = m.node_coords()
    u = inp.draw_u(w) + np.concatenate([0.0 * X[:, 0], 0.0 * X[:, 1], -0.1 * X[:, 2]])
    du = inp.draw_du(w)
    ref = Operator(m, w.mu, w.lam, w.bc).apply(u, du)
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(u), nhmf.NHMF_CACHE_FP32)
    errs = {}
    for name, strat in (("otf", nhmf.NHMF_ON_THE_FLY), ("cached", nhmf.NHMF_CACHED)):
        v32 = cuda(np.zeros(u.size, dtype=np.float32))
        prob.apply(cuda(du.astype(np.float32)), v32, nhmf.NHMF_FP32, strat)
        errs[name] = rel_l2(host(v32), ref)
    print(f"FP32 apply error at lambda 49, 10 % compression, Q{p}: {errs}")
    assert max(errs.values()) <= FP32_TOL, errs
    prob.close()


def test_strategies_agree(nhmf):
    w, u, du = case(5, 3, 2, lam=49.0)
    prob = nhmf.Problem.from_workload(w)
    prob.set_linearization(cuda(u), nhmf.NHMF_CACHE_FP64)
    a = cuda(np.zeros_like(u)); b = cuda(np.zeros_like(u))
    prob.apply(cuda(du), a, nhmf.NHMF_FP64, nhmf.NHMF_ON_THE_FLY)
    prob.apply(cuda(du), b, nhmf.NHMF_FP64, nhmf.NHMF_CACHED)
    assert rel_l2(host(a), host(b)) <= 1e-13


def test_nonpositive_jacobian_is_reported(nhmf):
    w, u, _ = case(3, 2, 0)
    prob = nhmf.Problem.from_workload(w)
    bad = u.copy()
    bad[: bad.size // 3] *= -3000.0       # folds elements: det F <= 0 somewhere
    with pytest.raises(nhmf.NhmfError) as ei:
        prob.set_linearization(cuda(bad), nhmf.NHMF_CACHE_FP64)
    assert ei.value.status == 4
    r = cuda(np.zeros_like(u))
    with pytest.raises(nhmf.NhmfError) as ei:
        prob.residual(cuda(bad), r)
    assert ei.value.status == 4
    prob.set_linearization(cuda(u), nhmf.NHMF_CACHE_FP64)  # the context stays usable


def test_call_order_and_argument_errors(nhmf):
    w, u, du = case(2, 1, 1)
    prob = nhmf.Problem.from_workload(w)
    v = cuda(np.zeros_like(u))
    with pytest.raises(nhmf.NhmfError) as ei:
        prob.apply(cuda(du), v)
    assert ei.value.status == 8
    prob.set_linearization(cuda(u), 0)
    with pytest.raises(nhmf.NhmfError) as ei:
        prob.apply(cuda(du), v, nhmf.NHMF_FP64, nhmf.NHMF_CACHED)
    assert ei.value.status == 8
    with pytest.raises(nhmf.NhmfError):
        nhmf.nhmf_create(0, 2, 1.0, 1.5, 0)
    with pytest.raises(nhmf.NhmfError):
        nhmf.nhmf_create(4, 5, 1.0, 1.5, 0)


@pytest.mark.parametrize("p", [1, 2])
def test_fp32_register_kernel_at_64_all_rows(nhmf, p):
    """N = 64: the FP32 applies run the one-thread-per-element kernel over 32-element tiles and
    the node gather; every row against the oracle (Q1), or the rows on and around the tile
    faces, the corners and the Dirichlet planes (Q2), both strategies, all three presets."""
    n_el = 64
    for bc in (0, 1, 2):
        w, u, du = case(n_el, p, bc, seed=7)
        m = Mesh(n_el, p)
        op = Operator(m, w.mu, w.lam, bc)
        if p == 1:
            rows = np.arange(w.n_dofs)
            ref = op.apply(u, du)
        else:
            M = w.n_nodes_1d
            pick = [0, 1, 2, 3, 4, 63, 64, 65, 127, 128, M - 1]     # node planes at tile faces and edges
            nodes = [i + M * (j + M * k) for i in pick for j in pick[:6] + [M - 1] for k in (0, 3, 4, 5, M - 1)]
            rows = np.array(sorted({c * M ** 3 + nd for nd in nodes for c in range(3)}))
            ref = op.apply_rows(u, du, rows)
        prob = nhmf.Problem.from_workload(w)
        prob.set_linearization(cuda(u), nhmf.NHMF_CACHE_FP32)
        for strat in (nhmf.NHMF_ON_THE_FLY, nhmf.NHMF_CACHED):
            v32 = cuda(np.zeros(u.size, dtype=np.float32))
            prob.apply(cuda(du.astype(np.float32)), v32, nhmf.NHMF_FP32, strat)
            got = host(v32)[rows]
            assert rel_l2(got, ref) <= FP32_TOL, (p, bc, strat, rel_l2(got, ref))
        prob.close()
