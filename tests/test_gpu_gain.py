"""What the trained U-Net gains over the solvers without it.

Compression of a Q2 16^3 cube (20 load steps of 0.5 %).  Load steps 1-5 run the plain FP64
Jacobi-CG solver and record training pairs (Newton (b, du), CG (r_j, x* - x_j), and
(K e, e) for random fields e at one lattice scale each); the network is trained on them;
steps 6-20 then run with and without it from the same state.  Every solver must reach the
same 1e-8 Newton tolerance and the same equilibrium; the iteration counts and times of each
are printed (the measured gain, which may be below 1), not asserted."""
import json
import time

import numpy as np
import pytest

from tests.gpu_util import cuda, host, lib_or_fail, rel_l2

pytestmark = pytest.mark.gpu


def test_learned_preconditioner_gain_is_measured():
    import torch
    from tests.unet_cases import flat_params, he_params
    nhmf = lib_or_fail()
    n_el, p, S, comp = 16, 2, 20, 0.1
    n = 3 * (p * n_el + 1) ** 3
    prob = nhmf.Problem(n_el, p, 1.0, 1.5, 2)
    nhmf.nhmf_unet_create(prob.ctx, 600)
    nhmf.nhmf_unet_set_params(prob.ctx, flat_params(he_params()))
    u = cuda(np.zeros(n))
    prob.solve(u, load_steps=S, compression=comp, last_step=5, record_pairs=1, cg_pair_every=8, synthetic_pairs=20)
    l0, l1 = nhmf.nhmf_unet_train(prob.ctx, 30, 1e-3)
    assert l1 < 0.5 * l0
    results, finals = {}, {}
    for name, solver in [("plain", nhmf.NHMF_SOLVER_JACOBI_CG), ("mixed", nhmf.NHMF_SOLVER_MIXED_FCG),
                         ("learned", nhmf.NHMF_SOLVER_LEARNED_FCG), ("mixed_learned", nhmf.NHMF_SOLVER_MIXED_LEARNED)]:
        uu = u.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = prob.solve(uu, load_steps=S, compression=comp, first_step=6, linear_rtol=1e-8, solver=solver)
        torch.cuda.synchronize()
        results[name] = {"seconds": time.perf_counter() - t0, "outer_iters": st["total_linear_iters"],
                         "inner_iters": st["total_inner_iters"], "fallbacks": sum(st["fallbacks"])}
        assert all(r <= 1e-8 for r in st["rel_residual"]), name
        finals[name] = host(uu)
    for name in results:
        assert rel_l2(finals[name], finals["plain"]) <= 1e-6, name
        results[name]["time_vs_plain"] = results[name]["seconds"] / results["plain"]["seconds"]
    print(json.dumps({"train_loss": [l0, l1], "solvers": results}))


def test_learned_multigrid_correction_gain_is_measured():
    """The network as a correction on top of the FP32 multigrid V-cycle V,
    z = V(r) + N(r - A V(r)), trained on the pairs (r_j - A V(r_j), x* - x_j - V(r_j)) that the
    mixed multigrid solves of load steps 1-5 record; steps 6-12 then run with and without the
    correction from the same state.  Both reach the 1e-8 Newton tolerance and the same
    equilibrium; iterations and times are printed (the measured ratio, which may be below 1)."""
    import torch
    nhmf = lib_or_fail()
    n_el, p, S, comp = 16, 2, 20, 0.1
    n = 3 * (p * n_el + 1) ** 3
    prob = nhmf.Problem(n_el, p, 1.0, 1.5, 2)
    nhmf.nhmf_unet_create(prob.ctx, 200)
    from tests.unet_cases import flat_params, he_params
    nhmf.nhmf_unet_set_params(prob.ctx, flat_params(he_params()))
    u = cuda(np.zeros(n))
    prob.solve(u, load_steps=S, compression=comp, last_step=5, solver=nhmf.NHMF_SOLVER_MIXED_GMG, record_pairs=1,
               cg_pair_every=4, linear_rtol=1e-8)
    npairs = nhmf.nhmf_unet_num_pairs(prob.ctx)
    assert npairs >= 10
    l0, l1 = nhmf.nhmf_unet_train(prob.ctx, 20, 1e-3)
    assert l1 < l0
    results, finals = {}, {}
    for name, solver in [("mixed_gmg", nhmf.NHMF_SOLVER_MIXED_GMG), ("mixed_gmg_learned", nhmf.NHMF_SOLVER_MIXED_GMG_LEARNED)]:
        uu = u.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = prob.solve(uu, load_steps=S, compression=comp, first_step=6, last_step=12, linear_rtol=1e-8, solver=solver)
        torch.cuda.synchronize()
        results[name] = {"seconds": time.perf_counter() - t0, "outer_iters": st["total_linear_iters"],
                         "vcycles": st["total_linear_iters"], "fallbacks": sum(st["fallbacks"])}
        assert all(r <= 1e-8 for r in st["rel_residual"]), name
        finals[name] = host(uu)
    assert rel_l2(finals["mixed_gmg_learned"], finals["mixed_gmg"]) <= 1e-6
    results["mixed_gmg_learned"]["time_vs_mixed_gmg"] = results["mixed_gmg_learned"]["seconds"] / results["mixed_gmg"]["seconds"]
    print(json.dumps({"pairs": npairs, "train_loss": [l0, l1], "solvers": results}))
