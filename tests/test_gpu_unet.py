"""The GPU U-Net against the oracle network: forward output, loss and parameter gradients
on the same weights and inputs.  The GPU stores weights, activations and activation
gradients in BF16 and accumulates in FP32; the oracle (quant=True) rounds to BF16 at the same
places and computes in FP64, so both take the ReLU decisions in the same precision.  What
remains is FP32 versus FP64 accumulation (about 1e-7 relative), which now and then moves a
stored value across a BF16 rounding boundary (one BF16 ulp, 2^-8); the bars are 2e-3 on the
forward output and loss and 1e-2 on each gradient tensor."""
import numpy as np
import pytest

import nhmf_inputs as inp
from oracle import unet as ounet
from oracle.mesh import Mesh
from tests.gpu_util import cuda, host, lib_or_fail, rel_l2

pytestmark = pytest.mark.gpu


def flat_params(params):
    out = []
    for name, kind, cin, cout in ounet.LAYERS:
        out.append(params[name + ".w"].reshape(-1))
        out.append(params[name + ".b"].reshape(-1))
    return np.concatenate(out)


def unflat(vec):
    out, k = {}, 0
    for name, kind, cin, cout in ounet.LAYERS:
        shape = ounet.weight_shape(kind, cin, cout)
        n = int(np.prod(shape))
        out[name + ".w"] = vec[k:k + n].reshape(shape); k += n
        out[name + ".b"] = vec[k:k + cout]; k += cout
    return out


def he_params(seed=5000, bias_scale=0.05):
    p = ounet.init_params(lambda k, n: inp.normal(seed + k, n))
    for i, (name, _, _, cout) in enumerate(ounet.LAYERS):
        p[name + ".b"] = bias_scale * inp.normal(seed + 100 + i, cout)
    return p


@pytest.fixture(scope="module")
def nhmf():
    return lib_or_fail()


@pytest.mark.parametrize("n_el,p,bc", [(4, 2, 2), (8, 2, 1), (4, 4, 0)])
def test_forward_loss_and_gradients_match_oracle(nhmf, n_el, p, bc):
    M = p * n_el + 1
    prob = nhmf.Problem(n_el, p, 1.0, 1.5, bc)
    nhmf.nhmf_unet_create(prob.ctx, 0)
    params = he_params()
    flat = flat_params(params)
    assert flat.size == nhmf.nhmf_unet_num_params(prob.ctx)
    nhmf.nhmf_unet_set_params(prob.ctx, flat)
    assert np.array_equal(nhmf.nhmf_unet_get_params(prob.ctx), flat.astype(np.float32))
    # oracle weights are the FP32 master weights rounded as the GPU stores them (BF16)
    x = inp.normal(11, 3 * M ** 3).astype(np.float32)
    e = inp.normal(12, 3 * M ** 3).astype(np.float32)
    xt, et = cuda(x), cuda(e)
    y = cuda(np.zeros(3 * M ** 3, dtype=np.float32))
    nhmf.nhmf_unet_forward(prob.ctx, xt, y)
    xo = x.astype(np.float64).reshape(3, M, M, M)
    eo = e.astype(np.float64).reshape(3, M, M, M)
    yo, acts = ounet.forward(params, xo, quant=True)
    assert rel_l2(host(y), yo.reshape(-1)) <= 2e-3
    free = (~Mesh(n_el, p).constrained(bc)).astype(np.float64).reshape(3, M, M, M)
    loss, g = nhmf.nhmf_unet_loss_grad(prob.ctx, xt, et)
    lo = ounet.loss(yo, eo, free)
    assert abs(loss - lo) <= 2e-3 * lo
    go = ounet.backward(params, acts, yo, eo, free, quant=True)
    gg = unflat(g.astype(np.float64))
    errs = {k: rel_l2(gg[k].reshape(-1), go[k].reshape(-1)) for k in go}
    assert max(errs.values()) <= 1e-2, errs


def test_adam_step_matches_oracle(nhmf):
    n_el, p, bc = 4, 2, 2
    M = p * n_el + 1
    prob = nhmf.Problem(n_el, p, 1.0, 1.5, bc)
    nhmf.nhmf_unet_create(prob.ctx, 4)
    params = he_params()
    nhmf.nhmf_unet_set_params(prob.ctx, flat_params(params))
    r = inp.normal(21, 3 * M ** 3)
    e = inp.normal(22, 3 * M ** 3)
    free = ~Mesh(n_el, p).constrained(bc)
    r[~free] = 0.0
    e[~free] = 0.0
    nhmf.nhmf_unet_record_pair(prob.ctx, cuda(r), cuda(e))
    assert nhmf.nhmf_unet_num_pairs(prob.ctx) == 1
    l0, l1 = nhmf.nhmf_unet_train(prob.ctx, 1, 1e-3)
    # oracle: the same pair normalised to unit RMS, one Adam step from the same weights
    xo = (r * np.sqrt(r.size) / np.linalg.norm(r)).reshape(3, M, M, M)
    eo = (e * np.sqrt(e.size) / np.linalg.norm(e)).reshape(3, M, M, M)
    yo, acts = ounet.forward(params, xo, quant=True)
    assert abs(l0 - ounet.loss(yo, eo, free.reshape(3, M, M, M).astype(float))) <= 2e-3 * l0
    go = ounet.backward(params, acts, yo, eo, free.reshape(3, M, M, M).astype(float), quant=True)
    st = {}
    p2 = {k: v.copy() for k, v in params.items()}
    ounet.adam_step(p2, go, st, lr=1e-3)
    new = unflat(nhmf.nhmf_unet_get_params(prob.ctx).astype(np.float64))
    # the first Adam step moves each weight by about lr * sign(g): compare the step direction
    for k in ("in.w", "e0.w", "m2.w", "out.w"):
        d_gpu = new[k] - params[k]
        d_ora = p2[k] - params[k]
        agree = np.mean(np.sign(d_gpu) == np.sign(d_ora))
        assert agree >= 0.9, (k, agree)


def test_training_reduces_loss_and_learned_solve_converges(nhmf):
    import torch
    n_el, p, S, comp = 4, 2, 4, 0.08
    prob = nhmf.Problem(n_el, p, 1.0, 1.5, 2)
    nhmf.nhmf_unet_create(prob.ctx, 64)
    nhmf.nhmf_unet_set_params(prob.ctx, flat_params(he_params()))
    n = 3 * (p * n_el + 1) ** 3
    u = cuda(np.zeros(n))
    prob.solve(u, load_steps=S, compression=comp, last_step=2, record_pairs=1, cg_pair_every=4)
    assert nhmf.nhmf_unet_num_pairs(prob.ctx) > 4
    l0, l1 = nhmf.nhmf_unet_train(prob.ctx, 20, 1e-3)
    assert l1 < l0
    u_plain = u.clone()
    prob.solve(u_plain, load_steps=S, compression=comp, first_step=3, linear_rtol=1e-8)
    u_learn = u.clone()
    st = prob.solve(u_learn, load_steps=S, compression=comp, first_step=3, linear_rtol=1e-8,
                    solver=nhmf.NHMF_SOLVER_LEARNED_FCG)
    assert all(r <= 1e-8 for r in st["rel_residual"])
    assert rel_l2(host(u_learn), host(u_plain)) <= 1e-6
