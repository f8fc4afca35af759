"""The GPU U-Net against the oracle network (forward output, loss, parameter gradients,
Adam, training).

Two kinds of parity:
* exact: sparse ternary weights (density 0.006, values -1/0/1, biases 0/1) and inputs in
  {-1, 0, 1} keep every activation, activation gradient and parameter gradient a small
  dyadic number, exactly representable in BF16 and summed exactly in FP32; the GPU must
  then reproduce the oracle bit for bit (this pins every gather, stride and transposition);
* rounded: He-initialised weights and normal inputs.  The GPU stores weights, activations
  and activation gradients in BF16; the oracle (quant=True) rounds at the same places in
  FP64.  One-ulp rounding differences (2^-8) cascade through the 11 layers, so two valid
  BF16 evaluations differ by about sqrt(11) * 2^-9 ~ 2e-3 to 3e-3 relative (each is about
  7.5e-3 from the exact FP64 network); the bars are 1e-2 on the output and loss and 8e-2 on
  each gradient tensor (the coarsest grids sum over 125 to 729 voxels only)."""
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


def ternary_params(seed=7000, density=0.006):
    p = {}
    for i, (name, kind, cin, cout) in enumerate(ounet.LAYERS):
        shape = ounet.weight_shape(kind, cin, cout)
        u = inp.uniform01(seed + i, int(np.prod(shape)))
        p[name + ".w"] = np.where(u < density / 2, -1.0, np.where(u < density, 1.0, 0.0)).reshape(shape)
        p[name + ".b"] = np.minimum(np.floor(inp.uniform01(seed + 50 + i, cout) * 3.0), 1.0)
    return p


@pytest.fixture(scope="module")
def nhmf():
    return lib_or_fail()


def run_gpu(nhmf, n_el, p, bc, params, x, e):
    M = p * n_el + 1
    prob = nhmf.Problem(n_el, p, 1.0, 1.5, bc)
    nhmf.nhmf_unet_create(prob.ctx, 0)
    flat = flat_params(params)
    assert flat.size == nhmf.nhmf_unet_num_params(prob.ctx)
    nhmf.nhmf_unet_set_params(prob.ctx, flat)
    assert np.array_equal(nhmf.nhmf_unet_get_params(prob.ctx), flat.astype(np.float32))
    xt, et = cuda(x.astype(np.float32)), cuda(e.astype(np.float32))
    y = cuda(np.zeros(3 * M ** 3, dtype=np.float32))
    nhmf.nhmf_unet_forward(prob.ctx, xt, y)
    loss, g = nhmf.nhmf_unet_loss_grad(prob.ctx, xt, et)
    return host(y), loss, unflat(g.astype(np.float64))


@pytest.mark.parametrize("n_el,p,bc", [(8, 2, 2), (16, 2, 1), (8, 4, 0)])
def test_exact_arithmetic_bit_parity(nhmf, n_el, p, bc):
    M = p * n_el + 1
    params = ternary_params()
    x = np.floor(inp.uniform01(123, 3 * M ** 3) * 3.0 - 1.0)
    e = np.zeros(3 * M ** 3)
    e[M ** 3 + (M // 2) * (1 + M + M * M)] = 4.0          # ||f e||^2 = 16: dy is dyadic
    y, loss, g = run_gpu(nhmf, n_el, p, bc, params, x, e)
    xo, eo = x.reshape(3, M, M, M), e.reshape(3, M, M, M)
    free = (~Mesh(n_el, p).constrained(bc)).astype(np.float64).reshape(3, M, M, M)
    yo, acts = ounet.forward(params, xo, quant=True)
    assert np.array_equal(y, yo.reshape(-1))
    assert loss == ounet.loss(yo, eo, free)
    go = ounet.backward(params, acts, yo, eo, free, quant=True)
    for k in go:
        assert np.array_equal(g[k], go[k]), k
    assert sum(np.count_nonzero(go[k]) for k in go if k.endswith(".w")) > 5000


@pytest.mark.parametrize("n_el,p,bc", [(8, 2, 2), (16, 2, 1), (8, 4, 0)])
def test_rounded_parity(nhmf, n_el, p, bc):
    M = p * n_el + 1
    params = he_params()
    x = inp.normal(11, 3 * M ** 3).astype(np.float32).astype(np.float64)
    e = inp.normal(12, 3 * M ** 3).astype(np.float32).astype(np.float64)
    y, loss, g = run_gpu(nhmf, n_el, p, bc, params, x, e)
    xo, eo = x.reshape(3, M, M, M), e.reshape(3, M, M, M)
    yo, acts = ounet.forward(params, xo, quant=True)
    assert np.mean(acts["t0"] > 0) > 0.2                    # the network is alive
    assert rel_l2(y, yo.reshape(-1)) <= 1e-2
    free = (~Mesh(n_el, p).constrained(bc)).astype(np.float64).reshape(3, M, M, M)
    lo = ounet.loss(yo, eo, free)
    assert abs(loss - lo) <= 1e-2 * lo
    go = ounet.backward(params, acts, yo, eo, free, quant=True)
    errs = {k: rel_l2(g[k].reshape(-1), go[k].reshape(-1)) for k in go}
    assert max(errs.values()) <= 8e-2, errs


def test_adam_step_matches_oracle(nhmf):
    n_el, p, bc = 8, 2, 2
    M = p * n_el + 1
    prob = nhmf.Problem(n_el, p, 1.0, 1.5, bc)
    nhmf.nhmf_unet_create(prob.ctx, 4)
    params = he_params()
    nhmf.nhmf_unet_set_params(prob.ctx, flat_params(params))
    free = ~Mesh(n_el, p).constrained(bc)
    r = np.where(free, inp.normal(21, 3 * M ** 3), 0.0)
    e = np.where(free, inp.normal(22, 3 * M ** 3), 0.0)
    nhmf.nhmf_unet_record_pair(prob.ctx, cuda(r), cuda(e))
    assert nhmf.nhmf_unet_num_pairs(prob.ctx) == 1
    lr = 1e-3
    l0, _ = nhmf.nhmf_unet_train(prob.ctx, 1, lr)
    xo = (r * np.sqrt(r.size) / np.linalg.norm(r)).reshape(3, M, M, M)
    eo = (e * np.sqrt(e.size) / np.linalg.norm(e)).reshape(3, M, M, M)
    fo = free.reshape(3, M, M, M).astype(float)
    yo, acts = ounet.forward(params, xo, quant=True)
    assert abs(l0 - ounet.loss(yo, eo, fo)) <= 1e-2 * l0
    go = ounet.backward(params, acts, yo, eo, fo, quant=True)
    p2 = {k: v.copy() for k, v in params.items()}
    ounet.adam_step(p2, go, {}, lr=lr)
    new = unflat(nhmf.nhmf_unet_get_params(prob.ctx).astype(np.float64))
    for k in go:
        big = np.abs(go[k]) > 0.2 * np.abs(go[k]).max()      # entries whose step is lr * sign(g)
        d_gpu = (new[k] - params[k])[big]
        d_ora = (p2[k] - params[k])[big]
        assert np.mean(np.abs(d_gpu - d_ora) <= 1e-2 * lr) >= 0.97, k


def test_training_reduces_loss_and_learned_solve_converges(nhmf):
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
