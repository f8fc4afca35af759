"""Pins of the oracle U-Net: convolutions against brute-force loops and torch's conv3d,
the adjoint relation between `down` and `up`, and finite differences of the loss."""
import numpy as np
import pytest

from oracle import unet

RNG = np.random.default_rng(3)


def brute_conv(x, W, b, stride):
    c, m = x.shape[0], x.shape[1]
    om = m if stride == 1 else (m - 1) // 2 + 1
    out = np.zeros((W.shape[0], om, om, om))
    for o in range(W.shape[0]):
        for z in range(om):
            for y in range(om):
                for xx in range(om):
                    s = b[o]
                    for ci in range(c):
                        for dz in (-1, 0, 1):
                            for dy in (-1, 0, 1):
                                for dx in (-1, 0, 1):
                                    zz, yy, x3 = stride * z + dz, stride * y + dy, stride * xx + dx
                                    if 0 <= zz < m and 0 <= yy < m and 0 <= x3 < m:
                                        s += W[o, ci, dz + 1, dy + 1, dx + 1] * x[ci, zz, yy, x3]
                    out[o, z, y, xx] = s
    return out


@pytest.mark.parametrize("stride", [1, 2])
def test_conv_brute_force(stride):
    x = RNG.standard_normal((2, 5, 5, 5))
    W = RNG.standard_normal((3, 2, 3, 3, 3))
    b = RNG.standard_normal(3)
    assert np.allclose(unet.conv(x, W, b, stride), brute_conv(x, W, b, stride), atol=1e-12)


def test_conv_matches_torch_conv3d():
    torch = pytest.importorskip("torch")
    x = RNG.standard_normal((4, 9, 9, 9))
    W = RNG.standard_normal((5, 4, 3, 3, 3))
    b = RNG.standard_normal(5)
    for stride in (1, 2):
        ref = torch.nn.functional.conv3d(torch.from_numpy(x)[None], torch.from_numpy(W), torch.from_numpy(b),
                                         stride=stride, padding=1)[0].numpy()
        assert np.allclose(unet.conv(x, W, b, stride), ref, atol=1e-12)
    y = RNG.standard_normal((4, 5, 5, 5))
    U = RNG.standard_normal((4, 5, 3, 3, 3))
    ref = torch.nn.functional.conv_transpose3d(torch.from_numpy(y)[None], torch.from_numpy(U), torch.from_numpy(b),
                                               stride=2, padding=1)[0].numpy()
    assert np.allclose(unet.up(y, U, b, 9), ref, atol=1e-12)


def test_up_is_adjoint_of_down():
    m = 9
    x = RNG.standard_normal((3, m, m, m))
    W = RNG.standard_normal((4, 3, 3, 3, 3))
    y = RNG.standard_normal((4, 5, 5, 5))
    zero3, zero4 = np.zeros(3), np.zeros(4)
    lhs = np.sum(unet.conv(x, W, zero4, 2) * y)
    rhs = np.sum(x * unet.up(y, W, zero3, m))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_backward_pieces_are_adjoints():
    x = RNG.standard_normal((3, 9, 9, 9))
    W = RNG.standard_normal((4, 3, 3, 3, 3))
    for stride in (1, 2):
        out = unet.conv(x, W, np.zeros(4), stride)
        g = RNG.standard_normal(out.shape)
        dx, dW, db = unet.conv_backward(x, W, g, stride)
        assert abs(np.sum(dx * x) - np.sum(g * out)) <= 1e-10 * abs(np.sum(g * out))   # linear in x
        assert abs(np.sum(dW * W) - np.sum(g * out)) <= 1e-10 * abs(np.sum(g * out))   # linear in W
        assert np.allclose(db, g.sum(axis=(1, 2, 3)))


def small_problem(m=9, seed=0):
    r = np.random.default_rng(seed)
    params = unet.init_params(lambda k, n: np.random.default_rng(100 + k).standard_normal(n))
    for k in params:
        if k.endswith(".b"):
            params[k] = 0.1 * r.standard_normal(params[k].shape)
    x = r.standard_normal((3, m, m, m))
    e = r.standard_normal((3, m, m, m))
    free = np.ones((3, m, m, m))
    free[:, 0] = 0.0
    return params, x, e, free


def test_network_gradient_finite_differences():
    params, x, e, free = small_problem()
    y, a = unet.forward(params, x)
    g = unet.backward(params, a, y, e, free)
    r = np.random.default_rng(9)
    h = 1e-6
    for name in ["in.w", "e0.w", "d1.w", "e1.w", "d2.w", "m2.w", "u1.w", "t1.w", "u0.w", "t0.w", "out.w",
                 "in.b", "m2.b", "u0.b", "out.b"]:
        for _ in range(3):
            idx = tuple(r.integers(0, s) for s in params[name].shape)
            p1 = {k: v.copy() for k, v in params.items()}
            p2 = {k: v.copy() for k, v in params.items()}
            p1[name][idx] += h
            p2[name][idx] -= h
            fd = (unet.loss(unet.forward(p1, x)[0], e, free) - unet.loss(unet.forward(p2, x)[0], e, free)) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 * max(1e-3, abs(fd)), (name, fd, g[name][idx])


def test_grid_sizes():
    params, x, e, free = small_problem(m=13)
    y, a = unet.forward(params, x)
    assert a["d1"].shape[1] == 7 and a["d2"].shape[1] == 4 and y.shape == (3, 13, 13, 13)


def test_adam_matches_closed_form_first_step():
    p = {"w": np.array([1.0, -2.0])}
    g = {"w": np.array([0.5, -0.25])}
    st = {}
    unet.adam_step(p, g, st, lr=0.1)
    # first Adam step moves each weight by lr * sign(g) (up to eps)
    assert np.allclose(p["w"], [1.0 - 0.1, -2.0 + 0.1], atol=1e-7)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.concatenate([RNG.standard_normal(10000) * 10.0 ** RNG.integers(-6, 6, 10000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8)]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(unet.bf16(x), ref)


def test_quantized_network_stays_close_to_exact():
    params, x, e, free = small_problem()
    y, _ = unet.forward(params, x)
    yq, _ = unet.forward(params, x, quant=True)
    assert np.linalg.norm(yq - y) <= 5e-2 * np.linalg.norm(y)
