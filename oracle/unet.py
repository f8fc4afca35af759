"""FP64 reference of the convolutional U-Net preconditioner (oracle; test infrastructure only).

The paper has no learned component; this network is the learned preconditioner the build
adds on the nodal grid of the Q_p mesh.  Definition (fixed here, and what the GPU kernels
must reproduce in BF16 with FP32 accumulation):

Arrays are channel-first [C, M, M, M] indexed [c, k, j, i] (x fastest), the DoF layout of the
mesh.  All convolutions are 3x3x3 cross-correlations with zero padding:
  conv(x; W, b)[o, v]    = b[o] + sum_c sum_d W[o, c, d] x[c, v + d],          d in {-1,0,1}^3
  down(x; W, b)[o, v']   = b[o] + sum_c sum_d W[o, c, d] x[c, 2 v' + d]          (stride 2)
  up(y; U, b)[o, v]      = b[o] + sum_c sum_{v', d: 2 v' + d = v} U[c, o, d] y[c, v']
(`up` is the adjoint of `down` for U = W, cropped to the fine grid).  Grids: M0 = M,
M1 = (M0 - 1)/2 + 1, M2 = (M1 - 1)/2 + 1; M - 1 must be divisible by 4.
W[o, c, d] is stored as W[o, c, dz + 1, dy + 1, dx + 1]; U as U[c, o, dz + 1, dy + 1, dx + 1].

Layers (C = 16 channels, ReLU r):
  a0 = r(conv(x; in))         3 -> C,  M0
  s0 = r(conv(a0; e0))        C -> C,  M0   (skip 0)
  d1 = r(down(s0; d1))        C -> C,  M1
  s1 = r(conv(d1; e1))        C -> C,  M1   (skip 1)
  d2 = r(down(s1; d2))        C -> C,  M2
  m2 = r(conv(d2; m2))        C -> C,  M2
  u1 = r(up(m2; u1) + s1)     C -> C,  M1
  t1 = r(conv(u1; t1))        C -> C,  M1
  u0 = r(up(t1; u0) + s0)     C -> C,  M0
  t0 = r(conv(u0; t0))        C -> C,  M0
  y  = conv(t0; out)          C -> 3,  M0   (linear)
Loss of one pair (x, e) with Dirichlet mask f (1 on free DoFs):
  L = ||f (y - e)||^2 / ||f e||^2.

With quant=True, forward and backward round to BF16 (round to nearest even) exactly where
the GPU kernels store BF16: the weights, the input, every activation, the loss gradient and
every activation gradient; arithmetic stays FP64.  The ReLU decisions and their masks are
then taken in the kernels' storage precision, which the parity tests need.
"""
from __future__ import annotations

import numpy as np

LAYERS = [  # name, kind, c_in, c_out
    ("in", "conv", 3, 16), ("e0", "conv", 16, 16), ("d1", "down", 16, 16), ("e1", "conv", 16, 16),
    ("d2", "down", 16, 16), ("m2", "conv", 16, 16), ("u1", "up", 16, 16), ("t1", "conv", 16, 16),
    ("u0", "up", 16, 16), ("t0", "conv", 16, 16), ("out", "conv", 16, 3),
]


def weight_shape(kind, cin, cout):
    return (cin, cout, 3, 3, 3) if kind == "up" else (cout, cin, 3, 3, 3)


def _taps():
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                yield dz, dy, dx


def _shift(x, dz, dy, dx, stride, out_m):
    """x[c, s v + d] for v in [0, out_m)^3 (zero outside), s = stride."""
    c, m = x.shape[0], x.shape[1]
    xp = np.zeros((c, m + 2, m + 2, m + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    sl = lambda d: slice(1 + d, 1 + d + stride * (out_m - 1) + 1, stride)
    return xp[:, sl(dz), sl(dy), sl(dx)]


def conv(x, W, b, stride=1):
    m = x.shape[1]
    om = m if stride == 1 else (m - 1) // 2 + 1
    out = np.broadcast_to(b[:, None, None, None], (W.shape[0], om, om, om)).copy()
    for dz, dy, dx in _taps():
        out += np.einsum("oc,czyx->ozyx", W[:, :, dz + 1, dy + 1, dx + 1], _shift(x, dz, dy, dx, stride, om))
    return out


def conv_backward(x, W, dout, stride=1):
    """(dx, dW, db) of conv/down for the upstream gradient dout."""
    m = x.shape[1]
    om = dout.shape[1]
    dW = np.zeros_like(W)
    dxp = np.zeros((x.shape[0], m + 2, m + 2, m + 2))
    for dz, dy, dx in _taps():
        xs = _shift(x, dz, dy, dx, stride, om)
        dW[:, :, dz + 1, dy + 1, dx + 1] = np.einsum("ozyx,czyx->oc", dout, xs)
        sl = lambda d: slice(1 + d, 1 + d + stride * (om - 1) + 1, stride)
        dxp[:, sl(dz), sl(dy), sl(dx)] += np.einsum("oc,ozyx->czyx", W[:, :, dz + 1, dy + 1, dx + 1], dout)
    return dxp[:, 1:-1, 1:-1, 1:-1], dW, dout.sum(axis=(1, 2, 3))


def up(y, U, b, out_m):
    """Transposed stride-2 convolution onto a grid of out_m points per direction."""
    co = U.shape[1]
    outp = np.zeros((co, out_m + 2, out_m + 2, out_m + 2))
    ym = y.shape[1]
    for dz, dy, dx in _taps():
        sl = lambda d: slice(1 + d, 1 + d + 2 * (ym - 1) + 1, 2)
        outp[:, sl(dz), sl(dy), sl(dx)] += np.einsum("co,czyx->ozyx", U[:, :, dz + 1, dy + 1, dx + 1], y)
    return outp[:, 1:-1, 1:-1, 1:-1] + b[:, None, None, None]


def up_backward(y, U, dout):
    """(dy, dU, db) of `up`."""
    ym = y.shape[1]
    dy_ = np.zeros_like(y)
    dU = np.zeros_like(U)
    for dz, dy, dx in _taps():
        ds = _shift(dout, dz, dy, dx, 2, ym)          # dout[o, 2 v' + d]
        dy_ += np.einsum("co,ozyx->czyx", U[:, :, dz + 1, dy + 1, dx + 1], ds)
        dU[:, :, dz + 1, dy + 1, dx + 1] = np.einsum("czyx,ozyx->co", y, ds)
    return dy_, dU, dout.sum(axis=(1, 2, 3))


def relu(z):
    return np.maximum(z, 0.0)


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _quantized(params):
    return {k: (bf16(v) if k.endswith(".w") else v) for k, v in params.items()}


def init_params(seed_normal, m_unused=None):
    """He-normal weights from a caller-supplied N(0,1) draw function, zero biases."""
    params = {}
    k = 0
    for name, kind, cin, cout in LAYERS:
        shape = weight_shape(kind, cin, cout)
        fan_in = cin * 27
        n = int(np.prod(shape))
        params[name + ".w"] = seed_normal(k, n).reshape(shape) * np.sqrt(2.0 / fan_in)
        params[name + ".b"] = np.zeros(cout)
        k += 1
    return params


def forward(params, x, quant=False):
    """y and the cache of activations for backward."""
    P = _quantized(params) if quant else params
    q = bf16 if quant else (lambda v: v)
    M0 = x.shape[1]
    M1 = (M0 - 1) // 2 + 1
    a = {}
    a["x"] = q(x)
    a["a0"] = q(relu(conv(a["x"], P["in.w"], P["in.b"])))
    a["s0"] = q(relu(conv(a["a0"], P["e0.w"], P["e0.b"])))
    a["d1"] = q(relu(conv(a["s0"], P["d1.w"], P["d1.b"], 2)))
    a["s1"] = q(relu(conv(a["d1"], P["e1.w"], P["e1.b"])))
    a["d2"] = q(relu(conv(a["s1"], P["d2.w"], P["d2.b"], 2)))
    a["m2"] = q(relu(conv(a["d2"], P["m2.w"], P["m2.b"])))
    a["u1"] = q(relu(up(a["m2"], P["u1.w"], P["u1.b"], M1) + a["s1"]))
    a["t1"] = q(relu(conv(a["u1"], P["t1.w"], P["t1.b"])))
    a["u0"] = q(relu(up(a["t1"], P["u0.w"], P["u0.b"], M0) + a["s0"]))
    a["t0"] = q(relu(conv(a["u0"], P["t0.w"], P["t0.b"])))
    y = conv(a["t0"], P["out.w"], P["out.b"])
    return y, a


def loss(y, e, free):
    d = free * (y - e)
    return float(np.sum(d * d) / np.sum((free * e) ** 2))


def backward(params, a, y, e, free, quant=False):
    """Gradients of the loss with respect to every parameter (dict like params)."""
    P = _quantized(params) if quant else params
    q = bf16 if quant else (lambda v: v)
    g = {}
    den = np.sum((free * e) ** 2)
    dy = q(2.0 * free * free * (y - e) / den)
    dt0, g["out.w"], g["out.b"] = conv_backward(a["t0"], P["out.w"], dy)
    dt0 = q(dt0 * (a["t0"] > 0))
    du0, g["t0.w"], g["t0.b"] = conv_backward(a["u0"], P["t0.w"], dt0)
    du0 = q(du0 * (a["u0"] > 0))               # through the ReLU of u0 (sum of up and skip)
    ds0 = du0.copy()
    dt1, g["u0.w"], g["u0.b"] = up_backward(a["t1"], P["u0.w"], du0)
    dt1 = q(dt1 * (a["t1"] > 0))
    du1, g["t1.w"], g["t1.b"] = conv_backward(a["u1"], P["t1.w"], dt1)
    du1 = q(du1 * (a["u1"] > 0))
    ds1 = du1.copy()
    dm2, g["u1.w"], g["u1.b"] = up_backward(a["m2"], P["u1.w"], du1)
    dm2 = q(dm2 * (a["m2"] > 0))
    dd2, g["m2.w"], g["m2.b"] = conv_backward(a["d2"], P["m2.w"], dm2)
    dd2 = q(dd2 * (a["d2"] > 0))
    ds1b, g["d2.w"], g["d2.b"] = conv_backward(a["s1"], P["d2.w"], dd2, 2)
    ds1 = q((ds1 + ds1b) * (a["s1"] > 0))
    dd1, g["e1.w"], g["e1.b"] = conv_backward(a["d1"], P["e1.w"], ds1)
    dd1 = q(dd1 * (a["d1"] > 0))
    ds0b, g["d1.w"], g["d1.b"] = conv_backward(a["s0"], P["d1.w"], dd1, 2)
    ds0 = q((ds0 + ds0b) * (a["s0"] > 0))
    da0, g["e0.w"], g["e0.b"] = conv_backward(a["a0"], P["e0.w"], ds0)
    da0 = q(da0 * (a["a0"] > 0))
    _, g["in.w"], g["in.b"] = conv_backward(a["x"], P["in.w"], da0)
    return g


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) of every parameter, in place."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m." + k, np.zeros_like(params[k]))
        v = state.setdefault("v." + k, np.zeros_like(params[k]))
        m[:] = b1 * m + (1 - b1) * grads[k]
        v[:] = b2 * v + (1 - b2) * grads[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        params[k] -= lr * mh / (np.sqrt(vh) + eps)
