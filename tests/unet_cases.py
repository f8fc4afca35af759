"""Seeded U-Net test cases shared by the GPU parity tests and the stored-value generator.

Parameters are built in the oracle network's shapes (`oracle.unet.LAYERS`) from the seeded
draws of `nhmf_inputs`; nothing here computes the network.

* He-initialised weights with small random biases and normal inputs ("rounded" cases);
* sparse ternary weights (values -1/0/1, density 0.006), biases 0/1, inputs in {-1, 0, 1} and
  a target that is one spike of 4 ("exact" cases): every activation is an integer, every
  activation gradient a multiple of 1/8, and every sum the kernels form stays below 2^21 in
  units of 1/8 (the largest sum of absolute terms is 1.5e5 at 65^3 and 6.0e5 at 129^3), so
  FP32 accumulation is exact in any order and BF16 rounding, where it happens, is the same
  round-to-nearest-even step on both sides.
"""
from __future__ import annotations

import hashlib

import numpy as np

import nhmf_inputs as inp
from oracle import unet as ounet


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


def exact_inputs(M):
    """(x, e) of the exact case on an M^3 grid, planar [3 M^3] FP64."""
    x = np.floor(inp.uniform01(123, 3 * M ** 3) * 3.0 - 1.0)
    e = np.zeros(3 * M ** 3)
    e[M ** 3 + (M // 2) * (1 + M + M * M)] = 4.0          # ||f e||^2 = 16: dy is a multiple of 1/8
    return x, e


def rounded_inputs(M):
    x = inp.normal(11, 3 * M ** 3).astype(np.float32).astype(np.float64)
    e = inp.normal(12, 3 * M ** 3).astype(np.float32).astype(np.float64)
    return x, e


def f32_digest(a) -> str:
    """SHA-256 of an array's FP32 bytes (C order) with -0.0 folded into +0.0."""
    b = np.ascontiguousarray(np.asarray(a, dtype=np.float32) + np.float32(0.0))
    return hashlib.sha256(b.tobytes()).hexdigest()


def sample_voxels(M, count=1024, seed=8100):
    """Voxel indices of the sampled-output check: the eight corners, then seeded uniform picks."""
    corners = [i + M * (j + M * k) for k in (0, M - 1) for j in (0, M - 1) for i in (0, M - 1)]
    picks = (inp.uniform01(seed, count - len(corners)) * M ** 3).astype(np.int64)
    return np.array(corners + list(picks), dtype=np.int64)
