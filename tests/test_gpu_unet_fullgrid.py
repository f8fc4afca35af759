"""The GPU U-Net on the production grid, 129^3 (the nodal grid of Q2 on 64^3 elements), against
the oracle network's stored results on the exact-arithmetic case (tests/golden/unet_exact_129.json,
written by tests/golden/make_unet_golden.py, which calls only the oracle).

On this grid every tensor-core kernel runs its production schedule: the stride-1
convolutions and their weight gradients walk z-columns of 8 tiles (129^3) and 3 tiles (65^3)
through the plane-slot ring, the transposed convolution onto 129^3 (and the backward-data
product of the stride-2 convolution from it) columns of 3 tiles, and every block loops over
several column units.  Exact arithmetic makes the comparison bit for bit: the whole output,
the loss and every parameter gradient (as SHA-256 digests of their FP32 bytes), with 1024
sampled output voxels stored as values for diagnosis."""
import json
import os

import numpy as np
import pytest

from tests.gpu_util import cuda, host, lib_or_fail
from tests.unet_cases import exact_inputs, f32_digest, flat_params, ternary_params, unflat

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "unet_exact_129.json")


def test_exact_arithmetic_129_matches_stored_oracle():
    nhmf = lib_or_fail()
    ref = json.load(open(GOLDEN))
    n_el, p, bc, M = (ref["case"][k] for k in ("n_el", "degree", "bc", "M"))
    params = ternary_params()
    x, e = exact_inputs(M)
    prob = nhmf.Problem(n_el, p, 1.0, 1.5, bc)
    nhmf.nhmf_unet_create(prob.ctx, 0)
    nhmf.nhmf_unet_set_params(prob.ctx, flat_params(params))
    xt, et = cuda(x.astype(np.float32)), cuda(e.astype(np.float32))
    y = cuda(np.zeros(3 * M ** 3, dtype=np.float32))
    nhmf.nhmf_unet_forward(prob.ctx, xt, y)
    loss, g = nhmf.nhmf_unet_loss_grad(prob.ctx, xt, et)
    yh = host(y)
    vox = np.array(ref["sample_voxels"])
    got = np.stack([yh[c * M ** 3 + vox] for c in range(3)], axis=1)
    want = np.array(ref["sample_y"])
    bad = np.nonzero(np.any(got != want, axis=1))[0]
    assert bad.size == 0, [(int(vox[i]), got[i].tolist(), want[i].tolist()) for i in bad[:8]]
    assert f32_digest(yh) == ref["y_digest"]
    assert loss == ref["loss"]
    gd = unflat(g.astype(np.float64))
    wrong = {k: (float(np.linalg.norm(gd[k])), ref["grad_norm"][k]) for k in ref["grad_digest"]
             if f32_digest(gd[k]) != ref["grad_digest"][k]}
    assert not wrong, wrong
    assert ref["grad_nonzeros"] > 5000
    prob.close()
