"""Writes unet_exact_129.json: the oracle network's results on the exact-arithmetic case at
the production grid, 129^3 (the nodal grid of Q2 on 64^3 elements), for the GPU test in
tests/test_gpu_unet_fullgrid.py.  Calls only `oracle.unet` (FP64, BF16 rounding where the
GPU stores BF16) and the seeded case builders of tests/unet_cases.py.

Stored: the loss; the output y at 1024 sampled voxels (3 channels each) and the SHA-256 of the
whole output and of every parameter gradient as FP32 (all exact: see tests/unet_cases.py);
the l2 norm of each gradient for diagnostics.  Takes about five minutes and 8 GB of memory.

    python tests/golden/make_unet_golden.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import unet as ounet  # noqa: E402
from oracle.mesh import Mesh  # noqa: E402
from tests import unet_cases as uc  # noqa: E402

N_EL, P, BC = 64, 2, 2


def main():
    M = P * N_EL + 1
    t0 = time.time()
    params = uc.ternary_params()
    x, e = uc.exact_inputs(M)
    xo, eo = x.reshape(3, M, M, M), e.reshape(3, M, M, M)
    free = (~Mesh(N_EL, P).constrained(BC)).astype(np.float64).reshape(3, M, M, M)
    y, acts = ounet.forward(params, xo, quant=True)
    loss = ounet.loss(y, eo, free)
    g = ounet.backward(params, acts, y, eo, free, quant=True)
    yf = y.reshape(-1)
    vox = uc.sample_voxels(M)
    out = {
        "source": __doc__.strip(),
        "case": {"n_el": N_EL, "degree": P, "bc": BC, "M": M, "params": "ternary_params(seed=7000, density=0.006)",
                 "inputs": "exact_inputs(M)"},
        "loss": loss,
        "y_digest": uc.f32_digest(yf),
        "sample_voxels": vox.tolist(),
        "sample_y": [[float(yf[c * M ** 3 + v]) for c in range(3)] for v in vox],
        "grad_digest": {k: uc.f32_digest(g[k]) for k in g},
        "grad_norm": {k: float(np.linalg.norm(g[k])) for k in g},
        "grad_nonzeros": int(sum(np.count_nonzero(g[k]) for k in g if k.endswith(".w"))),
        "seconds": None,
    }
    out["seconds"] = round(time.time() - t0, 1)
    with open(os.path.join(HERE, "unet_exact_129.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
