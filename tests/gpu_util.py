"""Helpers of the GPU parity tests: build/load the library, move arrays, compare."""
import numpy as np
import pytest


def lib_or_fail():
    import __graft_entry__ as g
    g.build()
    from paper_2505_15535_gb300 import nhmf
    return nhmf


def cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
