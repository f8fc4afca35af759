"""Host-side behaviour of the C ABI that needs no GPU (include/nhmf.h): the solver defaults
the header documents, argument checking of nhmf_create, and the absence of any CPU fallback
(creating a context without a CUDA device fails with a CUDA error)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nhmf():
    import __graft_entry__ as g
    g.build()
    from paper_2505_15535_gb300 import nhmf
    return nhmf


def header_struct(name):
    """Field lines of `typedef struct { ... } name;` in include/nhmf.h, comments kept."""
    text = open(os.path.join(ROOT, "include", "nhmf.h")).read()
    m = re.search(r"typedef struct \{(.*?)\}\s*" + name + ";", text, flags=re.S)
    assert m, name
    return m.group(1)


def documented_defaults():
    """field -> value for every `default <number>` the header states beside a field."""
    body = header_struct("nhmf_solve_opts")
    out = {}
    for m in re.finditer(r"^\s*[\w ]+?\b(\w+);\s*/\*(.*?)\*/", body, flags=re.S | re.M):
        field, comment = m.group(1), " ".join(m.group(2).split())
        d = re.search(r"\bdefault ([0-9][0-9.e+-]*)\b", comment)
        if d:
            out[field] = float(d.group(1))
    return out


def test_header_documents_the_numeric_defaults():
    d = documented_defaults()
    for field in ("newton_rtol", "newton_max_iter", "max_backtracks", "linear_rtol", "linear_max_iter",
                  "inner_rtol", "inner_max_iter", "check_every", "record_pairs", "cg_pair_every",
                  "synthetic_pairs", "seed", "smoother_degree", "smoother_range", "first_step"):
        assert field in d, field


def test_solve_opts_default_matches_the_header(nhmf):
    o = nhmf.nhmf_solve_opts_default()
    for field, value in documented_defaults().items():
        assert getattr(o, field) == pytest.approx(value, rel=0, abs=0), field
    # the defaults stated in words: "(defaults 10 and 0.9)", "NHMF_FP64 (default)", "default S"
    # (0: the last of the S load steps), and the function's own "(solver JACOBI_CG, strategy
    # CACHED, S = 1)"
    assert (o.learned_stall_window, o.learned_stall_factor) == (10, 0.9)
    assert o.outer_apply == nhmf.NHMF_FP64
    assert o.last_step == 0
    assert (o.solver, o.strategy, o.load_steps) == (nhmf.NHMF_SOLVER_JACOBI_CG, nhmf.NHMF_CACHED, 1)


def test_solve_opts_overrides_reject_unknown_fields(nhmf):
    o = nhmf.nhmf_solve_opts_default(smoother_degree=5, smoother_range=30.0)
    assert (o.smoother_degree, o.smoother_range) == (5, 30.0)
    with pytest.raises(AttributeError):
        nhmf.nhmf_solve_opts_default(smoother_degre=5)


VALID = dict(n_el=2, degree=2, mu=1.0, lambda_=1.5, bc=1, top_uz=0.0, model=0)


def create_raw(nhmf, **prm):
    p = nhmf.nhmf_params(**{**VALID, **prm})
    ctx = ctypes.c_void_p(12345)  # must come back null on failure
    st = nhmf.lib().nhmf_create(ctypes.byref(p), ctypes.byref(ctx))
    return st, ctx.value


@pytest.mark.parametrize("bad", [
    dict(n_el=0), dict(n_el=-3), dict(n_el=4097),
    dict(degree=0), dict(degree=5),
    dict(mu=0.0), dict(mu=-1.0), dict(mu=float("nan")),
    dict(lambda_=-0.5), dict(lambda_=float("nan")),
    dict(bc=-1), dict(bc=3),
    dict(model=2), dict(model=-1),
])
def test_create_rejects_invalid_parameters(nhmf, bad):
    st, ctx = create_raw(nhmf, **bad)
    assert st == nhmf.NHMF_ERR_ARG
    assert ctx is None


def test_create_rejects_null_pointers(nhmf):
    p = nhmf.nhmf_params(**VALID)
    ctx = ctypes.c_void_p()
    assert nhmf.lib().nhmf_create(None, ctypes.byref(ctx)) == nhmf.NHMF_ERR_ARG
    assert nhmf.lib().nhmf_create(ctypes.byref(p), None) == nhmf.NHMF_ERR_ARG


def test_no_cpu_fallback_without_a_device(nhmf):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    st, ctx = create_raw(nhmf)
    assert st == nhmf.NHMF_ERR_CUDA
    assert ctx is None
    with pytest.raises(nhmf.NhmfError):
        nhmf.nhmf_create(2, 2, 1.0, 1.5, 1)


def header_constants():
    """NHMF_* -> value for every enumerator and #define with an explicit value in the header."""
    text = open(os.path.join(ROOT, "include", "nhmf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(NHMF_[A-Z0-9_]+)\s*=\s*([0-9]+)(?:\s*<<\s*([0-9]+))?", text):
        out[m.group(1)] = int(m.group(2)) << int(m.group(3) or 0)
    for m in re.finditer(r"#define\s+(NHMF_[A-Z0-9_]+)\s+([0-9]+)\b", text):
        out[m.group(1)] = int(m.group(2))
    return out


def test_binding_constants_match_the_header(nhmf):
    consts = header_constants()
    assert len(consts) >= 40
    for k, v in consts.items():  # every named value, under the same name
        assert getattr(nhmf, k, None) == v, k
