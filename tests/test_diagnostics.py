"""Host-side diagnostics that need no GPU: the NHMF_INJECT syntax of the fault injection
(include/nhmf.h, "diagnostics").  The paths themselves run in tests/test_gpu_diagnostics.py."""
import pytest


@pytest.fixture(scope="module")
def nhmf():
    import __graft_entry__ as g
    g.build()
    from paper_2505_15535_gb300 import nhmf
    return nhmf


@pytest.mark.parametrize("spec, flags", [
    (None, 0),
    ("", 0),
    ("nan_in_du", 1),
    ("cg_stall", 2),
    ("unet_garbage", 4),
    ("cg_stall,unet_garbage", 6),
    (" nan_in_du , cg_stall ", 3),
    ("nan_in_du,,unet_garbage", 5),
])
def test_parse_inject_names(nhmf, spec, flags):
    assert nhmf.nhmf_parse_inject(spec) == flags


def test_parse_inject_marks_unknown_names(nhmf):
    assert nhmf.nhmf_parse_inject("bogus") == nhmf.NHMF_INJECT_UNKNOWN
    assert nhmf.nhmf_parse_inject("nan_in_du,nan_in_du_x") == nhmf.NHMF_INJECT_NAN_DU | nhmf.NHMF_INJECT_UNKNOWN
    assert nhmf.nhmf_parse_inject("NAN_IN_DU") == nhmf.NHMF_INJECT_UNKNOWN  # names are lower case
