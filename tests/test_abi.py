"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(nhmf_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def library():
    import __graft_entry__ as g
    g.build()
    from paper_2505_15535_gb300 import nhmf
    return ctypes.CDLL(nhmf.LIB_PATH)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ["nhmf_create", "nhmf_destroy", "nhmf_num_dofs", "nhmf_tangent_apply",
                     "nhmf_tangent_apply_at", "nhmf_residual", "nhmf_diagonal", "nhmf_set_linearization",
                     "nhmf_solve", "nhmf_unet_train", "nhmf_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(library):
    missing = [n for n in declared_functions() if not hasattr(library, n)]
    assert not missing, f"missing exports: {missing}"


def test_binding_covers_every_symbol():
    from paper_2505_15535_gb300 import nhmf
    for n in declared_functions():
        assert hasattr(nhmf, n), f"binding lacks {n}"
