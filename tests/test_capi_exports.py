"""The C-ABI library builds, loads without a GPU and exports every entry
point include/gcp.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gcp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gcp_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1512_07236_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 11, names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_1512_07236_gb300 import gcp
    assert sorted(gcp.EXPORTS) == _declared()


def test_status_strings_and_defaults(lib):
    from paper_1512_07236_gb300 import gcp
    L = gcp.load_library()
    assert L.gcp_status_string(0) == b"ok"
    assert L.gcp_status_string(2) == b"not converged"
    o = gcp.Options()
    L.gcp_default_options(ctypes.byref(o))
    assert o.prec == 0 and o.tol == 1e-12 and o.max_iter == 100 and o.use_graph == 1


def test_create_destroy_without_gpu(lib):
    """Handle creation allocates nothing on the device."""
    from paper_1512_07236_gb300 import gcp
    L = gcp.load_library()
    h = ctypes.c_void_p()
    assert L.gcp_create(ctypes.byref(h)) == 0
    assert L.gcp_destroy(h) == 0
    assert L.gcp_create(None) == 1
