"""The C-ABI library builds, loads, and exports every function ``include/hrr.h`` declares
(CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    return __graft_entry__._build_module().build()


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(hrr_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("hrr_create", "hrr_destroy", "hrr_build_light_tree", "hrr_set_shift_tile",
                 "hrr_cull", "hrr_range_min", "hrr_last_error"):
        assert name in d


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    import paper_1907_12343_gb300 as hrr
    assert set(_declared()) <= set(hrr.EXPORTED)


def test_status_strings(lib_path):
    import paper_1907_12343_gb300 as hrr
    assert hrr.hrr_status_string(hrr.HRR_ERR_OVERFLOW) == b"HRR_ERR_OVERFLOW"
    assert hrr.hrr_status_string(0) == b"HRR_OK"


def test_create_rejects_bad_device_without_gpu(lib_path):
    # no GPU here: creating a context must fail cleanly, never crash
    import paper_1907_12343_gb300 as hrr
    h = ctypes.c_void_p()
    st = hrr.hrr_create(ctypes.byref(h), 12345, None)
    assert st == hrr.HRR_ERR_INVALID_ARG and not h.value


def test_null_arguments_are_rejected(lib_path):
    import paper_1907_12343_gb300 as hrr
    assert hrr.hrr_destroy(None) == hrr.HRR_ERR_INVALID_ARG
    assert hrr.hrr_launch_count(None, None) == hrr.HRR_ERR_INVALID_ARG
    assert hrr.hrr_tree_perm(None, None) == hrr.HRR_ERR_INVALID_ARG


def test_default_tuning_is_the_documented_form(lib_path):
    # host code only: binary records with the head over the top six levels, a 256-entry
    # stack ring, 256-thread blocks, the branch-free range minimum, as many blocks as fit
    import paper_1907_12343_gb300 as hrr
    assert hrr.default_tuning() == {"rangemin_variant": 0, "blocks_per_sm": 0, "node_width": 2,
                                    "ring_entries": 256, "threads_per_block": 256, "top_levels": 6}
    t = hrr.hrr_tuning()
    assert hrr.hrr_default_tuning(None) == hrr.HRR_ERR_INVALID_ARG
    assert hrr.hrr_default_tuning(ctypes.byref(t)) == hrr.HRR_OK
