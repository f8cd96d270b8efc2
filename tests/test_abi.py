"""The C-ABI library loads without a GPU and exports every function that
include/mpn.h declares; the binding names match. No compute calls here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mpn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpn_[a-z_]+)\s*\(", src)))


def test_header_declares_core_calls():
    names = declared_functions()
    for must in ("mpn_create", "mpn_propagate", "mpn_trace", "mpn_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2004_00540_gb300 as pkg
    L = pkg.load()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert missing == []
    assert sorted(pkg.EXPORTS) == declared_functions()


def test_status_strings_and_variants_without_gpu():
    import paper_2004_00540_gb300 as pkg
    assert pkg.mpn_status_str(pkg.MPN_EOBSTACLE) == "target on an obstacle"
    assert pkg.mpn_status_str(99) == "unknown status"
    v0 = pkg.mpn_variant_info(0)
    assert v0["region_words"] * 32 >= 64 and v0["threads"] % 32 == 0
    assert pkg.mpn_variant_info(-1) is None


def test_argument_errors_need_no_gpu():
    import paper_2004_00540_gb300 as pkg
    L = pkg.load()
    out = ctypes.c_void_p()
    assert L.mpn_create(None, 4, 4, 0, None, ctypes.byref(out)) == pkg.MPN_EINVAL
    buf = (ctypes.c_uint8 * 16)()
    assert L.mpn_create(buf, 0, 4, 0, None, ctypes.byref(out)) == pkg.MPN_EINVAL
    assert L.mpn_create(buf, 4, 4, 8, None, ctypes.byref(out)) == pkg.MPN_EINVAL
    assert L.mpn_sync(None) == pkg.MPN_EINVAL
    assert L.mpn_get_distances(None, buf, 0) == pkg.MPN_EINVAL
    assert L.mpn_get_distances_async(None, buf, None) == pkg.MPN_EINVAL
    assert L.mpn_trace(None, None, 0, None, None, 0, None) == pkg.MPN_EINVAL
    assert L.mpn_launch_count() == 0


def test_tune_query_without_gpu():
    """The autotuner's table is host memory: nothing recorded yet for a size
    bucket means None; bad sizes and shapes are argument errors."""
    import paper_2004_00540_gb300 as pkg
    assert pkg.mpn_tune_query(3, 5, 0) is None
    with pytest.raises(pkg.MPNError):
        pkg.mpn_tune_query(0, 5, 0)
    with pytest.raises(pkg.MPNError):
        pkg.mpn_tune_query(64, 64, 999)
