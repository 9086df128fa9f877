"""Host-side checks of the C ABI (no GPU): the library builds and loads, exports every entry
point declared in include/spmv.h, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2107_12371_gb300 import build as gbuild
from paper_2107_12371_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"^\s*typedef[^;]*;", "", src, flags=re.M)  # callback types are not entry points
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                            src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    return capi.load(gbuild.build())


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["spmv_create", "spmv_destroy", "spmv_apply", "spmv_apply_multi",
                     "spmv_permute", "cg_solve", "spmv_server_create", "spmv_server_submit",
                     "spmv_server_poll", "spmv_server_destroy", "spmv_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared entry points
    for name in capi._SIGS:
        assert name in names


def test_status_strings(lib):
    for code in range(11):
        s = capi.spmv_status_string(code)
        assert s and s != "unknown status"
    assert capi.spmv_status_string(99) == "unknown status"


def test_default_options(lib):
    o = capi.spmv_default_options()
    assert (o.slice_height, o.block, o.reorder, o.precision, o.peripheral) == (64, 256, 0, 0, 1)
    c = capi.cg_default_options()
    assert c.rtol == 1e-10 and c.max_iter > 0 and c.check_every > 0


def test_create_rejects_bad_arguments_before_device_work(lib):
    h = ctypes.c_void_p()
    L = lib
    # out == NULL
    assert L.spmv_create(1, 1, 0, None, None, None, 0, None, None, None) == capi.SPMV_ERR_INVALID_ARG
    # a rectangular matrix cannot be renumbered symmetrically
    o = capi.spmv_default_options(reorder=capi.SPMV_REORDER_RCM)
    rp3 = (ctypes.c_int32 * 3)(0, 0, 0)
    assert L.spmv_create(2, 3, 0, rp3, None, None, 0, ctypes.byref(o), None, ctypes.byref(h)) == \
        capi.SPMV_ERR_INVALID_ARG
    assert h.value is None
    # negative sizes, missing arrays
    assert L.spmv_create(-1, -1, 0, None, None, None, 0, None, None, ctypes.byref(h)) == \
        capi.SPMV_ERR_INVALID_ARG
    rp = (ctypes.c_int32 * 3)(0, 1, 2)
    assert L.spmv_create(2, 2, 2, rp, None, None, 0, None, None, ctypes.byref(h)) == \
        capi.SPMV_ERR_INVALID_ARG
    # bad options
    for field, value in [("slice_height", 48), ("block", 100), ("variant", 7), ("reorder", 5),
                         ("precision", 3), ("window_words", -1), ("index_bits", 8),
                         ("sigma", 100), ("sigma", 8192), ("checks", 2)]:
        o = capi.spmv_default_options()
        setattr(o, field, value)
        assert L.spmv_create(2, 2, 0, rp, None, None, 0, ctypes.byref(o), None,
                             ctypes.byref(h)) == capi.SPMV_ERR_INVALID_ARG, field


def test_entry_points_reject_null_handles(lib):
    L = lib
    assert L.spmv_apply(None, None, None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_apply_f32(None, None, None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_apply_axpby(None, 1.0, None, 0.0, None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_apply_multi(None, 8, None, None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_permute(None, 0, 8, None, None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_get_info(None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_destroy(None) == capi.SPMV_OK
    assert L.cg_solve(None, None, None, None, None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_server_submit(None, 1, 0, None, None, None, None, None, None) == \
        capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_server_poll(None, 0, None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_server_cancel(None, 0) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_apply_host(None, None, None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_apply_host_async(None, None, None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_apply_chain_f32(None, None, None, None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_verify(None, None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_diag_checks(None, None, None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_device_status(None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_diag_bulk_timeout(None, None) == capi.SPMV_ERR_INVALID_ARG
    assert L.spmv_server_destroy(None) == capi.SPMV_OK


def test_binding_constants_match_the_header():
    """Every #define SPMV_* constant of the header that the binding names has the same value
    there, so the binding cannot drift from the C ABI."""
    src = open(os.path.join(ROOT, "include", "spmv.h")).read()
    defines = {name: int(val) for name, val in
               re.findall(r"^#define\s+(SPMV_[A-Z0-9_]+)\s+(-?\d+)", src, flags=re.M)}
    enums = dict(re.findall(r"\b(SPMV_(?:OK|ERR_[A-Z_]+))\s*=\s*(\d+)", src))
    checked = 0
    for name in dir(capi):
        if not name.startswith("SPMV_"):
            continue
        val = getattr(capi, name)
        if name in defines:
            assert val == defines[name], name
            checked += 1
        elif name in enums:
            assert val == int(enums[name]), name
            checked += 1
    assert checked >= 20
    for name in ("SPMV_VARIANT_SELL_BULK", "SPMV_PREC_DUAL", "SPMV_REORDER_RCM"):
        assert name in defines and hasattr(capi, name)
