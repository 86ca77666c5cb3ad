"""The C ABI on a machine without a GPU: the library builds and loads, exports
every function include/fastperm.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import re

import pytest

import paper_2602_00898_b300 as fp


def _declared():
    src = open(fp.HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fp_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("fp_create_from_faces", "fp_create_from_csr", "fp_permute", "fp_symbolic", "fp_destroy",
                 "fp_get_tree", "fp_get_patches", "fp_order_faces_host", "fp_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = fp.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_default_options_and_status_strings():
    o = fp.fp_default_options()
    assert (o.patch_cap, o.lloyd_rounds, o.seed, o.nd_level, o.schedule, o.dof_per_vertex, o.debug_dump,
            o.max_spin) == (512, 2, 0, 0, 0, 1, 0, 0)
    assert ctypes.sizeof(fp.fp_options) == 40
    L = fp.lib()
    for code, name in fp.STATUS.items():
        assert L.fp_status_string(code).decode() == name


@pytest.mark.parametrize("field,value", [("patch_cap", 0), ("lloyd_rounds", -1), ("nd_level", -2),
                                         ("nd_level", 25), ("schedule", 2), ("dof_per_vertex", 0),
                                         ("debug_dump", 2), ("debug_dump", -1), ("max_spin", -1)])
def test_bad_options_rejected_without_device(field, value):
    o = fp.fp_default_options(**{field: value})
    h = ctypes.c_void_p()
    st = fp.lib().fp_create_from_faces(None, 0, 10, ctypes.byref(o), None, ctypes.byref(h))
    assert st == 1 and not h.value
    assert "option" in fp.fp_last_error(None)


def test_null_out_and_negative_sizes_rejected():
    o = fp.fp_default_options()
    L = fp.lib()
    assert L.fp_create_from_faces(None, 0, 10, ctypes.byref(o), None, None) == 1
    h = ctypes.c_void_p()
    assert L.fp_create_from_faces(None, 5, 10, ctypes.byref(o), None, ctypes.byref(h)) == 1
    assert L.fp_create_from_faces(None, 0, -1, ctypes.byref(o), None, ctypes.byref(h)) == 1
    assert L.fp_create_from_csr(None, None, 6, ctypes.byref(o), None, ctypes.byref(h)) == 1
    o3 = fp.fp_default_options(dof_per_vertex=3)
    assert L.fp_create_from_csr(None, None, 7, ctypes.byref(o3), None, ctypes.byref(h)) == 1
    assert L.fp_permute(None, None, None) == 1
    assert L.fp_destroy(None) == 0
