"""The C-ABI library builds, loads and exports every symbol of include/dw.h.
Host-side argument checks run without a GPU (no compute calls here)."""
import ctypes
import os

import pytest

from helpers import header_functions

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dw():
    from paper_2001_05218_gb300 import build
    build.build()
    from paper_2001_05218_gb300 import dw as m
    return m


def test_header_declares_the_boundary():
    names = header_functions()
    for n in ["dw_field_alloc", "dw_apply", "dw_apply_dag", "dw_normal_apply", "dw_cg_solve",
              "dw_cg_solve_batched", "dw_cg_backward"]:
        assert n in names


def test_library_exports_every_declared_symbol(dw):
    lib = ctypes.CDLL(dw.LIB_PATH)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_field_bytes_and_shape_checks(dw):
    nb = ctypes.c_size_t()
    lat = dw.lattice((4, 4, 4, 4), 0.1)
    assert dw.dw_field_bytes(ctypes.byref(lat), dw.DW_SPINOR_FULL, dw.DW_F64, 0, 1, ctypes.byref(nb)) == dw.DW_OK
    assert nb.value == 256 * 12 * 16
    assert dw.dw_field_bytes(ctypes.byref(lat), dw.DW_SPINOR_EVEN, dw.DW_F16, 0, 3, ctypes.byref(nb)) == dw.DW_OK
    assert nb.value == 3 * 128 * 52
    assert dw.dw_field_bytes(ctypes.byref(lat), dw.DW_GAUGE, dw.DW_F32, 1, 1, ctypes.byref(nb)) == dw.DW_OK
    assert nb.value == 256 * 4 * 48
    bad = dw.lattice((4, 3, 4, 4), 0.1)
    assert dw.dw_field_bytes(ctypes.byref(bad), dw.DW_SPINOR_FULL, dw.DW_F64, 0, 1, ctypes.byref(nb)) == dw.DW_ERR_SHAPE
    assert "even" in dw.dw_last_error()
    assert dw.dw_field_bytes(ctypes.byref(lat), dw.DW_SPINOR_FULL, 9, 0, 1, ctypes.byref(nb)) == dw.DW_ERR_PRECISION
    assert dw.dw_field_bytes(ctypes.byref(lat), dw.DW_SPINOR_FULL, dw.DW_F64, 0, 0, ctypes.byref(nb)) == dw.DW_ERR_SHAPE
    tiny = dw.lattice((2, 2, 2, 2), 0.1)  # half volume 8: smallest allowed
    assert dw.dw_field_bytes(ctypes.byref(tiny), dw.DW_SPINOR_FULL, dw.DW_F64, 0, 1, ctypes.byref(nb)) == dw.DW_OK


def test_params_default_and_null_checks(dw):
    p = dw.params()
    assert abs(p.tol - 1e-10) < 1e-25 and p.inner == dw.DW_F32 and p.eo == 1 and p.delta == 0.0
    assert dw.dw_apply(None, None, None, None) == dw.DW_ERR_ARG
    assert dw.dw_cg_solve(None, None, None, ctypes.byref(p), None, None) == dw.DW_ERR_ARG
    assert dw.dw_field_free(None) == dw.DW_OK


def test_binding_has_same_names_as_header(dw):
    assert set(header_functions()) <= set(dw.symbols())


def test_field_bytes_rhs_range_and_fixed_point(dw):
    """nrhs spans 1..64 (per-block column gates are sized for 64); the
    fixed-point format has the 16-bit layout (52 bytes per spinor site,
    24 per 12-real link)."""
    nb = ctypes.c_size_t()
    lat = dw.lattice((4, 4, 4, 4), 0.1)
    assert dw.dw_field_bytes(ctypes.byref(lat), dw.DW_SPINOR_FULL, dw.DW_F16, 0, 64, ctypes.byref(nb)) == dw.DW_OK
    assert nb.value == 64 * 256 * 52
    assert dw.dw_field_bytes(ctypes.byref(lat), dw.DW_SPINOR_FULL, dw.DW_F16, 0, 65, ctypes.byref(nb)) == dw.DW_ERR_SHAPE
    assert dw.dw_field_bytes(ctypes.byref(lat), dw.DW_SPINOR_EVEN, dw.DW_I16, 0, 2, ctypes.byref(nb)) == dw.DW_OK
    assert nb.value == 2 * 128 * 52
    assert dw.dw_field_bytes(ctypes.byref(lat), dw.DW_GAUGE, dw.DW_I16, 1, 1, ctypes.byref(nb)) == dw.DW_OK
    assert nb.value == 256 * 4 * 24
