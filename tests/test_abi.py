"""The C-ABI library builds, loads and exports every entry point that
include/ftgemm.h declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ftgemm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    import paper_2305_01024_gb300.build as b
    return b.build()


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for must in ("ftgemm_create", "ftgemm_destroy", "ftgemm_gemm", "ftgemm_report_fetch",
                 "ftgemm_encode", "ftgemm_set_schedule", "ftgemm_get_schedule",
                 "ftgemm_set_threshold", "ftgemm_status_string", "ftgemm_group_create",
                 "ftgemm_group_tiles", "ftgemm_group_set_faults", "ftgemm_grouped_gemm",
                 "ftgemm_group_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_checks(libpath):
    import paper_2305_01024_gb300 as ft
    L = ft.lib()
    assert L.ftgemm_status_string(-1) == b"invalid argument"
    # NULL handle / NULL pointers are rejected before any device work
    assert L.ftgemm_gemm(None, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, 0, 3, None, None) == -1
    assert L.ftgemm_create(None, 0, None) == -1
    assert L.ftgemm_report_fetch(None, None) == -1
    assert L.ftgemm_set_schedule(None, None) == -1
    out = ctypes.c_void_p()
    assert L.ftgemm_group_create(None, 1, None, ft.BF16, ft.FT_TILE, ctypes.byref(out)) == -1
    assert L.ftgemm_grouped_gemm(None, None) == -1
    assert L.ftgemm_group_set_faults(None, None, None) == -1
    assert L.ftgemm_group_tiles(None, None, None) == -1
    assert L.ftgemm_group_destroy(None) == 0
    assert L.ftgemm_selftest_wait(None, 1000) == -1
    assert L.ftgemm_gemm_offline(None, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, None, 1, None, None) == -1
    assert L.ftgemm_gemm_nonfused(None, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, 256, None, None) == -1
    assert L.ftgemm_dgemm(None, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, ft.FT_BLOCK, 1, None, None) == -1
    one = (ctypes.c_double * 2)(1.0, 0.0)
    assert L.ftgemm_zgemm(None, 4, 4, 4, one, None, 4, None, 4, one, None, 4, ft.FT_BLOCK, 1, None, None,
                          None) == -1
    assert L.ftgemm_status_string(ft.ERR_UNRECOVERED) == b"every offline attempt detected a fault"
    assert b"NULL" in L.ftgemm_last_error() or len(L.ftgemm_last_error()) > 0


def test_every_handle_entry_point_rejects_null_before_device_work(libpath):
    # each call fails its argument check (NULL handle or NULL operands) and
    # returns FTGEMM_ERR_ARG with a message, without touching a device
    import paper_2305_01024_gb300 as ft
    L = ft.lib()
    sched = ft.Schedule()
    stats = ft.Stats()
    lv = ctypes.c_int(0)
    f = ctypes.c_float(0.0)
    calls = {
        "ftgemm_set_stream": lambda: L.ftgemm_set_stream(None, None),
        "ftgemm_get_schedule": lambda: L.ftgemm_get_schedule(None, 64, 64, 64, ft.F32, ft.FT_BLOCK,
                                                             ctypes.byref(sched)),
        "ftgemm_set_threshold": lambda: L.ftgemm_set_threshold(None, 0, 32.0, None, 0),
        "ftgemm_set_residual_sink": lambda: L.ftgemm_set_residual_sink(None, None, None, 0),
        "ftgemm_mlp_forward": lambda: L.ftgemm_mlp_forward(None, 8, None, None, None),
        "ftgemm_mlp_grad": lambda: L.ftgemm_mlp_grad(None, 8, None, None, None, None, ctypes.byref(f)),
        "ftgemm_mlp_train": lambda: L.ftgemm_mlp_train(None, 8, None, None, 1, 8, 1e-3, None, None),
        "ftgemm_set_fp8_scales": lambda: L.ftgemm_set_fp8_scales(None, 1.0, 1.0),
        "ftgemm_quantize": lambda: L.ftgemm_quantize(None, 8, None, None, ft.BF16, None),
        "ftgemm_autotune": lambda: L.ftgemm_autotune(None, 64, 64, 64, None, 64, None, 64, None, 64,
                                                     ft.FT_BLOCK, 1, ctypes.byref(sched), ctypes.byref(lv)),
        "ftgemm_encode": lambda: L.ftgemm_encode(None, 64, 64, 64, None, 64, None, 64, 16, 16,
                                                 None, None, None, None),
        "ftgemm_enable_timing": lambda: L.ftgemm_enable_timing(None, 1),
        "ftgemm_get_stats": lambda: L.ftgemm_get_stats(None, ctypes.byref(stats), 0),
    }
    for name, call in calls.items():
        assert call() == ft.ERR_ARG, name
        assert L.ftgemm_last_error(), name
    i64, vp = ctypes.c_int64, ctypes.c_void_p
    noalloc = L.ftgemm_gemm_noalloc
    noalloc.argtypes = [i64, i64, i64, ctypes.c_double, vp, i64, vp, i64, ctypes.c_double, vp, i64,
                        ctypes.c_int, vp, vp]
    noalloc.restype = ctypes.c_int
    assert noalloc(64, 64, 64, 1.0, None, 64, None, 64, 0.0, None, 64, ft.FT_BLOCK, None, None) == ft.ERR_ARG
    assert b"ftgemm_gemm_noalloc" in L.ftgemm_last_error()


def test_tensor_core_data_tile(libpath):
    # The 128 x 256 MMA tile gives up its last 3 (bf16) or 5 (e4m3) rows to
    # the pieces of e^T A and as many columns to those of B e at level TILE:
    # bf16 needs 3 pieces for the 24 significant bits of an fp32 checksum,
    # e4m3 5 pieces of scale steps of 16; the data columns are rounded down
    # to a multiple of 4 (16-byte stores of C); OFF computes the whole tile.
    import paper_2305_01024_gb300 as ft
    assert ft.tc_tile(ft.BF16, ft.FT_TILE) == (125, 252)
    assert ft.tc_tile(ft.E4M3, ft.FT_TILE) == (123, 248)
    assert ft.tc_tile(ft.BF16, ft.FT_OFF) == ft.tc_tile(ft.E4M3, ft.FT_OFF) == (128, 256)
    L = ft.lib()
    r = ctypes.c_int32()
    assert L.ftgemm_tc_tile(ft.F32, ft.FT_TILE, ctypes.byref(r), ctypes.byref(r)) == ft.ERR_UNSUPPORTED
    assert L.ftgemm_tc_tile(ft.BF16, ft.FT_BLOCK, ctypes.byref(r), ctypes.byref(r)) == ft.ERR_UNSUPPORTED
    assert L.ftgemm_tc_tile(ft.BF16, ft.FT_TILE, None, ctypes.byref(r)) == ft.ERR_ARG
