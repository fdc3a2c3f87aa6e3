"""The C-ABI library loads and exports every symbol include/rsvd.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rsvd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\brsvd_status\s+(rsvd_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1607_01649_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rsvd_create", "rsvd_destroy", "rsvd_workspace_size", "rsvd_fixed_rank",
                     "rsvd_adaptive_tol", "rsvd_query_status", "rsvd_last_error_detail"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    for name in declared_functions():
        assert hasattr(built_lib, name), name


def test_binding_covers_every_declared_symbol():
    import paper_1607_01649_gb300 as rs
    assert sorted(rs.EXPORTED) == declared_functions()


def test_params_struct_layout():
    import paper_1607_01649_gb300 as rs
    # int k, p, q, block, max_rank, probe_cols; double tol; uint64 seed; int prec, flags
    assert ctypes.sizeof(rs.Params) == 6 * 4 + 8 + 8 + 2 * 4
    assert rs.Params.tol.offset == 24 and rs.Params.seed.offset == 32 and rs.Params.prec.offset == 40


def test_create_without_device_is_an_error_not_a_crash(built_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    built_lib.rsvd_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    assert built_lib.rsvd_create(ctypes.byref(h), 0) != 0


def test_batched_variant_table_without_a_device(built_lib):
    """The launch-variant table is host data: every variant keeps a number of
    rows in flight that divides the binary64 fold length (256 rows), so the
    fold points, and with them the results, are the same in every variant."""
    n = ctypes.c_int()
    assert built_lib.rsvd_batched_variants(ctypes.byref(n)) == 0 and n.value >= 2
    seen = set()
    for v in range(n.value):
        a, b = ctypes.c_int(), ctypes.c_int()
        assert built_lib.rsvd_batched_variant_info(v, ctypes.byref(a), ctypes.byref(b)) == 0
        assert a.value in (4, 8, 16, 32) and 256 % a.value == 0 and 1 <= b.value <= 4
        seen.add((a.value, b.value))
    assert len(seen) == n.value
    a, b = ctypes.c_int(), ctypes.c_int()
    assert built_lib.rsvd_batched_variant_info(n.value, ctypes.byref(a), ctypes.byref(b)) != 0
    assert built_lib.rsvd_batched_variant_info(-1, ctypes.byref(a), ctypes.byref(b)) != 0


def test_binding_fails_loudly_without_the_library(monkeypatch):
    """No fallback: with librsvd.so absent the binding raises instead of
    computing anything another way."""
    import paper_1607_01649_gb300 as rs
    monkeypatch.setattr(rs, "_lib", None)
    monkeypatch.setattr(rs, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "librsvd.so"))
    with pytest.raises(ImportError, match="librsvd.so not found"):
        rs.load()
    with pytest.raises(ImportError):
        rs.handle(0)
