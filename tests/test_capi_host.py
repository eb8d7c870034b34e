"""The C-ABI library builds, loads and exports every symbol that
include/lbm.h declares; argument validation that runs before any CUDA call
is checked on the host (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1111_1129_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.load()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(capi.SIGNATURES), set(names) ^ set(capi.SIGNATURES)


def test_abi_version(lib):
    assert capi.lbm_abi_version() == 2


def test_host_side_validation(lib):
    ordering = capi.make_ordering(capi.LBM_ORDER_LEX)
    out = ctypes.c_void_p()
    dims = (ctypes.c_int32 * 3)(4, 4, 4)
    assert lib.lbm_build_sparse(None, dims, ordering, None, ctypes.byref(out)) == capi.LBM_EINVAL
    assert "flags" in capi.lbm_last_error()
    bad = (ctypes.c_int32 * 3)(4, 0, 4)
    assert lib.lbm_build_sparse(1, bad, ordering, None, ctypes.byref(out)) == capi.LBM_EINVAL
    huge = (ctypes.c_int32 * 3)(2048, 1024, 1024)
    assert lib.lbm_build_sparse(1, huge, ordering, None, ctypes.byref(out)) == capi.LBM_EOVERFLOW
    assert "2^31" in capi.lbm_last_error()
    weird = capi.make_ordering(9)
    assert lib.lbm_build_sparse(1, dims, weird, None, ctypes.byref(out)) == capi.LBM_EINVAL
    blk0 = capi.make_ordering(capi.LBM_ORDER_BLOCKED, (0, 2, 2))
    assert lib.lbm_ordering_keys(dims, blk0, 1, None) == capi.LBM_EINVAL
    assert lib.lbm_state_create(None, 0, 0, ctypes.byref(out)) == capi.LBM_EINVAL
    f = (ctypes.c_double * 3)(0, 0, 0)
    assert lib.lbm_step(None, 1, 1.0, 1.0, f) == capi.LBM_EINVAL
    m, q = ctypes.c_double(), ctypes.c_double()
    assert lib.lbm_reduce_flux(None, 0, ctypes.byref(m), ctypes.byref(q)) == capi.LBM_EINVAL
    lib.lbm_free(None)
    with pytest.raises(capi.LbmError) as ei:
        capi.lbm_build_sparse(0, (4, 4, 4), ordering, 0)
    assert ei.value.status == capi.LBM_EINVAL


def test_allocator_needs_both_functions(lib):
    alloc = capi.LBM_ALLOC_FN(lambda nbytes, stream, ctx: None)
    assert lib.lbm_set_allocator(alloc, capi.LBM_FREE_FN(), None) == capi.LBM_EINVAL
    assert "both" in capi.lbm_last_error()
    # back to the library's own allocator (no handle is alive here)
    assert lib.lbm_set_allocator(capi.LBM_ALLOC_FN(), capi.LBM_FREE_FN(), None) == capi.LBM_OK


def test_missing_library_is_an_error_not_a_fallback(monkeypatch, tmp_path):
    """Without the CUDA library every entry point fails loudly; nothing falls
    back to another implementation."""
    monkeypatch.setattr(capi, "_lib", None)
    monkeypatch.setattr(capi, "library_path", lambda: str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="is missing"):
        capi.load()
    with pytest.raises(RuntimeError, match="is missing"):
        capi.lbm_abi_version()
