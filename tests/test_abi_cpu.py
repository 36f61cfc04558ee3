"""The C-ABI library loads and exports every entry point include/lmep.h
declares; host-only validation paths answer without touching a GPU."""
import ctypes as C
import os

import pytest

from paper_2603_15964_gb300 import _lib


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2603_15964_gb300 import build
        build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _lib.declared_symbols()
    for required in ("lmep_create", "lmep_destroy", "lmep_build_operator", "lmep_expm",
                     "lmep_harvest_weights", "lmep_step", "lmep_step_batched", "lmep_batch_prepare",
                     "lmep_batch_workspace_bytes", "lmep_adjoint_step", "lmep_adjoint_scratch_bytes",
                     "lmep_sync_status", "lmep_status_string", "lmep_last_error", "lmep_fma_peak",
                     "lmep_version"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _lib.declared_symbols():
        assert hasattr(lib, name), name
    assert set(_lib.declared_symbols()) <= set(_lib._SIGS)


def test_host_only_calls(lib):
    assert lib.lmep_version().decode().startswith("lmep-gb300")
    assert lib.lmep_status_string(_lib.ERR_NONFINITE).decode() == "non-finite result"
    g = _lib.LmepGrid(1000, 0.01, 0, 9, 0, 0, 0, 0, 0.0, 0.0)
    out = C.c_size_t()
    assert lib.lmep_adjoint_scratch_bytes(C.byref(g), 0, C.byref(out)) == _lib.OK
    assert out.value >= 1000 * 10 * 8
    bad = _lib.LmepGrid(1000, 0.01, 0, 8, 0, 0, 0, 0, 0.0, 0.0)  # even stencil width
    assert lib.lmep_adjoint_scratch_bytes(C.byref(bad), 0, C.byref(out)) == _lib.ERR_INVALID
    assert "odd" in lib.lmep_last_error().decode()
    shifted = _lib.LmepGrid(1000, 0.01, 0, 9, 0, 0, 5, 0, 0.0, 0.0)  # |window_shift| > (n-1)/2
    assert lib.lmep_adjoint_scratch_bytes(C.byref(shifted), 0, C.byref(out)) == _lib.ERR_INVALID
    assert "window_shift" in lib.lmep_last_error().decode()
    reserved = _lib.LmepGrid(1000, 0.01, 0, 9, 0, 0, 0, 7, 0.0, 0.0)
    assert lib.lmep_adjoint_scratch_bytes(C.byref(reserved), 0, C.byref(out)) == _lib.ERR_INVALID


def test_batch_workspace_layout(lib):
    from paper_2603_15964_gb300 import Operator, lmep_batch_workspace_bytes
    Ns = [1024, 3000, 65536]
    hs = [2.0 / n for n in Ns]
    nbytes = lmep_batch_workspace_bytes(Ns, hs, ["periodic", "neumann", "periodic"], 9, "etdrk2",
                                        "allen_cahn", 1e-6, Operator(c2=1e-4), "mixed")
    tiles = sum((n + 2047) // 2048 for n in Ns)
    assert nbytes >= tiles * 8 + 3 * (32 + 8) + 3 * 9 * 3 * 9 * 4
    with pytest.raises(_lib.LmepError) as e:
        lmep_batch_workspace_bytes(Ns, hs, ["periodic", "dirichlet", "periodic"], 9, "etdrk2",
                                   "allen_cahn", 1e-6, Operator(c2=1e-4), "mixed")
    assert e.value.status == _lib.ERR_INVALID
