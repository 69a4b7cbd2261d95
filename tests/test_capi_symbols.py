"""The C-ABI library loads and exports every function include/ps.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ps_[A-Za-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libps():
    from paper_2502_08370_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    # the calls of the boundary: handles, slices and step counts, run to tolerance, state and
    # history, the plain comparator, the adjoint, batches and the autotuner
    for must in ("ps_grid_create", "ps_operator_create", "ps_splitting_create", "ps_problem_create",
                 "ps_problem_set_slices", "ps_run_parareal", "ps_get_state", "ps_get_history", "ps_last_error",
                 "ps_run_fine_sequential", "ps_adjoint", "ps_adjoint_vjp", "ps_batch_create", "ps_batch_add",
                 "ps_batch_run", "ps_batch_get_state", "ps_batch_destroy", "ps_autotune"):
        assert must in names, must


def test_every_declared_symbol_is_exported(libps):
    missing = [n for n in declared_functions() if not hasattr(libps, n)]
    assert not missing, missing


def test_abi_version_matches_header_and_binding(libps):
    import paper_2502_08370_gb300 as ps
    text = open(os.path.join(ROOT, "include", "ps.h")).read()
    header = int(re.search(r"#define PS_VERSION (\d+)", text).group(1))
    assert libps.ps_version() == header == ps.PS_VERSION


def test_binding_covers_the_header():
    import paper_2502_08370_gb300 as ps
    assert set(declared_functions()) <= set(ps.SIGNATURES), set(declared_functions()) - set(ps.SIGNATURES)


def test_host_side_validation_without_gpu(libps):
    """Argument checks run before any CUDA call: bad grids are rejected with a message."""
    import paper_2502_08370_gb300 as ps
    lib = ps.lib()
    h = ctypes.c_void_p()
    arr = (ctypes.c_int * 3)(0, 5, 1)
    assert lib.ps_grid_create(2, ctypes.byref(arr), ctypes.byref(h)) == 1
    assert b"grid size" in lib.ps_last_error()
    assert lib.ps_grid_create(4, ctypes.byref(arr), ctypes.byref(h)) == 1
    arr = (ctypes.c_int * 3)(5, 6, 7)
    assert lib.ps_grid_create(3, ctypes.byref(arr), ctypes.byref(h)) == 0
    assert lib.ps_grid_destroy(h) == 0
    # the wait-limit self-test validates its limit before touching the device
    assert lib.ps_selftest_wait_timeout(0, 0) == 1
    assert b"limit_us" in lib.ps_last_error()


def test_handle_calls_reject_null_handles(libps):
    """The new handle calls check their arguments before any CUDA call."""
    import paper_2502_08370_gb300 as ps
    lib = ps.lib()
    assert lib.ps_problem_set_slices(None, 4, 1, 4, 0) == 1
    assert lib.ps_batch_add(None, None, 0) == 1
    assert lib.ps_batch_get_state(None, 0, 0, None, 0) == 1
    h = ctypes.c_void_p()
    assert lib.ps_batch_create(None, -1, 0, ctypes.byref(h)) == 1
    assert lib.ps_adjoint(None, None, 1e-8, 0, None, None, 0, None, None) == 1
