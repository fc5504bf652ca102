"""The C ABI library builds for sm_103a, loads without a GPU and exports
every function that include/psc.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_1709_08681_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "psc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:psc_status|void|int|long long|const char \*)\s*(psc_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_function():
    lib = ctypes.CDLL(build.build())
    names = declared_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(_abi.EXPORTS) == names


def test_binding_loads_and_reports_argument_errors_without_a_device():
    L = _abi.lib()
    o = _abi.psc_solve_opts_default()
    assert o.max_iter == 50 and o.mode == _abi.PSC_LM_FULL and abs(o.block_gain - 0.5) < 1e-15
    # argument checks run before any CUDA call
    h = ctypes.c_void_p()
    st = L.psc_create(ctypes.byref(h), None, None, None, None, None)
    assert st == _abi.PSC_ERR_ARG and not h.value
    assert b"NULL" in L.psc_last_error(None)
    gd = _abi.psc_grid_desc(63, 128, 1e-5, 32, 20)    # odd image size
    st = L.psc_model_grid(ctypes.byref(gd), None, None, None)
    assert st == _abi.PSC_ERR_ARG
    assert L.psc_lm_restart(None) == _abi.PSC_ERR_ARG


def test_stack_calls_check_their_arguments_without_a_device():
    """The residual-w stack's calls refuse bad arguments before any CUDA call."""
    L = _abi.lib()
    D = ctypes.POINTER(ctypes.c_double)
    x = (ctypes.c_double * 8)()
    lo, hi = ctypes.c_double(), ctypes.c_double()
    assert L.psc_set_wstack(None, None, 0, 0.0, 1.0, 0.0, 0.0) == _abi.PSC_ERR_ARG        # no context
    assert L.psc_wstack_range(None, 10, 0.0, 0.0, ctypes.byref(lo), ctypes.byref(hi), None) == _abi.PSC_ERR_ARG
    assert L.psc_wstack_range(ctypes.addressof(x), 0, 0.0, 0.0, ctypes.byref(lo), ctypes.byref(hi),
                              None) == _abi.PSC_ERR_ARG                                 # no rows
    for n_planes, dw in ((1, 10.0), (4, 0.0), (4, float("nan"))):
        assert L.psc_model_grid_wstack(1, ctypes.cast(x, D), 64, 1e-5, n_planes, 0.0, dw, ctypes.addressof(x),
                                       None) == _abi.PSC_ERR_ARG
    assert L.psc_model_grid_wstack(1, ctypes.cast(x, D), 63, 1e-5, 4, 0.0, 10.0, ctypes.addressof(x),
                                   None) == _abi.PSC_ERR_ARG                            # odd grid
    assert b"n_grid" in L.psc_last_error(None)
