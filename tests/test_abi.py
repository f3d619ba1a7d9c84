"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and exports
every function include/wfq.h declares; the binding names the same set; calls that
fail argument checks before touching a device return the documented status."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "wfq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wfq_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2103_00438_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(wfq_\w+)", out))
    declared = set(_declared())
    assert declared, "no declarations parsed"
    assert declared <= exported, declared - exported


def test_binding_covers_header():
    from paper_2103_00438_gb300 import wfq
    assert sorted(wfq.EXPORTS) == _declared()


def test_library_loads_and_resolves(lib_path):
    L = ctypes.CDLL(lib_path)
    for name in _declared():
        assert getattr(L, name) is not None


def test_argument_errors_without_device(lib_path):
    from paper_2103_00438_gb300 import wfq
    L = wfq.load(lib_path)
    # NULL out-pointer is rejected before any CUDA call
    assert L.wfq_create(None, 0) == -1
    assert b"NULL" in L.wfq_last_error()
    # NULL handles
    assert L.wfq_build_geometry(None, 10, None, None, None, 0, None) == -1
    assert L.wfq_apply(None, 1, None, None, None, 0, None) == -1
    assert L.wfq_geometry_info(None, None, None, None) == -1
    assert L.wfq_destroy(None) == 0
    assert L.wfq_free_geometry(None) == 0


def test_sm103a_objects_built(lib_path):
    # every translation unit was compiled for sm_103a (ptxas log present and clean of spills
    # in the hot kernels)
    bdir = os.path.dirname(lib_path)
    logs = [f for f in os.listdir(bdir) if f.endswith(".o.log")]
    assert logs
    text = "".join(open(os.path.join(bdir, f)).read() for f in logs)
    assert "sm_103a" in text


def test_binding_buffer_layout_checks():
    """Caller buffers cross the ABI as plain pointers, so the binding must hand over
    C-contiguous memory of the right type: inputs are copied into that form, outputs
    that are not already in it are refused."""
    import numpy as np
    from paper_2103_00438_gb300 import wfq
    q = (np.arange(12.0) + 1j).reshape(4, 3)
    view = q[:, :1]                      # strided: its pointer would address q's row 0
    arr, ptr = wfq._buf(view, np.complex128, 4, 4, False, "q")
    assert arr.flags.c_contiguous and np.array_equal(arr.ravel(), q[:, 0]) and ptr == arr.ctypes.data
    arr, _ = wfq._buf(q.real, np.complex128, 4, 12, False, "x")     # converted to complex128
    assert arr.dtype == np.complex128
    with pytest.raises(ValueError):
        wfq._buf(np.empty((4, 6), np.complex128)[:, ::2], np.complex128, 4, 12, True, "y")
    with pytest.raises(ValueError):
        wfq._buf(np.empty((4, 3), np.complex64), np.complex128, 4, 12, True, "y")
    with pytest.raises(ValueError):
        wfq._buf(np.empty((5, 3), np.complex128), np.complex128, 4, 15, True, "y")
    out = np.empty((4, 3), np.complex128)
    assert wfq._buf(out, np.complex128, 4, 12, True, "y")[1] == out.ctypes.data
