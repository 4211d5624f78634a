"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/gravity.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

pytestmark = pytest.mark.abi


def _declared():
    src = open(os.path.join(ROOT, "include", "gravity.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"^\s*typedef[^;]*;", "", src, flags=re.M)     # function-pointer types
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("gravity_create", "gravity_destroy", "gravity_tree_build", "gravity_forces",
                 "gravity_direct", "leapfrog_step", "gravity_sync", "gravity_strerror",
                 "gravity_debug_export", "gravity_forces_host", "gravity_forces_host_batch",
                 "gravity_forces_vjp",
                 "leapfrog_adjoint", "gravity_diagnostics", "gravity_set_allocator",
                 "gravity_debug_set", "gravity_set_clouds", "gravity_batch_tree_build"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_1912_04197_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.gravity_strerror.restype = ctypes.c_char_p
    assert lib.gravity_strerror(-7) == b"no tree built"
    assert lib.gravity_strerror(0) == b"ok"


def test_params_default_needs_no_gpu():
    from paper_1912_04197_gb300 import build
    lib = ctypes.CDLL(build.build())
    buf = (ctypes.c_byte * 40)()
    lib.gravity_params_default(buf)
    G = ctypes.cast(buf, ctypes.POINTER(ctypes.c_double))[0]
    ints = ctypes.cast(ctypes.byref(buf, 8), ctypes.POINTER(ctypes.c_int32))
    assert G == 1.0 and [ints[i] for i in range(7)] == [0, 1, 0, 1, 0, -1, 1]
