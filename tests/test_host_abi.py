"""Host-side checks of the C-ABI library without a GPU: it loads, it exports
every function include/hram.h declares, the Python binding names exactly
those, and the host-only calls (status strings, workspace sizing) answer
without touching a device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import casegen
from paper_2609_05494_b300 import _lib
from paper_2609_05494_b300 import build as libbuild
from paper_2609_05494_b300.api import make_params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hram.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s*(hr_\w+)\s*\(", src,
                                 flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return C.CDLL(_lib.LIB_PATH)


def test_header_declares_the_binding_exports():
    names = declared()
    assert len(names) >= 28
    assert set(names) == set(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    lib.hr_status_str.restype = C.c_char_p
    lib.hr_status_str.argtypes = [C.c_int]
    for code in (_lib.HR_OK, _lib.HR_EINVAL, _lib.HR_ENOMEM, _lib.HR_ECUDA, _lib.HR_ENAN,
                 _lib.HR_EDT, _lib.HR_ERANGE, _lib.HR_EIO):
        assert lib.hr_status_str(code)


def test_workspace_bytes_is_host_only_and_grows_with_n(lib):
    p = make_params(casegen.config_parity())
    lib.hr_workspace_bytes.argtypes = [C.c_void_p, C.c_int64, C.POINTER(C.c_size_t)]
    a, b = C.c_size_t(), C.c_size_t()
    assert lib.hr_workspace_bytes(C.byref(p), 5625, C.byref(a)) == _lib.HR_OK
    assert lib.hr_workspace_bytes(C.byref(p), 4 * 5625, C.byref(b)) == _lib.HR_OK
    assert b.value > a.value > 5625 * 40
    bad = make_params(dict(casegen.config_parity(), dx=-1.0))
    assert lib.hr_workspace_bytes(C.byref(bad), 5625, C.byref(a)) == _lib.HR_EINVAL


def test_split_pass_flags_checked_on_the_host(lib):
    # the split pass: refused with the one-kernel flag, a pass variant, the
    # tangent mode or the 5 x 5 stencil; its lists enlarge the workspace,
    # at any size when asked for, from 262,144 particles by default
    lib.hr_workspace_bytes.argtypes = [C.c_void_p, C.c_int64, C.POINTER(C.c_size_t)]
    base = casegen.config_parity()
    n = C.c_size_t()

    def ws(flags, nf=5625, **kw):
        p = make_params(dict(base, **kw), flags)
        rc = lib.hr_workspace_bytes(C.byref(p), nf, C.byref(n))
        return rc, n.value

    S, F = _lib.HR_FLAG_PASS_SPLIT, _lib.HR_FLAG_PASS_FUSED
    for bad in (S | F, S | _lib.HR_FLAG_PASS_LANES2, S | _lib.HR_FLAG_NEWTON3,
                S | _lib.HR_FLAG_STAGE_POS, S | _lib.HR_FLAG_TANGENT):
        assert ws(bad, dt_mode=1)[0] == _lib.HR_EINVAL, bad
    assert ws(S, cell_factor=0.5)[0] == _lib.HR_EINVAL
    rc0, fused = ws(0)
    rc1, split = ws(S)
    assert rc0 == rc1 == _lib.HR_OK and split > fused
    big = 300000
    assert ws(0, big)[1] > ws(F, big)[1] == ws(F, big)[1]
    assert ws(0, big)[1] == ws(S, big)[1]


def test_jacobian_refuses_a_zero_parameter():
    from paper_2609_05494_b300.grad import jacobian
    p = casegen.config_parity()
    with pytest.raises(ValueError):
        jacobian([0.02, 1480.0, 0.0], p, np.zeros((4, 2), np.float32), 1)
