"""The C-ABI library builds, loads and exports every symbol include/bem.h
declares; host-side argument checks reject bad input before any device call
(no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1809_00845_gb300 import bem, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return bem.load_library()


def _declared():
    txt = open(os.path.join(ROOT, "include", "bem.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(bem_[a-z_]+)\s*\(", txt, re.M)))


def test_header_declares_the_abi():
    names = _declared()
    for n in ["bem_plan", "bem_apply", "bem_solve", "bem_destroy", "bem_status_string", "bem_set_bc"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) <= set(bem.EXPORTED) | set(_declared())


def test_status_strings(lib):
    for s in range(9):
        assert lib.bem_status_string(s)


def _plan_rc(dim, n, h, cell, w, normal, kernel=0, prec=1, flags=0, nu=0.3, mu=1.0):
    lib = bem.load_library()
    hnd = ctypes.c_void_p()
    nn = np.full(dim, n, dtype=np.int64) if np.isscalar(n) else np.asarray(n, dtype=np.int64)
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    normal = np.ascontiguousarray(normal, dtype=np.float64)
    rc = lib.bem_plan(ctypes.byref(hnd), dim, bem._ptr(nn), h, cell.shape[0], bem._ptr(cell), bem._ptr(w),
                      bem._ptr(normal), kernel, nu, mu, prec, flags, None)
    return rc, lib.bem_last_error().decode()


def test_rejects_bad_arguments_on_host(lib):
    cell = np.array([[1, 2], [3, 4]])
    w = np.ones(2)
    nrm = np.array([[1.0, 0.0], [0.0, 1.0]])
    assert _plan_rc(2, 8, 0.125, [[1, 2], [1, 2]], w, nrm)[0] == bem.BEM_ERR_ARG       # duplicate
    assert _plan_rc(2, 8, 0.125, [[1, 2], [8, 4]], w, nrm)[0] == bem.BEM_ERR_ARG       # outside the grid
    assert _plan_rc(2, 8, 0.125, [[1, -1], [3, 4]], w, nrm)[0] == bem.BEM_ERR_ARG      # negative index
    assert _plan_rc(2, 8, -1.0, cell, w, nrm)[0] == bem.BEM_ERR_ARG                    # h <= 0
    assert _plan_rc(2, 8, 0.125, cell, [1.0, np.nan], nrm)[0] == bem.BEM_ERR_ARG       # non-finite weight
    assert _plan_rc(2, 12, 1 / 12, cell, w, nrm)[0] == bem.BEM_ERR_UNSUPPORTED         # n not a power of two
    assert _plan_rc(3, 8, 0.125, cell, w, nrm)[0] == bem.BEM_ERR_ARG                   # dim vs kernel
    assert _plan_rc(2, 8, 0.125, cell, w, nrm, flags=6)[0] == bem.BEM_ERR_ARG          # unknown flags
    assert _plan_rc(2, 8, 0.125, cell, w, nrm, prec=9)[0] == bem.BEM_ERR_ARG           # precision
    assert _plan_rc(2, 8, 0.125, cell, w, nrm, prec=2)[0] == bem.BEM_ERR_UNSUPPORTED   # f32x2 below n = 256
    empty = np.zeros((0, 2))
    assert _plan_rc(2, 8, 0.125, empty, np.zeros(0), empty)[0] == bem.BEM_ERR_ARG       # empty boundary
    assert _plan_rc(2, 8, 0.125, cell, w, [[np.inf, 0.0], [0.0, 1.0]])[0] == bem.BEM_ERR_ARG  # non-finite normal
    assert _plan_rc(2, 2, 0.5, [[0, 1], [1, 0]], w, nrm)[0] == bem.BEM_ERR_UNSUPPORTED  # n < 4
    assert _plan_rc(2, [8, 16], 0.125, cell, w, nrm)[0] == bem.BEM_ERR_UNSUPPORTED     # unequal axes
    cell3 = np.array([[1, 2, 3], [3, 4, 5]])
    nrm3 = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    for nu, mu in ((0.5, 1.0), (-1.0, 1.0), (0.3, 0.0), (0.3, -2.0)):  # Kelvin material out of range
        assert _plan_rc(3, 16, 1 / 16, cell3, w, nrm3, kernel=2, nu=nu, mu=mu)[0] == bem.BEM_ERR_ARG
    for tc in (bem.BEM_TC_BF16X3, bem.BEM_TC_F16X3):  # tensor-core stages: 2D, n = 1024 ... 4096 only
        assert _plan_rc(2, 512, 1 / 512, cell, w, nrm, prec=tc)[0] == bem.BEM_ERR_UNSUPPORTED
        assert _plan_rc(2, 8192, 1 / 8192, cell, w, nrm, prec=tc)[0] == bem.BEM_ERR_UNSUPPORTED
        assert _plan_rc(3, 1024, 1 / 1024, cell3, w, nrm3, kernel=1, prec=tc)[0] == bem.BEM_ERR_UNSUPPORTED
    rc = lib.bem_plan(None, 2, None, 0.1, 1, None, None, None, 0, 0.3, 1.0, 1, 0, None)
    assert rc == bem.BEM_ERR_ARG
    assert lib.bem_apply(None, 0, None, None, 1, None) == bem.BEM_ERR_ARG
    assert lib.bem_destroy(None) == bem.BEM_OK
    assert lib.bem_device_status(None, None) == bem.BEM_ERR_ARG


def test_binding_calls_only_declared_functions():
    """Every library function the Python binding calls is declared in
    include/bem.h (the binding and the header cannot drift apart)."""
    src = open(os.path.join(ROOT, "paper_1809_00845_gb300", "bem.py")).read()
    called = set(re.findall(r"\.(bem_[a-z_]+)\b", src))
    assert called, "no library calls found"
    missing = sorted(called - set(_declared()))
    assert not missing, missing
