"""Argument checks of the Python binding that run before any library call
(CPU): an output the library would overrun, or an initial guess too short for
it to read, is refused with ValueError instead of being passed as a raw
pointer."""
import ctypes

import numpy as np
import pytest

from paper_1809_00845_gb300 import bem


def _shell_plan(nb=8, precision=bem.BEM_F32):
    """A Plan object with no device state (null handle): enough for the
    binding's own checks; any call that reaches the library gets BEM_ERR_ARG."""
    p = bem.Plan.__new__(bem.Plan)
    p.nb, p.ncomp, p.precision, p.dim, p.kernel = nb, 1, precision, 2, bem.BEM_LAPLACE_2D
    p._h = ctypes.c_void_p()
    return p


def test_output_tensor_checks():
    torch = pytest.importorskip("torch")
    x = torch.zeros(8, dtype=torch.float32)
    bem._check_out_tensor(x, torch.empty_like(x))  # what every caller passes
    bad = [torch.zeros(8, dtype=torch.float64), torch.zeros(7, dtype=torch.float32),
           torch.zeros(16, dtype=torch.float32)[::2], x, x.view(8)]
    for out in bad:
        with pytest.raises(ValueError):
            bem._check_out_tensor(x, out)
    big = torch.zeros(12, dtype=torch.float32)
    with pytest.raises(ValueError):  # partial overlap
        bem._check_out_tensor(big[:8], big[4:12])
    with pytest.raises(ValueError):
        bem._check_out_tensor(x, np.zeros(8, np.float32))


def test_apply_host_output_checks():
    p = _shell_plan()
    x = np.arange(8, dtype=np.float32)
    for out in (np.zeros(7, np.float32), np.zeros(8, np.float64), np.zeros(16, np.float32)[::2], x):
        with pytest.raises(ValueError):
            p.apply_host("single", x, out)
    ro = np.zeros(8, np.float32)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        p.apply_host("single", x, ro)
    with pytest.raises(ValueError):
        p.apply_host("single", np.zeros(7, np.float32))
    # a valid call reaches the library, which refuses the null plan
    with pytest.raises(bem.BemError) as e:
        p.apply_host("single", x, np.zeros(8, np.float32))
    assert e.value.status == bem.BEM_ERR_ARG


def test_solve_initial_guess_size():
    p = _shell_plan()
    bc = np.zeros(8, np.uint8)
    data = np.ones(8)
    with pytest.raises(ValueError):
        p.solve(bc, data, x0=np.zeros(7))
    with pytest.raises(ValueError):
        p.solve(bc[:7], data)
    with pytest.raises(bem.BemError) as e:
        p.solve(bc, data, x0=np.zeros(8))
    assert e.value.status == bem.BEM_ERR_ARG
