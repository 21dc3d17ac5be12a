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


def test_plan_geometry_shapes():
    cell = np.array([[1, 2], [3, 4]])
    w = np.ones(2)
    nrm = np.array([[1.0, 0.0], [0.0, 1.0]])
    for args in ((2, 8, 0.125, np.array([[1, 2, 3], [3, 4, 5]]), w, nrm),      # cell columns != dim
                 (2, 8, 0.125, np.array([1, 2, 3, 4]), w, nrm),                # cell not (nb, dim)
                 (2, 8, 0.125, cell, np.ones(3), nrm),                         # w size
                 (2, 8, 0.125, cell, w, np.ones(3)),                           # normal size
                 (2, [8, 8, 8], 0.125, cell, w, nrm)):                         # n per axis
        with pytest.raises(ValueError):
            bem.Plan(*args)
    with pytest.raises(ValueError):
        bem.Plan.from_panels(8, 0.125, np.zeros((3, 3)))


def test_boundary_condition_sizes():
    p = _shell_plan()
    with pytest.raises(ValueError):
        p.set_bc(np.zeros(7, np.uint8))
    with pytest.raises(ValueError):
        p.tune_preconditioner(np.zeros(8, np.uint8), np.ones(7))
    with pytest.raises(bem.BemError) as e:  # right size: the library refuses the null plan
        p.set_bc(np.zeros(8, np.uint8))
    assert e.value.status == bem.BEM_ERR_ARG


def test_batch_initial_guess_size():
    b = bem.Batch.__new__(bem.Batch)
    b.total, b.plans, b._h = 10, [None, None], ctypes.c_void_p()
    with pytest.raises(ValueError):
        b.solve(np.zeros(10, np.uint8), np.ones(10), x0=np.zeros(9))
    with pytest.raises(ValueError):
        b.solve(np.zeros(9, np.uint8), np.ones(10))


def test_network_batch_shapes():
    net = bem.Net.__new__(bem.Net)
    net.cin, net.nparams, net._h = 3, 10, ctypes.c_void_p()
    with pytest.raises(ValueError):
        net.set_params(np.zeros(9, np.float32))
    f = np.zeros((5, 3), np.float32)
    for feats, off in ((np.zeros((5, 4), np.float32), [0, 5]),   # channels != cin
                       (np.zeros(15, np.float32), [0, 5]),        # not (T, cin)
                       (f, [0, 3]),                               # does not end at T
                       (f, [1, 5]),                               # does not start at 0
                       (f, [0, 4, 2, 5]),                         # decreasing
                       (f, [0])):                                 # no sequence
        with pytest.raises(ValueError):
            net.forward(feats, np.asarray(off, np.int32))
    with pytest.raises(ValueError):
        net.gradient(f, np.array([0, 5], np.int32), np.zeros(4, np.float32))
    with pytest.raises(ValueError):
        net.train_step(f, np.array([0, 5], np.int32), np.zeros(6, np.float32))


def test_valid_arguments_pass_the_checks():
    """The shapes every caller uses pass: a valid network batch (host or torch
    CPU offsets), and valid geometry reaches the library (which, without a
    GPU, fails at its first CUDA call)."""
    torch = pytest.importorskip("torch")
    net = bem.Net.__new__(bem.Net)
    net.cin, net.nparams, net._h = 3, 10, ctypes.c_void_p()
    f = np.zeros((5, 3), np.float32)
    net._check_batch(f, np.array([0, 2, 5], np.int32), np.zeros(5, np.float32))
    net._check_batch(torch.zeros(5, 3), torch.tensor([0, 5], dtype=torch.int32), torch.zeros(5))
    net._check_batch(f.tolist(), [0, 5], [0.0] * 5)
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_1809_00845_gb300 import inputs as I
    b = I.curve_panels(64, I.circle_curve(0.35))
    with pytest.raises(bem.BemError) as e:
        bem.Plan.from_panel_boundary(b, "f32", 3, 3)
    assert e.value.status == bem.BEM_ERR_CUDA


def test_tensor_on_another_gpu_is_refused():
    """A plan records the GPU it was built on; a tensor on another GPU is
    refused before its pointer reaches the library (the kernels would run on
    the plan's GPU with addresses of the other one)."""
    torch = pytest.importorskip("torch")

    class FakeTensor:
        def __init__(self, dev):
            self.device = torch.device(dev)
    bem._check_tensor_device(0, FakeTensor("cuda:0"))
    bem._check_tensor_device(None, FakeTensor("cuda:3"))  # no device recorded (no CUDA at plan time)
    bem._check_tensor_device(1, FakeTensor("cpu"))       # host tensors are refused elsewhere
    with pytest.raises(ValueError):
        bem._check_tensor_device(0, FakeTensor("cuda:1"))
    with pytest.raises(ValueError):
        bem._check_tensor_device(2, FakeTensor("cuda:0"))
