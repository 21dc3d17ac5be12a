"""Thin Python binding of the C ABI in include/bem.h (argument marshalling only).

Every step of an apply or a solve runs in the CUDA kernels of libbem_gb300.so;
this module converts arrays, passes raw pointers and maps status codes to
exceptions.  PyTorch is used only to hold device memory and to name the
current CUDA stream.  There is no CPU fallback: if the library is missing the
import of the binding raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbem_gb300.so")

BEM_OK, BEM_ERR_ARG, BEM_ERR_CUDA, BEM_ERR_OOM, BEM_ERR_NOT_CONVERGED = 0, 1, 2, 3, 4
BEM_ERR_BREAKDOWN, BEM_ERR_NONFINITE, BEM_ERR_TIMEOUT, BEM_ERR_UNSUPPORTED = 5, 6, 7, 8
BEM_LAPLACE_2D, BEM_LAPLACE_3D, BEM_KELVIN_3D = 0, 1, 2
BEM_F64, BEM_F32, BEM_F32X2, BEM_TC_BF16X3, BEM_TC_F16X3 = 0, 1, 2, 3, 4
BEM_SINGLE, BEM_DOUBLE, BEM_SYSTEM = 0, 1, 2
BEM_PLAN_SINGLE_LAYER_ONLY, BEM_PLAN_THREE_PASS = 1, 2
BEM_TEST_WAIT_RUNS_OUT = 1
BEM_TEST_HOST_ARNOLDI = 2

KERNELS = {"laplace2d": BEM_LAPLACE_2D, "laplace3d": BEM_LAPLACE_3D, "kelvin3d": BEM_KELVIN_3D}
PRECISIONS = {"f64": BEM_F64, "f32": BEM_F32, "f32x2": BEM_F32X2, "tc_bf16x3": BEM_TC_BF16X3,
              "tc_f16x3": BEM_TC_F16X3}
# precisions whose plans take and return float32 vectors
F32_IO = (BEM_F32, BEM_TC_BF16X3, BEM_TC_F16X3)
LAYERS = {"single": BEM_SINGLE, "double": BEM_DOUBLE, "system": BEM_SYSTEM}

EXPORTED = ["bem_plan", "bem_plan_panels", "bem_set_bc", "bem_set_preconditioner", "bem_apply", "bem_apply_host", "bem_apply_static_scratch", "bem_solve",
            "bem_get_info", "bem_enable_refinement", "bem_set_kernel_timing", "bem_kernel_time", "bem_launches_per_apply", "bem_device_status", "bem_set_test_flags", "bem_destroy",
            "bem_status_string", "bem_last_error", "bem_batch_create", "bem_batch_buffers", "bem_batch_offset",
            "bem_batch_apply", "bem_batch_set_grouping", "bem_batch_launches", "bem_batch_destroy", "bem_batch_solve", "bem_tune_batch",
            "bem_tune_preconditioner", "bem_tune_shapes", "bem_net_create", "bem_net_destroy", "bem_net_num_params",
            "bem_net_get_params", "bem_net_set_params", "bem_net_forward", "bem_net_gradient", "bem_net_train_step",
            "bem_measure_peak", "bem_dtn_estimate", "bem_guess_features", "bem_guess_finish", "bem_fourier_features"]


class BemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("rel_residual_est", ctypes.c_double), ("seconds", ctypes.c_double), ("applies", ctypes.c_int),
                ("refine_steps", ctypes.c_int), ("rel_residual_fp64", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PlanInfo(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("ncomp", ctypes.c_int), ("n", ctypes.c_int64), ("N", ctypes.c_int64),
                ("nb", ctypes.c_int64), ("precision", ctypes.c_int), ("grid_ctas", ctypes.c_int),
                ("threads_per_cta", ctypes.c_int), ("scratch_bytes", ctypes.c_size_t),
                ("spectra_bytes", ctypes.c_size_t), ("plan_seconds", ctypes.c_double),
                ("grid_nodes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libbem_gb300.so; raise if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libbem_gb300.so not built ({path}); run paper_1809_00845_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I64, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    lib.bem_plan.argtypes = [ctypes.POINTER(P), I, P, D, I64, P, P, P, I, D, D, I, ctypes.c_uint32, P]
    lib.bem_plan_panels.argtypes = [ctypes.POINTER(P), I64, D, I64, P, I, I, I, ctypes.c_uint32, P]
    lib.bem_set_bc.argtypes = [P, P, D]
    lib.bem_set_preconditioner.argtypes = [P, I, I]
    lib.bem_enable_refinement.argtypes = [P, I]
    lib.bem_apply.argtypes = [P, I, P, P, I, P]
    lib.bem_apply_host.argtypes = [P, I, P, P, P]
    lib.bem_apply_static_scratch.argtypes = [P, I, P, P, P]
    lib.bem_solve.argtypes = [P, P, P, D, D, I, I, P, P, P, ctypes.POINTER(SolveInfo), P]
    lib.bem_get_info.argtypes = [P, ctypes.POINTER(PlanInfo)]
    lib.bem_set_kernel_timing.argtypes = [P, I]
    lib.bem_kernel_time.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(I64)]
    lib.bem_launches_per_apply.argtypes = [P, I]
    lib.bem_launches_per_apply.restype = I
    lib.bem_device_status.argtypes = [P, P]
    lib.bem_set_test_flags.argtypes = [P, ctypes.c_uint32]
    lib.bem_destroy.argtypes = [P]
    lib.bem_status_string.argtypes = [I]
    lib.bem_status_string.restype = ctypes.c_char_p
    lib.bem_batch_create.argtypes = [ctypes.POINTER(P), P, I, I, I, P]
    lib.bem_batch_buffers.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(ctypes.c_size_t)]
    lib.bem_batch_offset.argtypes = [P, I, ctypes.POINTER(ctypes.c_size_t)]
    lib.bem_batch_apply.argtypes = [P, P]
    lib.bem_batch_set_grouping.argtypes = [P, I]
    lib.bem_batch_launches.argtypes = [P]
    lib.bem_batch_launches.restype = I
    lib.bem_batch_destroy.argtypes = [P]
    lib.bem_batch_solve.argtypes = [P, P, P, D, D, I, I, P, P, P, ctypes.POINTER(SolveInfo), P]
    lib.bem_tune_batch.argtypes = [P, I, ctypes.POINTER(I)]
    lib.bem_tune_preconditioner.argtypes = [P, P, P, D, D, I, I, ctypes.POINTER(I)]
    lib.bem_tune_shapes.argtypes = [P, I, P, ctypes.POINTER(I), ctypes.POINTER(D)]
    lib.bem_tune_shapes.restype = I
    for name in ("bem_batch_create", "bem_batch_buffers", "bem_batch_offset", "bem_batch_apply", "bem_batch_destroy",
                 "bem_batch_set_grouping",
                 "bem_batch_solve", "bem_tune_batch", "bem_tune_preconditioner"):
        getattr(lib, name).restype = I
    lib.bem_net_create.argtypes = [ctypes.POINTER(P), I, I, I, I, P, ctypes.c_uint64]
    lib.bem_net_destroy.argtypes = [P]
    lib.bem_net_num_params.argtypes = [P]
    lib.bem_net_num_params.restype = I64
    lib.bem_net_get_params.argtypes = [P, P]
    lib.bem_net_set_params.argtypes = [P, P]
    lib.bem_net_forward.argtypes = [P, P, P, I, I64, P, P]
    lib.bem_net_gradient.argtypes = [P, P, P, I, I64, P, P, ctypes.POINTER(D), P]
    lib.bem_net_train_step.argtypes = [P, P, P, I, I64, P, ctypes.c_float, ctypes.POINTER(D), P]
    for name in ("bem_net_create", "bem_net_destroy", "bem_net_get_params", "bem_net_set_params", "bem_net_forward",
                 "bem_net_gradient", "bem_net_train_step"):
        getattr(lib, name).restype = I
    lib.bem_dtn_estimate.argtypes = [P, P, P, P, I, I64, I, P, P]
    lib.bem_dtn_estimate.restype = I
    lib.bem_guess_features.argtypes = [P, I, P, P, P, I, I64, ctypes.c_float, P, P]
    lib.bem_guess_features.restype = I
    lib.bem_guess_finish.argtypes = [P, P, P, P, P, I, I64, ctypes.c_float, P, P]
    lib.bem_guess_finish.restype = I
    lib.bem_fourier_features.argtypes = [P, I64, P, I, P, P]
    lib.bem_fourier_features.restype = I
    lib.bem_measure_peak.argtypes = [I, ctypes.POINTER(D), P]
    lib.bem_measure_peak.restype = I
    lib.bem_last_error.argtypes = []
    lib.bem_last_error.restype = ctypes.c_char_p
    for name in ("bem_plan", "bem_plan_panels", "bem_set_bc", "bem_set_preconditioner", "bem_enable_refinement", "bem_apply",
                 "bem_apply_static_scratch", "bem_apply_host", "bem_solve", "bem_get_info",
                 "bem_set_kernel_timing", "bem_kernel_time", "bem_device_status", "bem_set_test_flags",
                 "bem_destroy"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def _check(rc: int, allow=()):
    if rc != BEM_OK and rc not in allow:
        lib = load_library()
        raise BemError(rc, f"{lib.bem_status_string(rc).decode()}: {lib.bem_last_error().decode()}")
    return rc


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


_OFFSETS_CACHE = {}


def _device_offsets(oh):
    """A CUDA int32 copy of the host sequence offsets oh (already checked),
    reused while the same offsets come back (a few recent ones are kept), so
    repeated calls on one batch layout upload nothing."""
    import torch
    key = oh.astype(np.int32).tobytes()
    t = _OFFSETS_CACHE.get(key)
    if t is None:
        if len(_OFFSETS_CACHE) >= 16:
            _OFFSETS_CACHE.pop(next(iter(_OFFSETS_CACHE)))
        t = torch.from_numpy(np.frombuffer(key, dtype=np.int32).copy()).to("cuda")
        _OFFSETS_CACHE[key] = t
    return t


def _stream_ptr(stream):
    import torch
    if stream is None:
        if not torch.cuda.is_available():
            return ctypes.c_void_p(0)
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


@dataclass
class Geometry:
    dim: int
    n: int
    h: float
    cell: np.ndarray
    w: np.ndarray
    normal: np.ndarray


def _current_device():
    """Index of the current CUDA device (the one a plan is built on), or None."""
    import torch
    return torch.cuda.current_device() if torch.cuda.is_available() else None


def _check_tensor_device(plan_device, t):
    """A tensor handed to a plan's kernels must live on the plan's GPU (the
    library would otherwise launch on one device with pointers into another)."""
    if plan_device is not None and t.device.type == "cuda" and t.device.index is not None \
            and t.device.index != plan_device:
        raise ValueError(f"tensor on {t.device}, but the plan was built on cuda:{plan_device}")


def _check_out_tensor(x, out):
    """An output tensor for an apply of x: same device, dtype and size as x,
    contiguous, and not overlapping x (the library writes nb*ncomp values)."""
    import torch
    if not (isinstance(out, torch.Tensor) and out.device == x.device and out.dtype == x.dtype
            and out.is_contiguous() and out.numel() == x.numel()):
        raise ValueError("out must be a contiguous tensor on the input's device, of its dtype and size")
    nbytes = x.numel() * x.element_size()
    xa, oa = x.data_ptr(), out.data_ptr()
    if xa < oa + nbytes and oa < xa + nbytes:
        raise ValueError("out must not overlap the input")


class Plan:
    """Owning wrapper of a bem_plan_t."""

    def __init__(self, dim, n, h, cell, w, normal, kernel="laplace2d", precision="f32", nu=0.3, mu=1.0,
                 stream=None, flags=0):
        lib = load_library()
        self.kernel = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.dim = int(dim)
        self.ncomp = 3 if self.kernel == BEM_KELVIN_3D else 1
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.float64)
        normal = np.ascontiguousarray(normal, dtype=np.float64)
        self.nb = int(cell.shape[0]) if cell.ndim == 2 else -1
        nn = np.ascontiguousarray(np.full(self.dim, int(n), dtype=np.int64) if np.isscalar(n) else n,
                                  dtype=np.int64).reshape(-1)
        self._h = ctypes.c_void_p()
        if cell.ndim != 2 or cell.shape[1] != self.dim or w.size != self.nb or normal.size != self.nb * self.dim:
            raise ValueError("cell must be (nb, dim), w hold nb values and normal nb*dim values")
        if nn.size != self.dim:
            raise ValueError("n must be a scalar or hold dim grid sizes")
        rc = lib.bem_plan(ctypes.byref(self._h), self.dim, _ptr(nn), float(h), self.nb, _ptr(cell), _ptr(w),
                          _ptr(normal), self.kernel, float(nu), float(mu), self.precision, int(flags),
                          _stream_ptr(stream))
        _check(rc)
        self.torch_dtype = None
        self.device = _current_device()

    @classmethod
    def from_boundary(cls, b, kernel="laplace2d", precision="f32", **kw):
        return cls(b.dim, b.n, b.h, b.cell, b.w, b.normal, kernel=kernel, precision=precision, **kw)

    @classmethod
    def from_panels(cls, n, h, panels, precision="f32", order=3, near_radius=3, stream=None):
        """Accuracy-mode plan (bem_plan_panels): panels (nb, 4) = A.x, A.y, B.x, B.y."""
        lib = load_library()
        self = cls.__new__(cls)
        self.kernel = BEM_LAPLACE_2D
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.dim = 2
        self.ncomp = 1
        panels = np.ascontiguousarray(panels, dtype=np.float64)
        self._h = ctypes.c_void_p()
        if panels.ndim != 2 or panels.shape[1] != 4:
            raise ValueError("panels must be (nb, 4): A.x, A.y, B.x, B.y")
        self.nb = int(panels.shape[0])
        _check(lib.bem_plan_panels(ctypes.byref(self._h), int(n), float(h), self.nb, _ptr(panels), int(order),
                                   int(near_radius), self.precision, 0, _stream_ptr(stream)))
        self.torch_dtype = None
        self.device = _current_device()
        return self

    @classmethod
    def from_panel_boundary(cls, b, precision="f32", order=3, near_radius=3, stream=None):
        return cls.from_panels(b.n, b.h, b.panels, precision, order, near_radius, stream)

    # --------------------------------------------------------------- helpers
    @property
    def np_dtype(self):
        return np.float32 if self.precision in F32_IO else np.float64

    def _tdtype(self):
        import torch
        return torch.float32 if self.precision in F32_IO else torch.float64

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().bem_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ calls
    def set_bc(self, bc, c=0.5):
        bc = np.ascontiguousarray(bc, dtype=np.uint8).reshape(-1)
        if bc.size != self.nb * self.ncomp:
            raise ValueError("bc must hold nb*ncomp values")
        _check(load_library().bem_set_bc(self._h, _ptr(bc), float(c)))

    def set_preconditioner(self, kind="block", block_size=64):
        k = {"none": 0, "block": 1}[kind] if isinstance(kind, str) else int(kind)
        _check(load_library().bem_set_preconditioner(self._h, k, int(block_size)))

    def enable_refinement(self, enable=True):
        _check(load_library().bem_enable_refinement(self._h, 1 if enable else 0))

    def apply(self, layer, x, out=None, stream=None):
        """Device apply.  x: CUDA tensor of nb*ncomp plan-precision values, or
        of nbatch*nb*ncomp values (shape (nbatch, nb*ncomp) or flat): every
        vector through the same operator (bem_apply's nbatch)."""
        import torch
        lay = LAYERS[layer] if isinstance(layer, str) else int(layer)
        if not (isinstance(x, torch.Tensor) and x.is_cuda):
            raise TypeError("apply expects a CUDA tensor; use apply_host for host arrays")
        m = self.nb * self.ncomp
        if x.dtype != self._tdtype() or not x.is_contiguous() or x.numel() < m or x.numel() % m != 0:
            raise ValueError("input must be a contiguous tensor of nbatch*nb*ncomp values in the plan precision")
        _check_tensor_device(getattr(self, "device", None), x)
        if out is None:
            out = torch.empty_like(x)
        else:
            _check_out_tensor(x, out)
        _check(load_library().bem_apply(self._h, lay, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                        x.numel() // m, _stream_ptr(stream)))
        return out

    def apply_host(self, layer, x, out=None, stream=None):
        lay = LAYERS[layer] if isinstance(layer, str) else int(layer)
        x = np.ascontiguousarray(x, dtype=self.np_dtype).reshape(-1)
        if x.size != self.nb * self.ncomp:
            raise ValueError("input must hold nb*ncomp values")
        if out is None:
            out = np.empty_like(x)
        elif not (isinstance(out, np.ndarray) and out.dtype == x.dtype and out.size == x.size
                  and out.flags.c_contiguous and out.flags.writeable):
            raise ValueError("out must be a writeable contiguous array of nb*ncomp values in the plan precision")
        elif np.shares_memory(out, x):
            raise ValueError("out must not overlap the input")
        _check(load_library().bem_apply_host(self._h, lay, _ptr(x), _ptr(out), _stream_ptr(stream)))
        return out

    def solve(self, bc, data, c=0.5, tol=1e-6, max_iter=2000, restart=50, x0=None, stream=None,
              raise_on_nonconvergence=False):
        bc = np.ascontiguousarray(bc, dtype=np.uint8).reshape(-1)
        data = np.ascontiguousarray(data, dtype=np.float64).reshape(-1)
        m = self.nb * self.ncomp
        if bc.size != m or data.size != m:
            raise ValueError("bc and data must hold nb*ncomp values")
        u = np.empty(m)
        q = np.empty(m)
        x0p = None
        if x0 is not None:
            x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1)
            if x0.size != m:
                raise ValueError("x0 must hold nb*ncomp values")
            x0p = _ptr(x0)
        info = SolveInfo()
        rc = load_library().bem_solve(self._h, _ptr(bc), _ptr(data), float(c), float(tol), int(max_iter),
                                      int(restart), x0p, _ptr(u), _ptr(q), ctypes.byref(info), _stream_ptr(stream))
        allow = () if raise_on_nonconvergence else (BEM_ERR_NOT_CONVERGED,)
        _check(rc, allow)
        d = info.as_dict()
        d["status"] = rc
        return u, q, d

    def tune_preconditioner(self, bc, data, c=0.5, tol=1e-6, max_iter=2000, restart=100):
        """Measured block size of the block-Jacobi preconditioner (bem_tune_preconditioner)."""
        bc = np.ascontiguousarray(bc, dtype=np.uint8).reshape(-1)
        data = np.ascontiguousarray(data, dtype=np.float64).reshape(-1)
        if bc.size != self.nb * self.ncomp or data.size != self.nb * self.ncomp:
            raise ValueError("bc and data must hold nb*ncomp values")
        out = ctypes.c_int()
        _check(load_library().bem_tune_preconditioner(self._h, _ptr(bc), _ptr(data), float(c), float(tol),
                                                       int(max_iter), int(restart), ctypes.byref(out)))
        return out.value

    def tune_shapes(self, reps=20, stream=None):
        """Measured runtime launch shape of the apply (bem_tune_shapes): the
        cells per batch of the 2D fused walks or the lines per CTA of the 3D z
        pass; returns (chosen, ms per apply), (0, 0.0) when the plan has no
        such choice."""
        ch, ms = ctypes.c_int(), ctypes.c_double()
        _check(load_library().bem_tune_shapes(self._h, int(reps), _stream_ptr(stream), ctypes.byref(ch),
                                              ctypes.byref(ms)))
        return ch.value, ms.value

    def info(self):
        pi = PlanInfo()
        _check(load_library().bem_get_info(self._h, ctypes.byref(pi)))
        return pi.as_dict()

    def set_kernel_timing(self, enable: bool):
        _check(load_library().bem_set_kernel_timing(self._h, 1 if enable else 0))

    def kernel_time(self):
        ms = ctypes.c_double()
        cnt = ctypes.c_int64()
        _check(load_library().bem_kernel_time(self._h, ctypes.byref(ms), ctypes.byref(cnt)))
        return ms.value, cnt.value

    def launches_per_apply(self, layer="system"):
        lay = LAYERS[layer] if isinstance(layer, str) else int(layer)
        return int(load_library().bem_launches_per_apply(self._h, lay))

    def set_test_flags(self, flags: int):
        """Test hook for the bounded device waits (bem_set_test_flags)."""
        _check(load_library().bem_set_test_flags(self._h, int(flags)))

    def device_status(self, stream=None):
        """Raise BemError(BEM_ERR_TIMEOUT) if a kernel gave up a bounded device wait since the last check."""
        _check(load_library().bem_device_status(self._h, _stream_ptr(stream)))


class Batch:
    """One CUDA graph applying every plan's operator (bem_batch_*)."""

    def __init__(self, plans, layer="single", streams=4, stream=None):
        lib = load_library()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        lay = LAYERS[layer] if isinstance(layer, str) else int(layer)
        self._h = ctypes.c_void_p()
        _check(lib.bem_batch_create(ctypes.byref(self._h), arr, len(self.plans), lay, int(streams),
                                    _stream_ptr(stream)))
        din, dout, tot = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_size_t()
        _check(lib.bem_batch_buffers(self._h, ctypes.byref(din), ctypes.byref(dout), ctypes.byref(tot)))
        self.d_in, self.d_out, self.total = din.value, dout.value, tot.value
        self.offsets = []
        for i in range(len(self.plans)):
            o = ctypes.c_size_t()
            _check(lib.bem_batch_offset(self._h, i, ctypes.byref(o)))
            self.offsets.append(o.value)
        self.launches = int(lib.bem_batch_launches(self._h))

    def apply(self, stream=None):
        _check(load_library().bem_batch_apply(self._h, _stream_ptr(stream)))

    def set_grouping(self, enable: bool):
        """Grouped persistent launches per grid size (bem_batch_set_grouping)."""
        lib = load_library()
        _check(lib.bem_batch_set_grouping(self._h, 1 if enable else 0))
        self.launches = int(lib.bem_batch_launches(self._h))

    def tune(self, reps=10):
        """Measured number of capture streams (bem_tune_batch); returns it."""
        out = ctypes.c_int()
        _check(load_library().bem_tune_batch(self._h, int(reps), ctypes.byref(out)))
        return out.value

    def solve(self, bc, data, c=0.5, tol=1e-6, max_iter=2000, restart=100, x0=None, stream=None):
        """Lockstep GMRES over every plan's system (bem_batch_solve).  bc, data,
        x0 and the returned u, q are packed like the batch buffers; returns
        (u, q, [info dict per plan], status)."""
        bc = np.ascontiguousarray(bc, dtype=np.uint8).reshape(-1)
        data = np.ascontiguousarray(data, dtype=np.float64).reshape(-1)
        if bc.size != self.total or data.size != self.total:
            raise ValueError("bc and data must hold the batch's packed total of values")
        u = np.empty(self.total)
        q = np.empty(self.total)
        x0p = None
        if x0 is not None:
            x0 = np.ascontiguousarray(x0, dtype=np.float64).reshape(-1)
            if x0.size != self.total:
                raise ValueError("x0 must hold the batch's packed total of values")
            x0p = _ptr(x0)
        infos = (SolveInfo * len(self.plans))()
        rc = load_library().bem_batch_solve(self._h, _ptr(bc), _ptr(data), float(c), float(tol), int(max_iter),
                                            int(restart), x0p, _ptr(u), _ptr(q), infos, _stream_ptr(stream))
        _check(rc, (BEM_ERR_NOT_CONVERGED,))
        return u, q, [i.as_dict() for i in infos], rc

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().bem_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """Owning wrapper of a bem_net_t (learned initial guess network)."""

    def __init__(self, cin=7, hidden=64, layers=4, ksize=5, dilations=(1, 2, 4, 8), seed=0):
        lib = load_library()
        self.cin, self.hidden, self.layers, self.ksize = int(cin), int(hidden), int(layers), int(ksize)
        self.dilations = np.ascontiguousarray(dilations, dtype=np.int32)
        self._h = ctypes.c_void_p()
        _check(lib.bem_net_create(ctypes.byref(self._h), self.cin, self.hidden, self.layers, self.ksize,
                                  _ptr(self.dilations), int(seed)))
        self.nparams = int(lib.bem_net_num_params(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().bem_net_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.empty(self.nparams, dtype=np.float32)
        _check(load_library().bem_net_get_params(self._h, _ptr(out)))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32).reshape(-1)
        if p.size != self.nparams:
            raise ValueError(f"expected {self.nparams} parameters, got {p.size}")
        _check(load_library().bem_net_set_params(self._h, _ptr(p)))

    def _check_batch(self, feats, offsets, target=None):
        """Shapes of a batch: feats (T, cin), target T values; offsets (host
        or device) start at 0, do not decrease and end at T, so that the
        network kernels never index past feats or target."""
        import torch
        shape = tuple(feats.shape) if hasattr(feats, "shape") else np.shape(feats)
        if len(shape) != 2 or shape[1] != self.cin or shape[0] < 1:
            raise ValueError(f"feats must be (T, {self.cin})")
        T = shape[0]
        if isinstance(offsets, torch.Tensor) and offsets.is_cuda:
            o = offsets.reshape(-1)
            # two scalars and one flag come back to the host
            bad = o.numel() < 2 or int(o[0].item()) != 0 or int(o[-1].item()) != T or \
                bool((o[1:] < o[:-1]).any().item())
        else:
            o = offsets.numpy() if isinstance(offsets, torch.Tensor) else np.asarray(offsets)
            o = o.reshape(-1)
            bad = o.size < 2 or o[0] != 0 or o[-1] != T or bool(np.any(np.diff(o) < 0))
        if bad:
            raise ValueError("offsets must start at 0, not decrease and end at T")
        if target is not None and int(np.prod(target.shape if hasattr(target, "shape") else np.shape(target))) != T:
            raise ValueError("target must hold T values")

    @staticmethod
    def _dev(feats, offsets, target=None):
        import torch
        f = feats if isinstance(feats, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(feats, np.float32))
        if isinstance(offsets, torch.Tensor):
            o = offsets.to(device="cuda", dtype=torch.int32).contiguous()
        else:
            o = _device_offsets(np.asarray(offsets).reshape(-1))
        f = f.to(device="cuda", dtype=torch.float32).contiguous()
        t = None
        if target is not None:
            t = target if isinstance(target, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(target, np.float32))
            t = t.to(device="cuda", dtype=torch.float32).contiguous()
        return f, o, t

    def forward(self, feats, offsets, stream=None):
        import torch
        self._check_batch(feats, offsets)
        f, o, _ = self._dev(feats, offsets)
        T = f.shape[0]
        out = torch.empty(T, dtype=torch.float32, device="cuda")
        _check(load_library().bem_net_forward(self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(o.data_ptr()),
                                              o.numel() - 1, T, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def gradient(self, feats, offsets, target, stream=None):
        self._check_batch(feats, offsets, target)
        f, o, t = self._dev(feats, offsets, target)
        g = np.empty(self.nparams, dtype=np.float32)
        loss = ctypes.c_double()
        _check(load_library().bem_net_gradient(self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(o.data_ptr()),
                                               o.numel() - 1, f.shape[0], ctypes.c_void_p(t.data_ptr()), _ptr(g),
                                               ctypes.byref(loss), _stream_ptr(stream)))
        return loss.value, g

    def train_step(self, feats, offsets, target, lr=1e-3, stream=None):
        self._check_batch(feats, offsets, target)
        f, o, t = self._dev(feats, offsets, target)
        loss = ctypes.c_double()
        _check(load_library().bem_net_train_step(self._h, ctypes.c_void_p(f.data_ptr()),
                                                 ctypes.c_void_p(o.data_ptr()), o.numel() - 1, f.shape[0],
                                                 ctypes.c_void_p(t.data_ptr()), float(lr), ctypes.byref(loss),
                                                 _stream_ptr(stream)))
        return loss.value


def dtn_estimate(s, length, u, offsets, kmax, stream=None):
    """Arclength Dirichlet-to-Neumann estimate (bem_dtn_estimate) of a batch of
    closed curves: s, length, u hold T values (elements in arclength order,
    curve q at offsets[q] .. offsets[q+1]); returns a CUDA float32 tensor."""
    import torch
    def dev(a, dt):
        t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
        return t.to(device="cuda", dtype=dt).contiguous().reshape(-1)
    s, length, u = dev(s, torch.float32), dev(length, torch.float32), dev(u, torch.float32)
    oh = (offsets.cpu().numpy() if isinstance(offsets, torch.Tensor) else np.asarray(offsets)).reshape(-1)
    T = s.numel()
    if length.numel() != T or u.numel() != T or oh.size < 2 or oh[0] != 0 or oh[-1] != T or np.any(np.diff(oh) < 0):
        raise ValueError("s, length, u must hold T values; offsets start at 0, do not decrease and end at T")
    o = _device_offsets(oh)
    if not (1 <= int(kmax) <= 65535):
        raise ValueError("kmax must be in [1, 65535]")
    out = torch.empty(T, dtype=torch.float32, device="cuda")
    _check(load_library().bem_dtn_estimate(ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(length.data_ptr()),
                                           ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(o.data_ptr()),
                                           oh.size - 1, T, int(kmax), ctypes.c_void_p(out.data_ptr()),
                                           _stream_ptr(stream)))
    return out


def _seq_offsets(offsets, T):
    """Host copy of sequence offsets, checked: start at 0, do not decrease,
    end at T (so the kernels never index past their arrays)."""
    import torch
    oh = (offsets.cpu().numpy() if isinstance(offsets, torch.Tensor) else np.asarray(offsets)).reshape(-1)
    if oh.size < 2 or oh[0] != 0 or oh[-1] != T or np.any(np.diff(oh) < 0):
        raise ValueError("offsets must start at 0, not decrease and end at T")
    return oh


def _cuda_f32(a):
    import torch
    t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
    return t.to(device="cuda", dtype=torch.float32).contiguous()


def guess_features(geo, u, qd, offsets, radius, stream=None):
    """Input columns of the 2D guess network (bem_guess_features): geo (T, G)
    geometry columns, u and qd (T); returns a CUDA float32 tensor (T, G + 2)."""
    import torch
    g, u, qd = _cuda_f32(geo), _cuda_f32(u).reshape(-1), _cuda_f32(qd).reshape(-1)
    T = u.numel()
    if g.ndim != 2 or g.shape[0] != T or not (0 <= g.shape[1] <= 64) or qd.numel() != T:
        raise ValueError("geo must be (T, G) with G <= 64, u and qd T values")
    oh = _seq_offsets(offsets, T)
    out = torch.empty((T, g.shape[1] + 2), dtype=torch.float32, device="cuda")
    _check(load_library().bem_guess_features(ctypes.c_void_p(g.data_ptr()), int(g.shape[1]),
                                             ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(qd.data_ptr()),
                                             ctypes.c_void_p(_device_offsets(oh).data_ptr()), oh.size - 1, T,
                                             float(radius), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def guess_finish(qd, corr, u, length, offsets, cscale, stream=None):
    """The zero-flux guess from the network's output (bem_guess_finish); a
    CUDA float32 tensor (T)."""
    import torch
    qd, corr, u, ln = (_cuda_f32(a).reshape(-1) for a in (qd, corr, u, length))
    T = qd.numel()
    if corr.numel() != T or u.numel() != T or ln.numel() != T:
        raise ValueError("qd, corr, u, length must hold T values")
    oh = _seq_offsets(offsets, T)
    out = torch.empty(T, dtype=torch.float32, device="cuda")
    _check(load_library().bem_guess_finish(ctypes.c_void_p(qd.data_ptr()), ctypes.c_void_p(corr.data_ptr()),
                                           ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(ln.data_ptr()),
                                           ctypes.c_void_p(_device_offsets(oh).data_ptr()), oh.size - 1, T,
                                           float(cscale), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def fourier_features(points, B, stream=None):
    """Random Fourier features (bem_fourier_features) of points (T, 3) for the
    frequency matrix B (F, 3): a CUDA float32 tensor (T, 2F), sin and cos
    interleaved per frequency."""
    import torch
    p = points if isinstance(points, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(points))
    b = B if isinstance(B, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(B))
    p = p.to(device="cuda", dtype=torch.float32).contiguous()
    b = b.to(device="cuda", dtype=torch.float32).contiguous()
    if p.ndim != 2 or p.shape[1] != 3 or p.shape[0] < 1 or b.ndim != 2 or b.shape[1] != 3 or not (1 <= b.shape[0] <= 4096):
        raise ValueError("points must be (T, 3) and B (F, 3) with 1 <= F <= 4096")
    T, F = p.shape[0], b.shape[0]
    out = torch.empty((T, 2 * F), dtype=torch.float32, device="cuda")
    _check(load_library().bem_fourier_features(ctypes.c_void_p(p.data_ptr()), T, ctypes.c_void_p(b.data_ptr()), F,
                                               ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def measure_peak(kind="fp32", stream=None):
    """Measured arithmetic peak of the current GPU in TFLOP/s (bem_measure_peak):
    kind "fp32", "fp64" or "fp32x2" (packed pairs)."""
    k = {"fp32": 0, "fp64": 1, "fp32x2": 2}[kind]
    out = ctypes.c_double()
    _check(load_library().bem_measure_peak(k, ctypes.byref(out), _stream_ptr(stream)))
    return out.value


def bem_plan(dim, n, h, cell, w, normal, kernel="laplace2d", precision="f32", nu=0.3, mu=1.0, stream=None):
    return Plan(dim, n, h, cell, w, normal, kernel, precision, nu, mu, stream)


def bem_apply(plan: Plan, layer, x, out=None, stream=None):
    return plan.apply(layer, x, out, stream)


def bem_apply_host(plan: Plan, layer, x, out=None, stream=None):
    return plan.apply_host(layer, x, out, stream)


def bem_set_bc(plan: Plan, bc, c=0.5):
    return plan.set_bc(bc, c)


def bem_solve(plan: Plan, bc, data, c=0.5, tol=1e-6, max_iter=2000, restart=50, x0=None, stream=None):
    return plan.solve(bc, data, c, tol, max_iter, restart, x0, stream)


def bem_destroy(plan: Plan):
    plan.close()
