"""CPU FP64 oracle for the FFT-accelerated BEM operator (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs are the only callers.
The product path (the CUDA library and its Python binding) never imports this
module, and this module imports nothing from the product package.

Contents
--------
* ``apply``      direct O(N_b^2) sum of the discrete operator (C, OpenMP), the
                 plain definition of what the FFT path computes: Eq. 15 for
                 2D Laplace, its 3D analogue, and Eq. 7 plus the Kelvin traction
                 kernel for Navier (Eq. 8).
* ``matrix``     the same operator as a dense matrix.
* ``system``     the boundary-condition split of Eq. 4 / Eq. 8 into A x = b
                 (Dirichlet cells: flux/traction unknown; Neumann cells:
                 potential/displacement unknown), c = 1/2 on the boundary
                 (Section 2).
* ``solve_lu``   dense LU (LAPACK through numpy) of that system.
* ``L2``, ``C3`` closed-form cell-average constants of the singular cell.

Every function says which passage of the paper it follows.  Where the paper is
silent (singular cell value, traction kernel, padding) the module docstring of
``bem_oracle.c`` states the reading taken.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbem_oracle.so")
_lock = threading.Lock()
_lib = None

LAPLACE_2D, LAPLACE_3D, KELVIN_3D = 0, 1, 2
SINGLE, DOUBLE = 0, 1
KERNELS = {"laplace2d": LAPLACE_2D, "laplace3d": LAPLACE_3D, "kelvin3d": KELVIN_3D}


def build(force: bool = False) -> str:
    """Compile ``bem_oracle.c`` with gcc (-O2, OpenMP) into ``_build/``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            lib.bo_apply.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, P, ctypes.c_double, P, P,
                                     ctypes.c_double, ctypes.c_double, P, P, ctypes.c_int64, ctypes.c_int64]
            lib.bo_apply.restype = ctypes.c_int
            lib.bo_matrix.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, P, ctypes.c_double, P, P,
                                      ctypes.c_double, ctypes.c_double, P]
            lib.bo_matrix.restype = ctypes.c_int
            lib.bo_kernel_point.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_double, ctypes.c_double, P]
            lib.bo_kernel_point.restype = ctypes.c_int
            for name in ("bo_L2", "bo_C3"):
                getattr(lib, name).restype = ctypes.c_double
                getattr(lib, name).argtypes = []
            lib.bo_num_threads.restype = ctypes.c_int
            lib.bo_set_threads.argtypes = [ctypes.c_int]
            for name in ("bo_lap2d_U", "bo_lap2d_Q", "bo_lap3d_U", "bo_lap3d_Q"):
                getattr(lib, name).restype = ctypes.c_double
            lib.bo_lap2d_U.argtypes = [ctypes.c_double] * 3
            lib.bo_lap2d_Q.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
            lib.bo_lap3d_U.argtypes = [ctypes.c_double] * 4
            lib.bo_lap3d_Q.argtypes = [ctypes.c_int] + [ctypes.c_double] * 3
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def L2() -> float:
    """Mean of ln r over the unit square centred at 0 (singular 2D cell)."""
    return _load().bo_L2()


def C3() -> float:
    """Integral of 1/r over the unit cube centred at 0 (singular 3D cell)."""
    return _load().bo_C3()


def set_threads(n: int) -> None:
    _load().bo_set_threads(int(n))


def num_threads() -> int:
    return int(_load().bo_num_threads())


def _kernel_id(kernel) -> int:
    return KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


def _ncomp(kernel: int) -> int:
    return 3 if kernel == KELVIN_3D else 1


def _geom(cell, w, normal, dim):
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    normal = np.ascontiguousarray(normal, dtype=np.float64)
    assert cell.ndim == 2 and cell.shape[1] == dim
    assert normal.shape == cell.shape and w.shape == (cell.shape[0],)
    return cell, w, normal


def apply(kernel, layer: int, cell, h: float, w, normal, x, nu: float = 0.3, mu: float = 1.0,
          rows=None) -> np.ndarray:
    """Direct sum of the discrete single (layer=0) or double (layer=1) operator.

    Follows Eq. 15 (2D Laplace), its 3D analogue, and Eq. 7 / Eq. 8 (Kelvin).
    ``rows``: optional (row0, nrows) slice of target cells to evaluate.
    Returns out with shape (nrows,) or (nrows, 3).
    """
    k = _kernel_id(kernel)
    dim = 2 if k == LAPLACE_2D else 3
    nc = _ncomp(k)
    cell, w, normal = _geom(cell, w, normal, dim)
    nb = cell.shape[0]
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(nb * nc)
    row0, nrows = (0, nb) if rows is None else (int(rows[0]), int(rows[1]))
    out = np.zeros(nrows * nc, dtype=np.float64)
    rc = _load().bo_apply(k, int(layer), nb, _ptr(cell), float(h), _ptr(w), _ptr(normal), float(nu), float(mu),
                          _ptr(x), _ptr(out), row0, nrows)
    if rc != 0:
        raise ValueError("bo_apply rejected its arguments")
    return out if nc == 1 else out.reshape(nrows, nc)


def matrix(kernel, layer: int, cell, h: float, w, normal, nu: float = 0.3, mu: float = 1.0) -> np.ndarray:
    """Dense matrix of the discrete operator (weights included)."""
    k = _kernel_id(kernel)
    dim = 2 if k == LAPLACE_2D else 3
    nc = _ncomp(k)
    cell, w, normal = _geom(cell, w, normal, dim)
    nb = cell.shape[0]
    A = np.empty((nb * nc, nb * nc), dtype=np.float64)
    rc = _load().bo_matrix(k, int(layer), nb, _ptr(cell), float(h), _ptr(w), _ptr(normal), float(nu), float(mu),
                           _ptr(A))
    if rc != 0:
        raise ValueError("bo_matrix rejected its arguments")
    return A


def kernel_point(kernel, layer: int, d, n=None, nu: float = 0.3, mu: float = 1.0) -> np.ndarray:
    """Kernel block at a non-zero offset d = collocation - integration point."""
    k = _kernel_id(kernel)
    nc = _ncomp(k)
    d = np.ascontiguousarray(np.asarray(d, dtype=np.float64).reshape(-1)[:3].tolist() + [0.0] * 3,
                             dtype=np.float64)[:3]
    nn = np.zeros(3) if n is None else np.asarray(n, dtype=np.float64).reshape(-1)
    nn = np.ascontiguousarray(np.concatenate([nn, np.zeros(3)])[:3])
    blk = np.zeros(9, dtype=np.float64)
    _load().bo_kernel_point(k, int(layer), _ptr(d), _ptr(nn), float(nu), float(mu), _ptr(blk))
    return blk[0] if nc == 1 else blk.reshape(3, 3)


def double_sign(kernel) -> float:
    """Sign of the second integral in the BIE: Eq. 15 (Laplace) adds D u,
    Eq. 8 (Navier) subtracts T u."""
    return -1.0 if _kernel_id(kernel) == KELVIN_3D else 1.0


def system(kernel, cell, h, w, normal, bc, u_known, q_known, c: float = 0.5, nu: float = 0.3,
           mu: float = 1.0):
    """Dense A and b of the boundary-condition split of Eq. 4 / Eq. 8.

    With K1 the single-layer operator and K2 = +D (Laplace) or -T (Kelvin),
    the BIE at every boundary cell reads c u = K1 q + K2 u (c = 1/2 on the
    smooth boundary, Section 2).  For bc = 0 (Dirichlet: u known, q unknown)
    and bc = 1 (Neumann: q known, u unknown) the unknown x holds q on
    Dirichlet entries and u on Neumann entries:
        A x = K1 (x m_D) + K2 (x m_N) - c x m_N
        b   = c u m_D - K2 (u m_D) - K1 (q m_N).
    """
    k = _kernel_id(kernel)
    K1 = matrix(k, SINGLE, cell, h, w, normal, nu, mu)
    K2 = double_sign(k) * matrix(k, DOUBLE, cell, h, w, normal, nu, mu)
    bc = np.asarray(bc).reshape(-1).astype(np.float64)
    mN = bc
    mD = 1.0 - bc
    u = np.asarray(u_known, dtype=np.float64).reshape(-1)
    q = np.asarray(q_known, dtype=np.float64).reshape(-1)
    A = K1 * mD[None, :] + K2 * mN[None, :] - np.diag(c * mN)
    b = c * u * mD - K2 @ (u * mD) - K1 @ (q * mN)
    return A, b


def system_apply(kernel, cell, h, w, normal, bc, x, c: float = 0.5, nu: float = 0.3, mu: float = 1.0,
                 rows=None):
    """A x of ``system`` by direct sums (no dense matrix), for large N_b."""
    k = _kernel_id(kernel)
    nc = _ncomp(k)
    bc = np.asarray(bc).reshape(-1).astype(np.float64)
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    mN, mD = bc, 1.0 - bc
    y1 = apply(k, SINGLE, cell, h, w, normal, x * mD, nu, mu, rows).reshape(-1)
    y2 = apply(k, DOUBLE, cell, h, w, normal, x * mN, nu, mu, rows).reshape(-1)
    sl = slice(None) if rows is None else slice(rows[0] * nc, (rows[0] + rows[1]) * nc)
    return y1 + double_sign(k) * y2 - c * (x * mN)[sl]


def system_rhs(kernel, cell, h, w, normal, bc, u_known, q_known, c: float = 0.5, nu: float = 0.3,
               mu: float = 1.0):
    """b of ``system`` by direct sums."""
    k = _kernel_id(kernel)
    bc = np.asarray(bc).reshape(-1).astype(np.float64)
    mN, mD = bc, 1.0 - bc
    u = np.asarray(u_known, dtype=np.float64).reshape(-1)
    q = np.asarray(q_known, dtype=np.float64).reshape(-1)
    k1q = apply(k, SINGLE, cell, h, w, normal, q * mN, nu, mu).reshape(-1)
    k2u = apply(k, DOUBLE, cell, h, w, normal, u * mD, nu, mu).reshape(-1)
    return c * u * mD - double_sign(k) * k2u - k1q


def solve_lu(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Dense LU with partial pivoting (LAPACK gesv)."""
    return np.linalg.solve(A, b)
