"""bem_apply with several right-hand sides (nbatch) and the apply's host-side
argument checks (GPU).

The kernel spectra are fixed per plan (Section 4, Eq. 16), so one call applies
the operator to nbatch densities stored back to back.  Each vector must come
out as its own single apply does (the same kernels in the same order: equal
bit for bit) and match the CPU FP64 oracle within the parity bars (FP64
1e-12, FP32 2e-6).  Overlapping input and output ranges are refused before
any kernel runs.
"""
import ctypes

import numpy as np
import pytest

from paper_1809_00845_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_00845_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("prec,n,k", [("f32", 512, 4), ("f64", 64, 3), ("f32", 4096, 2)])
def test_nbatch_equals_single_applies_and_oracle(torch_cuda, oracle_mod, prec, n, k):
    torch = torch_cuda
    from paper_1809_00845_gb300.bem import Plan
    b = I.star_boundary(n)
    bc = I.mixed_bc_theta(b)
    plan = Plan.from_boundary(b, "laplace2d", prec)
    plan.set_bc(bc, 0.5)
    rng = np.random.default_rng(90 + n)
    X = rng.standard_normal((k, b.nb))
    xt = torch.from_numpy(X.astype(plan.np_dtype)).cuda()
    cnt = b.nb if b.nb <= 4000 else 256  # the full-size star: the first 256 target rows
    for layer in ("single", "double", "system"):
        Y = plan.apply(layer, xt).cpu().numpy().astype(np.float64)
        for r in range(k):
            y1 = plan.apply(layer, xt[r].contiguous()).cpu().numpy().astype(np.float64)
            assert np.array_equal(Y[r], y1), (layer, r)
            if layer == "system":
                ref = oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc, X[r], rows=(0, cnt))
            else:
                ref = oracle_mod.apply("laplace2d", 0 if layer == "single" else 1, b.cell, b.h, b.w, b.normal,
                                       X[r], rows=(0, cnt))
            ref = np.asarray(ref).reshape(-1)
            err = np.linalg.norm(Y[r][:cnt] - ref) / np.linalg.norm(ref)
            assert err <= TOL[prec], (layer, r, err)
    plan.close()


def test_overlapping_buffers_and_bad_nbatch_are_refused(torch_cuda):
    torch = torch_cuda
    from paper_1809_00845_gb300 import bem
    lib = bem.load_library()
    b = I.star_boundary(512)
    plan = bem.Plan.from_boundary(b, "laplace2d", "f32")
    buf = torch.zeros(3 * b.nb, dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    base = buf.data_ptr()
    # output starting one element into the input
    rc = lib.bem_apply(plan._h, bem.BEM_SINGLE, ctypes.c_void_p(base), ctypes.c_void_p(base + 4), 1, stream)
    assert rc == bem.BEM_ERR_ARG and b"overlap" in lib.bem_last_error()
    # two vectors in, the output starting at the second input vector
    rc = lib.bem_apply(plan._h, bem.BEM_SINGLE, ctypes.c_void_p(base), ctypes.c_void_p(base + 4 * b.nb), 2, stream)
    assert rc == bem.BEM_ERR_ARG
    rc = lib.bem_apply_static_scratch(plan._h, bem.BEM_SINGLE, ctypes.c_void_p(base), ctypes.c_void_p(base + 8),
                                      stream)
    assert rc == bem.BEM_ERR_ARG
    assert lib.bem_apply(plan._h, bem.BEM_SINGLE, ctypes.c_void_p(base), ctypes.c_void_p(base + 4 * b.nb), 0,
                         stream) == bem.BEM_ERR_ARG
    # adjacent, non-overlapping ranges are fine
    rc = lib.bem_apply(plan._h, bem.BEM_SINGLE, ctypes.c_void_p(base), ctypes.c_void_p(base + 4 * b.nb), 1, stream)
    assert rc == bem.BEM_OK, lib.bem_last_error()
    torch.cuda.synchronize()
    plan.close()


@pytest.mark.parametrize("n", [512, 4096])
def test_three_pass_form_matches_fused_and_oracle(torch_cuda, oracle_mod, n):
    """BEM_PLAN_THREE_PASS (the same operator through X/Y buffers in device
    memory instead of the fused column kernel) against the oracle (2e-6,
    sampled rows at full size) and the fused form (FP32 rounding apart)."""
    torch = torch_cuda
    from paper_1809_00845_gb300 import bem
    b = I.star_boundary(n)
    bc = I.mixed_bc_theta(b)
    rng = np.random.default_rng(70 + n)
    x = rng.standard_normal(b.nb)
    xt = torch.from_numpy(x.astype(np.float32)).cuda()
    fused = bem.Plan.from_boundary(b, "laplace2d", "f32")
    p3 = bem.Plan.from_boundary(b, "laplace2d", "f32", flags=bem.BEM_PLAN_THREE_PASS)
    cnt = b.nb if b.nb <= 4000 else 256
    for p in (fused, p3):
        p.set_bc(bc, 0.5)
    for layer in ("single", "double", "system"):
        y3 = p3.apply(layer, xt).cpu().numpy().astype(np.float64)
        yf = fused.apply(layer, xt).cpu().numpy().astype(np.float64)
        if layer == "system":
            ref = oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc, x, rows=(0, cnt))
        else:
            ref = oracle_mod.apply("laplace2d", 0 if layer == "single" else 1, b.cell, b.h, b.w, b.normal, x,
                                   rows=(0, cnt))
        ref = np.asarray(ref).reshape(-1)
        err = np.linalg.norm(y3[:cnt] - ref) / np.linalg.norm(ref)
        dif = np.linalg.norm(y3 - yf) / np.linalg.norm(yf)
        print(f"three-pass n={n} {layer}: rel L2 vs oracle {err:.2e}, vs fused {dif:.2e}")
        assert err <= 2e-6 and dif <= 2e-6, (layer, err, dif)
    fused.close()
    p3.close()
