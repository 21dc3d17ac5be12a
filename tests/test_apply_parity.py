"""Parity of the CUDA operator apply with the CPU FP64 oracle (GPU).

Bars: relative L2 <= 1e-12 for FP64 and double-float (f32x2) plans and
<= 2e-6 for FP32 plans on
random N(0,1) densities, element by element over every boundary cell.  Sizes
span one-thread columns (n = 4) through multi-pass transforms with a ragged
last pass (N = 2n = 2^k with k not a multiple of 4) up to the full 4096^2
star workload, where the oracle evaluates sampled target rows one by one.
"""
import numpy as np
import pytest

from paper_1809_00845_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6, "f32x2": 1e-12}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_00845_gb300 import build
    build.build()
    return torch


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def fp32_abs_bound(b, x, layer):
    """Absolute error bound of an FP32 FFT apply: its rounding error is
    relative to the whole convolution, about eps32 * log2(N^2) * max|K| *
    sum_j |w_j x_j|, not to the (possibly much smaller) values at the targets.
    Used for degenerate cell sets whose outputs cancel far below the kernel's
    near-field scale; random dense inputs are held to the relative bar."""
    import math
    h = b.h
    L2 = math.pi / 4 - 1.5 - 0.5 * math.log(2)
    if layer == "single":
        kmax = max(abs(-(math.log(h) + L2) / (2 * math.pi)), abs(math.log(h * b.n * 2 ** 0.5)) / (2 * math.pi))
    else:
        kmax = 1.0 / (2 * math.pi * h)
    return 6e-8 * math.log2((2 * b.n) ** 2) * kmax * float(np.sum(np.abs(b.w * np.asarray(x))))


def gpu_apply(torch, plan, layer, x):
    t = torch.from_numpy(np.asarray(x, dtype=plan.np_dtype)).cuda()
    y = plan.apply(layer, t)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


def _plan(b, prec):
    from paper_1809_00845_gb300.bem import Plan
    return Plan.from_boundary(b, "laplace2d", prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n,nb", [(4, 5), (8, 17), (16, 40), (32, 77), (64, 300), (128, 901), (256, 1500),
                                  (512, 2000)])
def test_random_cells_single_double(torch_cuda, oracle_mod, prec, n, nb):
    rng = np.random.default_rng(1000 + n)
    b = I.random_cells(n, nb, rng)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, prec)
    for layer, lid in (("single", 0), ("double", 1)):
        ref = oracle_mod.apply("laplace2d", lid, b.cell, b.h, b.w, b.normal, x)
        out = gpu_apply(torch_cuda, plan, layer, x)
        assert rel_l2(out, ref) <= TOL[prec], (layer, rel_l2(out, ref))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_system_operator_mixed_bc(torch_cuda, oracle_mod, prec):
    rng = np.random.default_rng(5)
    b = I.star_boundary(256)
    bc = I.mixed_bc_theta(b)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, prec)
    plan.set_bc(bc, 0.5)
    ref = oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc, x)
    out = gpu_apply(torch_cuda, plan, "system", x)
    assert rel_l2(out, ref) <= TOL[prec]
    # switching the BC pattern rebuilds the operator
    bc2 = 1 - bc
    plan.set_bc(bc2, 0.25)
    ref2 = oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc2, x, c=0.25)
    assert rel_l2(gpu_apply(torch_cuda, plan, "system", x), ref2) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n", [64, 256, 512])
def test_system_operator_uniform_bc(torch_cuda, oracle_mod, prec, n):
    """All-Dirichlet and all-Neumann data: the system operator leaves out the
    fields no cell feeds (U alone, or Q_x and Q_y alone) and must still be
    the oracle's BC-split operator (Eq. 15), on both column kernels (n < 256:
    the small-grid kernel; n >= 256: the four-step kernel)."""
    rng = np.random.default_rng(50 + n)
    b = I.star_boundary(n)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, prec)
    for fill, c in ((0, 0.5), (1, 0.5), (1, 0.25), (0, 0.5)):
        bc = np.full(b.nb, fill, np.uint8)
        plan.set_bc(bc, c)
        ref = oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc, x, c=c)
        err = rel_l2(gpu_apply(torch_cuda, plan, "system", x), ref)
        assert err <= TOL[prec], (fill, c, err)
    # back to mixed data: all three fields again
    bc = I.mixed_bc_theta(b)
    plan.set_bc(bc, 0.5)
    ref = oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc, x)
    assert rel_l2(gpu_apply(torch_cuda, plan, "system", x), ref) <= TOL[prec]
    plan.close()


def test_circle_config_f64(torch_cuda, oracle_mod):
    """Circle R = 0.35 on 128^2 (356 cells), FP64, single and double layer."""
    b = I.circle_boundary(128, 0.35)
    assert b.nb == 356
    rng = np.random.default_rng(7)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, "f64")
    for layer, lid in (("single", 0), ("double", 1)):
        ref = oracle_mod.apply("laplace2d", lid, b.cell, b.h, b.w, b.normal, x)
        assert rel_l2(gpu_apply(torch_cuda, plan, layer, x), ref) <= 1e-12


def test_edge_cases(torch_cuda, oracle_mod):
    # a single cell: only the singular-cell value; zero weights; a full plane (Eq. 9)
    from paper_1809_00845_gb300.bem import Plan
    for prec in ("f64", "f32"):
        one = I.Boundary(2, 8, np.array([[3, 5]], np.int32), np.array([0.125]), np.array([[0.6, 0.8]]),
                         np.zeros((1, 2)), np.zeros(1))
        p = _plan(one, prec)
        ref = oracle_mod.apply("laplace2d", 0, one.cell, one.h, one.w, one.normal, np.array([2.0]))
        assert rel_l2(gpu_apply(torch_cuda, p, "single", [2.0]), ref) <= TOL[prec]
        assert np.max(np.abs(gpu_apply(torch_cuda, p, "double", [2.0]))) <= 1e-12 * abs(ref[0]) * (1e6 if prec == "f32" else 1)
        rng = np.random.default_rng(9)
        full = I.full_plane_boundary(16, rng)
        x = rng.standard_normal(full.nb)
        p = _plan(full, prec)
        for layer, lid in (("single", 0), ("double", 1)):
            ref = oracle_mod.apply("laplace2d", lid, full.cell, full.h, full.w, full.normal, x)
            assert rel_l2(gpu_apply(torch_cuda, p, layer, x), ref) <= TOL[prec]
        # cells on the outermost rows/columns of the grid (largest offsets)
        corners = I.Boundary(2, 16, np.array([[0, 0], [15, 15], [0, 15], [15, 0], [7, 8]], np.int32),
                             np.full(5, 1 / 16), np.array([[1.0, 0.0]] * 5), np.zeros((5, 2)), np.zeros(5))
        x = rng.standard_normal(5)
        p = _plan(corners, prec)
        for layer, lid in (("single", 0), ("double", 1)):
            ref = oracle_mod.apply("laplace2d", lid, corners.cell, corners.h, corners.w, corners.normal, x)
            assert rel_l2(gpu_apply(torch_cuda, p, layer, x), ref) <= TOL[prec]


def test_linearity_and_repeatability(torch_cuda):
    b = I.circle_boundary(256, 0.3)
    rng = np.random.default_rng(3)
    x1, x2 = rng.standard_normal(b.nb), rng.standard_normal(b.nb)
    plan = _plan(b, "f64")
    y1 = gpu_apply(torch_cuda, plan, "single", x1)
    y2 = gpu_apply(torch_cuda, plan, "single", x2)
    y12 = gpu_apply(torch_cuda, plan, "single", 2.0 * x1 - 3.0 * x2)
    assert rel_l2(y12, 2.0 * y1 - 3.0 * y2) < 1e-13
    assert np.array_equal(gpu_apply(torch_cuda, plan, "single", x1), y1)


@pytest.mark.parametrize("prec", ["f32", "f64", "f32x2"])
def test_star_4096_full_size_sampled_rows(torch_cuda, oracle_mod, prec):
    """The 4096^2 star (padded 8192^2), mixed BCs, in the launch configuration
    the benchmark times; the oracle evaluates 3 x 256 target rows exactly."""
    b = I.star_boundary(4096)
    bc = I.mixed_bc_theta(b)
    rng = I.rng_for(1)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, prec)
    plan.set_bc(bc, 0.5)
    out = gpu_apply(torch_cuda, plan, "system", x)
    for row0 in (0, b.nb // 2, b.nb - 256):
        ref = oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc, x, rows=(row0, 256))
        assert rel_l2(out[row0:row0 + 256], ref) <= TOL[prec], row0
    s_out = gpu_apply(torch_cuda, plan, "single", x)
    ref = oracle_mod.apply("laplace2d", 0, b.cell, b.h, b.w, b.normal, x, rows=(1000, 256))
    assert rel_l2(s_out[1000:1256], ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32", "f32x2"])
def test_fourstep_kernel_edge_cases(torch_cuda, oracle_mod, prec):
    """n >= 256 uses the four-step column kernel: one cell, the four grid
    corners (largest offsets), and a dense random set where many rows carry
    several cells and thread row-ranges are uneven."""
    rng = np.random.default_rng(21)
    n = 256
    one = I.Boundary(2, n, np.array([[200, 3]], np.int32), np.array([1.0 / n]), np.array([[0.0, 1.0]]),
                     np.zeros((1, 2)), np.zeros(1))
    ref = oracle_mod.apply("laplace2d", 0, one.cell, one.h, one.w, one.normal, np.array([1.5]))
    assert rel_l2(gpu_apply(torch_cuda, _plan(one, prec), "single", [1.5]), ref) <= TOL[prec]
    corners = I.Boundary(2, n, np.array([[0, 0], [n - 1, n - 1], [0, n - 1], [n - 1, 0]], np.int32),
                         np.full(4, 1.0 / n), np.array([[0.6, 0.8]] * 4), np.zeros((4, 2)), np.zeros(4))
    x = rng.standard_normal(4)
    p = _plan(corners, prec)
    for layer, lid in (("single", 0), ("double", 1)):
        ref = oracle_mod.apply("laplace2d", lid, corners.cell, corners.h, corners.w, corners.normal, x)
        out = gpu_apply(torch_cuda, p, layer, x)
        if prec != "f32":
            assert rel_l2(out, ref) <= TOL[prec]
        else:  # four far-apart cells: outputs ~1e-4 of the near-field scale
            assert np.max(np.abs(out - ref)) <= fp32_abs_bound(corners, x, layer)
    dense = I.random_cells(n, 6000, rng)
    x = rng.standard_normal(dense.nb)
    p = _plan(dense, prec)
    bc = (rng.uniform(size=dense.nb) < 0.5).astype(np.uint8)
    p.set_bc(bc, 0.5)
    for layer, lid in (("single", 0), ("double", 1)):
        ref = oracle_mod.apply("laplace2d", lid, dense.cell, dense.h, dense.w, dense.normal, x)
        assert rel_l2(gpu_apply(torch_cuda, p, layer, x), ref) <= TOL[prec]
    ref = oracle_mod.system_apply("laplace2d", dense.cell, dense.h, dense.w, dense.normal, bc, x)
    assert rel_l2(gpu_apply(torch_cuda, p, "system", x), ref) <= TOL[prec]


@pytest.mark.parametrize("n,nb", [(256, 1500), (512, 2000), (1024, 3000), (2048, 5000)])
def test_f32x2_random_cells_single_double(torch_cuda, oracle_mod, n, nb):
    """Double-float plans (pairs of FP32 numbers, FP64 I/O) on every
    four-step grid size below the full one."""
    rng = np.random.default_rng(2000 + n)
    b = I.random_cells(n, nb, rng)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, "f32x2")
    for layer, lid in (("single", 0), ("double", 1)):
        ref = oracle_mod.apply("laplace2d", lid, b.cell, b.h, b.w, b.normal, x)
        out = gpu_apply(torch_cuda, plan, layer, x)
        assert rel_l2(out, ref) <= TOL["f32x2"], (layer, rel_l2(out, ref))


def test_fourstep_global_accumulators(torch_cuda, oracle_mod):
    """More cells than the shared-memory accumulators hold (n = 4096, FP32,
    20000 cells): per-CTA partial sums live in global memory."""
    rng = np.random.default_rng(33)
    b = I.random_cells(4096, 20000, rng)
    x = rng.standard_normal(b.nb)
    p = _plan(b, "f32")
    out = gpu_apply(torch_cuda, p, "single", x)
    ref = oracle_mod.apply("laplace2d", 0, b.cell, b.h, b.w, b.normal, x, rows=(5000, 400))
    assert rel_l2(out[5000:5400], ref) <= TOL["f32"]
