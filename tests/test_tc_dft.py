"""Tensor-core DFT stages (BEM_TC_BF16X3, BEM_TC_F16X3) against the CPU FP64
oracle (GPU).

The column kernel runs its radix-16 stages as split 16-bit products with
FP32 accumulation; everything else is the FP32 path.  Bars (relative L2 on
random N(0,1) densities, element by element):
  * FP16 hi + lo (22 significand bits per operand): 5e-6;
  * BF16 hi + lo (16 bits per operand): 1e-4.
Both follow from the operand split: per stage each product carries a relative
error of a few units of 2^-22 (FP16) or 2^-16 (BF16); six stages per
forward/inverse pair add about in quadrature, on top of the FP32 rounding of
the rest of the path.  Sizes: every grid the kernels exist for (n = 1024,
2048, 4096; 128, 256, 512 threads), ragged cell counts, the full 4096^2 star
in the benchmark's launch configuration (sampled oracle rows), and solves
with double-float residual refinement.
"""
import numpy as np
import pytest

from paper_1809_00845_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"tc_bf16x3": 1e-4, "tc_f16x3": 5e-6}
KINDS = list(TOL)


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


def gpu_apply(torch, plan, layer, x):
    t = torch.from_numpy(np.asarray(x, dtype=plan.np_dtype)).cuda()
    y = plan.apply(layer, t)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


def _plan(b, prec):
    from paper_1809_00845_gb300.bem import Plan
    return Plan.from_boundary(b, "laplace2d", prec)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n,nb", [(1024, 3001), (2048, 5003), (4096, 9000)])
def test_tc_random_cells_every_layer(torch_cuda, oracle_mod, kind, n, nb):
    rng = np.random.default_rng(4100 + n + nb)
    b = I.random_cells(n, nb, rng)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, kind)
    bc = (rng.uniform(size=b.nb) < 0.5).astype(np.uint8)
    plan.set_bc(bc, 0.5)
    errs = {}
    for layer, lid in (("single", 0), ("double", 1)):
        ref = oracle_mod.apply("laplace2d", lid, b.cell, b.h, b.w, b.normal, x)
        errs[layer] = rel_l2(gpu_apply(torch_cuda, plan, layer, x), ref)
    ref = oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc, x)
    errs["system"] = rel_l2(gpu_apply(torch_cuda, plan, "system", x), ref)
    print(f"{kind} n={n} nb={b.nb} rel L2 {errs}")
    plan.device_status()
    for layer, e in errs.items():
        assert e <= TOL[kind], (layer, e)


@pytest.mark.parametrize("kind", KINDS)
def test_tc_star_4096_full_size_sampled_rows(torch_cuda, oracle_mod, kind):
    """The 4096^2 star (padded 8192^2), mixed BCs, system operator; the oracle
    evaluates 3 x 256 target rows exactly."""
    b = I.star_boundary(4096)
    bc = I.mixed_bc_theta(b)
    rng = I.rng_for(1)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, kind)
    plan.set_bc(bc, 0.5)
    info = plan.info()
    from paper_1809_00845_gb300 import bem
    assert info["precision"] == bem.PRECISIONS[kind]
    assert info["threads_per_cta"] == 512
    out = gpu_apply(torch_cuda, plan, "system", x)
    errs = []
    for row0 in (0, b.nb // 2, b.nb - 256):
        ref = oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc, x, rows=(row0, 256))
        errs.append(rel_l2(out[row0:row0 + 256], ref))
    print(f"{kind} star 4096 sampled rel L2 {errs}")
    plan.device_status()
    assert max(errs) <= TOL[kind], errs


@pytest.mark.parametrize("kind", KINDS)
def test_tc_edge_cases(torch_cuda, oracle_mod, kind):
    """One cell; fewer cells than threads (most threads empty); rows split
    between threads (many cells per row); repeated applies agree bit for
    bit."""
    rng = np.random.default_rng(77)
    n = 1024
    one = I.Boundary(2, n, np.array([[300, 700]], np.int32), np.array([0.7 / n]), np.array([[0.6, 0.8]]),
                     np.array([[300.5 / n, 700.5 / n]]), np.zeros(1))
    plan = _plan(one, kind)
    x = np.array([1.3])
    ref = oracle_mod.apply("laplace2d", 0, one.cell, one.h, one.w, one.normal, x)
    assert rel_l2(gpu_apply(torch_cuda, plan, "single", x), ref) <= TOL[kind]
    few = I.random_cells(n, 57, rng)
    xf = rng.standard_normal(few.nb)
    plan = _plan(few, kind)
    ref = oracle_mod.apply("laplace2d", 0, few.cell, few.h, few.w, few.normal, xf)
    assert rel_l2(gpu_apply(torch_cuda, plan, "single", xf), ref) <= TOL[kind]
    # a dense band of rows: several hundred cells per row, split between threads
    ys, xs = np.meshgrid(np.arange(500, 504), np.arange(0, n, 2), indexing="ij")
    cell = np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.int32)
    band = I.Boundary(2, n, cell, np.full(len(cell), 1.0 / n), np.tile([0.0, 1.0], (len(cell), 1)),
                      (cell + 0.5) / n, np.zeros(len(cell)))
    xb = rng.standard_normal(band.nb)
    plan = _plan(band, kind)
    for layer, lid in (("single", 0), ("double", 1)):
        ref = oracle_mod.apply("laplace2d", lid, band.cell, band.h, band.w, band.normal, xb)
        y1 = gpu_apply(torch_cuda, plan, layer, xb)
        assert rel_l2(y1, ref) <= TOL[kind], layer
        assert np.array_equal(gpu_apply(torch_cuda, plan, layer, xb), y1)
    plan.device_status()


@pytest.mark.parametrize("kind", KINDS)
def test_tc_refined_solve_reaches_1e6(torch_cuda, oracle_mod, kind):
    """GMRES on the tensor-core operator with residuals from the double-float
    companion reaches relative residual 1e-6 against the FP64 oracle
    (star n = 1024, mixed BCs, u = e^x cos y)."""
    b = I.star_boundary(1024)
    u, q = I.boundary_data(b, I.field_expcos)
    bc = I.mixed_bc_theta(b)
    data = np.where(bc == 0, u, q)
    plan = _plan(b, kind)
    plan.enable_refinement(True)
    u_out, q_out, info = plan.solve(bc, data, tol=1e-6, restart=100, max_iter=1500)
    print(f"{kind} refined solve {info}")
    assert info["status"] == 0, info
    x = np.where(bc == 0, q_out, u_out)
    rhs = oracle_mod.system_rhs("laplace2d", b.cell, b.h, b.w, b.normal, bc, u * (bc == 0), q * (bc == 1))
    r = rhs - oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc, x)
    assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 2e-6


def test_tc_wait_that_runs_out_is_reported_and_the_context_survives(torch_cuda, oracle_mod):
    """The test hook makes every tensor-core stage issue nothing, so its
    bounded wait runs out (about a second; nothing faults, traps or hangs);
    the CTAs stop and free their tensor memory, bem_device_status reports
    BEM_ERR_TIMEOUT once, and the next apply without the hook is correct."""
    import time
    from paper_1809_00845_gb300 import bem
    b = I.star_boundary(1024)
    bc = I.mixed_bc_theta(b)
    x = np.random.default_rng(3).standard_normal(b.nb)
    plan = _plan(b, "tc_bf16x3")
    plan.set_bc(bc, 0.5)
    plan.set_test_flags(bem.BEM_TEST_WAIT_RUNS_OUT)
    t0 = time.perf_counter()
    gpu_apply(torch_cuda, plan, "system", x)
    elapsed = time.perf_counter() - t0
    with pytest.raises(bem.BemError) as e:
        plan.device_status()
    assert e.value.status == bem.BEM_ERR_TIMEOUT
    assert 0.5 < elapsed < 30.0, elapsed
    plan.device_status()  # the record was cleared
    plan.set_test_flags(0)
    out = gpu_apply(torch_cuda, plan, "system", x)
    plan.device_status()
    ref = oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc, x, rows=(0, 400))
    assert rel_l2(out[:400], ref) <= TOL["tc_bf16x3"]
