"""Parity of the 3D CUDA apply (3D Laplace, Kelvin) with the CPU FP64 oracle
(GPU).  Relative L2 <= 1e-12 (FP64 and double-float) / 2e-6 (FP32) on random
N(0,1) densities."""
import numpy as np
import pytest

from paper_1809_00845_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32x2": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_00845_gb300 import build
    build.build()
    return torch


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_apply(torch, plan, layer, x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=plan.np_dtype).reshape(-1)).cuda()
    y = plan.apply(layer, t)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


def _plan(b, kernel, prec, nu=0.3, mu=1.0):
    from paper_1809_00845_gb300.bem import Plan
    return Plan.from_boundary(b, kernel, prec, nu=nu, mu=mu)


@pytest.mark.parametrize("prec", ["f64", "f32", "f32x2"])
@pytest.mark.parametrize("n,nb", [(16, 60), (32, 400), (64, 1500)])
def test_laplace3d_random_cells(torch_cuda, oracle_mod, prec, n, nb):
    rng = np.random.default_rng(300 + n)
    b = I.random_cells(n, nb, rng, dim=3)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, "laplace3d", prec)
    for layer, lid in (("single", 0), ("double", 1)):
        ref = oracle_mod.apply("laplace3d", lid, b.cell, b.h, b.w, b.normal, x)
        assert rel_l2(gpu_apply(torch_cuda, plan, layer, x), ref) <= TOL[prec], layer
    bc = (rng.uniform(size=b.nb) < 0.4).astype(np.uint8)
    plan.set_bc(bc, 0.5)
    ref = oracle_mod.system_apply("laplace3d", b.cell, b.h, b.w, b.normal, bc, x)
    assert rel_l2(gpu_apply(torch_cuda, plan, "system", x), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32", "f32x2"])
@pytest.mark.parametrize("n,nb", [(16, 50), (32, 300)])
def test_kelvin_random_cells(torch_cuda, oracle_mod, prec, n, nb):
    rng = np.random.default_rng(700 + n)
    b = I.random_cells(n, nb, rng, dim=3)
    x = rng.standard_normal((b.nb, 3))
    plan = _plan(b, "kelvin3d", prec, nu=0.3, mu=1.0)
    for layer, lid in (("single", 0), ("double", 1)):
        ref = oracle_mod.apply("kelvin3d", lid, b.cell, b.h, b.w, b.normal, x, nu=0.3, mu=1.0)
        assert rel_l2(gpu_apply(torch_cuda, plan, layer, x), ref) <= TOL[prec], layer
    bc = (rng.uniform(size=(b.nb, 3)) < 0.5).astype(np.uint8)
    plan.set_bc(bc, 0.5)
    ref = oracle_mod.system_apply("kelvin3d", b.cell, b.h, b.w, b.normal, bc, x, nu=0.3, mu=1.0)
    assert rel_l2(gpu_apply(torch_cuda, plan, "system", x), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32", "f32x2"])
def test_system_operator_uniform_bc_3d(torch_cuda, oracle_mod, prec):
    """All-Dirichlet and all-Neumann data in 3D (Laplace and Kelvin, the
    latter also with one component Neumann everywhere): the system operator
    leaves out the fields no cell feeds and must still be the oracle's."""
    rng = np.random.default_rng(77)
    b = I.random_cells(32, 300, rng, dim=3)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, "laplace3d", prec)
    for fill in (0, 1, 0):
        bc = np.full(b.nb, fill, np.uint8)
        plan.set_bc(bc, 0.5)
        ref = oracle_mod.system_apply("laplace3d", b.cell, b.h, b.w, b.normal, bc, x)
        assert rel_l2(gpu_apply(torch_cuda, plan, "system", x), ref) <= TOL[prec], fill
    plan.close()
    xk = rng.standard_normal((b.nb, 3))
    plan = _plan(b, "kelvin3d", prec, nu=0.3, mu=1.0)
    patterns = [np.zeros((b.nb, 3), np.uint8), np.ones((b.nb, 3), np.uint8), np.zeros((b.nb, 3), np.uint8)]
    patterns[2][:, 1] = 1
    for bc in patterns:
        plan.set_bc(bc, 0.5)
        ref = oracle_mod.system_apply("kelvin3d", b.cell, b.h, b.w, b.normal, bc, xk, nu=0.3, mu=1.0)
        assert rel_l2(gpu_apply(torch_cuda, plan, "system", xk), ref) <= TOL[prec], bc[0]
    plan.close()


def test_kelvin_other_material(torch_cuda, oracle_mod):
    rng = np.random.default_rng(5)
    b = I.random_cells(16, 40, rng, dim=3)
    x = rng.standard_normal((b.nb, 3))
    plan = _plan(b, "kelvin3d", "f64", nu=0.15, mu=2.5)
    for layer, lid in (("single", 0), ("double", 1)):
        ref = oracle_mod.apply("kelvin3d", lid, b.cell, b.h, b.w, b.normal, x, nu=0.15, mu=2.5)
        assert rel_l2(gpu_apply(torch_cuda, plan, layer, x), ref) <= 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32", "f32x2"])
def test_ellipsoid_n64(torch_cuda, oracle_mod, prec):
    b = I.ellipsoid_boundary(64)
    rng = np.random.default_rng(8)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, "laplace3d", prec)
    for layer, lid in (("single", 0), ("double", 1)):
        ref = oracle_mod.apply("laplace3d", lid, b.cell, b.h, b.w, b.normal, x)
        assert rel_l2(gpu_apply(torch_cuda, plan, layer, x), ref) <= TOL[prec], layer


def test_ellipsoid_n256_full_size_sampled_rows(torch_cuda, oracle_mod):
    """The 256^3 ellipsoid (padded 512^3), FP32 single layer; the oracle
    evaluates 2 x 256 target rows exactly."""
    b = I.ellipsoid_boundary(256)
    rng = I.rng_for(2)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, "laplace3d", "f32")
    out = gpu_apply(torch_cuda, plan, "single", x)
    for row0 in (0, b.nb // 2):
        ref = oracle_mod.apply("laplace3d", 0, b.cell, b.h, b.w, b.normal, x, rows=(row0, 256))
        assert rel_l2(out[row0:row0 + 256], ref) <= TOL["f32"], row0


def test_cube_kelvin_n128_full_size_sampled_rows(torch_cuda, oracle_mod):
    """The Kelvin cube on 128^3 (padded 256^3), FP32 U and T operators."""
    b = I.cube_boundary(128)
    rng = I.rng_for(3)
    x = rng.standard_normal((b.nb, 3))
    plan = _plan(b, "kelvin3d", "f32")
    for layer, lid in (("single", 0), ("double", 1)):
        out = gpu_apply(torch_cuda, plan, layer, x).reshape(-1, 3)
        ref = oracle_mod.apply("kelvin3d", lid, b.cell, b.h, b.w, b.normal, x, rows=(1000, 128))
        assert rel_l2(out[1000:1128], ref) <= TOL["f32"], layer


@pytest.mark.parametrize("prec", ["f32", "f64", "f32x2"])
def test_largest_3d_grid_sampled_rows(torch_cuda, oracle_mod, prec):
    """The largest supported 3D grid, n = 512 (padded 1024^3: line FFTs span
    two warps, 8 planes per y-pass block), a small ellipsoid of 46k cells,
    single and double layer; the oracle evaluates sampled target rows."""
    b = I.ellipsoid_boundary(512, axes=(0.12, 0.1, 0.08))
    rng = I.rng_for(4)
    x = rng.standard_normal(b.nb)
    plan = _plan(b, "laplace3d", prec)
    for layer, lid in (("single", 0), ("double", 1)):
        out = gpu_apply(torch_cuda, plan, layer, x)
        for row0 in (0, b.nb - 200):
            ref = oracle_mod.apply("laplace3d", lid, b.cell, b.h, b.w, b.normal, x, rows=(row0, 200))
            assert rel_l2(out[row0:row0 + 200], ref) <= TOL[prec], (layer, row0)
