"""Exits of bem_solve other than convergence by iteration (GPU): non-finite
data, a solution that is already exact (the initial guess equals a previous
solution, or the data are zero), and an initial guess worse than zero (the
solver starts from zero instead, so the guess costs no iterations)."""
import numpy as np
import pytest

from paper_1809_00845_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_00845_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("prec,refine", [("f64", False), ("f32", True)])
def test_solve_exits(torch_cuda, prec, refine):
    from paper_1809_00845_gb300 import bem
    b = I.star_boundary(512)
    bc = I.mixed_bc_theta(b)
    u, q = I.boundary_data(b, I.field_expcos)
    data = np.where(bc == 0, u, q)
    p = bem.Plan.from_boundary(b, "laplace2d", prec)
    p.enable_refinement(refine)
    u1, q1, info = p.solve(bc, data, tol=1e-8, restart=100, max_iter=2000)
    assert info["status"] == bem.BEM_OK and info["iters"] > 5
    x_exact = np.where(bc == 0, q1, u1)
    # an exact start: no iteration, same answer
    u2, q2, info2 = p.solve(bc, data, tol=1e-6, restart=100, max_iter=2000, x0=x_exact)
    assert info2["status"] == bem.BEM_OK and info2["iters"] == 0, info2
    assert np.allclose(np.where(bc == 0, q2, u2), x_exact, rtol=0, atol=0)
    # zero data: the zero solution, at once
    _, q3, info3 = p.solve(bc, np.zeros_like(data), tol=1e-6, restart=100, max_iter=2000)
    assert info3["status"] == bem.BEM_OK and info3["iters"] == 0 and not np.any(q3)
    # a guess far worse than zero is replaced by zero: the same iterations as a zero start
    _, _, info4 = p.solve(bc, data, tol=1e-6, restart=100, max_iter=2000)
    bad = 1e3 * np.random.default_rng(5).standard_normal(b.nb)
    _, _, info5 = p.solve(bc, data, tol=1e-6, restart=100, max_iter=2000, x0=bad)
    assert info5["status"] == bem.BEM_OK
    assert info5["iters"] <= info4["iters"] + 2, (info4["iters"], info5["iters"])
    # non-finite data
    nan_data = data.copy()
    nan_data[7] = np.nan
    with pytest.raises(bem.BemError) as e:
        p.solve(bc, nan_data, tol=1e-6, restart=100, max_iter=2000)
    assert e.value.status == bem.BEM_ERR_NONFINITE
    # the plan is still usable afterwards
    _, _, info7 = p.solve(bc, data, tol=1e-6, restart=100, max_iter=2000)
    assert info7["status"] == bem.BEM_OK
    p.close()
