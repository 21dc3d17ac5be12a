"""Batched apply (one CUDA graph over many plans of uneven grid sizes) equals
the per-plan applies bit for bit (GPU)."""
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


@pytest.mark.parametrize("grouped", [False, True])
@pytest.mark.parametrize("layer", ["single", "system"])
def test_batch_equals_individual_applies(torch_cuda, layer, grouped):
    """Every segment of a batched apply equals the plan's own apply: bit for
    bit when each plan is applied on its own; with grouped launches (FP32
    four-step plans of a grid size share one persistent launch, so the columns
    are split over the CTAs differently) to FP32 rounding, and the same on
    every replay."""
    torch = torch_cuda
    from paper_1809_00845_gb300.bem import Batch, Plan
    rng = np.random.default_rng(42)
    plans, bounds = [], []
    sizes = (64, 128, 256, 512, 512, 1024, 256, 2048)
    for k, n in enumerate(sizes):
        b = I.curve_boundary(n, I.random_star_curve(rng))
        p = Plan.from_boundary(b, "laplace2d", "f32")
        if layer == "system":
            p.set_bc(I.mixed_bc_theta(b), 0.5)
        plans.append(p)
        bounds.append(b)
    batch = Batch(plans, layer, streams=4)
    batch.set_grouping(grouped)
    if grouped:
        # four-step plans (n >= 256) of one size share a launch: preps, one column launch, reductions
        counts = {n: sizes.count(n) for n in set(sizes) if n >= 256}
        expect = sum(2 * c + 1 if c > 1 else 3 * c for c in counts.values()) + 3 * sum(n < 256 for n in sizes)
        assert batch.launches == expect
    else:
        assert batch.launches == 3 * len(plans)
    src = torch.from_numpy(rng.standard_normal(batch.total).astype(np.float32)).cuda()
    raw_in = _as_tensor(torch, batch.d_in, batch.total)
    raw_out = _as_tensor(torch, batch.d_out, batch.total)
    raw_in.copy_(src)
    first = None
    for _ in range(2):
        batch.apply()
        torch.cuda.synchronize()
        if first is None:
            first = raw_out.clone()
        else:
            assert torch.equal(raw_out, first)
        for p, off in zip(plans, batch.offsets):
            seg = src[off:off + p.nb].contiguous()
            ref = p.apply(layer, seg)
            torch.cuda.synchronize()
            if grouped:
                got = raw_out[off:off + p.nb].double()
                assert float(torch.linalg.norm(got - ref.double()) / torch.linalg.norm(ref.double())) <= 1e-6
            else:
                assert torch.equal(raw_out[off:off + p.nb], ref)
    batch.close()


@pytest.mark.parametrize("kernel,sizes", [("laplace2d", (2048, 512)), ("laplace2d", (256, 64)),
                                           ("laplace3d", (32, 16))])
def test_larger_plan_still_applies_after_smaller_plan(torch_cuda, kernel, sizes):
    """A plan keeps working (bit for bit) after a plan of a smaller grid, whose
    kernels need less shared memory, has been made; the batch capture in
    random size order depends on this."""
    torch = torch_cuda
    from paper_1809_00845_gb300.bem import Plan
    rng = np.random.default_rng(7)
    if kernel == "laplace2d":
        big, small = (I.curve_boundary(n, I.random_star_curve(rng)) for n in sizes)
    else:
        big, small = (I.ellipsoid_boundary(n) for n in sizes)
    p = Plan.from_boundary(big, kernel, "f32")
    x = torch.from_numpy(rng.standard_normal(big.nb).astype(np.float32)).cuda()
    before = p.apply("single", x)
    torch.cuda.synchronize()
    q = Plan.from_boundary(small, kernel, "f32")
    q.apply("single", torch.ones(small.nb, dtype=torch.float32, device="cuda"))
    after = p.apply("single", x)
    torch.cuda.synchronize()
    assert torch.equal(before, after)
    p.close()
    q.close()


def _as_tensor(torch, ptr, numel):
    """A float32 CUDA tensor aliasing device memory at ptr (no copy)."""
    class _Cai:
        __cuda_array_interface__ = {"shape": (numel,), "typestr": "<f4", "data": (ptr, False), "version": 2}
    return torch.as_tensor(_Cai(), device="cuda")


@pytest.mark.parametrize("refine,tol,bound", [(False, 1e-5, 1e-4), (True, 1e-8, 2e-8)])
def test_batch_solve_matches_oracle_residuals(torch_cuda, oracle_mod, refine, tol, bound):
    """Lockstep batched GMRES over stars of several grid sizes and mixed
    boundary conditions: every system's solution has an oracle residual within
    the bound (FP32 plans; with refinement the residuals use the double-float
    companions)."""
    from paper_1809_00845_gb300.bem import Batch, Plan
    rng = np.random.default_rng(5)
    bounds, plans = [], []
    for n in (256, 512, 256, 1024, 512):
        b = I.curve_boundary(n, I.random_star_curve(rng))
        p = Plan.from_boundary(b, "laplace2d", "f32")
        p.set_bc(I.mixed_bc_theta(b), 0.5)
        if refine:
            p.enable_refinement(True)
        bounds.append(b)
        plans.append(p)
    batch = Batch(plans, "system", streams=4)
    bcs, datas, us, qs = [], [], [], []
    for b in bounds:
        u, q = I.boundary_data(b, I.field_expcos)
        bc = I.mixed_bc_theta(b)
        bcs.append(bc)
        datas.append(np.where(bc == 0, u, q))
        us.append(u)
        qs.append(q)
    u_out, q_out, infos, status = batch.solve(np.concatenate(bcs), np.concatenate(datas), tol=tol, restart=100,
                                              max_iter=1500)
    assert status == 0, infos
    for k, b in enumerate(bounds):
        o = batch.offsets[k]
        sl = slice(o, o + b.nb)
        bc = bcs[k]
        x = np.where(bc == 0, q_out[sl], u_out[sl])
        rhs = oracle_mod.system_rhs("laplace2d", b.cell, b.h, b.w, b.normal, bc, us[k] * (bc == 0), qs[k] * (bc == 1))
        r = rhs - oracle_mod.system_apply("laplace2d", b.cell, b.h, b.w, b.normal, bc, x)
        assert np.linalg.norm(r) / np.linalg.norm(rhs) <= bound, (k, infos[k])
        assert infos[k]["rel_residual"] <= tol
    # a second solve with other data reuses the captured graphs
    u2, q2, infos2, st2 = batch.solve(np.concatenate(bcs), 2.0 * np.concatenate(datas), tol=tol, restart=100,
                                      max_iter=1500)
    assert st2 == 0
    batch.close()


def test_batch_solve_equals_single_solves(torch_cuda):
    """The lockstep solve of a batch and per-plan bem_solve reach the same
    solutions (both to 1e-10 with FP64 plans)."""
    from paper_1809_00845_gb300.bem import Batch, Plan
    rng = np.random.default_rng(8)
    bounds = [I.curve_boundary(n, I.random_star_curve(rng)) for n in (256, 512)]
    plans = []
    for b in bounds:
        p = Plan.from_boundary(b, "laplace2d", "f64")
        p.set_bc(np.zeros(b.nb, np.uint8), 0.5)
        plans.append(p)
    batch = Batch(plans, "system", streams=2)
    datas = [I.boundary_data(b, I.field_x2y2)[0] for b in bounds]
    u, q, infos, st = batch.solve(np.zeros(batch.total, np.uint8), np.concatenate(datas), tol=1e-10, restart=100)
    assert st == 0
    for k, (b, p) in enumerate(zip(bounds, plans)):
        _, qk, ik = p.solve(np.zeros(b.nb, np.uint8), datas[k], tol=1e-10, restart=100)
        o = batch.offsets[k]
        assert np.linalg.norm(q[o:o + b.nb] - qk) / np.linalg.norm(qk) <= 1e-8
    batch.close()


def test_batch_solve_3d_and_initial_guess(torch_cuda, oracle_mod):
    """3D Laplace plans of two grid sizes in one batch (Dirichlet, FP64): the
    batched solution equals the dense LU solution of each system; starting
    from the solution itself ends at once with the same answer."""
    from paper_1809_00845_gb300.bem import Batch, Plan
    bounds = [I.ellipsoid_boundary(16), I.ellipsoid_boundary(32)]
    plans = []
    for b in bounds:
        p = Plan.from_boundary(b, "laplace3d", "f64")
        p.set_bc(np.zeros(b.nb, np.uint8), 0.5)
        plans.append(p)
    batch = Batch(plans, "system", streams=2)
    datas = [I.boundary_data(b, I.field_xy_z)[0] for b in bounds]
    bc = np.zeros(batch.total, np.uint8)
    u, q, infos, st = batch.solve(bc, np.concatenate(datas), tol=1e-11, restart=100, max_iter=500)
    assert st == 0, infos
    refs = []
    for k, b in enumerate(bounds):
        A, rhs = oracle_mod.system("laplace3d", b.cell, b.h, b.w, b.normal, np.zeros(b.nb, np.uint8), datas[k],
                                   np.zeros(b.nb))
        ref = oracle_mod.solve_lu(A, rhs)
        refs.append(ref)
        o = batch.offsets[k]
        assert np.linalg.norm(q[o:o + b.nb] - ref) / np.linalg.norm(ref) <= 1e-8
    u2, q2, infos2, st2 = batch.solve(bc, np.concatenate(datas), tol=1e-10, restart=100, max_iter=500,
                                      x0=np.concatenate(refs))
    assert st2 == 0 and infos2[0]["iters"] <= 2, infos2[0]
    assert np.linalg.norm(q2 - np.concatenate(refs)) / np.linalg.norm(np.concatenate(refs)) <= 1e-9
    batch.close()


def test_tuned_choices_are_cached_and_keep_results(torch_cuda):
    """The autotuner picks a stream count for a batch and a preconditioner
    block for a plan, stores them by shape (a second call returns at once with
    the same choice), and the tuned objects give the same results."""
    import time
    from paper_1809_00845_gb300.bem import Batch, Plan
    rng = np.random.default_rng(11)
    bounds = [I.curve_boundary(n, I.random_star_curve(rng)) for n in (512, 256, 1024, 512)]
    plans = [Plan.from_boundary(b, "laplace2d", "f32") for b in bounds]
    batch = Batch(plans, "single", streams=4)
    src = torch_cuda.from_numpy(rng.standard_normal(batch.total).astype(np.float32)).cuda()
    raw_in = _as_tensor(torch_cuda, batch.d_in, batch.total)
    raw_out = _as_tensor(torch_cuda, batch.d_out, batch.total)
    raw_in.copy_(src)
    batch.apply()
    torch_cuda.cuda.synchronize()
    before = raw_out.clone()
    s1 = batch.tune(reps=5)
    assert s1 in (1, 2, 4, 8)
    t0 = time.perf_counter()
    assert batch.tune(reps=5) == s1
    assert time.perf_counter() - t0 < 0.5
    batch.apply()
    torch_cuda.cuda.synchronize()
    assert torch_cuda.equal(raw_out, before)
    batch.close()
    b = bounds[2]
    u, q = I.boundary_data(b, I.field_expcos)
    bc = I.mixed_bc_theta(b)
    data = np.where(bc == 0, u, q)
    p = plans[2]
    bs = p.tune_preconditioner(bc, data, tol=1e-5)
    assert bs in (32, 64, 128)
    assert p.tune_preconditioner(bc, data, tol=1e-5) == bs
    _, _, info = p.solve(bc, data, tol=1e-5, restart=100)
    assert info["status"] == 0
