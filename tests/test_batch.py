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


@pytest.mark.parametrize("layer", ["single", "system"])
def test_batch_equals_individual_applies(torch_cuda, layer):
    torch = torch_cuda
    from paper_1809_00845_gb300.bem import Batch, Plan
    rng = np.random.default_rng(42)
    plans, bounds = [], []
    for k, n in enumerate((64, 128, 256, 512, 512, 1024, 256, 2048)):
        b = I.curve_boundary(n, I.random_star_curve(rng))
        p = Plan.from_boundary(b, "laplace2d", "f32")
        if layer == "system":
            p.set_bc(I.mixed_bc_theta(b), 0.5)
        plans.append(p)
        bounds.append(b)
    batch = Batch(plans, layer, streams=4)
    assert batch.launches == 3 * len(plans)
    src = torch.from_numpy(rng.standard_normal(batch.total).astype(np.float32)).cuda()
    raw_in = _as_tensor(torch, batch.d_in, batch.total)
    raw_out = _as_tensor(torch, batch.d_out, batch.total)
    raw_in.copy_(src)
    for _ in range(2):
        batch.apply()
        torch.cuda.synchronize()
        for p, off in zip(plans, batch.offsets):
            seg = src[off:off + p.nb].contiguous()
            ref = p.apply(layer, seg)
            torch.cuda.synchronize()
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
