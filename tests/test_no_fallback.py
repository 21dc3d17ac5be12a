"""The product path has no CPU fallback (CPU only): a missing library raises
on load, and without a usable CUDA device a plan fails with BEM_ERR_CUDA
instead of computing anything on the host."""
import pytest

from paper_1809_00845_gb300 import bem
from paper_1809_00845_gb300 import inputs as I


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(bem, "_lib", None)
    with pytest.raises(ImportError):
        bem.load_library(str(tmp_path / "libbem_gb300.so"))


def test_plan_without_a_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_1809_00845_gb300 import build
    build.build()
    with pytest.raises(bem.BemError) as e:
        bem.Plan.from_boundary(I.circle_boundary(128), "laplace2d", "f32")
    assert e.value.status == bem.BEM_ERR_CUDA
