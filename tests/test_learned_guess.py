"""The trained initial-guess network against zero-start GMRES on held-out
random stars (GPU).  Reports iterations and seconds to 1e-6 both ways; the
safeguarded guess (optimal scaling, alpha >= 0) must never start from a larger
residual than zero, and every solve must converge."""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_00845_gb300 import build
    build.build()
    return torch


def test_learned_guess_on_held_out_geometries(torch_cuda):
    from paper_1809_00845_gb300 import learned as L
    if not os.path.exists(L.WEIGHTS):
        pytest.skip("no trained weights (run python -m paper_1809_00845_gb300.learned)")
    net, meta = L.load()
    ev = L.evaluate(net, range(L.TEST_SEED0 + 100, L.TEST_SEED0 + 104), tscale=meta.get("tscale", 1.0))
    print(json.dumps({k: v for k, v in ev.items() if k != "rows"}))
    assert ev["all_converged"]
    for r in ev["rows"]:
        assert r["alpha"] >= 0.0
        assert r["guess_iters"] <= r["zero_iters"] + 3
