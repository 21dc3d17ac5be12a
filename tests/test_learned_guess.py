"""The trained initial-guess network against zero-start GMRES on held-out
random stars (GPU).  Reports iterations and seconds to 1e-6 from zero, from
the Dirichlet-to-Neumann estimate alone and from the network's guess (the
guess's own cost included); the guess must shorten the solve on average, in
iterations and in wall time, and every solve must converge."""
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
    assert meta["cin"] == L.NET_SHAPE["cin"]
    ev = L.evaluate(net, range(L.TEST_SEED0 + 100, L.TEST_SEED0 + 116), tscale=meta.get("tscale", 1.0))
    print(json.dumps({k: v for k, v in ev.items() if k != "rows"}))
    assert ev["all_converged"]
    assert ev["mean_iters_guess"] < ev["mean_iters_zero"]
    assert ev["mean_s_guess"] < ev["mean_s_zero"]
