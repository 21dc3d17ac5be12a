"""The learned-guess network's CUDA forward/backward/Adam kernels against the
CPU FP64 oracle with the same BF16 rounding points (GPU)."""
import numpy as np
import pytest

from oracle import net_oracle as N

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_00845_gb300 import build
    build.build()
    return torch


def _net(cin, hidden, layers, ksize, dil, seed=3):
    from paper_1809_00845_gb300.bem import Net
    return Net(cin, hidden, layers, ksize, dil, seed)


@pytest.mark.parametrize("shape", [(3, 8, 3, 3, (1, 2, 1)), (7, 64, 4, 5, (1, 3, 9, 27))])
def test_forward_and_gradient_match_oracle(torch_cuda, shape):
    cin, h, L, K, dil = shape
    net = _net(cin, h, L, K, dil)
    rng = np.random.default_rng(11)
    lens = [37, 120, 64] if h < 64 else [300, 517]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    T = int(off[-1])
    f = rng.standard_normal((T, cin)).astype(np.float32)
    tg = rng.standard_normal(T).astype(np.float32)
    p = net.get_params().astype(np.float64)
    y_gpu = net.forward(f, off).cpu().numpy()
    y_ref, _ = N.forward(p, f, off, cin, h, L, K, list(dil))
    assert np.linalg.norm(y_gpu - y_ref) / np.linalg.norm(y_ref) < 2e-3
    loss_gpu, g_gpu = net.gradient(f, off, tg)
    loss_ref, g_ref = N.loss_and_grad(p, f, off, tg, cin, h, L, K, list(dil))
    assert abs(loss_gpu - loss_ref) / loss_ref < 2e-3
    assert np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref) < 1e-2


def test_adam_steps_reduce_loss(torch_cuda):
    net = _net(3, 16, 3, 5, (1, 2, 4))
    rng = np.random.default_rng(2)
    off = np.array([0, 200, 450], np.int32)
    f = rng.standard_normal((450, 3)).astype(np.float32)
    tg = (0.5 * f[:, 0] - 0.25 * f[:, 1] * f[:, 2]).astype(np.float32)
    first = net.train_step(f, off, tg, lr=3e-3)
    for _ in range(150):
        last = net.train_step(f, off, tg, lr=3e-3)
    assert last < 0.2 * first
