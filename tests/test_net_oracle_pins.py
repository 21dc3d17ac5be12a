"""Pins of the learned-guess network oracle (CPU): BF16 rounding against its
definition, the circular convolution against scipy's wrap-mode correlation,
and the analytic gradient against central finite differences (FP64)."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import net_oracle as N


def test_bf16_round_to_nearest_even():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e38, 1e-40])
    got = N.bf16_round(vals)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even (1.0); 1 + 3*2^-8 -> 1 + 2^-6
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1.0 + 2 ** -6 and got[3] == -2.5
    # every result is exactly representable with an 8-bit significand
    m, e = np.frexp(got[np.isfinite(got) & (got != 0)])
    assert np.all(np.abs(m * 256 - np.round(m * 256)) == 0)


def test_circular_conv_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    L, cin, K = 23, 1, 5
    x = rng.standard_normal((L, cin))
    w = rng.standard_normal(K)
    params = np.concatenate([w, [0.0]])  # one layer, cout = 1, bias 0
    y, _ = N.forward(params, x, [0, L], cin, 1, 1, K, [1], bf16=False)
    ref = ndimage.correlate1d(x[:, 0], w, mode="wrap")
    assert np.allclose(y, ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dil", [[1, 1, 1], [1, 2, 4]])
def test_gradient_matches_finite_differences(dil):
    rng = np.random.default_rng(0)
    cin, h, L, K = 3, 4, 3, 3
    n = sum((1 if l == L - 1 else h) * (cin if l == 0 else h) * K + (1 if l == L - 1 else h) for l in range(L))
    p = rng.standard_normal(n) * 0.5
    off = [0, 9, 21]
    f = rng.standard_normal((21, cin))
    tg = rng.standard_normal(21)
    loss, g = N.loss_and_grad(p, f, off, tg, cin, h, L, K, dil, bf16=False)
    eps = 1e-6
    fd = np.zeros(n)
    for i in range(n):
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd[i] = (N.loss_and_grad(pp, f, off, tg, cin, h, L, K, dil, bf16=False)[0] -
                 N.loss_and_grad(pm, f, off, tg, cin, h, L, K, dil, bf16=False)[0]) / (2 * eps)
    assert np.linalg.norm(fd - g) / np.linalg.norm(g) < 1e-7


def test_bf16_rounding_points():
    """With rounding on, every layer input and every weight the forward uses
    is a BF16 value (the rounding points of the kernels), the first layer's
    input is the rounded features and the last layer's output is not rounded."""
    rng = np.random.default_rng(2)
    cin, h, L, K, dil = 3, 4, 3, 3, [1, 2, 4]
    n = sum((1 if l == L - 1 else h) * (cin if l == 0 else h) * K + (1 if l == L - 1 else h) for l in range(L))
    p = rng.standard_normal(n) * 0.5
    f = rng.standard_normal((21, cin))
    y, cache = N.forward(p, f, [0, 9, 21], cin, h, L, K, dil, bf16=True)
    assert np.array_equal(cache[0][0], N.bf16_round(f))
    for x, Wr, _ in cache:
        assert np.array_equal(x, N.bf16_round(x)) and np.array_equal(Wr, N.bf16_round(Wr))
    for l in range(1, L):
        assert np.array_equal(cache[l][0], N.bf16_round(np.maximum(cache[l - 1][2], 0.0)))
    assert not np.array_equal(y, N.bf16_round(y))
