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


def _circle_elements(R, nb, phase=0.3):
    """nb equal elements of a circle of radius R about (0.4, 0.6): midpoint
    angles, arclength positions of the midpoints, lengths."""
    th = phase + 2 * np.pi * (np.arange(nb) + 0.5) / nb
    length = np.full(nb, 2 * np.pi * R / nb)
    s = np.cumsum(length) - 0.5 * length
    return th, s, length


@pytest.mark.parametrize("m", [1, 2, 5, 17])
def test_dtn_estimate_is_the_circle_flux(m):
    """On a circle the estimate is the exact interior flux of a harmonic
    field: u = Re((z - c)^m) = R^m cos(m theta) has q = m R^(m-1) cos(m theta)."""
    R, nb = 0.27, 400
    th, s, length = _circle_elements(R, nb)
    u = R ** m * np.cos(m * th)
    q = N.dtn_estimate(s, length, u, [0, nb], kmax=nb // 2 - 1)
    exact = m * R ** (m - 1) * np.cos(m * th)
    # FP64 sums over ~200 modes whose multipliers reach 2 pi k / Lambda ~ 700
    assert np.allclose(q, exact, rtol=0, atol=1e-8 * np.abs(exact).max())


def test_dtn_estimate_constants_scaling_and_batches():
    rng = np.random.default_rng(4)
    th, s, length = _circle_elements(0.3, 256)
    assert np.allclose(N.dtn_estimate(s, length, np.full(256, 2.5), [0, 256], 100), 0.0, atol=1e-8)
    u = rng.standard_normal(256)
    q1 = N.dtn_estimate(s, length, u, [0, 256], 100)
    q2 = N.dtn_estimate(2 * s, 2 * length, u, [0, 256], 100)  # the same curve twice as large
    assert np.allclose(q2, q1 / 2, rtol=1e-12, atol=1e-12)
    # two curves in one batch are estimated independently
    _, s2, l2 = _circle_elements(0.2, 100)
    u2 = rng.standard_normal(100)
    both = N.dtn_estimate(np.concatenate([s, s2]), np.concatenate([length, l2]), np.concatenate([u, u2]),
                          [0, 256, 356], 40)
    assert np.allclose(both[:256], N.dtn_estimate(s, length, u, [0, 256], 40), rtol=1e-13, atol=1e-13)
    assert np.allclose(both[256:], N.dtn_estimate(s2, l2, u2, [0, 100], 40), rtol=1e-13, atol=1e-13)


def test_fourier_features_definition():
    """Features of points chosen so that b . p hits quarter periods: sin and
    cos in their slots, one frequency row per pair, the rows of B not
    transposed; sin^2 + cos^2 = 1 and integer shifts leave integer-frequency
    features unchanged."""
    B = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 0.5]])
    p = np.array([[0.25, 0.0, 0.0], [0.0, 0.125, 0.0], [0.0, 0.0, 1.0]])
    f = N.fourier_features(p, B)
    assert f.shape == (3, 6)
    np.testing.assert_allclose(f[0, 0:2], [1.0, 0.0], atol=1e-15)   # 2 pi * 0.25: sin 1, cos 0
    np.testing.assert_allclose(f[1, 2:4], [1.0, 0.0], atol=1e-15)   # 2 pi * 2 * 0.125
    np.testing.assert_allclose(f[2, 4:6], [0.0, -1.0], atol=1e-15)  # 2 pi * 0.5 * 1
    np.testing.assert_allclose(f[0, 2:6], [0.0, 1.0, 0.0, 1.0], atol=1e-15)  # other rows see b . p = 0
    rng = np.random.default_rng(3)
    pts = rng.uniform(size=(50, 3))
    Bi = rng.integers(-4, 5, size=(7, 3)).astype(np.float64)
    g = N.fourier_features(pts, Bi)
    np.testing.assert_allclose(g[:, 0::2] ** 2 + g[:, 1::2] ** 2, 1.0, atol=1e-14)
    np.testing.assert_allclose(N.fourier_features(pts + np.array([1.0, -2.0, 3.0]), Bi), g, atol=1e-12)


def test_guess_features_definition():
    """Hand-computed columns: a curve with u = (3, -4) (rms 3.5355...) and
    qd = (1, 2), radius 0.3; a second curve of zeros keeps scale 1; the
    geometry columns pass through in order."""
    geo = np.array([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]])
    u = np.array([3.0, -4.0, 0.0])
    qd = np.array([1.0, 2.0, 0.0])
    f = N.guess_features(geo, u, qd, [0, 2, 3], 0.3)
    s = np.sqrt(12.5)
    np.testing.assert_allclose(f[:, :2], geo, rtol=0, atol=0)
    np.testing.assert_allclose(f[:2, 2], [3 / s, -4 / s], rtol=1e-15)
    np.testing.assert_allclose(f[:2, 3], [0.3 / s, 0.6 / s], rtol=1e-15)
    np.testing.assert_array_equal(f[2, 2:], [0.0, 0.0])


def test_guess_finish_zero_flux_and_scaling():
    """The guess has zero length-weighted sum on every curve, leaves a
    zero-flux qd unchanged when corr = 0, is linear in corr with the factor
    cscale * rms(u), and a constant corr is removed entirely."""
    rng = np.random.default_rng(21)
    off = [0, 40, 100]
    length = rng.uniform(0.5, 2.0, 100)
    u = rng.standard_normal(100)
    corr = rng.standard_normal(100)
    qd = rng.standard_normal(100)
    for a, b in zip(off[:-1], off[1:]):
        qd[a:b] -= np.dot(length[a:b], qd[a:b]) / length[a:b].sum()
    out = N.guess_finish(qd, corr, u, length, off, 0.7)
    for a, b in zip(off[:-1], off[1:]):
        assert abs(np.dot(length[a:b], out[a:b])) < 1e-12 * length[a:b].sum()
    np.testing.assert_allclose(N.guess_finish(qd, np.zeros(100), u, length, off, 0.7), qd, atol=1e-14)
    np.testing.assert_allclose(N.guess_finish(qd, np.ones(100), u, length, off, 0.7), qd, atol=1e-14)
    d = N.guess_finish(qd, 2 * corr, u, length, off, 0.7) - N.guess_finish(qd, corr, u, length, off, 0.7)
    s0 = np.sqrt(np.mean(u[:40] ** 2))
    c0 = 0.7 * s0 * corr[:40]
    np.testing.assert_allclose(d[:40], c0 - np.dot(length[:40], c0) / length[:40].sum(), atol=1e-13)
