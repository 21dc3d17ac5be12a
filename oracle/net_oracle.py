"""CPU FP64 oracle of the learned-guess network (test infrastructure).

Plain numpy forward and backward of the circular 1D convolution network that
``bem_net_*`` implements, with the same rounding points: every layer input and
every weight rounded to BF16 (round to nearest even) before use, everything
else in FP64.  With ``bf16=False`` no rounding happens (pure FP64), which the
finite-difference check of the gradient uses.  Only the tests call it.

Layer l: y[t, o] = b[o] + sum_c sum_k W[o, c, k] x[(t + (k - K//2) d_l) mod L, c]
for each sequence of length L; ReLU between layers; loss = mean (y - target)^2.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, cin, hidden, layers, ksize):
    out, off = [], 0
    for l in range(layers):
        ci = cin if l == 0 else hidden
        co = 1 if l == layers - 1 else hidden
        W = np.asarray(params[off:off + co * ci * ksize], dtype=np.float64).reshape(co, ci, ksize)
        off += co * ci * ksize
        b = np.asarray(params[off:off + co], dtype=np.float64)
        off += co
        out.append((W, b))
    return out


def _conv(x, W, b, d, offsets):
    co, ci, K = W.shape
    y = np.empty((x.shape[0], co))
    for s in range(len(offsets) - 1):
        s0, s1 = offsets[s], offsets[s + 1]
        L = s1 - s0
        xs = x[s0:s1]
        acc = np.tile(b, (L, 1))
        for k in range(K):
            shift = (k - K // 2) * d
            idx = (np.arange(L) + shift) % L
            acc += xs[idx] @ W[:, :, k].T
        y[s0:s1] = acc
    return y


def forward(params, feats, offsets, cin, hidden, layers, ksize, dil, bf16=True):
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    layers_p = unpack(params, cin, hidden, layers, ksize)
    x = rnd(feats)
    cache = []
    for l, (W, b) in enumerate(layers_p):
        Wr = rnd(W)
        y = _conv(x, Wr, b, dil[l], offsets)
        cache.append((x, Wr, y))
        if l < layers - 1:
            x = rnd(np.maximum(y, 0.0))
    return y[:, 0], cache


def loss_and_grad(params, feats, offsets, target, cin, hidden, layers, ksize, dil, bf16=True):
    y, cache = forward(params, feats, offsets, cin, hidden, layers, ksize, dil, bf16)
    T = y.shape[0]
    e = y - target
    loss = float(np.mean(e * e))
    g = (2.0 * e / T)[:, None]
    grads = []
    for l in range(layers - 1, -1, -1):
        x, Wr, yl = cache[l]
        if l < layers - 1:
            g = g * (yl > 0)
        co, ci, K = Wr.shape
        gW = np.zeros_like(Wr)
        gx = np.zeros_like(x)
        for s in range(len(offsets) - 1):
            s0, s1 = offsets[s], offsets[s + 1]
            L = s1 - s0
            for k in range(K):
                shift = (k - K // 2) * dil[l]
                idx = (np.arange(L) + shift) % L
                gW[:, :, k] += g[s0:s1].T @ x[s0:s1][idx]
                np.add.at(gx, s0 + idx, g[s0:s1] @ Wr[:, :, k])
        gb = g.sum(axis=0)
        grads.append((gW, gb))
        g = gx
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.ravel())
        flat.append(gb.ravel())
    return loss, np.concatenate(flat)


def dtn_estimate(s, length, u, offsets, kmax):
    """Arclength Dirichlet-to-Neumann estimate of each closed curve of a batch
    (the learned guess's feature, ``bem_dtn_estimate``), FP64: with Lambda the
    curve length, uhat_k = (1/Lambda) sum_j l_j u_j exp(-2 pi i k s_j / Lambda)
    for k = 1..kmax and q_j = sum_k (2 pi k / Lambda) 2 Re(uhat_k
    exp(2 pi i k s_j / Lambda)): the interior Dirichlet-to-Neumann multiplier
    |k| / R of a circle of radius R = Lambda / (2 pi), applied mode by mode."""
    s = np.asarray(s, np.float64)
    length = np.asarray(length, np.float64)
    u = np.asarray(u, np.float64)
    out = np.zeros(s.size)
    k = np.arange(1, int(kmax) + 1)
    for q in range(len(offsets) - 1):
        a, b = int(offsets[q]), int(offsets[q + 1])
        lam = length[a:b].sum()
        if not lam > 0:
            continue
        E = np.exp(-2j * np.pi * np.outer(k, s[a:b]) / lam)  # (kmax, elements)
        uhat = E @ (length[a:b] * u[a:b]) / lam
        out[a:b] = ((2 * np.pi * k / lam)[:, None] * 2 * np.real(uhat[:, None] * np.conj(E))).sum(axis=0)
    return out


def fourier_features(points, B):
    """Random Fourier features of 3D points (the 3D point network's input
    encoding, ``bem_fourier_features``), FP64: for each point p and frequency
    row b of B, sin(2 pi b . p) and cos(2 pi b . p), interleaved per frequency
    -> (T, 2F)."""
    ph = 2 * np.pi * np.asarray(points, np.float64) @ np.asarray(B, np.float64).T  # (T, F)
    out = np.empty((ph.shape[0], 2 * ph.shape[1]))
    out[:, 0::2] = np.sin(ph)
    out[:, 1::2] = np.cos(ph)
    return out


def _rms_or_one(u):
    r = float(np.sqrt(np.mean(np.asarray(u, np.float64) ** 2))) if np.size(u) else 0.0
    return r if r > 0 else 1.0


def guess_features(geo, u, qd, offsets, radius):
    """Input columns of the 2D guess network (``bem_guess_features``), FP64:
    per curve, with s the root mean square of u over it (1 when zero), the
    geometry columns followed by u / s and radius * qd / s -> (T, G + 2)."""
    geo = np.asarray(geo, np.float64).reshape(len(u), -1)
    u = np.asarray(u, np.float64)
    qd = np.asarray(qd, np.float64)
    out = np.zeros((u.size, geo.shape[1] + 2))
    for q in range(len(offsets) - 1):
        a, b = int(offsets[q]), int(offsets[q + 1])
        s = _rms_or_one(u[a:b])
        out[a:b, :geo.shape[1]] = geo[a:b]
        out[a:b, -2] = u[a:b] / s
        out[a:b, -1] = radius * qd[a:b] / s
    return out


def guess_finish(qd, corr, u, length, offsets, cscale):
    """The learned guess (``bem_guess_finish``), FP64: per curve x = qd +
    cscale * s * corr (s the rms of u), shifted by the length-weighted mean of
    x so that sum_j length_j x_j = 0 (the zero net flux of a field harmonic
    inside the curve)."""
    qd, corr, u, length = (np.asarray(a, np.float64) for a in (qd, corr, u, length))
    out = np.zeros(qd.size)
    for q in range(len(offsets) - 1):
        a, b = int(offsets[q]), int(offsets[q + 1])
        x = qd[a:b] + cscale * _rms_or_one(u[a:b]) * corr[a:b]
        L = length[a:b].sum()
        out[a:b] = x - (np.dot(length[a:b], x) / L if L > 0 else 0.0)
    return out
