"""Learned GMRES initial guess for Dirichlet problems on random star curves.

Workload (batched-plus-learned configuration): star curves
r(theta) = 0.3 (1 + sum_{k=2..6} a_k cos(k theta + phi_k)), a_k ~ U(0, 0.05),
phi_k ~ U(0, 2 pi), on grids of uneven sizes n in {512, 1024, 2048}; harmonic
Dirichlet data from 8 multipoles placed outside the curve (centres at radius
0.45-0.7 from (0.5, 0.5); ln r and Re(e^{i alpha} / (z - s)^m), m = 1..3;
amplitudes N(0, 1)).  The unknown is the flux q on every boundary cell.

The network (``bem_net_*``, 4 circular conv layers, 64 channels, BF16) maps
per-cell features in arclength order
    (x - 1/2, y - 1/2, n_x, n_y, w/h, u/s, (D u)/s),  s = rms(u),
where D u is the double layer of the data applied with the FFT operator
itself, to the carried flux w q / (h s).  The operator only ever sees w_j q_j
(Section 4: the source weight), so q itself is ill-determined on cells that
hold a sliver of the curve while w q is not; the guess is x0 = pred h s / w.  Training targets are solutions of the FFT method (FP32 GMRES
with FP64 residual refinement to 1e-8).  At solve time the prediction is
passed to ``bem_solve`` as x0; zero-start GMRES remains the fallback and the
FP64 residual decides when the answer is good enough.

Everything that computes runs in the library's CUDA kernels; this module
prepares arrays and drives the loops.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "guess_net.npz")
NET_SHAPE = dict(cin=7, hidden=64, layers=4, ksize=5, dilations=(1, 3, 9, 27))
TRAIN_SEED0, TEST_SEED0 = 0, 10000
SIZES = (512, 1024, 2048)


def multipoles(rng: np.random.Generator, count: int = 8):
    """Harmonic field from `count` multipoles outside the disc of radius 0.45
    about (0.5, 0.5): returns u(p) for points p (..., 2)."""
    rad = rng.uniform(0.45, 0.7, size=count)
    ang = rng.uniform(0.0, 2 * math.pi, size=count)
    cen = 0.5 + 0.5j + rad * np.exp(1j * ang)
    kind = rng.integers(0, 4, size=count)  # 0: ln r, m = kind otherwise
    alpha = rng.uniform(0.0, 2 * math.pi, size=count)
    amp = rng.standard_normal(count)

    def u(p):
        z = p[..., 0] + 1j * p[..., 1]
        out = np.zeros(z.shape)
        for s, k, a, c in zip(cen, kind, alpha, amp):
            if k == 0:
                out += c * np.log(np.abs(z - s))
            else:
                out += c * np.real(np.exp(1j * a) / (z - s) ** int(k))
        return out

    return u


def geometry(seed: int, n: int | None = None) -> tuple:
    rng = np.random.Generator(np.random.PCG64(I.SEED_BASE + 4 + seed))
    curve = I.random_star_curve(rng)
    if n is None:
        n = int(rng.choice(SIZES))
    b = I.curve_boundary(n, curve)
    return b, rng


def features(b, u, du):
    s = float(np.sqrt(np.mean(u * u))) or 1.0
    f = np.stack([b.point[:, 0] - 0.5, b.point[:, 1] - 0.5, b.normal[:, 0], b.normal[:, 1], b.w / b.h, u / s,
                  du / s], axis=-1).astype(np.float32)
    return f, s


def _plan(b):
    from .bem import Plan
    p = Plan.from_boundary(b, "laplace2d", "f32")
    p.enable_refinement(True)
    return p


def double_layer(plan, u):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda()
    return plan.apply("double", x).cpu().numpy().astype(np.float64)


def generate(seeds, rhs_per_geometry=4, n=None, tol=1e-8, log=None):
    """Solve Dirichlet problems with the FFT method; returns a list of
    (features, target q/s) per solve."""
    data = []
    t0 = time.time()
    for k, seed in enumerate(seeds):
        b, rng = geometry(seed, n)
        plan = _plan(b)
        bc = np.zeros(b.nb, np.uint8)
        for _ in range(rhs_per_geometry):
            u = multipoles(rng)(b.point)
            du = double_layer(plan, u)
            _, q, info = plan.solve(bc, u, tol=tol, restart=100, max_iter=2000)
            if info["status"] != 0:
                continue
            f, s = features(b, u, du)
            data.append((f, (q * b.w / (b.h * s)).astype(np.float32)))
        plan.close()
        if log and (k + 1) % 100 == 0:
            log(f"generated {k + 1}/{len(seeds)} geometries, {len(data)} solves, {time.time() - t0:.0f} s")
    return data


def batches(data, batch, rng):
    idx = rng.permutation(len(data))
    for i in range(0, len(idx), batch):
        sel = idx[i:i + batch]
        feats = np.concatenate([data[j][0] for j in sel])
        tgt = np.concatenate([data[j][1] for j in sel])
        off = np.zeros(len(sel) + 1, np.int32)
        off[1:] = np.cumsum([data[j][0].shape[0] for j in sel])
        yield feats, off, tgt


def train(net, data, epochs=20, batch=16, lr=1e-3, seed=0, log=None):
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        lr_ep = lr * (0.5 * (1 + math.cos(math.pi * ep / max(epochs, 1))))
        losses = [net.train_step(f, o, t, lr=lr_ep) for f, o, t in batches(data, batch, rng)]
        hist.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    return hist


def target_scale(data):
    """Global scale of the training targets (their RMS), so that the network
    predicts O(1) values; stored with the weights."""
    return float(np.sqrt(np.mean(np.concatenate([t for _, t in data]) ** 2))) or 1.0


def predict(net, b, u, du, tscale=1.0):
    f, s = features(b, u, du)
    off = np.array([0, f.shape[0]], np.int32)
    return net.forward(f, off).cpu().numpy().astype(np.float64) * tscale * (s * b.h) / b.w


def safeguard(plan, bc, u, x0):
    """Scale the guess by the alpha minimising ||b - alpha A x0|| (one FP32
    apply of the BC-split operator and one of the right-hand side), so the
    starting residual never exceeds the zero start's; alpha = 0 falls back to
    zero-start GMRES."""
    import torch
    plan.set_bc(bc, 0.5)
    xt = torch.from_numpy(np.ascontiguousarray(x0, dtype=np.float32)).cuda()
    ax = plan.apply("system", xt).cpu().numpy().astype(np.float64)
    ut = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda()
    rhs = 0.5 * u - plan.apply("double", ut).cpu().numpy().astype(np.float64)
    den = float(ax @ ax)
    alpha = max(0.0, float(ax @ rhs) / den) if den > 0 else 0.0
    return alpha * x0, alpha


def evaluate(net, seeds, tol=1e-6, log=None, tscale=1.0):
    """Time to relative residual `tol` (FP32 GMRES + FP64 residual refinement,
    block-Jacobi preconditioner) from zero and from the network's guess."""
    import torch
    rows = []
    for seed in seeds:
        b, rng = geometry(seed)
        plan = _plan(b)
        u = multipoles(rng)(b.point)
        bc = np.zeros(b.nb, np.uint8)
        plan.solve(bc, u, tol=tol, restart=100, max_iter=2000)  # warm: preconditioner, companion
        torch.cuda.synchronize()
        _, _, z = plan.solve(bc, u, tol=tol, restart=100, max_iter=2000)
        t0 = time.perf_counter()
        du = double_layer(plan, u)
        x0, alpha = safeguard(plan, bc, u, predict(net, b, u, du, tscale))
        t_guess = time.perf_counter() - t0
        _, _, g = plan.solve(bc, u, tol=tol, restart=100, max_iter=2000, x0=x0)
        rows.append({"seed": seed, "n": b.n, "nb": b.nb, "zero_iters": z["iters"], "zero_s": z["seconds"],
                     "zero_status": z["status"], "guess_iters": g["iters"], "guess_s": g["seconds"] + t_guess,
                     "guess_status": g["status"], "guess_overhead_s": t_guess, "alpha": alpha})
        plan.close()
        if log:
            log(json.dumps(rows[-1]))
    zi = np.array([r["zero_iters"] for r in rows])
    gi = np.array([r["guess_iters"] for r in rows])
    zs = np.array([r["zero_s"] for r in rows])
    gs = np.array([r["guess_s"] for r in rows])
    return {"geometries": len(rows), "tol": tol, "mean_iters_zero": float(zi.mean()),
            "mean_iters_guess": float(gi.mean()), "mean_s_zero": float(zs.mean()), "mean_s_guess": float(gs.mean()),
            "speedup_time": float(zs.sum() / gs.sum()), "all_converged":
                bool(all(r["zero_status"] == 0 and r["guess_status"] == 0 for r in rows)), "rows": rows}


def save(net, path=WEIGHTS, meta=None):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, params=net.get_params(), meta=json.dumps({**NET_SHAPE, **(meta or {})}))


def load(path=WEIGHTS):
    from .bem import Net
    z = np.load(path, allow_pickle=False)
    meta = json.loads(str(z["meta"]))
    net = Net(meta["cin"], meta["hidden"], meta["layers"], meta["ksize"], meta["dilations"])
    net.set_params(z["params"])
    return net, meta


def main():
    ap = argparse.ArgumentParser(description="train / evaluate the learned initial guess")
    ap.add_argument("--geoms", type=int, default=2500)
    ap.add_argument("--rhs", type=int, default=4)
    ap.add_argument("--train-n", type=int, default=0, help="grid size of the training curves (0: mixed sizes)")
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--out", default=None, help="write the evaluation JSON here")
    args = ap.parse_args()
    import torch
    from .bem import Net
    torch.cuda.set_device(0)
    log = lambda m: print(m, flush=True)
    t0 = time.time()
    data = generate(range(TRAIN_SEED0, TRAIN_SEED0 + args.geoms), args.rhs, n=args.train_n or None, log=log)
    t_gen = time.time() - t0
    net = Net(**NET_SHAPE, seed=1)
    tscale = target_scale(data)
    data = [(f, t / tscale) for f, t in data]
    t0 = time.time()
    hist = train(net, data, epochs=args.epochs, log=log)
    t_train = time.time() - t0
    save(net, meta={"train_solves": len(data), "epochs": args.epochs, "final_loss": hist[-1], "tscale": tscale})
    ev = evaluate(net, range(TEST_SEED0, TEST_SEED0 + args.test), log=log, tscale=tscale)
    ev.update({"train_solves": len(data), "gen_s": t_gen, "train_s": t_train, "loss_history": hist})
    if args.out:
        with open(args.out, "w") as f:
            json.dump(ev, f, indent=1)
    with open(os.path.join(HERE, "weights", "guess_net_eval.json"), "w") as f:
        json.dump({k: v for k, v in ev.items() if k != "rows"}, f, indent=1)
    log(json.dumps({k: v for k, v in ev.items() if k != "rows"}))


if __name__ == "__main__":
    main()
