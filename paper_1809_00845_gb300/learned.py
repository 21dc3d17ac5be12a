"""Learned GMRES initial guess for Dirichlet problems on random star curves.

Workload (batched-plus-learned configuration): star curves
r(theta) = 0.3 (1 + sum_{k=2..6} a_k cos(k theta + phi_k)), a_k ~ U(0, 0.05),
phi_k ~ U(0, 2 pi), on grids of uneven sizes n in {512, 1024, 2048}; harmonic
Dirichlet data from 8 multipoles placed outside the curve (centres at radius
0.45-0.7 from (0.5, 0.5); ln r and Re(e^{i alpha} / (z - s)^m), m = 1..3;
amplitudes N(0, 1)).  The unknown is the flux q on every boundary element.

The guess is made for the accuracy-mode operator (flat panels, the paper's
grid convolution with precorrection, ``bem_plan_panels``), whose solution is
the smooth physical flux.  (The paper-form operator's solution on a curved
boundary is not: its discrete flux differs from the physical one by more than
the flux itself, so no function of the local data predicts it; a network
trained on it gave no gain.)

Guess = physics estimate + learned correction:
  * q_dtn, the arclength Dirichlet-to-Neumann estimate of the data
    (``bem_dtn_estimate``: the circle's multiplier 2 pi |k| / Lambda applied to
    the Fourier modes of u along the curve; exact on a circle, off by a smooth
    function on a star);
  * the network (``bem_net_*``, 4 circular conv layers, 64 channels, BF16) maps
    per-panel features in arclength order
        (x - 1/2, y - 1/2, n_x, n_y, L/h, u/s, a q_dtn/s),
    s = rms(u), a = 0.3 (the curves' radius), to the correction a (q - q_dtn)/s
    (an earlier form also took the double layer of the data as an input; the
    operator apply it cost per guess outweighed the iterations it saved);
  * the sum is shifted so that its flux integrates to zero over the curve
    (``bem_guess_finish``), as the flux of a field harmonic inside does.  The
    network's correction alone leaves a net flux of a few per cent, and the
    single layer weighs that constant mode most: measured on 12 held-out
    stars, the shift cuts the guess's initial residual from 0.13 to 0.05 of
    the zero start's (the estimate alone: 0.15).
Training targets are solutions of the method (FP32 GMRES with double-float
residual refinement to 1e-7).  At solve time the guess is passed to
``bem_solve`` as x0; the solver replaces a start whose residual exceeds the
zero start's by zero (zero-start GMRES remains the fallback) and the refined
residual decides when the answer is good enough.

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
RADIUS = 0.3             # length scale of the curves (feature and target scaling)
PANEL_ORDER, PANEL_R = 3, 3


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
    """Grid-cell boundary of random star `seed` (paper-form plans) and the
    generator that then draws its data."""
    rng = np.random.Generator(np.random.PCG64(I.SEED_BASE + 4 + seed))
    curve = I.random_star_curve(rng)
    if n is None:
        n = int(rng.choice(SIZES))
    b = I.curve_boundary(n, curve)
    return b, rng


def panel_geometry(seed: int, n: int | None = None) -> tuple:
    """The same star as flat panels (accuracy mode), and its data generator."""
    rng = np.random.Generator(np.random.PCG64(I.SEED_BASE + 4 + seed))
    curve = I.random_star_curve(rng)
    if n is None:
        n = int(rng.choice(SIZES))
    return I.curve_panels(n, curve), rng


def arclength(b):
    """Arclength position of each panel midpoint from the first vertex."""
    L = b.length
    return np.cumsum(L) - 0.5 * L


def dtn_modes(nb):
    """Fourier modes of the estimate: a quarter of the panels, at most 256 (the
    data's modes decay like e^{-k d / R} with d >= 0.075 the multipoles'
    distance from the curve and R = 0.3: below FP32 rounding long before)."""
    return max(1, min(nb // 4, 256))


def dtn(b, u):
    """Arclength Dirichlet-to-Neumann estimate of the data (library kernel)."""
    from .bem import dtn_estimate
    return dtn_estimate(arclength(b), b.length, u, [0, b.nb], dtn_modes(b.nb)).cpu().numpy().astype(np.float64)


def features(b, u, qd):
    s = float(np.sqrt(np.mean(u * u))) or 1.0
    m, nrm = b.mid, b.normal
    f = np.stack([m[:, 0] - 0.5, m[:, 1] - 0.5, nrm[:, 0], nrm[:, 1], b.length / b.h, u / s,
                  RADIUS * qd / s], axis=-1).astype(np.float32)
    return f, s


def _plan(b):
    from .bem import Plan
    p = Plan.from_panel_boundary(b, "f32", PANEL_ORDER, PANEL_R)
    p.enable_refinement(True)
    return p


def generate(seeds, rhs_per_geometry=8, n=None, tol=1e-7, log=None):
    """Solve Dirichlet problems with the FFT method (accuracy mode); returns a
    list of (features, target correction) per solve."""
    data = []
    t0 = time.time()
    for k, seed in enumerate(seeds):
        b, rng = panel_geometry(seed, n)
        plan = _plan(b)
        bc = np.zeros(b.nb, np.uint8)
        for _ in range(rhs_per_geometry):
            u = multipoles(rng)(b.mid)
            qd = dtn(b, u)
            _, q, info = plan.solve(bc, u, tol=tol, restart=100, max_iter=2000)
            if info["status"] != 0:
                continue
            f, s = features(b, u, qd)
            data.append((f, (RADIUS * (q - qd) / s).astype(np.float32)))
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


def predict(net, b, u, qd, tscale=1.0):
    """The guess q_dtn + the network's correction (host arrays)."""
    f, s = features(b, u, qd)
    off = np.array([0, f.shape[0]], np.int32)
    corr = net.forward(f, off).cpu().numpy().astype(np.float64) * tscale
    x = qd + corr * s / RADIUS
    return x - np.sum(b.length * x) / np.sum(b.length)


class Guesser:
    """The guess of one geometry, kept on the device: the geometry's feature
    columns and arclength data are uploaded once; per right-hand side the
    Dirichlet-to-Neumann estimate and the network run in the library's
    kernels and torch only stacks and scales columns.  Returns the
    host x0 for bem_solve (which replaces a start worse than zero by zero, so
    the guess never costs iterations)."""

    def __init__(self, net, plan, b, tscale=1.0):
        import torch
        self.net, self.plan, self.b, self.tscale = net, plan, b, tscale
        dev = torch.device("cuda")
        m, nrm = b.mid, b.normal
        geo = np.stack([m[:, 0] - 0.5, m[:, 1] - 0.5, nrm[:, 0], nrm[:, 1], b.length / b.h], axis=-1)
        self.geo = torch.from_numpy(geo.astype(np.float32)).to(dev)
        self.s = torch.from_numpy(arclength(b).astype(np.float32)).to(dev)
        self.len = torch.from_numpy(b.length.astype(np.float32)).to(dev)
        self.off = torch.tensor([0, b.nb], dtype=torch.int32, device=dev)
        self.off_host = np.array([0, b.nb], np.int32)
        self.kmax = dtn_modes(b.nb)

    def __call__(self, u, use_net=True):
        import torch
        from . import bem as B
        ut = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda()
        qd = B.dtn_estimate(self.s, self.len, ut, self.off_host, self.kmax)
        if use_net:
            f = B.guess_features(self.geo, ut, qd, self.off_host, RADIUS)
            corr = self.net.forward(f, self.off_host)
            # the network's correction carries a net flux, which the single
            # layer amplifies most; the guess drops it (zero for a field
            # harmonic inside)
            x0 = B.guess_finish(qd, corr, ut, self.len, self.off_host, self.tscale / RADIUS)
        else:
            x0 = qd
        return x0.double().cpu().numpy()


def evaluate(net, seeds, tol=1e-6, log=None, tscale=1.0):
    """Time to relative residual `tol` (FP32 GMRES + double-float residual
    refinement, block-Jacobi preconditioner) from zero, from the
    Dirichlet-to-Neumann estimate alone and from the network's guess; the
    guesses' own cost (estimate, features, network) is included."""
    import torch
    rows = []
    for seed in seeds:
        b, rng = panel_geometry(seed)
        plan = _plan(b)
        u = multipoles(rng)(b.mid)
        bc = np.zeros(b.nb, np.uint8)
        _, q_ref, _ = plan.solve(bc, u, tol=tol, restart=100, max_iter=2000)  # warm: preconditioner, companion
        torch.cuda.synchronize()
        _, _, z = plan.solve(bc, u, tol=tol, restart=100, max_iter=2000)
        guess = Guesser(net, plan, b, tscale)  # geometry arrays: once per plan
        guess(u)  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xd = guess(u, use_net=False)
        t_dtn = time.perf_counter() - t0
        _, _, d = plan.solve(bc, u, tol=tol, restart=100, max_iter=2000, x0=xd)
        t0 = time.perf_counter()
        x0 = guess(u)
        t_guess = time.perf_counter() - t0
        _, _, g = plan.solve(bc, u, tol=tol, restart=100, max_iter=2000, x0=x0)
        nq = float(np.linalg.norm(q_ref))
        rows.append({"seed": seed, "n": b.n, "nb": b.nb, "zero_iters": z["iters"], "zero_s": z["seconds"],
                     "zero_status": z["status"], "dtn_iters": d["iters"], "dtn_s": d["seconds"] + t_dtn,
                     "dtn_status": d["status"], "guess_iters": g["iters"], "guess_s": g["seconds"] + t_guess,
                     "guess_status": g["status"], "guess_overhead_s": t_guess,
                     "dtn_rel_err": float(np.linalg.norm(xd - q_ref) / nq),
                     "guess_rel_err": float(np.linalg.norm(x0 - q_ref) / nq)})
        plan.close()
        if log:
            log(json.dumps(rows[-1]))
    col = lambda k: np.array([r[k] for r in rows])
    return {"geometries": len(rows), "tol": tol, "operator": "accuracy mode (flat panels, order "
            f"{PANEL_ORDER}, R {PANEL_R}), FP32 + double-float refinement",
            "mean_iters_zero": float(col("zero_iters").mean()), "mean_iters_dtn": float(col("dtn_iters").mean()),
            "mean_iters_guess": float(col("guess_iters").mean()), "mean_s_zero": float(col("zero_s").mean()),
            "mean_s_dtn": float(col("dtn_s").mean()), "mean_s_guess": float(col("guess_s").mean()),
            "speedup_time": float(col("zero_s").sum() / col("guess_s").sum()),
            "mean_rel_err_dtn": float(col("dtn_rel_err").mean()),
            "mean_rel_err_guess": float(col("guess_rel_err").mean()),
            "all_converged": bool(all(r["zero_status"] == 0 and r["guess_status"] == 0 and r["dtn_status"] == 0
                                      for r in rows)), "rows": rows}


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
    ap.add_argument("--geoms", type=int, default=1250)
    ap.add_argument("--rhs", type=int, default=8)
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
