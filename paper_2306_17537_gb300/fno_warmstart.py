"""Learned warm start for the sub-domain solves: data from the solver, training with the library's FNO
kernels (include/ie_fno.h), and a cold-versus-warm comparison at equal accuracy.

    python -m paper_2306_17537_gb300.fno_warmstart [--n 64] [--train 1800] [--test 200] [--epochs 30]

1. Data: ``inputs.config4_item(seed)`` blocks (n^3 crops of the 128x128x256 dipping-TI model, 400 kHz),
   each solved to FP64 residual ``--tol`` by ie_solve (one sub-domain, mixed precision, cold start).
   The encoding of include/ie_fno.h turns (contrast, b = incident field, solution E) into the network
   input a (12 channels) and target t (6 channels, the scattered part E - b scaled by sqrt(N)/|b|).
2. Training: Adam on the mean relative L2 loss, mini-batches drawn without replacement per epoch,
   cosine step-size decay; every step is ie_fno_train_step (forward, backward, Adam on the GPU).
3. Evaluation on held-out seeds: each block is solved cold (E := b, the method without the network)
   and warm (E := b + |b|/sqrt(N) FNO(a), the network's inference included in the timed region) to the
   same FP64 residual; GMRES iterations, matvecs and solves/s are reported for both.

Prints one JSON object. The same functions serve the GPU test of the warm start at a small size.
"""
from __future__ import annotations

import argparse
import json
import math
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np


def _make_item(args):
    from . import inputs

    seed, n = args
    return seed, np.ascontiguousarray(inputs.config4_item(seed, n).sigma6)


def item_stream(seeds, n, workers):
    """(seed, sigma6) in seed order; generated by a spawn-started process pool when workers > 1, with at
    most 4 * workers models held ahead of the consumer."""
    seeds = list(seeds)
    if workers <= 1:
        for s in seeds:
            yield _make_item((s, n))
        return
    import multiprocessing as mp
    from collections import deque

    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as pool:
        pending = deque()
        it = iter(seeds)
        for s in it:
            pending.append(pool.submit(_make_item, (s, n)))
            if len(pending) >= 4 * workers:
                break
        while pending:
            yield pending.popleft().result()
            nxt = next(it, None)
            if nxt is not None:
                pending.append(pool.submit(_make_item, (nxt, n)))


class Data:
    """Network inputs and targets resident on the device: a [count][N][12], t [count][N][6] FP32."""

    def __init__(self, torch, count, n):
        dev = torch.device("cuda", torch.cuda.current_device())
        self.a = torch.empty((count, n ** 3, 12), dtype=torch.float32, device=dev)
        self.t = torch.empty((count, n ** 3, 6), dtype=torch.float32, device=dev)
        self.iters = np.zeros(count, dtype=np.int64)
        self.ok = np.zeros(count, dtype=bool)


def solve_opts(ie, restart, max_inner, max_outer, contraction=False):
    return ie.make_opts(restart=restart, max_inner=max_inner, max_outer=max_outer, contraction=contraction)


def generate(torch, ie, net, ctx, wl0, models, data, tol, opts):
    """Solve every model (cold start) within the work cap of ``opts`` and store its encoded input and
    target in ``data``; data.ok marks the blocks that reached ``tol`` (the others are not trained on)."""
    dev = data.a.device
    N = wl0.grid.n
    b = torch.empty((3, N), dtype=torch.complex128, device=dev)
    E = torch.empty_like(b)
    bn = torch.empty(1, dtype=torch.float64, device=dev)
    s6_d = torch.empty((N, 6), dtype=torch.float64, device=dev)
    src = wl0.sources[0]
    ctx.incident_field_dev(src, b)
    t0 = time.perf_counter()
    for k, (seed, s6) in enumerate(models):
        s6_d.copy_(torch.from_numpy(s6.reshape(N, 6)))
        ctx.set_contrast_dev(s6_d)
        _, info, st = ctx.solve([src], [], ie.IE_DD_NONE, tol, opts, allow_noconv=True)
        ctx.get_field_dev(E)
        net.encode(s6_d, wl0.sigma0, b, data.a[k], bn)
        net.encode_target(E, b, bn, data.t[k])
        data.iters[k] = info.gmres_iters_total
        data.ok[k] = st == ie.IE_OK
    torch.cuda.synchronize()
    return time.perf_counter() - t0


def train(torch, net, data, train_idx, batch, epochs, lr, seed=0, log=None):
    """Adam with cosine decay over ``epochs`` passes of the samples train_idx; returns the loss curve."""
    rng = np.random.default_rng(seed)
    train_idx = np.asarray(train_idx)
    steps_per_epoch = max(1, len(train_idx) // batch)
    total = epochs * steps_per_epoch
    a_b = torch.empty((batch,) + tuple(data.a.shape[1:]), dtype=torch.float32, device=data.a.device)
    t_b = torch.empty((batch,) + tuple(data.t.shape[1:]), dtype=torch.float32, device=data.t.device)
    curve = []
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        order = train_idx[rng.permutation(len(train_idx))]
        acc = 0.0
        for s in range(steps_per_epoch):
            idx = torch.from_numpy(order[s * batch:(s + 1) * batch]).to(data.a.device)
            torch.index_select(data.a, 0, idx, out=a_b)
            torch.index_select(data.t, 0, idx, out=t_b)
            step_lr = lr * 0.5 * (1.0 + math.cos(math.pi * step / total))
            acc += net.train_step(batch, a_b, t_b, step_lr)
            step += 1
        curve.append(acc / steps_per_epoch)
        if log:
            log(f"epoch {ep}: train loss {curve[-1]:.4f}")
    torch.cuda.synchronize()
    return curve, time.perf_counter() - t0, step


def test_loss(torch, net, data, idx):
    """Mean relative L2 error of the prediction on the samples idx."""
    u = torch.empty_like(data.t[0:1])
    errs = []
    for k in idx:
        net.forward(1, data.a[k:k + 1], u)
        errs.append(float(torch.linalg.vector_norm(u - data.t[k:k + 1]) / torch.linalg.vector_norm(data.t[k:k + 1])))
    return float(np.mean(errs)) if errs else float("nan")


def compare(torch, ie, net, ctx, wl0, models, tol, opts):
    """Cold and warm solves of the same blocks to the same FP64 residual, each within the work cap of
    ``opts``. Per mode: blocks that reached tol, iterations and time; iteration means are over the
    blocks both modes solved."""
    dev = torch.device("cuda", torch.cuda.current_device())
    N = wl0.grid.n
    b = torch.empty((3, N), dtype=torch.complex128, device=dev)
    x0 = torch.empty_like(b)
    bn = torch.empty(1, dtype=torch.float64, device=dev)
    a = torch.empty((1, N, 12), dtype=torch.float32, device=dev)
    u = torch.empty((1, N, 6), dtype=torch.float32, device=dev)
    s6_d = torch.empty((N, 6), dtype=torch.float64, device=dev)
    src = wl0.sources[0]
    out = {"cold": {"iters": [], "matvecs": [], "e": [], "ok": [], "seconds": 0.0},
           "warm": {"iters": [], "matvecs": [], "e": [], "ok": [], "seconds": 0.0, "used": 0,
                    "initial_e_cold": [], "initial_e_warm": []}}
    for seed, s6 in models:
        s6_d.copy_(torch.from_numpy(s6.reshape(N, 6)))
        ctx.set_contrast_dev(s6_d)
        torch.cuda.synchronize()
        for mode in ("cold", "warm"):
            t0 = time.perf_counter()
            if mode == "warm":
                ctx.incident_field_dev(src, b)
                net.encode(s6_d, wl0.sigma0, b, a[0], bn)
                net.forward(1, a, u)
                net.decode(u[0], b, bn, x0)
                ctx.set_initial_field_dev(x0)
            _, info, st = ctx.solve([src], [], ie.IE_DD_NONE, tol, opts, allow_noconv=True)
            dt = time.perf_counter() - t0
            r = out[mode]
            r["ok"].append(st == ie.IE_OK)
            r["seconds"] += dt
            r["iters"].append(int(info.gmres_iters_total))
            r["matvecs"].append(int(info.matvecs))
            r["e"].append(float(info.final_rel_residual))
            if mode == "warm":
                r["used"] += int(info.warm_start_used)
                r["initial_e_cold"].append(float(info.cold_rel_residual))
                r["initial_e_warm"].append(float(info.warm_rel_residual))
    both = np.array(out["cold"]["ok"], bool) & np.array(out["warm"]["ok"], bool)
    for r in out.values():
        ok = np.array(r["ok"], bool)
        r["solved"] = int(ok.sum())
        r["blocks"] = len(ok)
        # solves/s counts the blocks that reached tol, over the time spent on all blocks
        r["solves_per_s"] = r["solved"] / r["seconds"] if r["seconds"] > 0 else float("nan")
        r["mean_iters"] = float(np.mean(np.array(r["iters"])[both])) if both.any() else float("nan")
        r["max_e_solved"] = float(np.max(np.array(r["e"])[ok])) if ok.any() else float("nan")
        r.pop("ok")
    return out


def init_flat(ie, n, modes, width, layers, hidden, seed):
    """Initial parameters with the layouts of include/ie_fno.h (uniform fan-in scaling, zero biases,
    spectral weights uniform in [0, 1/width^2) per real and imaginary part)."""
    rng = np.random.default_rng(seed)

    def lin(i, o):
        return rng.uniform(-1, 1, (i, o)) / np.sqrt(i)

    shp = (modes, 2 * modes, 2 * modes, width, width)
    R = [(rng.uniform(0, 1, shp) + 1j * rng.uniform(0, 1, shp)) / (width * width) for _ in range(layers)]
    parts = ([lin(12, width), np.zeros(width)] + [lin(width, width) for _ in range(layers)]
             + [np.zeros(width) for _ in range(layers)] + R
             + [lin(width, hidden), np.zeros(hidden), lin(hidden, 6), np.zeros(6)])
    return ie.fno_flat(parts)


def run(n=64, n_train=1800, n_test=200, epochs=30, batch=8, lr=2e-3, modes=12, width=32, layers=4, hidden=128,
        tol=1e-6, restart=40, max_inner=8000, max_outer=6, workers=8, seed0=0, log=None, contraction=False):
    import torch

    from . import ie, inputs

    torch.cuda.set_device(0)
    wl0 = inputs.config4_item(seed0, n)
    res = {"n": n, "train": n_train, "test": n_test, "epochs": epochs, "batch": batch, "lr": lr,
           "net": {"modes": modes, "width": width, "layers": layers, "hidden": hidden, "storage": "bf16"},
           "solver": {"tol": tol, "restart": restart, "max_inner": max_inner, "max_outer": max_outer,
                      "precision": "mixed (complex64 GMRES, FP64-accurate residual)",
                      "operator": "contraction" if contraction else "conventional"}}
    opts_of = lambda: solve_opts(ie, restart, max_inner, max_outer, contraction)  # noqa: E731
    with ie.Context(wl0.grid, wl0.grid.h, wl0.sigma0, wl0.freq) as ctx, \
            ie.FNO(n, modes=modes, width=width, layers=layers, hidden=hidden, batch_max=batch, bf16=True) as net:
        net.set_params(init_flat(ie, n, modes, width, layers, hidden, seed0))
        res["params"] = net.param_count()
        data = Data(torch, n_train + n_test, n)
        models = item_stream(range(seed0, seed0 + n_train + n_test), n, workers)
        res["gen_seconds"] = generate(torch, ie, net, ctx, wl0, models, data, tol, opts_of())
        res["gen_solved"] = int(data.ok.sum())
        res["gen_median_iters"] = float(np.median(data.iters[data.ok])) if data.ok.any() else float("nan")
        train_idx = np.flatnonzero(data.ok[:n_train])
        test_idx = n_train + np.flatnonzero(data.ok[n_train:])
        curve, secs, steps = train(torch, net, data, train_idx, batch, epochs, lr, seed0, log)
        res.update(train_loss=[round(v, 5) for v in curve], train_seconds=secs, train_steps=steps,
                   ms_per_train_step=1e3 * secs / max(steps, 1))
        res["test_rel_l2"] = test_loss(torch, net, data, test_idx)
        res["train_rel_l2"] = test_loss(torch, net, data, train_idx[:len(test_idx)])
        test_models = item_stream(range(seed0 + n_train, seed0 + n_train + n_test), n, workers)
        cmp = compare(torch, ie, net, ctx, wl0, test_models, tol, opts_of())
    for k in ("cold", "warm"):
        cmp[k].pop("e")
    res["compare"] = cmp
    res["iteration_ratio"] = cmp["warm"]["mean_iters"] / cmp["cold"]["mean_iters"]
    res["solved_cold_warm"] = [cmp["cold"]["solved"], cmp["warm"]["solved"]]
    res["speedup"] = cmp["warm"]["solves_per_s"] / cmp["cold"]["solves_per_s"]
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--train", type=int, default=1800)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--modes", type=int, default=12)
    ap.add_argument("--width", type=int, default=32)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--hidden", type=int, default=128)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--max-inner", type=int, default=8000)
    ap.add_argument("--max-outer", type=int, default=6)
    ap.add_argument("--contraction", action="store_true", help="block solves on the contraction form")
    ap.add_argument("--full-lists", action="store_true", help="keep per-solve iteration lists in the output")
    a = ap.parse_args(argv)
    res = run(a.n, a.train, a.test, a.epochs, a.batch, a.lr, a.modes, a.width, a.layers, a.hidden,
              max_inner=a.max_inner, max_outer=a.max_outer, workers=a.workers, log=lambda s: print(s, flush=True),
              contraction=a.contraction)
    if not a.full_lists:
        for k in ("cold", "warm"):
            for key in ("iters", "matvecs", "initial_e_cold", "initial_e_warm"):
                v = res["compare"][k].pop(key, None)
                if v:
                    res["compare"][k][key + "_mean"] = float(np.mean(v))
    print(json.dumps(res))


if __name__ == "__main__":
    main()
