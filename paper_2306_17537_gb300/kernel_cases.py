"""Small, fixed invocations of single parts of the path, for kernel profiling and quick timing.

    python -m paper_2306_17537_gb300.kernel_cases matvec   --n 128 [--shape nx,ny,nz] [--fp64 | --dfloat] [--reps 5]
        repeated sub-domain operator y = (I - G dsigma) x on an n^3 (or nx x ny x nz) grid, complex64
        by default, complex128 or double-float (the outer-residual kernels) on request
    python -m paper_2306_17537_gb300.kernel_cases gmres    --scale 2 [--iters 60]
        one restarted GMRES(30) run on a sub-domain of the 128x128x256 workload divided by `scale`
    python -m paper_2306_17537_gb300.kernel_cases solve    --scale 2
        one complete forward solve (Algorithm 1) of the same workload
    python -m paper_2306_17537_gb300.kernel_cases fno      --n 64 [--reps 10]
        forward passes of the warm-start network (4 layers, width 32, 12 modes, hidden 128, BF16, batch 8)
        with the pointwise maps on the CUDA cores, then on the tensor cores (ie_fno_set_tensor_cores)
    python -m paper_2306_17537_gb300.kernel_cases large    --scale 1 [--position 5]
        one warm-up and one measured solve of the 256x256x512 benchmark model as bench.py solves it
        (flexible GMRES over concurrent block-Jacobi sweeps); prints the measured solve's launch count, so
        a launch list of the whole run can be cut to its last launches
    python -m paper_2306_17537_gb300.kernel_cases batch    --positions 8 [--scale 1] [--lanes 4]
        the batched logging workload: positions x {100 kHz, 2 MHz} tool-aligned windows, block Jacobi,
        solved with ie_solve_batch (lanes contexts per frequency), then one at a time for comparison;
        contraction form; --conc runs each window's two sub-domain solves in flight together

Each prints the elapsed device time and the per-kernel-class accounting of the library.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def _ctx(grid, sigma0, freq, s6):
    from . import ie

    ctx = ie.Context(grid, grid.h, sigma0, freq)
    ctx.set_contrast(s6)
    return ctx


def main(argv=None):
    import torch

    from . import ie, inputs

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["matvec", "gmres", "solve", "batch", "large", "fno"])
    ap.add_argument("--position", type=int, default=5)
    ap.add_argument("--positions", type=int, default=8)
    ap.add_argument("--lanes", type=int, default=4)
    ap.add_argument("--freqs", default="1e5,2e6", help="batch case: comma-separated frequencies")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--shape", default=None, help="matvec case: nx,ny,nz instead of n^3")
    ap.add_argument("--scale", type=int, default=2)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--iters", type=int, default=60)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--dfloat", action="store_true")
    ap.add_argument("--conc", action="store_true", help="batch case: sub-domain solves of a sweep in flight together")
    ap.add_argument("--graph", action="store_true", help="batch case: each block GMRES as one CUDA graph")
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    out = {"case": a.case}
    if a.case == "matvec":
        nx, ny, nz = [int(v) for v in a.shape.split(",")] if a.shape else (a.n, a.n, a.n)
        g = inputs.centred_grid(nx, ny, nz, 0.25)
        s6 = inputs.dipping_ti_with_ellipsoids(g, 0)
        ctx = _ctx(g, 0.1, 4.0e5, s6)
        ctx.set_stream(stream)
        nb = 3 * g.n
        if a.fp64 or a.dfloat:
            x = inputs.random_field((3, g.nz, g.ny, g.nx), 1)
            ctx.profile_enable(True)
            for _ in range(a.reps):
                ctx.matvec(x, precision=ie.IE_PREC_FP64 if a.fp64 else ie.IE_PREC_DFLOAT)
        else:
            x = torch.randn(nb, dtype=torch.complex64, device=dev)
            y = torch.empty_like(x)
            ctx.matvec_dev(x, y)
            torch.cuda.synchronize()
            ctx.profile_enable(True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(a.reps):
                ctx.matvec_dev(x, y)
            e1.record(stream)
            torch.cuda.synchronize()
            out["ms_per_matvec"] = e0.elapsed_time(e1) / a.reps
    elif a.case == "gmres":
        wl = inputs.config2(0, scale=a.scale)
        ctx = _ctx(wl.grid, wl.sigma0, wl.freq, wl.sigma6)
        nz = wl.grid.nz // 2
        b = inputs.random_field((3, nz, wl.grid.ny, wl.grid.nx), 2)
        ctx.profile_enable(True)
        _, its, rr, st = ctx.gmres(b, nz=nz, tol=1e-14, restart=30, max_iter=a.iters,
                                   precision=ie.IE_PREC_FP64 if a.fp64 else ie.IE_PREC_MIXED)
        out.update({"iters": its, "rel_res": rr})
    elif a.case == "batch":
        import time

        scale = a.scale if a.scale > 0 else 1
        freqs = [float(v) for v in a.freqs.split(",")]
        probs = [inputs.config3_item(0, p, f, n_positions=a.positions, scale=scale)
                 for f in freqs for p in range(a.positions)]
        ctxs = {}
        for w in probs:
            lst = ctxs.setdefault(w.freq, [])
            if len(lst) < a.lanes:
                lst.append(ie.Context(w.grid, w.grid.h, w.sigma0, w.freq))
        batch, count = [], {}
        for w in probs:
            k = count.get(w.freq, 0)
            count[w.freq] = k + 1
            batch.append(dict(ctx=ctxs[w.freq][k % a.lanes], sigma6=w.sigma6, sources=w.sources,
                              receivers=w.receivers, dd_mode=ie.IE_DD_JACOBI, tol=w.tol,
                              opts=ie.make_opts(z_split=w.z_split, restart=w.restart, max_inner=4000, max_outer=60,
                                                contraction=True, concurrent_blocks=a.conc, graph=a.graph)))
        ie.solve_batch(batch[:2])  # warm-up: spectra of every sub-domain height, tile tuning
        for mode, conc in (("concurrent", 0), ("one at a time", 1)):
            t0 = time.perf_counter()
            res = ie.solve_batch(batch, max_concurrent=conc)
            dt = time.perf_counter() - t0
            out[mode] = {"solves": len(batch), "seconds": round(dt, 3), "solves_per_s": round(len(batch) / dt, 4),
                         "all_ok": all(r[2] == ie.IE_OK for r in res),
                         "max_rel_residual": max(r[1].final_rel_residual for r in res),
                         "gmres_iters": [r[1].gmres_iters_total for r in res]}
        ctx = next(iter(ctxs.values()))[0]
    elif a.case == "fno":
        from . import fno_warmstart

        n, B = a.n, 8
        with ie.FNO(n, modes=12, width=32, layers=4, cin=12, cout=6, hidden=128, batch_max=B, bf16=True) as net:
            net.set_stream(stream)
            net.set_params(fno_warmstart.init_flat(ie, n, 12, 32, 4, 128, 0))
            x = torch.randn((B, n ** 3, 12), dtype=torch.float32, device=dev)
            u = torch.empty((B, n ** 3, 6), dtype=torch.float32, device=dev)
            res = {}
            for on in (False, True):
                net.set_tensor_cores(on)
                net.forward(B, x, u)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(a.reps):
                    net.forward(B, x, u)
                e1.record(stream)
                torch.cuda.synchronize()
                res["tensor_cores" if on else "cuda_cores"] = {"ms_per_forward": e0.elapsed_time(e1) / a.reps,
                                                               "u_norm": float(u.norm())}
            out.update(res)
        print(json.dumps(out))
        return
    elif a.case == "large":
        wl = inputs.config5(0, a.position, scale=max(a.scale, 1))
        ctx = _ctx(wl.grid, wl.sigma0, wl.freq, wl.sigma6)
        ctx.set_stream(stream)
        opts = ie.make_opts(z_split=wl.z_split, restart=wl.restart, max_inner=4000, max_outer=60, contraction=True,
                            concurrent_blocks=True, outer_krylov=True, outer_restart=20, outer_inner_tol=0.3)
        ctx.solve(wl.sources, wl.receivers, ie.IE_DD_JACOBI, wl.tol, opts)  # warm-up: spectra, workers, tiles
        torch.cuda.synchronize()
        ctx.profile_enable(True)
        H, info, st = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_JACOBI, wl.tol, opts)
        out.update({"status": int(st), "sweeps": info.outer_iters, "gmres_iters": info.gmres_iters_total,
                    "e": info.final_rel_residual, "seconds": info.seconds,
                    "launches_measured": int(sum(v[0] for v in ctx.profile_read().values()))})
    else:
        wl = inputs.config2(0, scale=a.scale)
        ctx = _ctx(wl.grid, wl.sigma0, wl.freq, wl.sigma6)
        ctx.profile_enable(True)
        H, info, st = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_GAUSS_SEIDEL, wl.tol,
                                ie.make_opts(z_split=wl.z_split, max_inner=4000, max_outer=60))
        out.update({"sweeps": info.outer_iters, "gmres_iters": info.gmres_iters_total,
                    "e": info.final_rel_residual, "seconds": info.seconds})
    out["tuned_tiles"] = ie.tuned_tiles().strip().splitlines()
    prof = ctx.profile_read()
    out["kernels"] = {k: {"launches": v[0], "ms": round(v[1], 3), "GB": round(v[2] / 1e9, 4)}
                      for k, v in prof.items() if v[0]}
    print(json.dumps(out))
    ctx.close()


if __name__ == "__main__":
    main()
