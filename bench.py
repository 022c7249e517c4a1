#!/usr/bin/env python3
"""Benchmark of the IE forward model: tool-position solves per second at e <= 1e-6 (eq. 9, FP64-verified).

Default workload (`--workload c5`, the largest single-GPU configuration): 256 x 256 x 512 cells of
0.25 m (33.5 M cells, 100.7 M complex unknowns) split into 8 sub-domains of 256 x 256 x 64 along the
tool axis; 7 dipping TI layers offset by a fault plus 5 isotropic ellipsoids (seeded); coaxial z
magnetic dipole with receivers 0.5/1/2 m above it at 16 positions 2 m apart along the axis; 2 MHz;
sigma0 = 0.1 S/m. Solver: block Jacobi over the 8 sub-domains with all block solves in flight together
(concurrent worker streams; block tolerance 0.3), used as the preconditioner of a flexible GMRES(20)
outer iteration on the whole-grid system (the Krylov acceleration the paper proposes for its fixed-point sweeps), block GMRES
on the contraction form of the operator, complex64 FFT convolution and Krylov vectors, FP64-accurate
(double-float) whole-grid residuals. One step = one tool position's solve (incident field, DD solve,
receivers); the model is uploaded (ie_set_contrast_dev / ie_set_contrast) at the first step of every
cycle of 16 positions, inside the timed region. Green spectra (ie_create) depend only on grid, cell
size, background and frequency and are computed once before timing, as the paper precomputes them
(Section 2.2). Inputs (fields 1.6 GB, Krylov bases tens of GB) are far larger than the 129 MB L2.

`--workload c2`: the 128 x 128 x 256 two-sub-domain block Gauss-Seidel configuration (Algorithm 1 with
the adaptive tolerance, contraction form), one tool position, 400 kHz; it is also timed as a variant of
the default line.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}] [--workload c5|c2]
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "IE forward solves/sec at 1e-6 rel. residual; matvec HBM GB/s vs peak"
UNIT = "solves/s"
POSITIONS_C5 = 16


class BenchWorkload:
    """One benchmark configuration: the seeded model, the tool positions a step cycles through, the DD
    mode and solver options (as plain values; the GB300 arm turns them into ie_opts), the sub-domain
    whose operator bandwidth is reported, and a one-line description."""

    def __init__(self, key: str, seed: int, scale: int = 1, operator: str = "contraction", restart=None):
        from paper_2306_17537_gb300 import inputs

        self.key = key
        contraction = operator == "contraction"
        if key == "c5":
            self.items = [inputs.config5(seed, p, n_positions=POSITIONS_C5, scale=scale) for p in range(POSITIONS_C5)]
            wl = self.items[0]
            self.dd = "jacobi"
            self.opts = dict(z_split=wl.z_split, restart=restart or wl.restart, max_inner=4000, max_outer=60,
                             contraction=contraction, concurrent_blocks=True, outer_krylov=True, outer_restart=20,
                             outer_inner_tol=0.3)
            g = wl.grid
            self.description = (f"DD {g.nx}x{g.ny}x{g.nz} @0.25 m, 8 sub-domains block Jacobi (all block solves in "
                                f"flight together) preconditioning flexible GMRES(20), 7 faulted TI layers + 5 "
                                f"ellipsoids, {POSITIONS_C5} tool positions, 2 MHz, tol 1e-6")
            self.dd_text = "flexible GMRES(20) outer iteration, preconditioner: one concurrent block-Jacobi sweep (block tol 0.3)"
        elif key == "c2":
            self.items = [inputs.config2(seed, scale=scale)]
            wl = self.items[0]
            self.dd = "gs"
            self.opts = dict(z_split=wl.z_split, restart=restart or wl.restart, max_inner=4000, max_outer=60,
                             contraction=contraction)
            g = wl.grid
            self.description = (f"DD {g.nx}x{g.ny}x{g.nz} @0.25 m, 2 sub-domains block Gauss-Seidel adaptive (GS-A), "
                                f"5 dipping TI layers + 2 ellipsoids, 1 coaxial tool position, 400 kHz, tol 1e-6")
            self.dd_text = "block Gauss-Seidel fixed-point sweeps (Algorithm 1), adaptive block tol e/10"
        else:
            raise ValueError(key)
        self.grid = wl.grid
        self.sigma6 = wl.sigma6
        self.sigma0, self.freq, self.tol = wl.sigma0, wl.freq, wl.tol
        self.split = wl.z_split
        self.block = (self.split[0], self.split[1])  # the sub-domain whose operator is timed alone

    def item(self, step: int):
        return self.items[step % len(self.items)]

    def uploads_model(self, step: int) -> bool:
        """The model is (re)uploaded at the first position of every cycle of positions."""
        return step % len(self.items) == 0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16, help="timed steps (default: one cycle of the 16 tool positions)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--scale", type=int, default=1, help="divide the grid by this factor (testing only)")
    ap.add_argument("--restart", type=int, default=None, help="GMRES restart length (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--operator", default="contraction", choices=["contraction", "conventional"],
                    help="operator form GMRES iterates on inside the sub-domain solves")
    ap.add_argument("--workload", default="c5", choices=["c5", "c2"])
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------------------------ ranks
def rank_seed(seed: int, rank: int) -> int:
    """Weak scaling: every rank solves its own tool position (an independent seeded model)."""
    return seed + rank


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (timings: the job is as slow as its slowest rank)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps: int, world: int, t_ms_max: float) -> float:
    """Whole-job solves per second: all ranks' steps over the slowest rank's time."""
    return steps * world / (t_ms_max / 1000.0)


# ------------------------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power) if power else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_record(kernel_class: str):
    """Per-launch DRAM traffic of a kernel from the committed ncu summary, or None when the kernel
    source changed since the capture (the summary stores a hash of the sources it covers)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    import hashlib

    rec = json.load(open(p)).get(kernel_class)
    if not rec:
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if h.hexdigest() != rec["sha256"]:
        return None
    return rec


# ------------------------------------------------------------------------------------ CPU oracle
def oracle_block_sample(bw, nz, n_apply=1, contraction=True):
    """Time the CPU oracle's operator of one z slab of `nz` planes at the bottom of the model (the
    contraction or the conventional form): spectra setup + n_apply applications (seconds each)."""
    import numpy as np

    from oracle import contraction as oc
    from oracle import operator as oop

    g = bw.grid
    s6 = bw.sigma6[:nz]
    t0 = time.perf_counter()
    if contraction:
        op = oc.ContractionOperator(s6, g.h, bw.freq, bw.sigma0)
    else:
        op = oop.FFTOperator(oop.contrast(s6, bw.sigma0), g.h, bw.freq, bw.sigma0)
    t1 = time.perf_counter()
    x = np.ones((3, nz, g.ny, g.nx), dtype=np.complex128)
    for _ in range(n_apply):
        x = op(x)
    t2 = time.perf_counter()
    return t1 - t0, (t2 - t1) / n_apply


def padded_volume(g, nz):
    """Padded FFT volume of a slab of nz planes (the pass model's cost scale of one application)."""
    def p2(n):
        v = 1
        while v < 2 * n:
            v *= 2
        return v
    return p2(g.nx) * p2(g.ny) * p2(nz)


def cpu_cores():
    return os.cpu_count() or 1


def c1_full_solves(ie, torch, dev, stream, reps=3):
    """The 16^3 whole-domain configuration (complex128 GMRES(30) to 1e-8, seed 0) solved in full by the
    GPU (mean of `reps` solves, CUDA events) and by the CPU oracle (one timed solve): a directly timed
    solve on both sides, next to the scaled sample of the headline workload."""
    import numpy as np

    from oracle import solve as osolve
    from paper_2306_17537_gb300 import inputs

    wl = inputs.config1(0)
    g = wl.grid
    with ie.Context(g, g.h, wl.sigma0, wl.freq) as c1:
        c1.set_stream(stream)
        c1.set_contrast(wl.sigma6)
        opts = ie.make_opts(restart=30, max_inner=20000, max_outer=20, precision=ie.IE_PREC_FP64)
        c1.solve(wl.sources, wl.receivers, ie.IE_DD_NONE, wl.tol, opts)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            Hg, ginfo, gst = c1.solve(wl.sources, wl.receivers, ie.IE_DD_NONE, wl.tol, opts)
        b.record(stream)
        torch.cuda.synchronize(dev)
        gpu_s = a.elapsed_time(b) / 1e3 / reps
    t0 = time.perf_counter()
    Ho, oinfo = osolve.forward(g, wl.sigma6, wl.sigma0, wl.freq, wl.sources, wl.receivers, method="gmres",
                               tol=wl.tol, restart=wl.restart, max_inner=20000)
    oracle_s = time.perf_counter() - t0
    return {"workload": "16^3 @0.5 m whole domain, 3 VTI layers, 100 kHz, complex128 GMRES(30) to 1e-8, seed 0",
            "oracle_s": round(oracle_s, 3), "oracle_gmres_iters": int(oinfo.gmres_iters),
            "oracle_rel_residual": float(oinfo.rel_residual),
            "gpu_s": round(gpu_s, 5), "gpu_status": int(gst), "gpu_gmres_iters": int(ginfo.gmres_iters_total),
            "gpu_rel_residual": float(ginfo.final_rel_residual),
            "max_rel_diff_H": float(np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho))),
            "oracle_over_gpu": round(oracle_s / gpu_s, 1)}


# ------------------------------------------------------------------------------------ GB300 arm
def timed(stream, torch, dev, fn, steps, world, dist):
    """Run fn(k) for k = 0..steps-1 between CUDA events on `stream` (barrier + synchronize on both
    sides); returns (ms, results)."""
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = [fn(k) for k in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    return e0.elapsed_time(e1), res


def run_gb300(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2306_17537_gb300 import ie

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    # weak scaling: every rank solves its own seeded model (independent problems), no data exchange
    bw = BenchWorkload(args.workload, rank_seed(args.seed, rank), args.scale, args.operator, args.restart)
    g = bw.grid
    dd_mode = {"jacobi": ie.IE_DD_JACOBI, "gs": ie.IE_DD_GAUSS_SEIDEL}[bw.dd]
    stream = torch.cuda.current_stream(dev)
    t_setup0 = time.perf_counter()
    ctx = ie.Context(g, g.h, bw.sigma0, bw.freq)
    ctx.set_stream(stream)
    setup_s = time.perf_counter() - t_setup0
    s6_dev = torch.from_numpy(np.ascontiguousarray(bw.sigma6)).to(dev)
    opts = ie.make_opts(precision=ie.IE_PREC_MIXED, **bw.opts)

    def step_dev(k):
        if bw.uploads_model(k):
            ctx.set_contrast_dev(s6_dev)
        it = bw.item(k)
        return ctx.solve(it.sources, it.receivers, dd_mode, bw.tol, opts)

    for k in range(args.warmup):
        step_dev(k)
    # ----------------------------------------------------------------- timed region (device inputs)
    # no launch accounting inside: the per-kernel breakdown comes from a separate profiled pass below
    ctx.profile_enable(False)
    clocks = ClockSampler(local)
    clocks.start()
    t_ms, results = timed(stream, torch, dev, step_dev, args.steps, world, dist)
    clk = clocks.stop()
    t_ms_max = max_over_ranks(t_ms, dev)
    infos = [r[1] for r in results]
    failed = [k for k, (_, inf, stk) in enumerate(results) if stk != ie.IE_OK or not (inf.final_rel_residual <= bw.tol)]
    value = job_throughput(args.steps, world, t_ms_max) if not failed else None
    H, _, st = results[-1]
    # ----------------------------------------------------------------- end to end (host buffers)
    # the same steps with every input from pinned host memory (the model at the first position of a
    # cycle, sources and receivers every step) and the receiver fields back on the host every step
    s6_host = torch.from_numpy(np.ascontiguousarray(bw.sigma6)).pin_memory().numpy()
    h2d_total, d2h_total = 0, 0

    def step_host(k):
        nonlocal h2d_total, d2h_total
        if bw.uploads_model(k):
            ctx.set_contrast(s6_host)
            h2d_total += s6_host.nbytes
        it = bw.item(k)
        r = ctx.solve(it.sources, it.receivers, dd_mode, bw.tol, opts)
        h2d_total += it.receivers.nbytes + 48 * len(it.sources)
        d2h_total += r[0].nbytes
        return r

    e_ms, e_res = timed(stream, torch, dev, step_host, args.steps, world, dist)
    e2e_ok = all(stk == ie.IE_OK and inf.final_rel_residual <= bw.tol for _, inf, stk in e_res)
    e2e_value = job_throughput(args.steps, world, max_over_ranks(e_ms, dev)) if e2e_ok else None
    # ----------------------------------------------------------------- profiled pass (per-kernel times)
    # per-launch CUDA events around every kernel of the same solves, with the sub-domain solves of a
    # sweep one after another (the same arithmetic, bit-identical results) so that no two timed launches
    # overlap; these steps are not part of `value`
    prof_steps = max(1, min(args.steps, 3))
    popts = ie.make_opts(precision=ie.IE_PREC_MIXED, **dict(bw.opts, concurrent_blocks=False))

    def step_prof(k):
        if bw.uploads_model(k):
            ctx.set_contrast_dev(s6_dev)
        it = bw.item(k)
        return ctx.solve(it.sources, it.receivers, dd_mode, bw.tol, popts)

    step_prof(0)
    torch.cuda.synchronize(dev)
    ctx.profile_enable(True)
    p_ms, _ = timed(stream, torch, dev, step_prof, prof_steps, 1, dist)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    # ----------------------------------------------------------------- variants (a step or a few each)
    variants = {}

    def variant(name, vopts, steps, note, ctx_=None, items=None, dd=None, reupload=True):
        c_ = ctx_ or ctx
        its_ = items or bw.items
        dd_ = dd if dd is not None else dd_mode
        vo = ie.make_opts(precision=ie.IE_PREC_MIXED, **vopts)

        def vstep(k):
            if reupload and k == 0:
                c_.set_contrast_dev(s6_dev) if c_ is ctx else None
            it = its_[k % len(its_)]
            return c_.solve(it.sources, it.receivers, dd_, it.tol, vo)

        vstep(0)
        v_ms, vres = timed(stream, torch, dev, vstep, steps, world, dist)
        Hv, vinfo, vst = vres[-1]
        ref = results[(steps - 1) % len(results)][0] if c_ is ctx else None
        variants[name] = {"note": note, "value": round(job_throughput(steps, world, max_over_ranks(v_ms, dev)), 4),
                          "unit": UNIT, "steps": steps, "ms_per_step": round(v_ms / steps, 2), "status": int(vst),
                          "outer_iters": vinfo.outer_iters, "gmres_iters": vinfo.gmres_iters_total,
                          "final_rel_residual": vinfo.final_rel_residual}
        if ref is not None and ref.shape == Hv.shape:
            variants[name]["max_rel_diff_H_vs_headline"] = float(np.max(np.abs(Hv - ref)) / np.max(np.abs(ref)))

    v_steps = max(1, min(args.steps, 2))
    if bw.key == "c5":
        variant("sequential_blocks", dict(bw.opts, concurrent_blocks=False), v_steps,
                "the same solve with the block solves of each sweep one after another")
        variant("device_graph_blocks", dict(bw.opts, graph=True), v_steps,
                "the same solve with every block's GMRES as one CUDA graph, all launched before the first wait")
        c2 = BenchWorkload("c2", rank_seed(args.seed, rank), args.scale, args.operator)
        with ie.Context(c2.grid, c2.grid.h, c2.sigma0, c2.freq) as cctx:
            cctx.set_stream(stream)
            cctx.set_contrast(c2.sigma6)
            variant("c2_gauss_seidel", c2.opts, max(1, min(args.steps, 3)), c2.description, ctx_=cctx,
                    items=c2.items, dd=ie.IE_DD_GAUSS_SEIDEL, reupload=False)
    else:
        other = "conventional" if args.operator == "contraction" else "contraction"
        variant(other, dict(bw.opts, contraction=(other == "contraction")), v_steps, f"{other} operator form")
        variant("fgmres_outer", dict(bw.opts, outer_krylov=True, outer_restart=20, outer_inner_tol=0.1), v_steps,
                "flexible GMRES(20) preconditioned by one GS sweep, block tol 0.1")
    # ----------------------------------------------------------------- sub-domain operator bandwidth
    z0, z1 = bw.block
    nzb = z1 - z0
    nb = 3 * nzb * g.ny * g.nx
    ctx.set_contrast_dev(s6_dev)
    x = torch.randn(nb, dtype=torch.complex64, device=dev)
    y = torch.empty_like(x)
    for _ in range(3):
        ctx.matvec_dev(x, y, z0=z0, nz=nzb)
    torch.cuda.synchronize(dev)
    ctx.profile_enable(True)
    reps = 20
    mv_ms, _ = timed(stream, torch, dev, lambda k: ctx.matvec_dev(x, y, z0=z0, nz=nzb), reps, 1, dist)
    mv_ms /= reps
    mprof = ctx.profile_read()
    ctx.profile_enable(False)
    mv_bytes = sum(mprof[k][2] for k in ("P1_c64", "P2_c64", "P3_c64", "P4_c64", "P5_c64")) / reps
    n_block = nzb * g.ny * g.nx
    peak, peak_kind = measured_peaks()
    # ----------------------------------------------------------------- roofline of the dominant kernel
    dom = max(prof, key=lambda k: prof[k][1])
    launches, ms, by = prof[dom]
    achieved = (by / 1e9) / (ms / 1e3) if ms > 0 else 0.0
    tr = traffic_record(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                # DRAM bytes per launch: the captured launch's DRAM-to-algorithmic ratio times this class's mean
                # algorithmic bytes per launch (the capture is of the sub-domain launch; see profiles/traffic.json)
                "traffic": (round(tr["dram_per_algorithmic_byte"] * by / max(launches, 1)) if tr else None),
                "traffic_capture": (tr["workload"] if tr else None),
                "algorithmic_bytes_per_launch": by / max(launches, 1), "avg_launch_us": 1e3 * ms / max(launches, 1),
                "launches": launches}
    total_ms = sum(v[1] for v in prof.values())
    breakdown = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / total_ms, 4) if total_ms else 0,
                     "GBps": round((v[2] / 1e9) / (v[1] / 1e3), 1) if v[1] > 0 else None}
                 for k, v in prof.items() if v[0] > 0}
    gpu_launches = int(round(sum(v[0] for v in prof.values()) * args.steps / prof_steps))
    last = infos[-1]
    # ----------------------------------------------------------------- CPU oracle baseline
    cpu_baseline = None
    contraction = args.operator == "contraction"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if bw.key == "c5":
            nzs = max(1, nzb // 4)  # a quarter of a sub-domain: a bounded sample
            t_setup, t_apply = oracle_block_sample(bw, nzs, 1, contraction)
            unit_v = padded_volume(g, nzs)
            blk = padded_volume(g, nzb) / unit_v
            whole = padded_volume(g, g.nz) / unit_v
            whole_apps = last.outer_iters + 2 + last.outer_iters // 20
            est = t_setup * (blk + whole) + t_apply * (last.matvecs * blk + whole_apps * whole)
            sample = (f"CPU FP64 oracle: spectra ({t_setup:.1f} s) and one operator application ({t_apply:.1f} s) of a "
                      f"{g.nx}x{g.ny}x{nzs} slab of the model, scaled by padded FFT volume to this solve's "
                      f"{last.matvecs} sub-domain applications ({blk:.0f}x the slab), {whole_apps} whole-grid "
                      f"applications ({whole:.0f}x) and one spectra setup of each size: an extrapolation; "
                      f"the directly timed full solve is timed_full_solve")
        else:
            t_setup, t_apply = oracle_block_sample(bw, nzb, 1, contraction)
            applications = last.matvecs + 2 * (last.outer_iters + 1) + last.outer_iters
            est = 3 * t_setup + t_apply * applications
            sample = (f"CPU FP64 oracle: spectra of one {g.nx}x{g.ny}x{nzb} sub-domain ({t_setup:.1f} s) + one operator "
                      f"application ({t_apply:.1f} s), scaled to this solve's {applications} sub-domain-operator "
                      f"equivalents and 3 spectra setups: an extrapolation; the directly timed full solve is "
                      f"timed_full_solve")
        cpu_baseline = {"value": 1.0 / est, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": sample,
                        "seconds_per_solve_estimate": est, "timed_full_solve": c1_full_solves(ie, torch, dev, stream)}
    out = {
        "metric": METRIC, "value": (round(value, 4) if value is not None else None), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_ms_max / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64",
        "data": "synthetic (seeded generator)",
        "config": {"workload": bw.description, "grid": [g.nx, g.ny, g.nz], "h_m": g.h, "sub_domains": bw.split,
                   "dd": bw.dd_text, "precision": "complex64 conv/Krylov + FP64-accurate refinement",
                   "operator": args.operator, "restart": bw.opts["restart"], "tol": bw.tol, "freq_hz": bw.freq,
                   "sigma0": bw.sigma0, "seed": args.seed, "positions": len(bw.items),
                   "setup_s_excluded": round(setup_s, 3), "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"{world} independent models (one per GPU)"},
        "e2e": {"value": (round(e2e_value, 4) if e2e_value is not None else None), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d_total / args.steps), "d2h_bytes_per_step": int(d2h_total / args.steps)},
        "roofline": roofline,
        "matvec": {"sub_domain": [g.nx, g.ny, nzb], "ms": round(mv_ms, 4), "algorithmic_GB": round(mv_bytes / 1e9, 4),
                   "GBps": round(mv_bytes / 1e9 / (mv_ms / 1e3), 1),
                   "frac_of_peak": round(mv_bytes / 1e9 / (mv_ms / 1e3) / peak, 4),
                   "bytes_per_voxel": round(mv_bytes / n_block, 1),
                   # compulsory traffic of one application: read x and the contrast, the Green octant, write y
                   "compulsory_GBps": round(120.0 * n_block / 1e9 / (mv_ms / 1e3), 1)},
        "solve": {"status": int(st), "all_steps_converged": not failed, "failed_steps": failed,
                  "profiled_pass": {"steps": prof_steps, "ms_per_step": round(p_ms / prof_steps, 2),
                                    "blocks": "one after another (per-launch events do not overlap)"},
                  "outer_iters": last.outer_iters, "gmres_iters": last.gmres_iters_total, "matvecs": last.matvecs,
                  "reorth_passes": last.reorth_passes, "final_rel_residual": last.final_rel_residual,
                  "ms_per_position": [round(1e3 * inf.seconds, 1) for inf in infos],
                  "residual_history": [float(v) for v in last.history()],
                  "H_rx_z": [[float(H[0, r, 2].real), float(H[0, r, 2].imag)] for r in range(H.shape[1])]},
        "variants": variants,
        "kernels": breakdown,
        "tuned_tiles": ie.tuned_tiles().strip().splitlines(),
        "gpu_launches": gpu_launches,
        "clocks": clk,
        "cpu_baseline": cpu_baseline,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------ reference arm
# Operator applications of one solve, as the GB300 arm counts them (sub-domain applications of GMRES,
# whole-grid applications of the outer iteration and residuals), used only to scale the reference arm's
# CPU sample to solves/s, because that arm runs without the GB300 one.
# (The conventional large-model count is the contraction one times 2.5, the ratio of the two forms'
# applications measured on the 128x128x256 model.)
REF_COUNTS = {("c5", "contraction"): (513, 17), ("c5", "conventional"): (1282, 17),
              ("c2", "contraction"): (260, 11), ("c2", "conventional"): (650, 11)}


def run_reference(args):
    """The CPU FP64 oracle as the reference arm: its spectra once, then each step times one bounded sample
    (one application of the oracle's operator, in the selected form, on a slab of the workload's model:
    a quarter of a 256x256x64 sub-domain for c5, a whole 128^3 sub-domain for c2), converted to solves/s
    by padded FFT volume and the operator-application counts of one solve (REF_COUNTS): an extrapolation,
    stated as such in the line."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    from oracle import contraction as oc
    from oracle import operator as oop

    bw = BenchWorkload(args.workload, args.seed, args.scale, args.operator)
    g = bw.grid
    nzb = bw.block[1] - bw.block[0]
    nzs = max(1, nzb // 4) if bw.key == "c5" else nzb
    s6 = bw.sigma6[:nzs]
    t0 = time.perf_counter()
    if args.operator == "contraction":
        op = oc.ContractionOperator(s6, g.h, bw.freq, bw.sigma0)
    else:
        op = oop.FFTOperator(oop.contrast(s6, bw.sigma0), g.h, bw.freq, bw.sigma0)
    t_setup = time.perf_counter() - t0
    x = np.ones((3, nzs, g.ny, g.nx), dtype=np.complex128)
    for _ in range(min(args.warmup, 1)):
        op(x)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        op(x)
        times.append(time.perf_counter() - t0)
    t_apply = sum(times) / len(times)
    n_block, n_whole = REF_COUNTS[(bw.key, args.operator)]
    unit_v = padded_volume(g, nzs)
    blk, whole = padded_volume(g, nzb) / unit_v, padded_volume(g, g.nz) / unit_v
    est = t_setup * (blk + whole) + t_apply * (n_block * blk + n_whole * whole)
    value = 1.0 / est
    sample = (f"one application of the CPU FP64 oracle's operator on a {g.nx}x{g.ny}x{nzs} slab per step (mean "
              f"{t_apply:.2f} s; spectra {t_setup:.1f} s), scaled by padded FFT volume to {n_block} sub-domain and "
              f"{n_whole} whole-grid applications and one spectra setup of each size per solve: an extrapolation")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * t_apply, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic (seeded generator)",
           "config": {"workload": bw.description, "seed": args.seed, "operator": args.operator}, "impl": "reference",
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gb300(a)
