#!/usr/bin/env python
"""Throughput of the DG diffusion -> Sigma path on the 40 um cell workload.

Workload (one GPU): 40x40 um periodic cell of 256x256 elements, p = 3
(16 GLL nodes per element), Gamma(2, 0.5 um) disks at a seeded packing in
[0.5, 0.7], tiled into a 7x7-cell absorbing window (1792^2 elements), 64
seeded Gaussian start densities (sigma0 = 0.2 um), D = 2 um^2/ms.

One bench step = R SSP-RK3 time steps of all 64 densities followed by the
FP64 moment reduction and the covariance (every row of the hot path after
the one-off geometry set-up).  ``value`` is DoF-steps/s (active nodes x
densities x RK steps per second), timed with CUDA events on the library's
stream with the state already resident.  ``e2e`` times the user's call
sequence through the C ABI with host buffers: start points copied in
(dg_set_sources, which re-initialises the densities), R steps, covariance
copied out.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--precision f32|f64] [--rk R]
Under torchrun each rank runs its own 64 densities (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import dginputs  # noqa: E402

METRIC = "DoF-steps/s"
BYTES_PER_DOF_STEP = {"f32": 32, "f64": 64}   # 8 state accesses per RK step
# pixel triangles in two launches per stage: the q pass reads u and writes q (2
# values per DoF), the divergence pass reads q, u (and u0 in stages 2, 3) and
# writes the result: 3 + 4 + 3 + 5 + 3 + 5 = 23 accesses per RK step; in one
# launch per stage q stays on chip: the method's 8 accesses
BYTES_PER_DOF_STEP_TRI = {"f32": 92, "f64": 184}


def flops_per_dof_step_tri(p: int) -> float:
    """Dense element matrices per pixel and stage: G (4 N^2 FMAs per pass),
    the liftings (6 N (p+1) per pass) and the normal products (12 N), over
    the 2 N DoF of a pixel, 2 flops per FMA, 3 stages."""
    N = (p + 1) * (p + 2) // 2
    fma_pixel = 8 * N * N + 12 * N * (p + 1) + 12 * N
    return 3 * 2 * fma_pixel / (2 * N)


def flops_per_dof_step(p: int) -> float:
    """Sum-factorised FMAs per element and stage: volume 2n^3, own face
    derivatives 4n^2, lifting 4n^2, fluxes ~4n^2 -> 2 flops each, per node,
    times 3 stages."""
    n = p + 1
    return 3 * 2 * (2 * n ** 3 + 12 * n ** 2) / n ** 2


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace('.', '').isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace('.', '').isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) > 8:
                for k, nm in enumerate(names):
                    if r[5 + k].lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _traffic_record(kernel_src: str):
    """DRAM bytes per launch of the stage kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    return rec if rec.get("kernel_sha") == h else None


def workload_config(w, tri, window_elements, active_elements, densities, rk):
    """The workload's identity (the same for both arms of the benchmark)."""
    return {"workload": w.name + ("_triangles" if tri else ""), "p": w.p,
            "element": "triangle" if tri else "square", "window_elements": int(window_elements),
            "active_elements": int(active_elements), "densities_per_gpu": int(densities),
            "rk_steps_per_bench_step": int(rk),
            "l2": "state (>=16 GB) larger than L2, no flush"}


def run_reference(args, world, rank):
    """The oracle (plain FP64 C, OpenMP over elements) on host cores, each
    step a bounded sample of the workload: one of its densities carried R RK
    steps on the full 1792^2-element window (the sample cpu_baseline times)."""
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    w = dginputs.workload_cell40(args.seed, m=args.densities)
    cell = O.mask_disks(w.L, w.n_cell, w.disks.cx, w.disks.cy, w.disks.r)
    act = O.window_mask(cell, w.tiles)
    mesh = O.Mesh(p=w.p, active=act, h=w.h, x0=w.origin, y0=w.origin, k0=w.D)
    dof = int(act.sum()) * (w.p + 1) ** 2
    u = O.init_gaussian(mesh, *w.sources[0], w.sigma0)
    dt = 1e-4
    R = args.rk
    for _ in range(args.warmup):
        u = O.rk3(mesh, u, R, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = O.rk3(mesh, u, R, dt)
    el = time.perf_counter() - t0
    v = dof * R * args.steps / el
    cores = O.threads()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DoF-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, False, act.size, act.sum(), len(w.sources), R),
            "cpu_baseline": {"value": v, "unit": "DoF-steps/s", "cores": cores,
                             "kind": "oracle", "cpu": _host_cpu(),
                             "sample": f"1 of {len(w.sources)} densities x {R} SSP-RK3 steps per "
                                       "bench step on the full window"},
            "e2e": {"value": v, "unit": "DoF-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _host_cpu() -> str:
    """Host CPU model (where /proc/cpuinfo names it) and logical CPU count."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return f"{model or platform.machine()}, {os.cpu_count()} logical CPUs"


def cpu_baseline_sample(w, seconds_target=20.0, threads=None):
    """Oracle DoF-steps/s on a bounded sample: one density of the workload,
    RK steps on the full window until ~seconds_target of CPU work, on all
    host cores (threads=None) or on the given number of threads."""
    import oracle as O
    O.build()
    before = O.threads()
    if threads:
        O.set_threads(threads)
    try:
        cell = O.mask_disks(w.L, w.n_cell, w.disks.cx, w.disks.cy, w.disks.r)
        act = O.window_mask(cell, w.tiles)
        mesh = O.Mesh(p=w.p, active=act, h=w.h, x0=w.origin, y0=w.origin, k0=w.D)
        dof = int(act.sum()) * (w.p + 1) ** 2
        u = O.init_gaussian(mesh, *w.sources[0], w.sigma0)
        t0 = time.perf_counter()
        u = O.rk3(mesh, u, 1, 1e-4)
        one = time.perf_counter() - t0
        n = max(1, min(20, int(seconds_target / max(one, 1e-3)) - 1))
        t0 = time.perf_counter()
        u = O.rk3(mesh, u, n, 1e-4)
        el = time.perf_counter() - t0
        cores = O.threads()
    finally:
        O.set_threads(before)
    return {"value": dof * n / el, "unit": "DoF-steps/s", "cores": cores, "kind": "oracle",
            "cpu": _host_cpu(),
            "sample": f"1 of {len(w.sources)} densities x {n} SSP-RK3 steps on the full "
                      f"{act.shape[0]}^2 window"}


def fp64_roofline(p, tri, dof, stage_ms):
    """FP64 stage kernel against the FP64 pipe (2 FMA/clk/SM on GB300):
    152 x 2 x 2 flop x 2.07 GHz = 1.26 TFLOP/s, by algorithmic flops."""
    peak = 152 * 2 * 2 * 2.07e9 / 1e12
    fl = flops_per_dof_step_tri(p) if tri else flops_per_dof_step(p)
    ach = fl * dof / 3.0 / (stage_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "peak_source": "derived from unit counts and max clock"}


def sigma_solve(dg, w, s, dev, args, rnd, r_factor=10.0):
    """Sigma solves/s measured on the bench context: every density carried
    from its start to Delta = args.solve_delta on the growing window
    (radius factor 10, the library's setting for p = 3), Sigma formed, host
    wall clock around propagate_to + covariance.  Then the plain FP64 path
    solves the first few densities the same way (its rate per density), and
    the FP32 Sigma of those densities (dg_mixture_covariance of their FP32
    moments) is compared with the FP64 one."""
    import torch
    delta, nd = args.solve_delta, max(1, min(args.solve_fp64_densities, len(w.sources)))
    s.set_growing_window(r_factor)
    s.set_sources(w.sources)
    mom0 = s.moments()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    s.propagate_to(delta)
    sig32, mu32, mass32 = s.covariance()
    t32 = time.perf_counter() - t0
    steps = s.info().steps
    mom = s.moments()
    sub32, _ = s.mixture_covariance(mom[:nd], mom0[:nd])
    s.set_growing_window(0.0)
    with dg.DGSolver(p=w.p, precision=dg.DG_FP64, D=w.D, sigma0=w.sigma0, device=dev) as d64:
        d64.set_geometry_disks(w.disks.cx, w.disks.cy, w.disks.r, w.L, w.n_cell, w.tiles)
        d64.set_growing_window(r_factor)
        d64.set_sources(w.sources[:nd])
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        d64.propagate_to(delta)
        sig64, _, _ = d64.covariance()
        t64 = time.perf_counter() - t0
    m = len(w.sources)
    return {"delta_ms": delta, "densities": m, "rk_steps": steps, "seconds": t32,
            "sigma_solves_per_s": m / t32, "sigma": sig32.tolist(), "mu": mu32.tolist(),
            "free_value": 2 * w.D * delta, "growing_window_r": r_factor,
            "fp64_densities": nd, "fp64_seconds": t64, "fp64_sigma_solves_per_s": nd / t64,
            "sigma_fp64_subset": sig64.tolist(), "sigma_fp32_subset": sub32.tolist(),
            "sigma_rel_err_vs_fp64": float(np.abs(sub32 - sig64).max() / np.abs(sig64).max()),
            "what": "measured: start densities to Delta, growing window, Sigma; FP32 default "
                    "path vs the plain FP64 GPU path on the same densities"}


def _batch_member(args_tuple):
    seed, delta = args_tuple
    return dginputs.workload_batch_member(seed, delta=delta)


def run_batch(args):
    """Uneven-geometry batch: seeded geometries with 64..256 elements per cell
    side (h = 0.156 um), p in {2, 3, 4}, packing 0.40-0.75, Gamma shape
    1.5-3.0, 16 densities each, windows sized for Delta = --batch-delta ms
    (1 ms: 512 geometries, ~130 GB of FP32 state; the 20 ms windows of the
    full batch would need ~700 GB).  Geometries of equal p share one context
    (one launch per RK stage for all of them); geometries are added in seed
    order while the FP32 state stays under --batch-gb.  The same geometries
    are then run one context each (one launch per stage and geometry)."""
    import multiprocessing as mp
    # the geometries are drawn on the host cores before CUDA starts
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        cands = pool.map(_batch_member, [(sd, args.batch_delta) for sd in range(args.batch_geometries)])
    import torch
    import paper_1907_06191_gb300 as dg
    from paper_1907_06191_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    budget = args.batch_gb * 2 ** 30
    members, used = [], 0.0
    for w in cands:
        npe = (w.p + 1) ** 2
        est = w.n_window ** 2 * (1 - w.disks.packing) * npe * 16 * 4 * 3
        if used + est > budget:
            break
        members.append(w)
        used += est
    groups = {}
    for w in members:
        groups.setdefault(w.p, []).append(w)
    stream = torch.cuda.Stream(device=0)
    ctxs = []
    for p, ws in sorted(groups.items()):
        s = dg.DGSolver(p=p, precision=dg.DG_FP32, D=2.0, sigma0=0.2, device=0)
        s.set_stream(stream.cuda_stream)
        s.set_launch(args.launch)
        s.set_geometry_batch([(w.disks.cx, w.disks.cy, w.disks.r) for w in ws],
                             [w.L for w in ws], [w.n_cell for w in ws], [w.tiles for w in ws])
        s.set_sources(np.stack([w.sources for w in ws]))
        dt, _ = s.query_dt()
        ctxs.append((s, dt, s.info()))
    dof = sum(inf.dof_per_source * inf.m for _, _, inf in ctxs)
    R = args.rk

    def step_all():
        for s, dt, _ in ctxs:
            s.step(R, dt)
        for s, _, _ in ctxs:
            s.covariance_batch()

    for _ in range(args.warmup):
        step_all()
    torch.cuda.synchronize()
    launches = {str(inf.p): s.get_launch() for s, _, inf in ctxs}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step_all()
        e1.record(stream)
        e1.synchronize()
    ms = e0.elapsed_time(e1)
    batched = dof * R * args.steps / (ms * 1e-3)
    dt_of = dict((inf.p, dt) for s, dt, inf in ctxs)
    for s, _, _ in ctxs:
        s.close()
    # the same geometries one context each
    singles = []
    for w in members:
        s = dg.DGSolver(p=w.p, precision=dg.DG_FP32, D=2.0, sigma0=0.2, device=0)
        s.set_stream(stream.cuda_stream)
        s.set_launch(args.launch)
        s.set_geometry_disks(w.disks.cx, w.disks.cy, w.disks.r, w.L, w.n_cell, w.tiles)
        s.set_sources(w.sources)
        singles.append((s, dt_of[w.p]))
    for _ in range(max(1, args.warmup)):
        for s, dt in singles:
            s.step(R, dt)
            s.covariance()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        for s, dt in singles:
            s.step(R, dt)
        for s, dt in singles:
            s.covariance()
    e1.record(stream)
    e1.synchronize()
    ms1 = e0.elapsed_time(e1)
    for s, _ in singles:
        s.close()
    unbatched = dof * R * args.steps / (ms1 * 1e-3)
    line = {"metric": METRIC, "value": batched, "unit": "DoF-steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batch_uneven_p234", "geometries": len(members),
                       "geometries_requested": args.batch_geometries,
                       "delta_ms": args.batch_delta,
                       "per_p": {str(p): len(ws) for p, ws in groups.items()},
                       "densities_per_geometry": 16, "rk_steps_per_bench_step": R,
                       "dof": dof, "state_gb": used / 2 ** 30,
                       "window_elements_min_max": [min(w.n_window for w in members) ** 2,
                                                   max(w.n_window for w in members) ** 2],
                       "launch_blocks_per_sm": launches,
                       "l2": "state larger than L2, no flush"},
            "unbatched_value": unbatched, "batched_over_unbatched": batched / unbatched,
            "unbatched_ms_per_step": ms1 / args.steps,
            "gpu_launches": args.steps * len(ctxs) * (3 * R + 3),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def _surrogate_member(args_tuple):
    seed, m = args_tuple
    return dginputs.workload_surrogate_member(seed, m=m)


def run_surrogate(args):
    """Learned covariance surrogate: DG Sigma of seeded 10 um cells (batched
    FP32 solves, Delta = 1..5 ms) trains the CNN; held-out cells test it.
    value = Sigma evaluations/s of batch-4096 network inference; the DG
    rate on the same cells and the network's error against DG are reported
    beside it."""
    import torch
    import paper_1907_06191_gb300 as dg
    from paper_1907_06191_gb300 import _build, surrogate as sgm
    _build.build()
    torch.cuda.set_device(0)
    ntr, nte, ms = args.sg_train, args.sg_test, args.sg_sources
    t_start = time.perf_counter()
    phases = {}

    def mark(name):
        phases[name] = round(time.perf_counter() - t_start, 2)
        print(f"[surrogate] {name}: {phases[name]} s", file=sys.stderr, flush=True)

    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        ws_tr = pool.map(_surrogate_member, [(s, ms) for s in range(ntr)], chunksize=16)
        ws_te = pool.map(_surrogate_member, [(100000 + s, ms) for s in range(nte)], chunksize=16)
    mark("cells drawn")
    sig_tr, t_tr = sgm.dg_sigma(ws_tr)
    mark("DG training set")
    sig_te, t_te = sgm.dg_sigma(ws_te)
    mark("DG held-out set")
    # the reference's own noise: the same held-out cells with an independent set
    # of start points (the network sees the substrate, not the start points)
    ws_te2 = []
    for w in ws_te:
        lo, hi = dginputs.source_box(w.L, w.tiles, w.sigma0, w.D, max(w.deltas))
        src = dginputs.sample_sources(w.meta["seed"] + 555, w.disks, ms, lo, hi, margin=w.h)
        ws_te2.append(dginputs.Workload(w.name, w.p, w.L, w.n_cell, w.tiles, w.D, w.sigma0,
                                        w.deltas, w.disks, src, w.meta))
    sig_te2, _ = sgm.dg_sigma(ws_te2)
    mark("DG held-out set, second start points")
    occ, cond, tgt = sgm.build_samples(ws_tr, sig_tr)
    occ_e, cond_e, tgt_e = sgm.build_samples(ws_te, 0.5 * (sig_te + sig_te2))
    _, _, tgt_a = sgm.build_samples(ws_te, sig_te)
    _, _, tgt_b = sgm.build_samples(ws_te, sig_te2)
    dg_noise = np.linalg.norm(tgt_a - tgt_b, axis=1) / np.linalg.norm(tgt_e, axis=1)
    to = lambda a, dt: torch.from_numpy(a).to("cuda:0", dt)
    net = dg.Surrogate(max_batch=4096, seed=1, device=0)
    t0 = time.perf_counter()
    mark("samples built")
    hist = sgm.train(net, to(occ, torch.uint8), to(cond, torch.float32), to(tgt, torch.float32),
                     epochs=args.sg_epochs)
    t_train = time.perf_counter() - t0
    mark("trained")
    # held-out error against the DG solve (the reference)
    pe = torch.zeros((occ_e.shape[0], 3), device="cuda:0")
    oe, ce = to(occ_e, torch.uint8), to(cond_e, torch.float32)
    for b0 in range(0, oe.shape[0], 4096):
        net.predict(oe[b0:b0 + 4096], ce[b0:b0 + 4096], pe[b0:b0 + 4096])
    pred = pe.cpu().numpy()
    rel = np.linalg.norm(pred - tgt_e, axis=1) / np.linalg.norm(tgt_e, axis=1)
    # reference point: least squares on the packing fraction and log(D Delta)
    base = sgm.packing_fit(ws_tr, tgt, ws_te)
    rel_base = np.linalg.norm(base - tgt_e, axis=1) / np.linalg.norm(tgt_e, axis=1)
    # batch-4096 inference throughput (inputs resident)
    B = 4096
    reps = (B + oe.shape[0] - 1) // oe.shape[0]
    ob = oe.repeat(reps, 1, 1)[:B].contiguous()
    cb = ce.repeat(reps, 1)[:B].contiguous()
    out = torch.zeros((B, 3), device="cuda:0")
    for _ in range(args.warmup):
        net.predict(ob, cb, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        net.predict(ob, cb, out)
    e1.record()
    e1.synchronize()
    ms_step = e0.elapsed_time(e1) / args.steps
    value = B / (ms_step * 1e-3)
    dg_rate = (nte * len(ws_te[0].deltas)) / t_te
    line = {"metric": "Sigma evaluations/s", "value": value, "unit": "Sigma/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": "surrogate_cell10_p2", "batch": B, "train_geometries": ntr,
                       "test_geometries": nte, "deltas_ms": ws_tr[0].deltas,
                       "params": net.param_count(), "epochs": args.sg_epochs,
                       "l2": "batch inputs 64 MB, resident"},
            "dg_sigma_per_s": dg_rate, "speedup_vs_dg": value / dg_rate,
            "heldout_rel_err": {"mean": float(rel.mean()), "p95": float(np.percentile(rel, 95)),
                                "max": float(rel.max()),
                                "vs": "mean of two DG solves with independent start points"},
            "packing_fit_rel_err": {"mean": float(rel_base.mean()),
                                    "p95": float(np.percentile(rel_base, 95))},
            "dg_reference_noise": {"mean": float(dg_noise.mean()), "p95": float(np.percentile(dg_noise, 95)),
                               "what": "relative difference of the two DG solves"},
            "sources_per_geometry": ms,
            "train_loss_first_last": [hist[0], hist[-1]], "train_seconds": t_train,
            "phase_seconds": phases,
            "dg_seconds_train_set": t_tr}
    net.close()
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--element", default="square", choices=["square", "triangle"],
                    help="square GLL elements or the paper's pixel triangles (p <= 3)")
    ap.add_argument("--rounding", default="stochastic", choices=["stochastic", "nearest"],
                    help="rounding of the FP32 state (library default: stochastic)")
    ap.add_argument("--rk", type=int, default=20, help="RK3 steps per bench step")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--densities", type=int, default=64,
                    help="start points per GPU (64 = the workload; fewer for profiling)")
    ap.add_argument("--launch", type=int, default=-1,
                    help="stage-kernel launch shape: -1 tuned (library default), 0 one block "
                         "per chunk, k persistent blocks per SM")
    ap.add_argument("--contraction", type=int, default=0,
                    help="FP32 p = 5 element contractions: 0 CUDA cores (library default), "
                         "1 tensor cores, -1 tuned")
    ap.add_argument("--triangle-fusion", type=int, default=1,
                    help="pixel triangles: 1 one launch per stage (library default where "
                         "available), 0 two launches")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="bench steps of the plain FP64 GPU path timed beside the FP32 path")
    ap.add_argument("--solve-delta", type=float, default=None,
                    help="measure Sigma solves/s: every density to this Delta (ms) on the "
                         "growing window (0: skip; default 5 on the 40 um cell workload, "
                         "0 otherwise)")
    ap.add_argument("--solve-fp64-densities", type=int, default=2,
                    help="densities solved in FP64 for the comparator rate and the error")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--check-delta", type=float, default=0.0,
                    help="compare FP32 with the FP64 GPU path over a solve to this Delta (ms) "
                         "on 4 densities instead of over R steps")
    ap.add_argument("--growing-window", type=float, default=0.0,
                    help="with --full-delta: also solve on the growing window of this radius "
                         "factor and report its time and Sigma against the fixed window")
    ap.add_argument("--full-delta", type=float, default=0.0,
                    help="after the timed steps, solve every density to each of the workload's "
                         "diffusion times up to this Delta (ms) and report Sigma and the time")
    ap.add_argument("--workload", default="cell40", choices=["cell40", "batch", "p5", "surrogate"])
    ap.add_argument("--sg-train", type=int, default=4000,
                    help="training cells (x 5 diffusion times = DG samples)")
    ap.add_argument("--sg-test", type=int, default=1000, help="held-out cells")
    ap.add_argument("--sg-epochs", type=int, default=30)
    ap.add_argument("--sg-sources", type=int, default=16)
    ap.add_argument("--batch-geometries", type=int, default=512)
    ap.add_argument("--batch-gb", type=float, default=200.0)
    ap.add_argument("--batch-delta", type=float, default=1.0,
                    help="diffusion time (ms) the batch windows are sized for")
    args = ap.parse_args()
    if args.solve_delta is None:
        args.solve_delta = 5.0 if args.workload == "cell40" else 0.0
    world, rank, local = _dist()
    if args.workload == "batch" and args.impl == "ours":
        return run_batch(args) if rank == 0 else 0
    if args.workload == "surrogate" and args.impl == "ours":
        return run_surrogate(args) if rank == 0 else 0

    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    import paper_1907_06191_gb300 as dg
    from paper_1907_06191_gb300 import _build
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        tdist.barrier()
        _build.build()
    torch.cuda.set_device(local)
    dev = local

    if args.workload == "p5":
        w = dginputs.workload_p5(args.seed, m=32)
    else:
        w = dginputs.workload_cell40(args.seed, m=64)
    w.sources = w.sources[:args.densities]
    # weak scaling: every rank its own 64 start points
    if world > 1:
        from dginputs import sample_sources, source_box
        lo, hi = source_box(w.L, w.tiles, w.sigma0, w.D, max(w.deltas))
        w.sources = sample_sources(args.seed + 7919 + 1000 * rank, w.disks, args.densities, lo, hi,
                                   margin=w.h)
    prec = dg.DG_FP32 if args.precision == "f32" else dg.DG_FP64
    rnd = dg.DG_ROUND_STOCHASTIC if args.rounding == "stochastic" else dg.DG_ROUND_NEAREST
    tri = args.element == "triangle"
    if tri:
        w.p = min(w.p, 3)
    s = dg.DGSolver(p=w.p, precision=prec, D=w.D, sigma0=w.sigma0, device=dev, rounding=rnd,
                    element=dg.DG_ELEMENT_TRIANGLE if tri else dg.DG_ELEMENT_SQUARE)
    s.set_geometry_disks(w.disks.cx, w.disks.cy, w.disks.r, w.L, w.n_cell, w.tiles)
    s.set_launch(args.launch)
    s.set_contraction(args.contraction)
    if tri:
        s.set_triangle_fusion(args.triangle_fusion)
    tri_fused = bool(tri and s.get_triangle_fusion())
    stream = torch.cuda.Stream(device=dev)
    s.set_stream(stream.cuda_stream)
    s.set_sources(w.sources)
    dt, rho = s.query_dt()
    inf = s.info()
    m = inf.m
    dof = inf.dof_per_source * m
    R = args.rk

    def bench_step():
        s.step(R, dt)
        s.covariance()

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize(dev)
    launch_used = s.get_launch()
    contraction_used = s.get_contraction()

    # device-timed region: state resident (16 GB > L2, no flush needed)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(dev) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            bench_step()
        ev1.record(stream)
        ev1.synchronize()
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([ms], device=f"cuda:{dev}")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms = float(t.item())
    total_dof_steps = dof * R * args.steps * world
    value = total_dof_steps / (ms * 1e-3)

    # stage kernel alone: R RK steps = 3R launches of the fused stage kernel
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(R, dt)
    e1.record(stream)
    e1.synchronize()
    stage_ms = e0.elapsed_time(e1) / (3 * R)
    # algorithmic bytes: the method's 8 state accesses per DoF-step (the
    # triangles' two-pass design moves more, reported beside as design traffic)
    bytes_per_launch = BYTES_PER_DOF_STEP[args.precision] * dof / 3.0
    peaks, src = _peaks()
    achieved = bytes_per_launch / (stage_ms * 1e-3) / 1e9
    rec = _traffic_record(os.path.join(ROOT, "paper_1907_06191_gb300", "csrc", "dg_stage.cuh"))
    traffic = None
    if rec and rec.get("precision") == args.precision and rec.get("p") == w.p and not tri:
        traffic = rec["dram_bytes_per_launch_per_dof"] * dof
    if args.precision == "f64":
        roofline = fp64_roofline(w.p, tri, dof, stage_ms)
        roofline["traffic"] = traffic
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                    "peak_source": f"{src} hbm_gbs"}
        if tri and not tri_fused:
            design = BYTES_PER_DOF_STEP_TRI[args.precision] * dof / 3.0 / (stage_ms * 1e-3) / 1e9
            roofline["design_bytes_per_dof_step"] = BYTES_PER_DOF_STEP_TRI[args.precision]
            roofline["design_achieved"] = design
            roofline["design_frac"] = design / peaks["hbm_gbs"]
            roofline["note"] = ("achieved counts the method's 32 B per DoF-step; the two-pass "
                                "triangle design moves 92 B (q written and read back)")
        elif tri:
            roofline["note"] = ("one launch per stage: q stays in shared memory, the design "
                                "moves the method's 32 B per DoF-step (plus halo reads)")

    # e2e through the C ABI with host buffers
    xy_host = torch.from_numpy(np.ascontiguousarray(w.sources)).pin_memory()
    torch.cuda.synchronize(dev)
    if world > 1:
        tdist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.set_sources(xy_host.numpy())
        s.step(R, dt)
        sig, mu, mass = s.covariance()
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=f"cuda:{dev}")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": total_dof_steps / e2e_s, "unit": "DoF-steps/s",
           "h2d_bytes_per_step": int(m * 2 * 8),
           "d2h_bytes_per_step": int(5 * 8 + m * 8)}

    # agreement with the FP64 GPU path on the same steps
    check = None
    fp64 = None
    if args.check_delta and args.precision == "f32" and rank == 0:
        # a longer solve: the first 4 densities to Delta in both precisions
        nd = 4
        res = {}
        for pr in (dg.DG_FP32, dg.DG_FP64):
            with dg.DGSolver(p=w.p, precision=pr, D=w.D, sigma0=w.sigma0, device=dev,
                             rounding=rnd, element=s.cfg.element) as c2:
                c2.set_geometry_disks(w.disks.cx, w.disks.cy, w.disks.r, w.L, w.n_cell, w.tiles)
                c2.set_sources(w.sources[:nd])
                t0 = time.perf_counter()
                c2.propagate_to(args.check_delta)
                secs = time.perf_counter() - t0
                sg3, mu2, mass = c2.covariance()
                res[pr] = (sg3, mass, secs, c2.info().steps)
        s32, m32, t32, n32 = res[dg.DG_FP32]
        s64, m64, t64, n64 = res[dg.DG_FP64]
        check = {"delta_ms": args.check_delta, "densities": nd, "rk_steps": n32,
                 "sigma_fp64": s64.tolist(), "sigma_fp32": s32.tolist(),
                 "sigma_rel_err": float(np.abs(s32 - s64).max() / np.abs(s64).max()),
                 "mass_rel_err": float(np.abs(m32 - m64).max() / np.abs(m64).max()),
                 "seconds_fp32": t32, "seconds_fp64": t64}
    elif not args.no_check and args.precision == "f32" and rank == 0:
        # the plain FP64 GPU path on the same workload: timed (the metric's
        # comparator), then the same R steps from the same start compared
        s.set_sources(w.sources)
        s.step(R, dt)
        sig32 = s.covariance()[0]
        mom32 = s.moments()
        with dg.DGSolver(p=w.p, precision=dg.DG_FP64, D=w.D, sigma0=w.sigma0, device=dev,
                         element=s.cfg.element) as d64:
            d64.set_geometry_disks(w.disks.cx, w.disks.cy, w.disks.r, w.L, w.n_cell, w.tiles)
            d64.set_stream(stream.cuda_stream)
            d64.set_sources(w.sources)
            d64.step(R, dt)
            d64.covariance()
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(args.fp64_steps):
                d64.step(R, dt)
                d64.covariance()
            e1.record(stream)
            e1.synchronize()
            ms64 = e0.elapsed_time(e1)
            e0.record(stream)
            d64.step(1, dt)
            e1.record(stream)
            e1.synchronize()
            stage64 = e0.elapsed_time(e1) / 3.0
            d64.set_sources(w.sources)
            d64.step(R, dt)
            sig64 = d64.covariance()[0]
            mom64 = d64.moments()
        m2_32 = mom32[:, 3:] / mom32[:, :1]
        m2_64 = mom64[:, 3:] / mom64[:, :1]
        check = {"steps": R, "sigma_rel_err": float(np.abs(sig32 - sig64).max() / np.abs(sig64).max()),
                 "second_moment_rel_err": float(np.abs(m2_32 - m2_64).max() / np.abs(m2_64).max())}
        fp64 = {"value": dof * R * args.fp64_steps / (ms64 * 1e-3), "unit": "DoF-steps/s",
                "steps": args.fp64_steps, "ms_per_step": ms64 / args.fp64_steps,
                "roofline": fp64_roofline(w.p, tri, dof, stage64),
                "what": "the plain FP64 GPU path, same workload and bench step, timed in this run"}

    # measured Sigma solves: every density carried to the workload's first
    # diffusion time on the growing window, the FP32 path timed end to end;
    # a few densities in FP64 give the comparator's rate and the error
    solve = None
    if args.solve_delta > 0 and rank == 0 and not tri:
        solve = sigma_solve(dg, w, s, dev, args, rnd)

    full = None
    if args.full_delta > 0 and rank == 0:
        def full_solve(r_factor):
            s.set_growing_window(r_factor)
            s.set_sources(w.sources)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            snaps = []
            for d in [d for d in w.deltas if d <= args.full_delta]:
                s.propagate_to(d)
                sg3, mu2, mass = s.covariance()
                snaps.append({"delta_ms": d, "elapsed_s": time.perf_counter() - t0,
                              "rk_steps": s.info().steps, "sigma": sg3.tolist(), "mu": mu2.tolist(),
                              "mass_min": float(mass.min()), "mass_max": float(mass.max()),
                              "free_value": 2 * w.D * d})
            el = time.perf_counter() - t0
            s.set_growing_window(0.0)
            return {"snapshots": snaps, "seconds": el, "densities": m,
                    "sigma_solves_per_s_measured": m / el,
                    "note": "one propagation through every snapshot; solves = densities "
                            "carried to the last Delta"}
        full = full_solve(0.0)
        if args.growing_window > 0:
            g = full_solve(args.growing_window)
            g["r_factor"] = args.growing_window
            g["sigma_rel_diff_vs_fixed"] = [
                float(np.abs(np.array(a["sigma"]) - np.array(b["sigma"])).max()
                      / np.abs(np.array(b["sigma"])).max())
                for a, b in zip(g["snapshots"], full["snapshots"])]
            g["speedup_vs_fixed"] = full["seconds"] / g["seconds"]
            full["growing_window"] = g
    # multi-GPU: the densities of every rank form one mixture; the one
    # exchange is the moment gather, then Sigma on each rank's device
    sharded = None
    if world > 1:
        from dginputs import sample_sources, source_box
        from paper_1907_06191_gb300.multi import sharded_covariance
        lo, hi = source_box(w.L, w.tiles, w.sigma0, w.D, max(w.deltas))
        every = np.concatenate([sample_sources(args.seed + 7919 + 1000 * r, w.disks, args.densities,
                                               lo, hi, margin=w.h) for r in range(world)])
        s3, mu2, gm, _ = sharded_covariance(s, every, lambda c: c.step(R, dt), device=f"cuda:{dev}")
        sharded = {"ranks": world, "densities": int(gm.shape[0]), "rk_steps": R,
                   "sigma": s3.tolist(), "mu": mu2.tolist(),
                   "what": "start points of all ranks, one moment all-gather, dg_mixture_covariance"}
    s.close()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": "DoF-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.precision, "data": "synthetic",
        "config": workload_config(w, tri, inf.nx * inf.ny, inf.n_active, m, R),
        "run": {"rounding": args.rounding if args.precision == "f32" else "nearest",
                "dof_per_density": inf.dof_per_source, "dt_ms": dt, "rho_per_ms": rho,
                "packing": w.disks.packing, "disks": w.disks.n,
                "halo_max_per_block": inf.halo_max, "launch_blocks_per_sm": launch_used,
                "contraction": "tensor cores (FP16 hi/lo split, FP32 accumulation)"
                if contraction_used else "CUDA cores",
                "triangle_stage": None if not tri else
                ("one launch per stage" if tri_fused else "two launches per stage (q through device memory)")},
        "sigma_solves_per_s": solve["sigma_solves_per_s"] if solve else None,
        "sigma_solve": solve,
        "fp64_value": fp64["value"] if fp64 else None,
        "fp64_path": fp64,
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": args.steps * (3 * R + 3),
        "clocks": clk.summary(),
        "fp64_check": check,
    }
    if full is not None:
        line["full_solve"] = full
    if sharded is not None:
        line["sharded_sigma"] = sharded
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline_sample(w)
        line["cpu_baseline_1thread"] = cpu_baseline_sample(w, seconds_target=10.0, threads=1)
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
