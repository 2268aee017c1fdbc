#!/usr/bin/env python3
"""Throughput of the direct point-catalog SHT on GB300 (arXiv:2312.12285).

One step = one pass of the whole forward hot path over the workload:
point preparation, per-(point, m) seed and phase, l-recurrence and
accumulation into a_lm (analysis kernel), reduction over chunks, shot noise,
pseudo-C_l and 32 log-spaced bandpowers.  The metric is nominal
points x modes per second (modes = (lmax+1)(lmax+2)/2 per point).

Default workload: 1e6 lognormal galaxies + 9e6 randoms in a 40%-sky cap mask,
lmax = 2048, FP32 recurrence with FP64-accurate seed and phase.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every catalog is split into N
contiguous shards, each rank transforms its shard and the partial a_lm are
summed with one NCCL all-reduce (the sum over points is the only exchange).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "a_lm points*modes/s at lmax=2048, mixed vs FP64 at C_l err 1e-4; roofline %"
UNIT = "points*modes/s"
FLOPS_PER_POINT_MODE = 7  # recurrence: 1 mul + 1 FMA; accumulation: 2 FMA (Sec. 2.2 / App. A)
FP32_LANES_PER_SM = 128
FP64_TFLOPS_NOMINAL = 1.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=3, help="workload configuration (3 = lmax 2048, 1e7 points)")
    ap.add_argument("--scale", type=float, default=1.0, help="scale the point counts (profiling runs)")
    ap.add_argument("--lmax", type=int, default=None)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "mixed", "interp"],
                    help="interp = the interpolated route (samples in theta, default 16 per multipole)")
    ap.add_argument("--columns", type=int, default=0,
                    help="weight columns on the workload's point set (pointsht_alm_columns); 0 = catalog form")
    ap.add_argument("--mixed-kernel", default="mma.sync", choices=["mma.sync", "tcgen05", "tcgen05:8x32",
                                                                     "tcgen05:4x64", "tcgen05:2x128"],
                    help="weight-column contraction kernel of --columns / --precision mixed")
    ap.add_argument("--no-ladder", action="store_true", help="skip the mixed / FP32 / FP64 comparison")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint (gradient) measurement")
    ap.add_argument("--no-coupling", action="store_true", help="skip the mode-coupling matrix measurement")
    ap.add_argument("--no-spin2", action="store_true", help="skip the spin-2 (shear) transform measurement")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batching workload (16 tomographic bins + shared randoms, lmax 1536)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle sample points (0 = automatic)")
    ap.add_argument("--graph", action="store_true", help="capture one step in a CUDA graph and replay it")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
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
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s in sm if s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------- helpers --
def load_workload(args):
    from paper_2312_12285_gb300 import catalogs
    wl = catalogs.config(args.config, scale=args.scale, lmax=args.lmax)
    if args.precision == "fp64":
        for c in wl.catalogs:
            c.x, c.phi, c.w = (v.astype("float64") for v in (c.x, c.phi, c.w))
    return wl


def workload_name(wl, args) -> str:
    parts = [f"{c.name} {c.n:.3g}" for c in wl.catalogs]
    return f"{wl.name}: " + " + ".join(parts) + f", lmax {wl.lmax}, {args.precision}"


def oracle_sample(wl, target_pm: float):
    """A bounded sample of the workload: the first points of every catalog in
    proportion to its size, about target_pm points*modes in total."""
    nm = wl.nmodes
    ntot = wl.npoints
    npts = max(len(wl.catalogs), int(target_pm / nm))
    frac = min(1.0, npts / ntot)
    out = []
    for c in wl.catalogs:
        k = max(1, int(round(c.n * frac)))
        out.append((c.x[:k], c.phi[:k], c.w[:k], c.coeff, c.field))
    return out


def run_oracle(sample, lmax, nfield=1):
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    alms = []
    for f in range(nfield):
        sel = [(x, p, w, co) for (x, p, w, co, fi) in sample if fi == f]
        alms.append(oracle.field_alm(sel, lmax) if sel else np.zeros(oracle.nmodes(lmax), np.complex128))
    dt = time.perf_counter() - t0
    return alms, dt


# --------------------------------------------------------------- reference --
def reference_arm(args):
    """The FP64 CPU oracle timed on this machine's host cores, each step a
    bounded sample of the same workload (the paper's method written plainly)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = load_workload(args)
    L = wl.lmax
    target = 3.0e9 if L >= 1024 else 5.0e8
    sample = oracle_sample(wl, target)
    npts = sum(s[0].shape[0] for s in sample)
    pm = npts * wl.nmodes
    for _ in range(args.warmup):
        run_oracle(sample, L, wl.nfield)
    times = []
    for _ in range(args.steps):
        _, dt = run_oracle(sample, L, wl.nfield)
        times.append(dt)
    t = sum(times) / len(times)
    val = pm / t
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(wl, args), "points": wl.npoints, "lmax": L, "nmodes": wl.nmodes},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {npts} points of the workload (proportional per catalog), "
                                   f"all {wl.nmodes} modes, FP64 C oracle, OpenMP"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- ours --
def ours(args):
    import numpy as np
    import torch

    from paper_2312_12285_gb300 import catalogs, ops
    from paper_2312_12285_gb300.sharding import allreduce_sum, shard_array as shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    wl = load_workload(args)
    L = wl.lmax
    prec = args.precision
    # this rank's shard of every catalog
    cats_np = [(shard(c.x, rank, world), shard(c.phi, rank, world), shard(c.w, rank, world), c.field, c.coeff)
               for c in wl.catalogs]
    n_rank = sum(c[0].shape[0] for c in cats_np)
    cats = [ops.Cat(torch.from_numpy(np.ascontiguousarray(x)).to(dev), torch.from_numpy(np.ascontiguousarray(p)).to(dev),
                    torch.from_numpy(np.ascontiguousarray(w)).to(dev), f, co) for (x, p, w, f, co) in cats_np]
    nfield = wl.nfield
    plan = ops.get_plan(L, dev)
    ws = torch.empty(ops.workspace_bytes(plan, cats, nfield, "fp32" if prec == "interp" else prec),
                     dtype=torch.uint8, device=dev)
    out = torch.empty((nfield, plan.nmodes), dtype=torch.complex128, device=dev)
    edges = torch.from_numpy(catalogs.log_bin_edges(L, 32).astype(np.int32)).to(dev)

    # fields formed from the sources: D_b - alpha_b R for a shared random catalog
    coef = None
    if isinstance(wl.extra.get("alpha"), list):
        nb = wl.extra["nbins"]
        cm = np.zeros((nb, nfield))
        for b in range(nb):
            cm[b, b] = 1.0
            cm[b, nb] = -wl.extra["alpha"][b]
        coef = torch.from_numpy(cm).to(dev)
    nout = nfield if coef is None else coef.shape[0]

    if prec == "interp":
        nt = ops.ntheta_for_tolerance(L, 1e-4)
        ws = torch.empty(max(ws.numel(), ops.workspace_bytes_interp(plan, cats, nfield, nt)), dtype=torch.uint8,
                         device=dev)

    def step(cs=cats):
        if prec == "interp":
            a = ops.alm_interp(plan, cs, nfield, nt, out=out, workspace=ws)
        else:
            a = ops.alm_raw(plan, cs, nfield, prec, out=out, workspace=ws)
        noise = ops.shot_noise_raw(cs, nfield, "fp32" if prec == "interp" else prec, dev, workspace=ws)
        if dist is not None:
            allreduce_sum([a, noise])
        if coef is not None:
            a, noise = ops.combine_raw(a, coef, noise)
        cl = ops.cl_raw(a, noise)
        cb = ops.bin_raw(cl, edges)
        return cl, cb

    # prep (pads, hist, scan, scatter), analysis, reduce, 2 x shot noise, [combine x2], C_l, bins
    # interp: prep, hist, 2 scans, scatter, bin, fold, [pad], positions, transform, reduce, combine;
    # then noise 2, C_l, bins
    launches_per_step = 10 + (2 if coef is not None else 0)
    if prec == "interp":
        launches_per_step = nfield * (11 + (1 if (nt // 2) % 1024 else 0)) + 4 + (2 if coef is not None else 0)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    plan.check()
    gstep = ops.GraphStep(step) if args.graph else None

    evk = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a_, b_ in evk:  # create the event handles before they are handed to the library
        a_.record()
        b_.record()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0.record()
    for k in range(args.steps):
        if gstep is not None:
            gstep.replay()
        else:
            plan.set_timing_events(evk[k][0], evk[k][1])
            step()
    e1.record()
    torch.cuda.synchronize()
    plan.set_timing_events(None, None)
    clocks = sampler.stop()
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    # with a graph the analysis kernel is not bracketed separately: its time is
    # bounded by the step time (it is > 99.9% of a step)
    kms = ms if gstep is not None else sum(a.elapsed_time(b) for a, b in evk) / args.steps
    if dist is not None:
        t = torch.tensor([ms, kms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, kms = float(t[0]), float(t[1])
    plan.check()

    total_pm = wl.npoints * wl.nmodes
    value = total_pm / (ms / 1e3)
    props = torch.cuda.get_device_properties(dev)
    sm_max = None
    try:
        sm_max = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz")
    except Exception:
        pass
    sm_max = sm_max or 2070.0
    if prec == "fp64":
        # FP64 pipe: the nominal dense FP64 rate of the part (profiling recipe's table)
        peak = FP64_TFLOPS_NOMINAL
        peak_src = "nominal GB300 FP64 1.25 TFLOP/s (recipe table; a DFMA loop measured 1.18)"
    else:
        peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12  # TFLOP/s FP32
        peak_src = (f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz "
                    f"(recipe unit counts and clock)")
    achieved = FLOPS_PER_POINT_MODE * n_rank * wl.nmodes / (kms / 1e3) / 1e12
    if prec == "interp":
        # algorithmic flops of the interpolated route: binning 22 per (point, m)
        # (4 spline weights x complex MAC, phase rotation), transform of the
        # samples 27 per (sample, mode) (recurrence, 6 columns x complex MAC)
        achieved = (22.0 * n_rank * (L + 1) + 27.0 * nt * wl.nmodes) / (kms / 1e3) / 1e12

    # ---- end to end through the public API, host buffers in pinned memory ----
    e2e = None
    if not args.no_e2e:
        host = [(torch.from_numpy(np.ascontiguousarray(x)).pin_memory(), torch.from_numpy(np.ascontiguousarray(p)).pin_memory(),
                 torch.from_numpy(np.ascontiguousarray(w)).pin_memory()) for (x, p, w, f, co) in cats_np]
        dcats = [ops.Cat(torch.empty_like(h[0], device=dev), torch.empty_like(h[1], device=dev),
                         torch.empty_like(h[2], device=dev), c.field, c.coeff) for h, c in zip(host, cats)]
        cl_h = torch.empty((nout * (nout + 1) // 2, L + 1), dtype=torch.float64).pin_memory()
        cb_h = torch.empty((nout * (nout + 1) // 2, 32), dtype=torch.float64).pin_memory()
        h2d = sum(sum(t.numel() * t.element_size() for t in h) for h in host)
        d2h = cl_h.numel() * 8 + cb_h.numel() * 8

        def e2e_step():
            for h, d in zip(host, dcats):
                d.x.copy_(h[0], non_blocking=True)
                d.phi.copy_(h[1], non_blocking=True)
                d.w.copy_(h[2], non_blocking=True)
            cl, cb = step(dcats)
            cl_h.copy_(cl, non_blocking=True)
            cb_h.copy_(cb, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for _ in range(args.steps):
            e2e_step()
        s1.record()
        torch.cuda.synchronize()
        ems = s0.elapsed_time(s1) / args.steps
        if dist is not None:
            t = torch.tensor([ems], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t[0])
        e2e = {"value": total_pm / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": ems}

    # ---- CPU oracle baseline and accuracy on a bounded sample (rank 0, N = 1) ----
    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        target = args.cpu_sample * wl.nmodes if args.cpu_sample else (1.2e10 if L >= 1024 else 1e9)
        sample = oracle_sample(wl, target)
        npts = sum(s[0].shape[0] for s in sample)
        ref, dt = run_oracle(sample, L, nfield)
        cpu = {"value": npts * wl.nmodes / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"first {npts} points of the workload (proportional per catalog), all {wl.nmodes} "
                         f"modes, {dt:.1f} s"}
        import oracle
        scats = [ops.Cat(torch.from_numpy(np.ascontiguousarray(x)).to(dev), torch.from_numpy(np.ascontiguousarray(p)).to(dev),
                         torch.from_numpy(np.ascontiguousarray(w)).to(dev), f, co) for (x, p, w, co, f) in sample]
        a = (ops.alm_interp(plan, scats, nfield, nt) if prec == "interp" else
             ops.alm_raw(plan, scats, nfield, prec)).cpu().numpy()
        errs = []
        for f in range(nfield):
            tot = oracle.cl(ref[f], ref[f], L)
            errs.append(float(np.max(np.abs(oracle.cl(a[f], a[f], L)[1:] - tot[1:]) / tot[1:])))
        accuracy = {"cl_err_vs_fp64_oracle": max(errs), "alm_rel_err_per_l": max(
            oracle.rel_err_per_l(a[f], ref[f], L) for f in range(nfield)),
            "sample_points": npts, "definition": "max over 1<=l<=lmax of |C_l - C_l^ref| / C_l^ref"}
        ladder_sample = (sample, ref[0]) if nfield == 1 else None
    adjoint = None
    if rank == 0 and world == 1 and not args.no_adjoint and prec in ("fp32", "fp64") and coef is None:
        adjoint = adjoint_measure(plan, cats, nfield, prec, out, ws, edges, L, peak, peak_src)
    coupling = None
    if rank == 0 and world == 1 and not args.no_coupling and prec == "fp32" and coef is None:
        coupling = coupling_measure(plan, wl, dev, L)
    spin2 = None
    if rank == 0 and world == 1 and not args.no_spin2 and prec == "fp32" and coef is None:
        spin2 = spin2_measure(plan, wl, dev, L, peak, peak_src)
    skipped = None
    if prec == "fp32" and coef is None:
        # fraction of (point, m, l) accumulation steps skipped below the FP32 range (one untimed call)
        cnt = torch.zeros(2, dtype=torch.int64, device=dev)
        plan.set_skip_counters(cnt)
        ops.alm_raw(plan, cats, nfield, prec, out=out, workspace=ws)
        torch.cuda.synchronize()
        plan.set_skip_counters(None)
        plan.check()
        c = cnt.cpu().tolist()
        skipped = {"fraction": c[0] / max(1, c[1]), "blocks_skipped": c[0], "blocks": c[1],
                   "what": "16-step recurrence blocks of a warp whose points were all below the FP32 range: "
                           "accumulation not executed (exact zeros), counted by the kernel"}
    batched = None
    if rank == 0 and world == 1 and not args.no_batched and prec == "fp32" and args.config == 3:
        batched = batched_measure(dev, peak, peak_src)
    ladder = None
    if rank == 0 and world == 1 and not args.no_ladder and prec == "fp32" and wl.nfield == 1:
        ladder = precision_ladder(wl, plan, dev, value, accuracy["cl_err_vs_fp64_oracle"] if accuracy else None,
                                  ladder_sample if accuracy else None)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "interp": "f32 + f16 hi/lo"}[prec],
            "data": "synthetic",
            "config": {"workload": workload_name(wl, args), "points": wl.npoints, "lmax": L, "nmodes": wl.nmodes,
                       "fields": nfield, "l2": "inputs larger than L2 (prepared points 24 B x 1e7 = 240 MB)",
                       "modes_counted": "nominal (lmax+1)(lmax+2)/2 per point; accumulation skipped in 16-step "
                                        "blocks where every point of a warp is below the FP32 range (exact zeros)",
                       "accumulation_skipped": skipped,
                       "parallelism": f"points sharded over {world} GPU(s), one all-reduce of a_lm",
                       "cuda_graph": bool(gstep is not None)},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": None,  # DRAM bytes come from an ncu capture, not from this run
                         "kernel": ("analysis_kernel (FP64, 4 points/lane, 4 warps/CTA)" if prec == "fp64" else
                                    "interpolated route: sort, ip_bin, ip_fold, analysis_mixed_kernel<8> table "
                                    "mode, combine (timed together; algorithmic flops against the FP32 peak)"
                                    if prec == "interp" else
                                    "analysis_kernel (FP32, 16 points/lane in f32x2 pairs, 4 warps/CTA)"),
                         "kernel_ms": kms,
                         "peak_source": peak_src},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
            "accuracy": accuracy,
            "precision_ladder": ladder,
            "adjoint": adjoint,
            "coupling": coupling,
            "spin2": spin2,
            "batched": batched,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def coupling_terms(L: int, Lw: int) -> int:
    """Terms of Eq. chat the coupling kernel sums: pairs l <= l' <= L, lambda
    from l' - l to min(l + l', Lw) in steps of 2 (the parity of l + l')."""
    import numpy as np
    lp = np.arange(L + 1)
    tot = 0
    for l in range(L + 1):
        q = lp[l:]
        hi = np.minimum(l + q, Lw)
        lo = q - l
        hi = hi - ((hi - lo) % 2)
        tot += int(np.sum(np.where(hi >= lo, (hi - lo) // 2 + 1, 0)))
    return tot


def coupling_measure(plan, wl, dev, L):
    """The mode-coupling row (Sec. 2.1): W_l of the workload's randoms (scaled
    by alpha) up to lmax, then M_ll' (Eq. chat) for 0 <= l, l' <= lmax, timed
    with CUDA events (one warm-up, three timed calls).  FP64 pipe bound: per
    term one multiply and one FMA = 3 flops."""
    import torch

    from paper_2312_12285_gb300 import ops
    rnd = [c for c in wl.catalogs if c.name == "randoms"]
    if not rnd:
        return None
    c = rnd[0]
    cat = ops.Cat(torch.from_numpy(c.x).to(dev), torch.from_numpy(c.phi).to(dev), torch.from_numpy(c.w).to(dev), 0,
                  abs(c.coeff))
    W = ops.window_cl(plan, [cat], "fp32", subtract_noise=True)
    M = ops.coupling(W, L)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        ops.coupling(W, L)
    e1.record()
    torch.cuda.synchronize()
    plan.check()
    ms = e0.elapsed_time(e1) / 3
    terms = coupling_terms(L, L)
    ach = 3.0 * terms / (ms / 1e3) / 1e12
    return {"value": terms / (ms / 1e3), "unit": "3j terms/s", "ms": ms, "terms": terms, "lmax": L, "lmax_w": L,
            "finite": bool(torch.isfinite(M).all()),
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                         "frac": ach / FP64_TFLOPS_NOMINAL,
                         "kernel": "cp_coupling_kernel (FP64: one multiply + one FMA per term)",
                         "peak_source": "nominal FP64 1.25 TFLOP/s"},
            "what": "M_ll' (Eq. chat) from the randoms' window spectrum, lmax = lmax_w = workload lmax"}


def spin2_measure(plan, wl, dev, L, peak, peak_src):
    """The spin-2 row: E_lm, B_lm of a synthetic shear field (a smooth
    random-wave pattern plus shape noise, seeded) carried by the workload's
    galaxies, lmax = workload lmax, timed with CUDA events (one warm-up, one
    timed call).  Algorithmic flops per point x mode, both spins: recurrence
    2 x (t = A' x + B': 2, tau = t p1 + p2: 2) = 8, accumulation 2 x 2 FMA = 8."""
    import numpy as np
    import torch

    from paper_2312_12285_gb300 import ops
    gal = [c for c in wl.catalogs if c.name == "galaxies"]
    if not gal:
        return None
    g = gal[0]
    rng = np.random.default_rng(31)
    th = np.arccos(g.x.astype(np.float64))
    g1 = (0.05 * np.cos(7 * th + 3 * g.phi) + 0.2 * rng.standard_normal(g.n)).astype(np.float32)
    g2 = (0.05 * np.sin(5 * th - 2 * g.phi) + 0.2 * rng.standard_normal(g.n)).astype(np.float32)
    cat = ops.ShearCat(*(torch.from_numpy(a).to(dev) for a in (g.x, g.phi, g.w, g1, g2)), 0, 1.0)
    E, B = ops.alm_spin2(plan, [cat], 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ops.alm_spin2(plan, [cat], 1)
    e1.record()
    torch.cuda.synchronize()
    plan.check()
    ms = e0.elapsed_time(e1)
    nm = (L + 1) * (L + 2) // 2
    pm = g.n * nm / (ms / 1e3)
    ach = 16.0 * pm / 1e12
    return {"value": pm, "unit": UNIT + " (E and B)", "ms": ms, "points": g.n, "lmax": L,
            "finite": bool(torch.isfinite(E).all() and torch.isfinite(B).all()),
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "kernel": "s2_analysis_kernel (one f32x2 recurrence per point for both spins, "
                                   "16 flops per point x mode)", "peak_source": peak_src},
            "what": "E_lm, B_lm of a synthetic shear field on the workload's galaxies (Sec. 4 spin-2 variant)"}


def adjoint_measure(plan, cats, nfield, prec, out, ws, edges, L, peak, peak_src):
    """The adjoint row: gradient of L = sum_b g_b C_b (32 log-spaced bandpowers,
    shot noise removed) with respect to every weight, i.e. bin_backward ->
    cl_backward -> alm_backward (the point-evaluation synthesis kernel), timed
    with CUDA events after one warm-up."""
    import numpy as np
    import torch

    from paper_2312_12285_gb300 import catalogs, ops
    a = ops.alm_raw(plan, cats, nfield, prec, out=out, workspace=ws)
    noise = ops.shot_noise_raw(cats, nfield, prec, a.device, workspace=ws)
    a = a.clone()
    gb = torch.from_numpy(catalogs.rng_for(5, 7).standard_normal((nfield * (nfield + 1) // 2, edges.shape[0] - 1))
                          ).to(a.device)

    def backward():
        gcl = ops.bin_backward_raw(gb, edges, L)
        galm, gnoise = ops.cl_backward_raw(a, gcl, want_noise=True)
        return ops.alm_backward_raw(plan, cats, nfield, prec, galm, gnoise, workspace=ws)

    backward()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    grads = backward()
    e1.record()
    torch.cuda.synchronize()
    plan.check()
    ms = e0.elapsed_time(e1)
    npts = sum(int(c.x.shape[0]) for c in cats)
    nm = (L + 1) * (L + 2) // 2
    ach = FLOPS_PER_POINT_MODE * npts * nm / (ms / 1e3) / 1e12
    finite = bool(all(torch.isfinite(g).all() for g in grads))
    return {"value": npts * nm / (ms / 1e3), "unit": UNIT, "ms": ms, "grad_finite": finite,
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "kernel": ("adjoint_sorted_kernel (|x|-sorted, packed f32x2" if prec == "fp32" else
                                    "adjoint_kernel (catalog order") +
                                   "; point-evaluation synthesis, 7 flops per point x mode: "
                                   "recurrence 3, accumulation 4)", "peak_source": peak_src},
            "what": "d(sum_b g_b C_b)/dw_i for every object: bin_backward, cl_backward, alm_backward"}


# ------------------------------------------------------- weight columns --
def mixed_mma_flops_per_point_mode(F: int) -> float:
    """Tensor-core flops the mixed kernel issues per point x mode of one pass:
    per 16 points x 8 multipoles, 2 (4-column kernel) or 3 (8-column kernel)
    m16n8k16 MMAs of 2 x 16 x 8 x 16 flops."""
    nmma = 2 if F <= 4 else 3
    return nmma * 2 * 16 * 8 * 16 / (16 * 8)


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def time_columns(plan, xd, pd, Wd, prec, reps, warm=1):
    """Device time (ms) of pointsht_alm_columns: whole call and kernel(s) alone."""
    import torch

    from paper_2312_12285_gb300 import ops
    n, F = int(xd.shape[0]), int(Wd.shape[0])
    ws = torch.empty(max(256, ops.workspace_bytes_columns(plan, n, F, prec)), dtype=torch.uint8, device=xd.device)
    out = torch.empty((F, plan.nmodes), dtype=torch.complex128, device=xd.device)
    for _ in range(warm):
        ops.alm_columns(plan, xd, pd, Wd, prec, out=out, workspace=ws)
    torch.cuda.synchronize()
    evk = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a_, b_ in evk:
        a_.record()
        b_.record()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(reps):
        plan.set_timing_events(evk[k][0], evk[k][1])
        ops.alm_columns(plan, xd, pd, Wd, prec, out=out, workspace=ws)
    e1.record()
    torch.cuda.synchronize()
    plan.set_timing_events(None, None)
    plan.check()
    return e0.elapsed_time(e1) / reps, sum(a.elapsed_time(b) for a, b in evk) / reps, out


def batched_measure(dev, peak, peak_src, steps_fp32=2, steps_interp=5, cpu_pm=1.0e10):
    """The batching workload: 16 tomographic bins of uneven sizes (10^U[5,7]
    galaxies) plus 2e7 shared randoms, lmax 1536, all 17 source fields in one
    call, combined into the 16 FKP fields D_b - alpha_b R (Sec. 2.1), all 136
    auto and cross pseudo-C_l with shot noise removed.  Timed through the plain
    FP32 path (the whole step captured in one CUDA graph) and through the
    interpolated route (tensor-core contraction of theta-sample tables,
    ntheta from the 1e-4 C_l budget); each with its device time, an end-to-end
    time through the public API with host buffers, its roofline, and its C_l
    error against the FP64 oracle on a bounded sample of the workload."""
    import numpy as np
    import torch

    import oracle
    from paper_2312_12285_gb300 import catalogs, ops
    wl = catalogs.config(4)
    L, M = wl.lmax, wl.nmodes
    nb = wl.extra["nbins"]
    nsrc = wl.nfield
    cm = np.zeros((nb, nsrc))
    for b in range(nb):
        cm[b, b] = 1.0
        cm[b, nb] = -wl.extra["alpha"][b]
    coef = torch.from_numpy(cm).to(dev)
    host = [tuple(torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for v in (c.x, c.phi, c.w))
            for c in wl.catalogs]
    cats = [ops.Cat(h[0].to(dev), h[1].to(dev), h[2].to(dev), c.field, c.coeff) for h, c in zip(host, wl.catalogs)]
    plan = ops.get_plan(L, dev)
    h2d = sum(sum(t.numel() * t.element_size() for t in h) for h in host)
    npair = nb * (nb + 1) // 2
    cl_h = torch.empty((npair, L + 1), dtype=torch.float64).pin_memory()
    total_pm = wl.npoints * M
    res = {"workload": f"tomographic: 16 bins ({min(c.n for c in wl.catalogs[:nb])}..{max(c.n for c in wl.catalogs[:nb])} "
                       f"galaxies) + 2e7 shared randoms = {wl.npoints} points, lmax {L}, 17 source fields -> "
                       f"{nb} FKP fields, {npair} spectra",
           "points": wl.npoints, "lmax": L, "unit": UNIT}

    def timed(fn, steps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        plan.check()
        return e0.elapsed_time(e1) / steps

    # ---- plain FP32 path, one CUDA graph per step ----
    step = ops.GraphStep(ops.make_pipeline(plan, cats, nsrc, "fp32", coef=coef), warmup=1)
    ms = timed(step.replay, steps_fp32)
    dcats = [ops.Cat(torch.empty_like(c.x), torch.empty_like(c.phi), torch.empty_like(c.w), c.field, c.coeff)
             for c in cats]
    fn_e2e = ops.make_pipeline(plan, dcats, nsrc, "fp32", coef=coef)

    def e2e_fp32():
        for h, d in zip(host, dcats):
            d.x.copy_(h[0], non_blocking=True)
            d.phi.copy_(h[1], non_blocking=True)
            d.w.copy_(h[2], non_blocking=True)
        cl_h.copy_(fn_e2e()[0], non_blocking=True)
    ems = timed(e2e_fp32, 1)
    del fn_e2e
    ach = FLOPS_PER_POINT_MODE * total_pm / (ms / 1e3) / 1e12
    res["fp32"] = {"value": total_pm / (ms / 1e3), "ms_per_step": ms,
                   "e2e": {"value": total_pm / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                           "d2h_bytes_per_step": int(cl_h.numel() * 8), "ms_per_step": ems},
                   "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                                "traffic": None, "peak_source": peak_src,
                                "kernel": "analysis_kernel (FP32, one persistent launch over all 17 fields), "
                                          "timed as the whole graph step"},
                   "gpu_launches_per_step": 12}
    del step
    # ---- interpolated route ----
    nt = ops.ntheta_for_tolerance(L, 1e-4)
    wsi = torch.empty(ops.workspace_bytes_interp(plan, cats, nsrc, nt), dtype=torch.uint8, device=dev)
    outi = torch.empty((nsrc, plan.nmodes), dtype=torch.complex128, device=dev)
    nws = torch.empty(512 * len(cats) + 256, dtype=torch.uint8, device=dev)

    def istep(cs=cats):
        a = ops.alm_interp(plan, cs, nsrc, nt, out=outi, workspace=wsi)
        noise = ops.shot_noise_raw(cs, nsrc, "fp32", dev, workspace=nws)
        af, nf = ops.combine_raw(a, coef, noise)
        return ops.cl_raw(af, nf)
    ims = timed(istep, steps_interp)

    def e2e_interp():
        for h, d in zip(host, dcats):
            d.x.copy_(h[0], non_blocking=True)
            d.phi.copy_(h[1], non_blocking=True)
            d.w.copy_(h[2], non_blocking=True)
        cl_h.copy_(istep(dcats), non_blocking=True)
    iems = timed(e2e_interp, steps_interp)
    iach = (22.0 * wl.npoints * (L + 1) + 27.0 * nt * M * nsrc) / (ims / 1e3) / 1e12
    res["interp"] = {"value": total_pm / (ims / 1e3), "ms_per_step": ims, "ntheta": nt,
                     "ntheta_rule": "smallest even N with 4.3e-6 (16 lmax / N)^4 <= 1e-4 / 4 (h^4 model)",
                     "e2e": {"value": total_pm / (iems / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                             "d2h_bytes_per_step": int(cl_h.numel() * 8), "ms_per_step": iems},
                     "roofline": {"bound": "alu", "achieved": iach, "peak": peak, "unit": "TFLOP/s",
                                  "frac": iach / peak, "traffic": None, "peak_source": peak_src,
                                  "kernel": "interpolated route (sort, ip_bin, ip_fold, analysis_mixed_kernel<8> "
                                            "table mode per field, reduce, combine), algorithmic flops: 22 per "
                                            "(point, m) binning + 27 per (sample, mode) per field"}}
    res["interp_speedup_vs_fp32"] = res["interp"]["value"] / res["fp32"]["value"]
    del wsi, outi, dcats
    # ---- C_l error of both routes against the FP64 oracle on a bounded sample ----
    sample = oracle_sample(wl, cpu_pm)
    t0 = time.perf_counter()
    ref = [oracle.alm(x, p, w.astype(np.float64), L) for (x, p, w, co, f) in sample]
    cpu_s = time.perf_counter() - t0
    scats = [ops.Cat(*(torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (x, p, w)), f, co)
             for (x, p, w, co, f) in sample]
    alpha = wl.extra["alpha"]
    fk = [ref[b] - alpha[b] * ref[nb] for b in range(nb)]
    tot = [oracle.cl(fk[b], fk[b], L) for b in range(nb)]
    noise_s = ops.shot_noise_raw(scats, nsrc, "fp32", dev)

    def cl_err(a_src):
        af, nf = ops.combine_raw(a_src, coef, noise_s)
        cl = ops.cl_raw(af, nf).cpu().numpy()
        nfh = nf.cpu().numpy()
        worst, p_ = 0.0, 0
        for f in range(nb):
            for g in range(f, nb):
                want = oracle.cl(fk[f], fk[g], L) - nfh[f, g]
                worst = max(worst, float(np.max(np.abs(cl[p_][1:] - want[1:]) / np.sqrt(tot[f][1:] * tot[g][1:]))))
                p_ += 1
        return worst
    res["fp32"]["cl_err_vs_fp64_oracle"] = cl_err(ops.alm_raw(plan, scats, nsrc, "fp32"))
    res["interp"]["cl_err_vs_fp64_oracle"] = cl_err(ops.alm_interp(plan, scats, nsrc, nt))
    plan.check()
    npts = sum(s[0].shape[0] for s in sample)
    res["cl_err_definition"] = ("max over the 136 pairs (f, g) and 1 <= l <= lmax of |C_l^fg - ref| / "
                                "sqrt(C_l^ff C_l^gg) (totals before shot-noise subtraction)")
    res["oracle_sample"] = f"first {npts} points of every catalog in proportion, all {M} modes, {cpu_s:.1f} s"
    del cats, host
    return res


def precision_ladder(wl, plan, dev, fp32_value, fp32_cl_err, sample):
    """Mixed path for F = 1, 4, 8 weight columns on the workload's point set
    (per-column throughput, speed-up over the plain FP32 path at the same F,
    C_l error against the FP64 oracle on the bench sample), the interpolated
    route on the whole workload, and the FP64 path on a 1% subsample."""
    import numpy as np
    import torch

    import oracle
    from paper_2312_12285_gb300 import catalogs, ops
    L, M = wl.lmax, wl.nmodes
    res = {"F": [], "mixed_value": [], "mixed_kernel_ms": [], "fp32_value": [],
           "speedup_vs_fp32": [], "unit": "columns x " + UNIT}
    for F in (1, 4, 8):
        x, phi, W = catalogs.weight_columns(wl, F)
        n = x.shape[0]
        xd, pd, Wd = (torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (x, phi, W))
        ms, kms, _ = time_columns(plan, xd, pd, Wd, "mixed", reps=1)
        v = F * n * M / (ms / 1e3)  # column x point x mode throughput
        f32 = fp32_value
        if F == 4:
            fms, _, _ = time_columns(plan, xd, pd, Wd, "fp32", reps=1, warm=0)
            f32 = F * n * M / (fms / 1e3)
        res["F"].append(F)
        res["mixed_value"].append(v)
        res["mixed_kernel_ms"].append(kms)
        res["fp32_value"].append(f32)
        res["speedup_vs_fp32"].append(v / f32)
        del xd, pd, Wd
    res["fp32_value_note"] = ("F = 1 and 8: the catalog-form FP32 measurement of this line (the plain "
                                        "path runs one transform per column); F = 4: measured through "
                                        "pointsht_alm_columns with POINTSHT_FP32")
    # accuracy of the mixed path (the workload's field as one column) on the bench sample
    if sample is not None:
        smp, ref = sample
        xs = np.concatenate([c[0] for c in smp]).astype(np.float32)
        ps = np.concatenate([c[1] for c in smp]).astype(np.float32)
        ws_ = np.concatenate([(c[2].astype(np.float64) * c[3]) for c in smp]).astype(np.float32)
        a = ops.alm_columns(plan, torch.from_numpy(xs).to(dev), torch.from_numpy(ps).to(dev),
                            torch.from_numpy(ws_[None, :].copy()).to(dev), "mixed").cpu().numpy()[0]
        tot = oracle.cl(ref, ref, L)
        res["mixed_cl_err_vs_fp64_oracle"] = float(np.max(np.abs(oracle.cl(a, a, L)[1:] - tot[1:]) / tot[1:]))
        res["mixed_alm_rel_err_per_l"] = oracle.rel_err_per_l(a, ref, L)
    res["fp32_cl_err_vs_fp64_oracle"] = fp32_cl_err
    # interpolated route (App. "Interpolation", samples in theta), whole workload
    cats = [ops.Cat(*(torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (c.x, c.phi, c.w)), c.field,
                    c.coeff) for c in wl.catalogs]
    nt = ops.ntheta_for_tolerance(L, 1e-4)
    wsi = torch.empty(ops.workspace_bytes_interp(plan, cats, wl.nfield, nt), dtype=torch.uint8, device=dev)
    outi = ops.alm_interp(plan, cats, wl.nfield, nt, workspace=wsi)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        ops.alm_interp(plan, cats, wl.nfield, nt, out=outi, workspace=wsi)
    e1.record()
    torch.cuda.synchronize()
    plan.check()
    ims = e0.elapsed_time(e1) / 3
    res["interp_value"] = wl.npoints * M / (ims / 1e3)
    res["interp_ms"] = ims
    res["interp_ntheta"] = nt
    res["interp_speedup_vs_fp32"] = res["interp_value"] / fp32_value
    del wsi, outi, cats
    if sample is not None:
        scats = [ops.Cat(*(torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (c[0], c[1], c[2])), 0, c[3])
                 for c in smp]
        a = ops.alm_interp(plan, scats, 1, nt).cpu().numpy()[0]
        res["interp_cl_err_vs_fp64_oracle"] = float(np.max(np.abs(oracle.cl(a, a, L)[1:] - tot[1:]) / tot[1:]))
        res["interp_alm_rel_err_per_l"] = oracle.rel_err_per_l(a, ref, L)
    # FP64 path (catalog form) on the first 1% of every catalog
    sub = [ops.Cat(*(torch.from_numpy(np.ascontiguousarray(v[:max(1, c.n // 100)].astype(np.float64))).to(dev)
                     for v in (c.x, c.phi, c.w)), c.field, c.coeff) for c in wl.catalogs]
    nsub = sum(int(c.x.shape[0]) for c in sub)
    ops.alm_raw(plan, sub, wl.nfield, "fp64")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ops.alm_raw(plan, sub, wl.nfield, "fp64")
    e1.record()
    torch.cuda.synchronize()
    res["fp64_value"] = nsub * M / (e0.elapsed_time(e1) / 1e3)
    res["fp64_sample_points"] = nsub
    res["mixed_vs_fp64"] = [v / res["fp64_value"] for v in res["mixed_value"]]
    return res


def ours_columns(args):
    """F weight columns on the workload's point set through pointsht_alm_columns
    (jackknife columns of the field: column 0 the field, column k the field with
    the k-th of F-1 azimuthal wedges removed), then shot noise, C_l of all
    column pairs and bandpowers.  value = F x points x modes / s."""
    import numpy as np
    import torch

    from paper_2312_12285_gb300 import catalogs, ops
    from paper_2312_12285_gb300.sharding import allreduce_sum, shard_array as shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    prec = args.precision if args.precision in ("mixed", "fp32") else "mixed"
    F = max(1, args.columns)
    wl = load_workload(args)
    L, M = wl.lmax, wl.nmodes
    x, phi, W = catalogs.weight_columns(wl, F)
    xs, ps = shard(x, rank, world), shard(phi, rank, world)
    Ws = np.ascontiguousarray(np.stack([shard(W[f], rank, world) for f in range(F)]))
    n_rank = xs.shape[0]
    xd, pd, Wd = (torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (xs, ps, Ws))
    plan = ops.get_plan(L, dev)
    plan.set_mixed_kernel(args.mixed_kernel)
    ws = torch.empty(max(256, ops.workspace_bytes_columns(plan, n_rank, F, prec)), dtype=torch.uint8, device=dev)
    wsn = torch.empty(512 * F + 256, dtype=torch.uint8, device=dev)
    out = torch.empty((F, M), dtype=torch.complex128, device=dev)
    edges = torch.from_numpy(catalogs.log_bin_edges(L, 32).astype(np.int32)).to(dev)

    def step(xd=xd, pd=pd, Wd=Wd):
        a = ops.alm_columns(plan, xd, pd, Wd, prec, out=out, workspace=ws)
        noise = ops.shot_noise_raw([ops.Cat(xd, pd, Wd[f], f, 1.0) for f in range(F)], F, "fp32", dev, workspace=wsn)
        if dist is not None:
            allreduce_sum([a, noise])
        cl = ops.cl_raw(a, noise)
        return cl, ops.bin_raw(cl, edges)

    npass = (F + 7) // 8
    # mixed: hist, scan, pad, scatter + (analysis, reduce) per pass; fp32: pads, hist, scan, scatter, analysis,
    # reduce; then 2 x shot noise, C_l, bins
    launches_per_step = (4 + 2 * npass + 4) if prec == "mixed" else (6 + 4)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    plan.check()
    evk = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a_, b_ in evk:
        a_.record()
        b_.record()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0.record()
    for k in range(args.steps):
        plan.set_timing_events(evk[k][0], evk[k][1])
        step()
    e1.record()
    torch.cuda.synchronize()
    plan.set_timing_events(None, None)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    kms = sum(a.elapsed_time(b) for a, b in evk) / args.steps
    if dist is not None:
        t = torch.tensor([ms, kms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, kms = float(t[0]), float(t[1])
    plan.check()
    total = F * wl.npoints * M
    value = total / (ms / 1e3)
    peaks = measured_peaks()
    if prec == "mixed":
        bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
        src = ("measured bf16_tflops_sustained (MEASURED_PEAKS.json; fp16 has the bf16 rate)" if bf16 else
               "fallback 1.7 PFLOP/s sustained bf16 (fp16 has the bf16 rate)")
        bf16 = bf16 or 1700.0
        per_pass = [min(8, F - 8 * i) for i in range(npass)]
        if args.mixed_kernel == "mma.sync":
            flops_pm = sum(mixed_mma_flops_per_point_mode(c) for c in per_pass)
        else:
            # tcgen05: per 16 points x 32 multipoles two M = 128, N = 32, K = 16 MMAs (hi, lo'),
            # whatever the number of columns (rows beyond 4 F are zero)
            flops_pm = npass * 2 * (2 * 128 * 32 * 16) / (16 * 32)
        achieved = flops_pm * n_rank * M / (kms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": bf16, "unit": "TFLOP/s", "frac": achieved / bf16,
                "traffic": None, "kernel": ("analysis_mixed_kernel (mma.sync m16n8k16 fp16 hi+lo, FP32 recurrence)"
                                            if args.mixed_kernel == "mma.sync" else
                                            f"analysis_tc_kernel ({args.mixed_kernel}: tcgen05.mma M=128 fp16 hi+lo, "
                                            "TMEM accumulators, FP32 recurrence)"),
                "kernel_ms": kms, "peak_source": src,
                "note": "tensor flops issued (hi x hi + lo x hi + hi x lo products, 16-row MMAs); the kernel is "
                        "bound by the FP32 recurrence and the fp16 split on the FP32/ALU pipes, not by the tensor pipe"}
    else:
        props = torch.cuda.get_device_properties(dev)
        peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * (peaks.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
        achieved = FLOPS_PER_POINT_MODE * F * n_rank * M / (kms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": "analysis_kernel (FP32)", "kernel_ms": kms,
                "peak_source": "derived: SMs x 128 FP32 lanes x 2 flop x max SM clock"}

    e2e = None
    if not args.no_e2e:
        hx, hp, hW = (torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for v in (xs, ps, Ws))
        cl_h = torch.empty((F * (F + 1) // 2, L + 1), dtype=torch.float64).pin_memory()
        cb_h = torch.empty((F * (F + 1) // 2, 32), dtype=torch.float64).pin_memory()
        dx, dp, dW = torch.empty_like(xd), torch.empty_like(pd), torch.empty_like(Wd)

        def e2e_step():
            dx.copy_(hx, non_blocking=True)
            dp.copy_(hp, non_blocking=True)
            dW.copy_(hW, non_blocking=True)
            cl, cb = step(dx, dp, dW)
            cl_h.copy_(cl, non_blocking=True)
            cb_h.copy_(cb, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for _ in range(args.steps):
            e2e_step()
        s1.record()
        torch.cuda.synchronize()
        ems = s0.elapsed_time(s1) / args.steps
        if dist is not None:
            t = torch.tensor([ems], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t[0])
        h2d = sum(t.numel() * t.element_size() for t in (hx, hp, hW))
        e2e = {"value": total / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int((cl_h.numel() + cb_h.numel()) * 8), "ms_per_step": ems}

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        target = args.cpu_sample * M if args.cpu_sample else (1.2e10 if L >= 1024 else 1e9)
        npts = max(1, int(target / M / F))
        t0 = time.perf_counter()
        refs = [oracle.alm(x[:npts], phi[:npts], W[f, :npts], L) for f in range(F)]
        dt = time.perf_counter() - t0
        cpu = {"value": F * npts * M / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"first {npts} points of the point set, {F} weight columns, all {M} modes, {dt:.1f} s"}
        a = ops.alm_columns(plan, torch.from_numpy(x[:npts].copy()).to(dev), torch.from_numpy(phi[:npts].copy()).to(dev),
                            torch.from_numpy(np.ascontiguousarray(W[:, :npts])).to(dev), prec).cpu().numpy()
        errs = []
        for f in range(F):
            tot = oracle.cl(refs[f], refs[f], L)
            errs.append(float(np.max(np.abs(oracle.cl(a[f], a[f], L)[1:] - tot[1:]) / tot[1:])))
        accuracy = {"cl_err_vs_fp64_oracle": max(errs),
                    "alm_rel_err_per_l": max(oracle.rel_err_per_l(a[f], refs[f], L) for f in range(F)),
                    "sample_points": npts,
                    "definition": "max over columns and 1<=l<=lmax of |C_l - C_l^ref| / C_l^ref"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f16 hi+lo, f32 acc" if prec == "mixed" else "f32", "data": "synthetic",
            "config": {"workload": workload_name(wl, args) + f", {F} weight columns (jackknife: the field, and "
                                                              f"the field minus each of {max(1, F - 1)} azimuthal "
                                                              f"wedges)",
                       "points": wl.npoints, "lmax": L, "nmodes": M, "columns": F,
                       "l2": "inputs larger than L2", "value_counts": "columns x points x modes",
                       "parallelism": f"points sharded over {world} GPU(s), one all-reduce of a_lm"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks, "accuracy": accuracy,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def spawn_ranks(args) -> int:
    """--gpus N > 1 outside torchrun: start N ranks on this node, one per GPU
    (torch.distributed.run, rendezvous on 127.0.0.1), and return their exit
    status; an error if this node has fewer than N GPUs."""
    import socket

    import torch
    if torch.cuda.device_count() < args.gpus:
        print(json.dumps({"error": f"--gpus {args.gpus}: this node has {torch.cuda.device_count()} GPU(s)"}),
              flush=True)
        return 2
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(spawn_ranks(args))
    if args.impl == "reference":
        reference_arm(args)
    elif args.columns > 0 or args.precision == "mixed":
        ours_columns(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
