"""Autotuner for the FP32 analysis kernel: picks the kernel variant and the
accumulation chunk size by timing candidates on the caller's own catalogs (a
bounded subsample of them), and caches the choice per (device, lmax,
precision, fields, size bucket) in a JSON file.

Cache file: $POINTSHT_TUNING_CACHE, else ~/.cache/pointsht/tuning.json.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import ops

# (variant, chunk_log2); variant as in pointsht_plan_set_tuning
# Only the default variant (116) carries the near-pole form of the recurrence,
# so the tuner varies the accumulation chunk.
CANDIDATES = [(116, 0), (116, 16), (116, 18), (116, 20)]


def cache_path() -> str:
    return os.environ.get("POINTSHT_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pointsht", "tuning.json"))


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _save(d):
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def key(plan: ops.Plan, cats, nfield: int, precision: str) -> str:
    n = sum(int(c.x.shape[0]) for c in cats)
    props = torch.cuda.get_device_properties(plan.device)
    return (f"{props.name}|sm{props.major}{props.minor}|L{plan.lmax}|{precision}|F{nfield}|"
            f"N2^{int(round(math.log2(max(n, 1))))}")


def _subsample(cats, max_points: int):
    n = sum(int(c.x.shape[0]) for c in cats)
    if n <= max_points:
        return cats
    frac = max_points / n
    out = []
    for c in cats:
        k = max(1, int(c.x.shape[0] * frac))
        out.append(ops.Cat(c.x[:k].contiguous(), c.phi[:k].contiguous(), c.w[:k].contiguous(), c.field, c.coeff))
    return out


def tune(plan: ops.Plan, cats, nfield: int = 1, precision: str = "fp32", reps: int = 2,
         target_point_modes: float = 2e12, force: bool = False, candidates=CANDIDATES):
    """Choose and set the plan's tuning for these catalogs; returns
    (variant, chunk_log2, {candidate: ms})."""
    if precision == "fp64":
        return 0, 0, {}
    k = key(plan, cats, nfield, precision)
    cache = _load()
    if not force and k in cache:
        v, c = cache[k]["variant"], cache[k]["chunk_log2"]
        plan.set_tuning(v, c)
        return v, c, cache[k].get("ms", {})
    sub = _subsample(cats, max(32_768, int(target_point_modes / plan.nmodes)))
    out = torch.empty((nfield, plan.nmodes), dtype=torch.complex128, device=plan.device)
    times = {}
    for v, c in candidates:
        plan.set_tuning(v, c)
        ws = torch.empty(ops.workspace_bytes(plan, sub, nfield, precision), dtype=torch.uint8, device=plan.device)
        ops.alm_raw(plan, sub, nfield, precision, out=out, workspace=ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ops.alm_raw(plan, sub, nfield, precision, out=out, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        times[f"{v}/{c}"] = e0.elapsed_time(e1) / reps
        del ws
    best = min(times, key=times.get)
    v, c = (int(t) for t in best.split("/"))
    plan.set_tuning(v, c)
    cache[k] = {"variant": v, "chunk_log2": c, "ms": times}
    _save(cache)
    return v, c, times
