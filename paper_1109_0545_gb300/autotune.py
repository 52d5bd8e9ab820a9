"""Autotuners of the evaluation kernel's tile shape and of the path tracker's shape.

The evaluation kernel (one lane per point) splits its work into tasks of one 32-point
tile times a group of rows, run by persistent warps.  Two knobs set the shape:
``rows_per_task`` (polynomials per task: smaller tasks balance the SMs better, larger
ones keep a tile's points in L1 longer) and ``blocks_per_sm`` (resident 4-warp blocks,
capped by register occupancy).  The autotuner times ``hc_eval_jac`` on the caller's own
system and points for each candidate, keeps the fastest, and caches the choice per
(GPU, system shape, precision, point count) in a JSON file.

Every candidate computes bit-identical results: a point's arithmetic does not depend
on how tasks are cut (the summation order is per point), which the tests check.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

from . import hc

CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1109_0545_gb300", "autotune.json")
ROWS = (0, 1, 2, 4, 8, 16)
BLOCKS = (0, 2, 3, 4, 6, 8)


def _key(gpu: str, info: dict, npts: int, jac: bool) -> str:
    shape = f"{gpu}|n{info['n']}|p{info['npoly']}|m{info['nmon']}|v{info['nvar']}|L{info['prec']}|e{info['max_exp']}|{npts}|{int(jac)}"
    return hashlib.sha1(shape.encode()).hexdigest()[:16] + "|" + shape


def _load_cache() -> dict:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save_cache(c: dict) -> None:
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(c, fh, indent=1)
        os.replace(tmp, CACHE)
    except OSError:
        pass


def tune_eval(sysh: "hc.System", x, f, J, npts: int, t: float = 0.5, reps: int = 2,
              use_cache: bool = True, candidates=None) -> dict:
    """Pick (rows_per_task, blocks_per_sm) for hc_eval_jac on these buffers and apply it
    with hc_set_tiles.  Returns {"rows_per_task", "blocks_per_sm", "ms", "tried"}."""
    import torch
    gpu = torch.cuda.get_device_name()
    info = sysh.info()
    key = _key(gpu, info, npts, J is not None)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        best = cache[key]
        hc.hc_set_tiles(best["rows_per_task"], best["blocks_per_sm"])
        return dict(best, cached=True)
    cands = candidates or [(r, b) for r in ROWS for b in BLOCKS]
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tried = []
    for r, b in cands:
        hc.hc_set_tiles(r, b)
        hc.hc_eval_jac(sysh, npts, t, x, f, J, stream)   # warm-up
        ms = 1e30
        for _ in range(reps):
            ev0.record(stream)
            hc.hc_eval_jac(sysh, npts, t, x, f, J, stream)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = min(ms, ev0.elapsed_time(ev1))
        tried.append({"rows_per_task": r, "blocks_per_sm": b, "ms": ms})
    best = min(tried, key=lambda d: d["ms"])
    hc.hc_set_tiles(best["rows_per_task"], best["blocks_per_sm"])
    out = {"rows_per_task": best["rows_per_task"], "blocks_per_sm": best["blocks_per_sm"],
           "ms": best["ms"], "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    if use_cache:
        cache[key] = out
        _save_cache(cache)
    return dict(out, cached=False, tried=tried)


# tracker shapes searched: threads per path block x blocks per SM (0: all that fit) x
# FP64 factors in shared (0) or global (2) memory
TRACK_TB = (64, 128, 256, 512)
TRACK_BPS = (0, 2, 3, 4, 6)
TRACK_FACTORS = (0, 2)
GRID_CHUNKS = (16, 32, 64, 128)


def _track_key(gpu: str, handles, opts, what: str) -> str:
    infos = [h.info() for h in handles]
    ns = sorted(i["n"] for i in infos)
    shape = (f"{gpu}|{what}|paths{len(handles)}|n{ns[0]}-{ns[-1]}|m{sum(i['nmon'] for i in infos)}"
             f"|L{infos[0]['prec']}|lu{opts.lu_mode}|pred{opts.predictor}|cap{opts.max_steps}")
    return hashlib.sha1(shape.encode()).hexdigest()[:16] + "|" + shape


def tune_track(handles, x0, opts, reps: int = 1, use_cache: bool = True, candidates=None) -> dict:
    """Pick (threads_per_block, blocks_per_sm, factors) of the block engine by timing
    hc_track_path on the caller's own paths (handles, start points x0, options; a stage
    cap in opts.max_steps keeps the sample short), then apply it with hc_set_track_tiles.
    Every candidate computes the same results bit for bit (tested).  Returns the choice,
    its seconds and the candidates tried."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _track_key(gpu, handles, opts, "block")
    cache = _load_cache() if use_cache else {}
    prev = hc.hc_get_track_tiles()
    if key in cache:
        best = cache[key]
        hc.hc_set_track_tiles(best["threads_per_block"], best["blocks_per_sm"], best["factors"], prev["grid_chunk"])
        return dict(best, cached=True)
    cands = candidates or [(t, b, f) for t in TRACK_TB for b in TRACK_BPS for f in TRACK_FACTORS]
    x1 = torch.zeros_like(x0)
    tried = []
    for t, b, f in cands:
        hc.hc_set_track_tiles(t, b, f, prev["grid_chunk"])
        best_s = 1e30
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hc.hc_track_path(handles, x0, x1, opts)
            best_s = min(best_s, time.perf_counter() - t0)
        tried.append({"threads_per_block": t, "blocks_per_sm": b, "factors": f, "s": best_s})
    best = min(tried, key=lambda d: d["s"])
    hc.hc_set_track_tiles(best["threads_per_block"], best["blocks_per_sm"], best["factors"], prev["grid_chunk"])
    out = {k: best[k] for k in ("threads_per_block", "blocks_per_sm", "factors", "s")}
    out["when"] = time.strftime("%Y-%m-%dT%H:%M:%S")
    if use_cache:
        cache[key] = out
        _save_cache(cache)
    return dict(out, cached=False, tried=tried)


def tune_grid_chunk(handle, x0, opts, use_cache: bool = True, candidates=GRID_CHUNKS) -> dict:
    """Pick the whole-GPU engine's chunk length by timing a few stages of hc_track_path
    (HC_TRACK_GRID, opts.max_steps stages) on the caller's path; applied with
    hc_set_track_tiles.  Returns the choice, its seconds and the candidates tried."""
    import torch
    gpu = torch.cuda.get_device_name()
    key = _track_key(gpu, [handle], opts, "grid")
    cache = _load_cache() if use_cache else {}
    prev = hc.hc_get_track_tiles()
    if key in cache:
        best = cache[key]
        hc.hc_set_track_tiles(prev["threads_per_block"], prev["blocks_per_sm"], prev["factors"], best["grid_chunk"])
        return dict(best, cached=True)
    x1 = torch.zeros_like(x0)
    tried = []
    for c in candidates:
        hc.hc_set_track_tiles(prev["threads_per_block"], prev["blocks_per_sm"], prev["factors"], c)
        hc.hc_track_path([handle], x0, x1, opts)      # warm-up (graph capture, allocation)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hc.hc_track_path([handle], x0, x1, opts)
        tried.append({"grid_chunk": c, "s": time.perf_counter() - t0})
    best = min(tried, key=lambda d: d["s"])
    hc.hc_set_track_tiles(prev["threads_per_block"], prev["blocks_per_sm"], prev["factors"], best["grid_chunk"])
    out = {"grid_chunk": best["grid_chunk"], "s": best["s"], "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    if use_cache:
        cache[key] = out
        _save_cache(cache)
    return dict(out, cached=False, tried=tried)
