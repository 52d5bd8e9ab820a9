#!/usr/bin/env python
"""Benchmark of the hot path: one Newton step (Alg. 4.1 loop body: evaluation of the
homotopy and its full Jacobian by the scheme of Sec. 6, residual, FP64 LU + DD
refinement of the Newton system, update) at every point of the eval-throughput
workload -- n = 32 unknowns, 32 polynomials x 128 monomials, 6 variables per monomial,
exponents 1..4, unit-circle coefficients, 65,536 points on the unit torus, complex
double-double -- through the C-ABI library.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  Under torchrun each rank runs its own 65,536 points
(independent problems, weak scaling, no collective on the data path); the timing is
barrier-bracketed and the max over ranks.  ``--impl reference`` times the CPU oracle
on the host cores instead (bounded sample per step).
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
sys.path.insert(0, ROOT)

METRIC = "DD eval+Jacobian points/s, path steps/s vs plain GPU at 1e-28; FP64 roof %"
WORKLOAD = ("Newton step (eval+Jacobian+homotopy, FP64 LU + DD refinement, update) per point; "
            "n=32, 32x128 monomials, k=6, exponents 1..4, unit-circle coefficients, "
            "65,536 unit-torus points, complex double-double, seed 2")
T_HOM = 0.5
MAX_REFINE = 6
L2_NOTE = ("GPU arm: a 256 MiB buffer written between timed steps (L2 is 129 MB); "
           "host arm: a fresh sample of points every step")


def workload_config(npts: int, s, world: int) -> dict:
    """The config of the JSON line, the same for the GPU arm and the reference arm."""
    return {"workload": WORKLOAD, "npts": npts, "n": s.n, "monomials": s.nmon,
            "precision": "complex double-double", "lu": "FP64 LU + DD refinement",
            "max_refine": MAX_REFINE, "t": T_HOM, "parallelism": f"dp{world}", "l2": L2_NOTE}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--npts", type=int, default=65536)
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--full-uneven", action="store_true",
                    help="also track all 8,192 systems of the uneven-path family (about a minute more)")
    ap.add_argument("--profile-shared", action="store_true",
                    help="only run the shared-monomial evaluation of Table 1's system (for ncu)")
    ap.add_argument("--profile-large-path", action="store_true",
                    help="only run 2 stages of the large QD path on the whole GPU (for ncu)")
    ap.add_argument("--profile-tracker", action="store_true",
                    help="only run a short graph-stepped tracking of 8 uneven paths (for ncu)")
    return ap.parse_args()


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id: str | None):
        self.proc = None
        self.path = None
        self.dev_id = dev_id

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.dev_id:
                cmd += ["-i", self.dev_id]
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------ CPU arm
def oracle_points_per_s(s, pts, gamma, budget_s: float, lu_mode: int = 1):
    """Time the oracle's threaded Newton step on a bounded sample of the points."""
    import numpy as np

    import oracle
    from paper_1109_0545_gb300 import synth
    cores = os.cpu_count() or 1
    g = np.array([gamma.real, gamma.imag])
    # calibrate on one point per core
    probe = synth.limbs(pts[:cores], 2)
    t0 = time.perf_counter()
    oracle.newton_threads(s.as_dict(), s.coef_limbs(2), probe, T_HOM, g, lu_mode, MAX_REFINE, cores)
    per_wave = max(time.perf_counter() - t0, 1e-3)
    waves = max(1, int(budget_s / per_wave))
    n = min(len(pts), waves * cores)
    sample = synth.limbs(pts[:n], 2)
    t0 = time.perf_counter()
    oracle.newton_threads(s.as_dict(), s.coef_limbs(2), sample, T_HOM, g, lu_mode, MAX_REFINE, cores)
    dt = time.perf_counter() - t0
    return n / dt, cores, n, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1109_0545_gb300 import synth
    s, pts, gamma = synth.eval_throughput(2, npts=args.npts)
    steps = []
    cores = os.cpu_count() or 1
    budget = 2.0
    for k in range(args.warmup + args.steps):
        v, cores, n, dt = oracle_points_per_s(s, pts, gamma, budget)
        if k >= args.warmup:
            steps.append((n, dt))
    tot_n = sum(n for n, _ in steps)
    tot_t = sum(t for _, t in steps)
    value = tot_n / tot_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / max(len(steps), 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.npts, s, args.gpus),
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": f"{steps[0][0] if steps else 0} points per step "
                                   f"(about {budget:.0f} s of oracle work), all host cores"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ GPU arm
def captured_traffic(npts: int):
    """DRAM bytes of one evaluation launch from the committed ncu summary, scaled by
    points -- or None once the kernel sources differ from the captured ones."""
    import hashlib
    import re
    path = os.path.join(ROOT, "profiles", "eval_jac_dd_8192pts_ncu.md")
    srcs = ["points.cuh", "mp.cuh", "hc_eval.cu"]
    try:
        text = open(path).read()
        h = hashlib.sha256()
        for name in srcs:
            with open(os.path.join(ROOT, "paper_1109_0545_gb300", "csrc", name), "rb") as fh:
                h.update(fh.read())
        sha = re.search(r"counters_source_sha256:\s*([0-9a-f]+)", text).group(1)
        per_pt = float(re.search(r"dram_bytes_per_point:\s*([0-9.]+)", text).group(1))
    except (OSError, AttributeError):
        return None
    if not h.hexdigest().startswith(sha):
        return None
    return per_pt * npts


PROPOSER = os.path.join(ROOT, "paper_1109_0545_gb300", "data", "proposer_weights.npy")


def tracker_bench(torch, hc, synth, peak_gops=None, npaths=608, uneven_paths=2432, cap=200, plain_sample=16,
                  full_uneven=False):
    """Path steps/s and paths/s of the batched tracker (all paths in one persistent
    kernel, FP64 LU + DD refinement; secant, quadratic, tangent, and quadratic + learned step
    proposer) against the plain GPU tracker (all-DD elimination, secant, plain step
    control, one path per launch).  Two families: the uneven-path family (n 10..64,
    20..200 monomials per polynomial, k 2..8, exponents 1..3, seed 3; uneven_paths = 2432
    systems, four waves of four blocks on each of 152 SMs), whose paths all diverge,
    tracked for at most `cap` stages each (path steps/s); and its regular variant (a pure
    power and a constant per polynomial, seed 33; npaths = 608, one wave), tracked to the
    end (paths/s, end points compared with the batched all-DD tracker's at 1e-28); with
    full_uneven, also all 8,192 systems of the uneven family, 200 stages each.  FP64 throughput: the
    Newton iterations of all paths (end game included) times the FP64 instructions of one
    iteration without its refinement sweeps (`opcount.newton_iteration_ops`, a lower bound)
    per second, against the measured FP64 peak."""
    import numpy as np
    from paper_1109_0545_gb300 import opcount
    prop = None
    if os.path.exists(PROPOSER):
        prop = torch.from_numpy(np.load(PROPOSER).astype(np.float32)).cuda()

    def run(handles, systems, opts):
        """One tracking call on already loaded systems (loading is outside the timing)."""
        x0 = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(s.n), 2) for s in systems])).cuda()
        x1 = torch.zeros_like(x0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats = hc.hc_track_path(handles, x0, x1, opts)
        dt = time.perf_counter() - t0
        ends = hc.unpack_paths(x1.cpu().numpy(), [s.n for s in systems], 2)
        return stats, ends, dt

    rng = np.random.default_rng(33)
    reg = []
    for j in range(npaths):
        n = int(rng.integers(10, 65))
        reg.append((synth.regular_system(rng, n, (20, 200), (2, 8), (1, 3), lead=1),
                    synth.unit_complex(rng)))
    fams = {"uneven": ([synth.uneven_path_system(3, j) for j in range(uneven_paths)], dict(max_steps=cap)),
            "uneven_regular": (reg, {})}
    variants = [("batched_secant", dict(lu_mode=hc.HC_LU_FP64_REFINE)),
                ("batched_quadratic", dict(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_QUADRATIC)),
                ("batched_tangent", dict(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_TANGENT))]
    if prop is not None:
        variants.append(("batched_quadratic_proposer",
                         dict(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_QUADRATIC,
                              proposer=prop.data_ptr())))
    from paper_1109_0545_gb300 import autotune
    # the shape of each family's runs, tuned on the family itself: the uneven family on all
    # its paths capped at 40 stages (its rate per stage does not depend on the cap); the
    # regular variant, one wave of paths run to their ends whose makespan is set by the
    # longest, on the whole run with three shapes
    tune = {"uneven": (dict(max_steps=40), [(t, b, 0) for t in (64, 128, 256) for b in (0, 2, 3)] + [(512, 0, 0)]),
            "uneven_regular": (dict(predictor=hc.HC_PRED_QUADRATIC),
                               [(128, 0, 0), (256, 0, 0), (256, 1, 0), (512, 0, 0)])}
    out = {}
    for name, (fam, extra) in fams.items():
        systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
        handles = [hc.system_from(sy, 2, g) for sy, g in fam]
        topts, cands = tune[name]
        x0t = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(sy.n), 2) for sy in systems])).cuda()
        tiles = autotune.tune_track(handles, x0t, hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, **topts),
                                    use_cache=False, candidates=cands)
        del x0t
        npaths = len(systems)
        it_ops = [opcount.newton_iteration_ops(sy, 2) for sy in systems]
        plain = hc.hc_track_opts_default(lu_mode=hc.HC_LU_NATIVE, **extra)
        p_steps, p_dt = 0, 0.0
        for j in range(plain_sample):
            pst, _, pdt = run(handles[j:j + 1], systems[j:j + 1], plain)
            p_steps += pst[0]["n_corr"]
            p_dt += pdt
        ref_st, ref_ends, ref_dt = run(handles, systems, plain)
        ref_steps = sum(x["n_corr"] for x in ref_st)
        res = {"paths": npaths, "stage_cap": extra.get("max_steps"),
               "tiles": {k: tiles[k] for k in ("threads_per_block", "blocks_per_sm", "factors")},
               "tile_candidates": tiles["tried"],
               "plain_one_path_per_launch": {"path_steps_per_s": p_steps / p_dt,
                                             "paths_per_s": plain_sample / p_dt,
                                             "sample_paths": plain_sample},
               "batched_all_dd_secant": {"path_steps_per_s": ref_steps / ref_dt,
                                         "paths_per_s": npaths / ref_dt,
                                         "ok_paths": sum(1 for x in ref_st if x["status"] == hc.HC_OK),
                                         "status_hist": np.bincount([x["status"] for x in ref_st],
                                                                    minlength=7).tolist()}}
        for vname, kw in variants:
            st, ends, dt = run(handles, systems, hc.hc_track_opts_default(**kw, **extra))
            steps = sum(x["n_corr"] for x in st)
            same = sum(1 for p in range(npaths) if st[p]["status"] == hc.HC_OK and ref_st[p]["status"] == hc.HC_OK
                       and np.abs((ends[p] - ref_ends[p]).sum(-1)).max()
                       <= 1e-28 * max(1.0, np.abs(ref_ends[p].sum(-1)).max()))
            gops = sum((x["newton_its"] + x["end_its"]) * w for x, w in zip(st, it_ops)) / dt / 1e9
            res[vname] = {"path_steps_per_s": steps / dt, "paths_per_s": npaths / dt,
                          "fp64_gops_at_least": gops,
                          "fp64_frac_of_measured_peak_at_least": gops / peak_gops if peak_gops else None,
                          "speedup_steps_vs_batched_all_dd": (steps / dt) / (ref_steps / ref_dt),
                          "speedup_paths_vs_batched_all_dd": (npaths / dt) / (npaths / ref_dt),
                          "speedup_steps_vs_plain": (steps / dt) / (p_steps / p_dt),
                          "speedup_paths_vs_plain": (npaths / dt) / (plain_sample / p_dt),
                          "mean_stages": steps / npaths,
                          "ok_paths": sum(1 for x in st if x["status"] == hc.HC_OK),
                          "same_end_point_as_batched_all_dd_1e-28": same,
                          "status_hist": np.bincount([x["status"] for x in st], minlength=7).tolist()}
        for h in handles:
            h.free()
        hc.hc_set_track_tiles(0, 0, 0, 0)
        out[name] = res
    if not full_uneven:
        return out
    # the full uneven-path workload: 8,192 systems, 200 stages each, batched secant tracker
    fam = [synth.uneven_path_system(3, j) for j in range(8192)]
    systems = [f[0] for f in fam]
    handles = [hc.system_from(sy, 2, g) for sy, g in fam]
    st, _, dt = run(handles, systems, hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, max_steps=cap))
    for h in handles:
        h.free()
    steps = sum(x["n_corr"] for x in st)
    gops = sum((x["newton_its"] + x["end_its"]) * opcount.newton_iteration_ops(sy, 2)
               for x, sy in zip(st, systems)) / dt / 1e9
    out["uneven_8192_paths"] = {"paths": 8192, "stage_cap": cap, "path_steps_per_s": steps / dt,
                                "seconds": dt, "fp64_gops_at_least": gops,
                                "fp64_frac_of_measured_peak_at_least": gops / peak_gops if peak_gops else None,
                                "speedup_steps_vs_plain":
                                    (steps / dt) / out["uneven"]["plain_one_path_per_launch"]["path_steps_per_s"]}
    return out


def large_path_bench(torch, hc, synth):
    """The large single path (n = 96, 96 x 1024 monomials, k = 12, exponents 1..5, complex
    QD, FP64 LU with QD refinement, seed 4) tracked on the whole GPU from t = 0 until it
    stops: corrector stages, seconds, stages per second, status and the t reached.  (Its
    stages are compared with the QD oracle in tests/test_gpu_grid.py.)"""
    import numpy as np
    from paper_1109_0545_gb300 import autotune
    s, g = synth.large_path_qd(4)
    h = hc.system_from(s, 4, g)
    x0 = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(s.n), 4)])).cuda()
    x1 = torch.zeros_like(x0)
    o = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, mode=hc.HC_TRACK_GRID,
                                 eps=1e-58, eps_end=1e-58, eps_end_x=1e-58)
    # the chunk length of the entry sums, tuned on 8 stages of this path
    o8 = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, mode=hc.HC_TRACK_GRID, max_steps=8,
                                  eps=1e-58, eps_end=1e-58, eps_end_x=1e-58)
    chunk = autotune.tune_grid_chunk(h, x0, o8, use_cache=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = hc.hc_track_path([h], x0, x1, o)[0]
    dt = time.perf_counter() - t0
    z = hc.unpack_paths(x1.cpu().numpy(), [s.n], 4)[0]
    h.free()
    hc.hc_set_track_tiles(0, 0, 0, 0)
    return {"n": s.n, "monomials": s.nmon, "grid_chunk": chunk["grid_chunk"], "status": hc.STATUS_NAMES[st["status"]],
            "stages": int(st["n_corr"]), "accepted": int(st["n_succ"]), "newton_its": int(st["newton_its"]),
            "t_end": st["t_end"], "min_step": st["min_step"], "seconds": dt, "stages_per_s": st["n_corr"] / dt,
            "max_abs_z_end": float(np.abs(z[:, 0, 0] + 1j * z[:, 1, 0]).max())}


def single_path_bench(torch, hc, synth):
    """The single-path workload (n = 8, 8 polynomials of 12 monomials plus a constant, k = 3,
    exponents 1..3, complex DD, seed 1) on one block: the plain tracker (all-DD elimination,
    secant predictor) and the FP64-LU tracker with the quadratic predictor.  Path steps
    (corrector stages) per second and microseconds per stage; the end point's agreement with
    the oracle is checked in tests/test_gpu_track.py."""
    import numpy as np
    from paper_1109_0545_gb300 import autotune
    s, g = synth.single_path_dd(1)
    h = hc.system_from(s, 2, g)
    out = {"n": s.n, "monomials": s.nmon}
    xt = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(s.n), 2)])).cuda()
    tiles = autotune.tune_track([h], xt, hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE,
                                                                  predictor=hc.HC_PRED_QUADRATIC),
                                use_cache=False, candidates=[(64, 0, 0), (128, 0, 0), (256, 0, 0)])
    out["threads_per_block"] = tiles["threads_per_block"]
    for name, kw in (("plain_all_dd_secant", dict(lu_mode=hc.HC_LU_NATIVE)),
                     ("fp64_refine_quadratic", dict(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_QUADRATIC))):
        x0 = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(s.n), 2)])).cuda()
        x1 = torch.zeros_like(x0)
        o = hc.hc_track_opts_default(**kw)
        hc.hc_track_path([h], x0, x1, o)            # warm-up (module load, allocations)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = hc.hc_track_path([h], x0, x1, o)[0]
        dt = time.perf_counter() - t0
        out[name] = {"status": hc.STATUS_NAMES[st["status"]], "stages": int(st["n_corr"]),
                     "accepted": int(st["n_succ"]), "newton_its": int(st["newton_its"]),
                     "path_steps_per_s": st["n_corr"] / dt, "us_per_step": 1e6 * dt / max(st["n_corr"], 1),
                     "seconds": dt}
    h.free()
    hc.hc_set_track_tiles(0, 0, 0, 0)
    return out


def paper_tables_bench(torch, hc, synth):
    """One-path runs in complex QD (the paper's precision) on the shapes of its one-path
    experiments, regular variant (a constant and x_i^(D+1) added per polynomial so that the
    path ends at a root).  Table 4: n = 40, 40 monomials of degree 2 per polynomial, and of
    degree 20; quadratic predictor; on one 128-thread block and on the whole GPU
    (HC_TRACK_GRID); the paper's times on 8 cores of a 2011 Xeon are context.  Tables 2-3:
    n = 20, 20 monomials of degree 10 per polynomial, three systems tracked together,
    secant against quadratic predictor: successful / total corrector stages, average and
    minimal accepted step, time; and the tangent (Euler) predictor beside them."""
    import numpy as np

    def run(systems, gammas, **kw):
        handles = [hc.system_from(s, 4, g) for s, g in zip(systems, gammas)]
        x0 = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(s.n), 4) for s in systems])).cuda()
        x1 = torch.zeros_like(x0)
        o = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, eps=1e-58, eps_end=1e-58,
                                     eps_end_x=1e-58, **kw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = hc.hc_track_path(handles, x0, x1, o)
        dt = time.perf_counter() - t0
        for h in handles:
            h.free()
        return st, dt

    def summary(st, dt):
        return {"seconds": dt, "status": [hc.STATUS_NAMES[x["status"]] for x in st],
                "succ_corrs": [int(x["n_succ"]) for x in st], "corrs": [int(x["n_corr"]) for x in st],
                "avg_step": [x["avg_step"] for x in st], "min_step": [x["min_step"] for x in st],
                "newton_its": [int(x["newton_its"]) for x in st],
                "stages_per_s": sum(x["n_corr"] for x in st) / dt}

    out = {}
    paper_s = {2: 62.257, 20: 1942.671}
    for deg in (2, 20):
        s, g = synth.paper_dim_degree(40, 40, 40, deg)
        r = {"n": 40, "monomials": s.nmon, "degree": deg, "paper_8_cores_s": paper_s[deg]}
        for eng, mode in (("one_block", hc.HC_TRACK_PERSISTENT), ("whole_gpu", hc.HC_TRACK_GRID)):
            st, dt = run([s], [g], predictor=hc.HC_PRED_QUADRATIC, mode=mode)
            r[eng] = summary(st, dt)
        out[f"table4_dim40_deg{deg}_qd"] = r
    fam = [synth.paper_dim_degree(20 + j, 20, 20, 10) for j in range(3)]
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    r = {"n": 20, "monomials": systems[0].nmon, "degree": 10, "systems": 3}
    for name, pred in (("secant", hc.HC_PRED_SECANT), ("quadratic", hc.HC_PRED_QUADRATIC),
                       ("tangent", hc.HC_PRED_TANGENT)):
        st, dt = run(systems, gammas, predictor=pred)
        r[name] = summary(st, dt)
    out["tables23_dim20_deg10_qd"] = r
    return out


def common_support_bench(torch, hc, synth, peak_gops=None, npts=8192):
    """The system behind Table 1 (40 variables, one support of 200 monomials shared by all
    40 polynomials, degree 40 on average and 80 at most), complex DD, at npts unit-torus
    points: evaluation with Jacobian in the per-term and in the shared-monomial scheme
    (points/s, and FP64 instructions per second from the library's per-point counts
    against the measured peak), and the split of a Newton step (FP64 LU + DD refinement)
    between evaluation and solve, the split Table 1 reports."""
    import numpy as np
    s, gamma = synth.common_support_system(1)
    rng = np.random.default_rng(77)
    pts = synth.torus_points(rng, npts, s.n)
    sysh = hc.system_from(s, 2, gamma)
    x0 = torch.from_numpy(hc.to_soa(pts, 2)).cuda()
    x = x0.clone()
    f = torch.empty((2, 2, s.npoly, npts), dtype=torch.float64, device="cuda")
    J = torch.empty((2, 2, s.npoly, s.n, npts), dtype=torch.float64, device="cuda")
    res = torch.zeros(npts, dtype=torch.float64, device="cuda")
    st = torch.zeros(npts, dtype=torch.int32, device="cuda")
    sw = torch.zeros(npts, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    _, ops_term, ops_shared = sysh.eval_mode()

    def timed(fn, reps=3):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        best = 1e30
        for _ in range(reps):
            x.copy_(x0)
            ev0.record(stream)
            fn()
            ev1.record(stream)
            torch.cuda.synchronize()
            best = min(best, ev0.elapsed_time(ev1))
        return best

    out = {"n": s.n, "monomials": s.nmon, "distinct_monomials": 200, "npts": npts,
           "fp64_per_point_per_term": ops_term, "fp64_per_point_shared": ops_shared}
    for name, mode, ops in (("per_term", hc.HC_EVAL_PER_TERM, ops_term), ("shared", hc.HC_EVAL_SHARED, ops_shared)):
        sysh.set_eval_mode(mode)
        ms_eval = timed(lambda: hc.hc_eval_jac(sysh, npts, 0.5, x, f, J, stream))
        ms_newton = timed(lambda: hc.hc_newton_step(sysh, npts, 0.5, x, hc.HC_LU_FP64_REFINE, 4, res, st, sw, stream))
        gops = ops * npts / (ms_eval * 1e-3) / 1e9
        out[name] = {"eval_points_per_s": npts / (ms_eval * 1e-3), "eval_ms": ms_eval,
                     "newton_step_ms": ms_newton, "eval_share_of_newton_step": ms_eval / ms_newton,
                     "eval_fp64_gops": gops, "eval_fp64_frac_of_measured_peak": gops / peak_gops if peak_gops else None}
    out["shared_speedup"] = out["per_term"]["eval_ms"] / out["shared"]["eval_ms"]
    sysh.free()
    return out


def quality_up_bench(torch, hc, synth, npaths=456):
    """Quality up (Sec. 2): the same 456 regular-variant paths tracked in complex double,
    double-double and quad-double (FP64 LU with refinement, quadratic predictor, corrector
    tolerances 1e-12 / 1e-26 / 1e-58).  Quality Q = correct decimal places of the end
    points (median over converged paths; the QD end points are the reference for double
    and DD, the DD ones bound QD from below at its own tolerance).  The paper's quality up
    at fixed time (`quality.py`, Sec. 2): p* = ceil(T_QD / T_DD) GPUs let QD match the time
    of DD on one GPU (optimal speedup assumed, as in the paper), and y(p) runs linearly from
    y(1) = 1 to y(p*) = Q_QD / Q_DD; reported for p = 8 GPUs."""
    import numpy as np
    rng = np.random.default_rng(44)
    fam = []
    for _ in range(npaths):
        n = int(rng.integers(10, 65))
        fam.append((synth.regular_system(rng, n, (20, 200), (2, 8), (1, 3), lead=1), synth.unit_complex(rng)))
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    eps = {1: 1e-12, 2: 1e-26, 4: 1e-58}
    runs = {}
    for L in (1, 2, 4):
        handles = [hc.system_from(sy, L, g) for sy, g in fam]
        x0 = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(sy.n), L) for sy in systems])).cuda()
        x1 = torch.zeros_like(x0)
        o = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_QUADRATIC,
                                     eps=eps[L], eps_end=eps[L], eps_end_x=eps[L])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = hc.hc_track_path(handles, x0, x1, o)
        dt = time.perf_counter() - t0
        runs[L] = (st, hc.unpack_paths(x1.cpu().numpy(), [sy.n for sy in systems], L), dt)
        for h in handles:
            h.free()
    q_st, q_end, _ = runs[4]

    def digits(L):
        st, ends, _ = runs[L]
        d = []
        for p in range(npaths):
            if st[p]["status"] != hc.HC_OK or q_st[p]["status"] != hc.HC_OK:
                continue
            ref = q_end[p]
            g = np.zeros_like(ref)
            g[..., :L] = ends[p]
            # the leading limbs of two close values subtract exactly, so the sum of the
            # limb differences is the difference to far below its own size
            diff = np.abs((g - ref).sum(-1)).max()
            scale = np.abs(ref[..., 0]).max()
            d.append(-np.log10(max(diff / scale, 1e-64)))
        return float(np.median(d)) if d else None

    out = {"paths": npaths}
    for L, name in ((1, "double"), (2, "double_double"), (4, "quad_double")):
        st, _, dt = runs[L]
        out[name] = {"seconds": dt, "paths_per_s": npaths / dt, "ok_paths": sum(1 for x in st if x["status"] == hc.HC_OK)}
    out["double"]["digits_vs_qd"] = digits(1)
    out["double_double"]["digits_vs_qd"] = digits(2)
    # QD's own quality: its corrector tolerance (the end game stops at 1e-58 relative)
    from paper_1109_0545_gb300 import quality
    q_dd = out["double_double"]["digits_vs_qd"]
    q_qd = 58.0
    out["quad_double"]["digits"] = q_qd
    ratio, p_star = quality.processors_for_fixed_time(out["double_double"]["seconds"],
                                                      out["quad_double"]["seconds"], 1)
    out["qd_time_over_dd_time"] = ratio
    out["qd_gpus_for_dd_time"] = p_star
    if q_dd:
        out["quality_up_8_gpus"] = quality.quality_up(8, p_star, q_qd / q_dd)
    return out


def mlp_bench(torch, hc, steps=200, batch=8192, nrec=65536):
    """The step proposer's kernels: one training step (k_mlp_grad + k_mlp_reduce +
    k_mlp_adamw on a batch of 8,192 feature records, the batch of the proposer's training)
    and inference (k_mlp_forward) on 65,536 records, on seeded synthetic records of the
    logged shapes.  Times from CUDA events on the launching stream."""
    import numpy as np
    from paper_1109_0545_gb300 import learn
    rng = np.random.default_rng(55)
    X = torch.from_numpy(rng.normal(0.0, 0.5, (nrec, hc.HC_MLP_IN)).astype(np.float32)).cuda()
    r = torch.from_numpy(rng.uniform(-1.5, 1.5, nrec).astype(np.float32)).cuda()
    a = torch.from_numpy((rng.uniform(size=nrec) < 0.75).astype(np.int32)).cuda()
    p = torch.from_numpy(learn.init_params(0)).cuda()
    m1, m2, g = torch.zeros_like(p), torch.zeros_like(p), torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    out = torch.empty(nrec, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def train_step(k):
        hc.hc_mlp_grad(p, batch, X, r, a, learn.KAPPA, g, loss, stream)
        hc.hc_mlp_adamw(p, m1, m2, g, k, 1e-3, 0.9, 0.999, 1e-8, 1e-4, stream)

    for k in range(1, 6):
        train_step(k)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for k in range(6, 6 + steps):
        train_step(k)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_train = ev0.elapsed_time(ev1) / steps
    hc.hc_mlp_forward(p, nrec, X, out, stream)
    ev0.record(stream)
    for _ in range(10):
        hc.hc_mlp_forward(p, nrec, X, out, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_fwd = ev0.elapsed_time(ev1) / 10
    return {"train_step_ms": ms_train, "train_records_per_s": batch / (ms_train * 1e-3),
            "batch": batch, "forward_ms_65536_records": ms_fwd,
            "forward_records_per_s": nrec / (ms_fwd * 1e-3)}


def compact_extras(ex: dict) -> dict:
    """The secondary figures in a few hundred bytes (the full record is printed on the line
    before the main one)."""
    def r(v, d=3):
        return None if v is None else float(f"{v:.{d}g}")

    out = {}
    tr = ex.get("tracker", {})
    for fam, res in tr.items():
        if not isinstance(res, dict) or "batched_all_dd_secant" not in res:
            continue
        key = "paths_per_s" if fam == "uneven_regular" else "path_steps_per_s"
        row = {"unit": key, "paths": res["paths"], "cap": res.get("stage_cap"), "tiles": res.get("tiles"),
               "plain_1_per_launch": r(res["plain_one_path_per_launch"][key]),
               "plain_sample_paths": res["plain_one_path_per_launch"]["sample_paths"],
               "batched_all_dd": r(res["batched_all_dd_secant"][key])}
        for v in ("batched_secant", "batched_quadratic", "batched_tangent", "batched_quadratic_proposer"):
            if v in res:
                row[v.replace("batched_", "mixed_")] = r(res[v][key])
        if "batched_secant" in res:
            row["mixed_vs_all_dd_equal_batching"] = r(res["batched_secant"][key] / res["batched_all_dd_secant"][key])
            row["ok_paths_mixed"] = res["batched_secant"]["ok_paths"]
            row["same_end_points_1e-28"] = res["batched_secant"]["same_end_point_as_batched_all_dd_1e-28"]
        out[f"tracker_{fam}"] = row
    if "uneven_8192_paths" in tr:
        out["tracker_uneven_8192"] = {"path_steps_per_s": r(tr["uneven_8192_paths"]["path_steps_per_s"])}
    lp = ex.get("large_path_qd_n96")
    if lp:
        out["large_path_qd_n96"] = {k: (r(v, 9) if isinstance(v, float) else v) for k, v in lp.items()
                                    if k in ("status", "stages", "seconds", "stages_per_s", "t_end", "grid_chunk")}
    sp = ex.get("single_path_n8")
    if sp:
        out["single_path_n8_stages_per_s"] = {k: r(v["path_steps_per_s"]) for k, v in sp.items() if isinstance(v, dict)}
    pt = ex.get("paper_tables", {})
    for k in ("table4_dim40_deg2_qd", "table4_dim40_deg20_qd"):
        if k in pt:
            out[k + "_s"] = {"one_block": r(pt[k]["one_block"]["seconds"]), "whole_gpu": r(pt[k]["whole_gpu"]["seconds"]),
                             "paper_8_cores": pt[k]["paper_8_cores_s"]}
    cs = ex.get("common_support_table1")
    if cs:
        out["table1_eval_points_per_s"] = {"per_term": r(cs["per_term"]["eval_points_per_s"]),
                                           "shared": r(cs["shared"]["eval_points_per_s"])}
    q = ex.get("quality_up")
    if q:
        out["quality_up_8_gpus"] = r(q.get("quality_up_8_gpus"))
    for k in ("eval_jac_points_per_s", "eval_jac_qd_points_per_s", "newton_native_dd_lu_points_per_s"):
        if k in ex:
            out[k] = r(ex[k])
    return out


def rank_points(rank: int, npts: int, n: int, default):
    """The points rank `rank` evaluates: rank 0 the workload's own, every other rank its
    own seeded draw of the same size (independent problems: weak scaling)."""
    import numpy as np
    from paper_1109_0545_gb300 import synth
    if rank == 0:
        return default
    return synth.torus_points(np.random.default_rng([2, rank]), npts, n)


def shard_range(nunits: int, rank: int, world: int) -> tuple[int, int]:
    """The block of independent units (paths, points) rank `rank` of `world` takes: the
    first nunits % world ranks take one more; no unit is shared, so the ranks need no
    exchange until the results are gathered."""
    base, extra = divmod(nunits, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def gather_stats(stats: list, dist) -> list:
    """The per-unit results of every rank, in rank order, on every rank (the one gather of
    a sharded run)."""
    if dist is None:
        return list(stats)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, list(stats))
    return [x for part in parts for x in part]


def sharded_tracker(torch, hc, synth, fam, opts, dist=None, rank: int = 0, world: int = 1, L: int = 2):
    """Paths shard in blocks over the ranks (shard_range): each rank tracks its own block
    in one hc_track_path call on its own GPU, and the per-path statistics and end points
    gather once, in rank order (gather_stats).  fam: list of (system, gamma).  Returns
    (statistics of every path, end points of every path, this rank's seconds)."""
    import numpy as np
    lo, hi = shard_range(len(fam), rank, world)
    mine = fam[lo:hi]
    rows, dt = [], 0.0
    if mine:
        handles = [hc.system_from(sy, L, g) for sy, g in mine]
        x0 = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(sy.n), L) for sy, _ in mine])).cuda()
        x1 = torch.zeros_like(x0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats = hc.hc_track_path(handles, x0, x1, opts)
        dt = time.perf_counter() - t0
        ends = hc.unpack_paths(x1.cpu().numpy(), [sy.n for sy, _ in mine], L)
        rows = [(st, e.tolist()) for st, e in zip(stats, ends)]
        for h in handles:
            h.free()
    rows = gather_stats(rows, dist)
    return [r[0] for r in rows], [np.array(r[1]) for r in rows], dt


def max_over_ranks(ms: float, dist, device=None) -> float:
    """The slowest rank's time (the job's time); the only collective of the bench."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_gpu(args):
    import numpy as np
    import torch

    from paper_1109_0545_gb300 import hc, opcount, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    hc.load(build_if_missing=False)

    L = 2
    npts = args.npts
    s, pts, gamma = synth.eval_throughput(2, npts=npts)
    pts = rank_points(rank, npts, s.n, pts)
    sysh = hc.system_from(s, L, gamma)
    stream = torch.cuda.current_stream()
    x0 = torch.from_numpy(hc.to_soa(pts, L)).cuda()
    x = x0.clone()
    res = torch.zeros(npts, dtype=torch.float64, device="cuda")
    st = torch.zeros(npts, dtype=torch.int32, device="cuda")
    sw = torch.zeros(npts, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2

    def step(lu=hc.HC_LU_FP64_REFINE):
        hc.hc_newton_step(sysh, npts, T_HOM, x, lu, MAX_REFINE, res, st, sw, stream)

    # tile shape of the evaluation kernel, tuned on this workload (outside the timing)
    from paper_1109_0545_gb300 import autotune
    fbuf = torch.empty((2, L, s.npoly, npts), dtype=torch.float64, device="cuda")
    jbuf = torch.empty((2, L, s.npoly, s.n, npts), dtype=torch.float64, device="cuda")
    tiles = autotune.tune_eval(sysh, x0, fbuf, jbuf, npts, T_HOM, reps=1, use_cache=False,
                               candidates=[(0, 0), (1, 4), (2, 4), (4, 4), (1, 6), (2, 6),
                                           (4, 6), (8, 6), (1, 8), (2, 8)])
    del fbuf, jbuf
    tiles.pop("tried", None)
    for _ in range(max(args.warmup, 0)):
        x.copy_(x0)
        step()
    torch.cuda.synchronize()
    peak_gops = hc.hc_probe_fp64_peak()

    dev_id = None
    try:
        dev_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        dev_id = None
    clocks = ClockSampler(dev_id)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    hc.hc_prof_read()          # drop anything recorded earlier
    hc.hc_prof_enable(True)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        x.copy_(x0)            # restore the input point set (outside the step's events)
        flush.zero_()          # evict L2 between timed steps
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    hc.hc_prof_enable(False)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = sum(step_ms)
    eval_ms, eval_launches = hc.hc_prof_read()
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    value = npts * world * args.steps / (total_ms * 1e-3)
    status = st.cpu().numpy()
    sweeps = sw.cpu().numpy()

    ops_pt = opcount.eval_ops_per_point(s, L)
    eval_avg_ms = eval_ms / max(eval_launches, 1)
    achieved = ops_pt * npts / (eval_avg_ms * 1e-3) / 1e9
    roofline = {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": peak_gops,
                "unit": "G FP64 instr/s", "frac": achieved / peak_gops,
                "peak_source": "measured live (hc_probe_fp64_peak, independent DFMA chains)",
                "kernel": "k_eval_pts<DD,jacobian>", "ops_per_point": ops_pt,
                "kernel_ms": eval_avg_ms, "traffic": captured_traffic(npts),
                "traffic_note": "ncu dram read+write per launch, 8,192-point capture scaled by points"}
    if roofline["traffic"] and eval_avg_ms > 0:
        # the secondary counter: DRAM bytes per second of the evaluation kernel (the HBM is idle)
        roofline["hbm_gbs"] = roofline["traffic"] / (eval_avg_ms * 1e-3) / 1e9
    # against the FP64 issue rate the profiler states as the peak (2 FP64 thread
    # instructions per clock per SM) at the median SM clock of the timed region
    mhz = clk.get("sm_mhz") if isinstance(clk, dict) else None
    if mhz:
        nominal = 2.0 * torch.cuda.get_device_properties(local).multi_processor_count * mhz * 1e6 / 1e9
        roofline["nominal_peak"] = nominal
        roofline["frac_of_nominal"] = achieved / nominal

    extras = {}
    # the secondary measurements are single-GPU figures: with several ranks they would hold
    # every GPU for minutes, so they run at N = 1 only
    if not args.no_extras and world == 1:
        # the plain all-DD elimination, and evaluation alone, same points
        def timed(fn, reps=3):
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            best = 1e30
            for _ in range(reps):
                x.copy_(x0)
                flush.zero_()
                ev0.record(stream)
                fn()
                ev1.record(stream)
                torch.cuda.synchronize()
                best = min(best, ev0.elapsed_time(ev1))
            return best
        ms_native = timed(lambda: step(hc.HC_LU_NATIVE))
        f = torch.empty((2, L, s.npoly, npts), dtype=torch.float64, device="cuda")
        J = torch.empty((2, L, s.npoly, s.n, npts), dtype=torch.float64, device="cuda")
        ms_eval = timed(lambda: hc.hc_eval_jac(sysh, npts, T_HOM, x, f, J, stream))
        del f, J
        # complex QD evaluation throughput on 16,384 of the points
        q = 16384
        sysq = hc.system_from(s, 4, gamma)
        xq = torch.from_numpy(hc.to_soa(pts[:q], 4)).cuda()
        fq = torch.empty((2, 4, s.npoly, q), dtype=torch.float64, device="cuda")
        Jq = torch.empty((2, 4, s.npoly, s.n, q), dtype=torch.float64, device="cuda")
        hc.hc_eval_jac(sysq, q, T_HOM, xq, fq, Jq, stream)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        hc.hc_eval_jac(sysq, q, T_HOM, xq, fq, Jq, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_qd = ev0.elapsed_time(ev1)
        del fq, Jq
        # refinement sweeps per accuracy level: one Newton step (FP64 LU + refinement) at
        # the same 16,384 points in complex double and QD (DD: the timed step above)
        sweeps_by_prec = {}
        for Lq, hq in ((1, hc.system_from(s, 1, gamma)), (4, sysq)):
            xl = torch.from_numpy(hc.to_soa(pts[:q], Lq)).cuda()
            rl = torch.zeros(q, dtype=torch.float64, device="cuda")
            sl = torch.zeros(q, dtype=torch.int32, device="cuda")
            wl = torch.zeros(q, dtype=torch.int32, device="cuda")
            hc.hc_newton_step(hq, q, T_HOM, xl, hc.HC_LU_FP64_REFINE, MAX_REFINE, rl, sl, wl, stream)
            torch.cuda.synchronize()
            sweeps_by_prec[{1: "double", 4: "quad_double"}[Lq]] = np.bincount(
                wl.cpu().numpy(), minlength=MAX_REFINE + 1).tolist()
            hq.free()
            del xl, rl, sl, wl
        del xq
        extras = {"tracker": tracker_bench(torch, hc, synth, peak_gops, full_uneven=args.full_uneven),
                  "large_path_qd_n96": large_path_bench(torch, hc, synth),
                  "single_path_n8": single_path_bench(torch, hc, synth),
                  "paper_tables": paper_tables_bench(torch, hc, synth),
                  "common_support_table1": common_support_bench(torch, hc, synth, peak_gops),
                  "quality_up": quality_up_bench(torch, hc, synth),
                  "proposer_mlp": mlp_bench(torch, hc),
                  "eval_jac_qd_points_per_s": q / (ms_qd * 1e-3),
                  "eval_jac_qd_fp64_gops": opcount.eval_ops_per_point(s, 4) * q / (ms_qd * 1e-3) / 1e9,
                  "newton_native_dd_lu_points_per_s": npts / (ms_native * 1e-3),
                  "eval_jac_points_per_s": npts / (ms_eval * 1e-3),
                  "refine_sweeps_hist": np.bincount(sweeps, minlength=MAX_REFINE + 1).tolist(),
                  "refine_sweeps_hist_16384pts": sweeps_by_prec,
                  "status_ok_frac": float(np.mean(status == hc.HC_OK))}

    # end to end through the public API with host buffers (pinned), copies timed
    x_host = torch.from_numpy(hc.to_soa(pts, L)).pin_memory()
    x_out = torch.empty_like(x_host).pin_memory()
    st_host = torch.empty(npts, dtype=torch.int32).pin_memory()
    res_host = torch.empty(npts, dtype=torch.float64).pin_memory()
    e2e_steps = min(args.steps, 5)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        x.copy_(x_host, non_blocking=True)
        step()
        x_out.copy_(x, non_blocking=True)
        st_host.copy_(st, non_blocking=True)
        res_host.copy_(res, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = x_host.numel() * 8
    d2h = x_out.numel() * 8 + npts * 4 + npts * 8
    e2e = {"value": npts * e2e_steps / e2e_s, "unit": "points/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    # the tracker sharded over the ranks (weak scaling: 2,432 paths of the uneven family per
    # rank, 40 corrector stages each, FP64 LU + DD refinement; one gather of the results)
    shard = None
    if not args.no_extras:
        fam = [synth.uneven_path_system(3, j) for j in range(2432 * world)]
        sst, _, sdt = sharded_tracker(torch, hc, synth, fam,
                                      hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, max_steps=40),
                                      dist, rank, world)
        sdt = max_over_ranks(sdt * 1e3, dist, "cuda") * 1e-3
        shard = {"paths": len(fam), "paths_per_rank": 2432, "stage_cap": 40,
                 "path_steps_per_s": sum(x["n_corr"] for x in sst) / sdt, "seconds": sdt,
                 "gathered_paths": len(sst)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_extras:
        v, cores, n, dt = oracle_points_per_s(s, pts, gamma, budget_s=15.0)
        cpu = {"value": v, "unit": "points/s", "cores": cores, "kind": "oracle",
               "sample": f"{n} of {npts} points, one Newton step each (FP64 LU + DD "
                         f"refinement), {dt:.1f} s on {cores} threads"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(npts, s, world),
            "eval_tiles": tiles,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": 3 * args.steps, "clocks": clk, "wall_s": t_wall,
            "tracker_sharded": shard,
            "extras": compact_extras(extras),
        }
        if extras:
            # the full record of the secondary measurements, before the main line
            print(json.dumps({"bench_detail": extras}), flush=True)
        print(json.dumps(line), flush=True)
    sysh.free()
    if dist:
        dist.destroy_process_group()


def profile_tracker():
    """A short tracking run for profiling: 8 paths of the uneven-path family, graph mode
    (one launch per stage), 6 corrector stages each."""
    import numpy as np
    import torch

    from paper_1109_0545_gb300 import hc, synth
    hc.load(build_if_missing=False)
    fam = [synth.uneven_path_system(3, j) for j in range(8)]
    handles = [hc.system_from(s, 2, g) for s, g in fam]
    x0 = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(s.n), 2) for s, _ in fam])).cuda()
    x1 = torch.zeros_like(x0)
    o = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, mode=hc.HC_TRACK_GRAPH,
                                 graph_steps=2, max_steps=6)
    st = hc.hc_track_path(handles, x0, x1, o)
    torch.cuda.synchronize()
    print(json.dumps({"profile_tracker": [x["n_corr"] for x in st]}))


def profile_shared():
    """Two evaluations with Jacobian of Table 1's common-support system (40 x 40, 200 shared
    monomials) in DD at 8,192 points, shared-monomial scheme (for profiling)."""
    import numpy as np
    import torch

    from paper_1109_0545_gb300 import hc, synth
    hc.load(build_if_missing=False)
    s, gamma = synth.common_support_system(1)
    npts = 8192
    pts = synth.torus_points(np.random.default_rng(77), npts, s.n)
    h = hc.system_from(s, 2, gamma)
    h.set_eval_mode(hc.HC_EVAL_SHARED)
    x = torch.from_numpy(hc.to_soa(pts, 2)).cuda()
    f = torch.empty((2, 2, s.npoly, npts), dtype=torch.float64, device="cuda")
    J = torch.empty((2, 2, s.npoly, s.n, npts), dtype=torch.float64, device="cuda")
    for _ in range(2):
        hc.hc_eval_jac(h, npts, 0.5, x, f, J)
    torch.cuda.synchronize()
    print(json.dumps({"profile_shared": npts}))


def profile_large_path():
    """Two corrector stages of the large QD path (n = 96, 98,304 monomials) on the whole GPU
    (for profiling)."""
    import numpy as np
    import torch

    from paper_1109_0545_gb300 import hc, synth
    hc.load(build_if_missing=False)
    s, g = synth.large_path_qd(4)
    h = hc.system_from(s, 4, g)
    x0 = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(s.n), 4)])).cuda()
    x1 = torch.zeros_like(x0)
    o = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, mode=hc.HC_TRACK_GRID, max_steps=2,
                                 eps=1e-58, eps_end=1e-58, eps_end_x=1e-58)
    st = hc.hc_track_path([h], x0, x1, o)
    torch.cuda.synchronize()
    print(json.dumps({"profile_large_path": int(st[0]["n_corr"])}))


def main():
    args = parse()
    if args.profile_tracker:
        profile_tracker()
        return
    if args.profile_shared:
        profile_shared()
        return
    if args.profile_large_path:
        profile_large_path()
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
