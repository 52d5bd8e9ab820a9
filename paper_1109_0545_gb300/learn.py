"""Training and evaluation of the learned step-size proposer.

The proposer's network, loss and features are defined in ``include/hc.h``.  Here:
logged corrector stages of the plain tracker (``hc_track_path`` with a log buffer) are
turned into feature records, the network is trained with the library's own kernels
(``hc_mlp_grad`` for the forward/backward pass, ``hc_mlp_adamw`` for the update), and
the tracker runs with and without the trained proposer.  The arithmetic of the method
never changes: the DD corrector judges every step either way.

    python -m paper_1109_0545_gb300.learn --out result.json   # the full experiment
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import hc, synth

KAPPA = 4.0


def features(recs: np.ndarray, n: int, lambda0: float):
    """Feature records of one path's log (its first n stages): for each stage s >= 1,
    the features before stage s (history s-1, s-2, s-3), the attempted log2 step ratio
    r = log2(lambda_s / lambda_{s-1}) and the outcome.  Same definition as the kernel."""
    recs = recs[:n]
    X, r, a = [], [], []
    for s in range(1, n):
        f = np.zeros(12, dtype=np.float64)
        f[0] = recs["t"][s]
        for j in range(3):
            q = s - 1 - j
            if q >= 0:
                lam, it, res = recs["lam"][q], recs["iters"][q], recs["res_last"][q]
            else:
                lam, it, res = lambda0, 0, 0.0
            f[1 + j] = math.log2(lam / lambda0) / 8.0
            f[4 + j] = it / 4.0
            f[7 + j] = min(max(math.log10(res), -40.0), 5.0) / 10.0 if res > 0 else -4.0
        pcd = recs["pc_dist"][s - 1]
        f[10] = min(max(math.log10(pcd), -40.0), 5.0) / 10.0 if pcd > 0 else -4.0
        f[11] = recs["cond_log10"][s - 1] / 4.0
        X.append(f)
        r.append(math.log2(recs["lam"][s] / recs["lam"][s - 1]))
        a.append(int(recs["accepted"][s]))
    return (np.array(X, dtype=np.float32).reshape(-1, 12), np.array(r, dtype=np.float32),
            np.array(a, dtype=np.int32))


def run_tracker(torch, systems, gammas, opts, log_cap=0):
    handles = [hc.system_from(s, 2, g) for s, g in zip(systems, gammas)]
    x0 = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(s.n), 2) for s in systems])).cuda()
    x1 = torch.zeros_like(x0)
    log = None
    if log_cap:
        log = torch.zeros(len(systems) * log_cap * hc.STEP_RECORD_DTYPE.itemsize,
                          dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stats = hc.hc_track_path(handles, x0, x1, opts, log, log_cap)
    dt = time.perf_counter() - t0
    ends = hc.unpack_paths(x1.cpu().numpy(), [s.n for s in systems], 2)
    recs = (log.cpu().numpy().view(hc.STEP_RECORD_DTYPE).reshape(len(systems), log_cap)
            if log_cap else None)
    for h in handles:
        h.free()
    return stats, ends, recs, dt


def collect(torch, systems, gammas, opts, log_cap=4096, batch=512):
    """Feature records from the plain tracker's logs over the given systems."""
    Xs, rs, as_ = [], [], []
    for b0 in range(0, len(systems), batch):
        st, _, recs, _ = run_tracker(torch, systems[b0:b0 + batch], gammas[b0:b0 + batch], opts, log_cap)
        for p, s in enumerate(st):
            X, r, a = features(recs[p], min(s["n_corr"], log_cap), opts.lambda0)
            Xs.append(X)
            rs.append(r)
            as_.append(a)
    return np.concatenate(Xs), np.concatenate(rs), np.concatenate(as_)


def init_params(seed=0) -> np.ndarray:
    """He-style initial weights N(0, 2/fan_in) (output layer N(0, 1/fan_in)), biases 0."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, math.sqrt(2 / 12), (64, 12))
    W2 = rng.normal(0, math.sqrt(2 / 64), (64, 64))
    W3 = rng.normal(0, math.sqrt(1 / 64), 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3,
                           np.zeros(1)]).astype(np.float32)


def train(torch, X, r, a, steps=2000, batch=8192, lr=2e-3, wd=1e-4, seed=0):
    """Mini-batch AdamW on the library's kernels; the learning rate decays by cosine to
    lr/20.  Returns (params on the device, per-step losses)."""
    dev = "cuda"
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    rd = torch.from_numpy(np.ascontiguousarray(r)).to(dev)
    ad = torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    p = torch.from_numpy(init_params(seed)).to(dev)
    m1 = torch.zeros_like(p)
    m2 = torch.zeros_like(p)
    g = torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    rng = np.random.default_rng(seed + 1)
    N = X.shape[0]
    losses = []
    stream = torch.cuda.current_stream()
    for step in range(1, steps + 1):
        idx = torch.from_numpy(rng.integers(0, N, size=min(batch, N)).astype(np.int64)).to(dev)
        xb = Xd[idx].contiguous()
        rb = rd[idx].contiguous()
        ab = ad[idx].contiguous()
        hc.hc_mlp_grad(p, xb.shape[0], xb, rb, ab, KAPPA, g, loss, stream)
        cur = lr * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * (step - 1) / steps)))
        hc.hc_mlp_adamw(p, m1, m2, g, step, cur, 0.9, 0.999, 1e-8, wd, stream)
        if step % 50 == 0 or step == steps:
            losses.append(float(loss.item()))
    return p, losses


def evaluate(torch, systems, gammas, params, margin=0.5, lu_mode=hc.HC_LU_FP64_REFINE):
    """The tracker with the plain controller and with the proposer on the same paths."""
    out = {}
    for name, prop in (("plain", None), ("proposer", params)):
        o = hc.hc_track_opts_default(lu_mode=lu_mode)
        if prop is not None:
            o.proposer = prop.data_ptr()
            o.proposer_margin = margin
        st, ends, _, dt = run_tracker(torch, systems, gammas, o)
        ok = [x["status"] == hc.HC_OK for x in st]
        out[name] = {"stats": st, "ends": ends, "seconds": dt,
                     "mean_stages": float(np.mean([x["n_corr"] for x in st])),
                     "mean_rejected": float(np.mean([x["n_corr"] - x["n_succ"] for x in st])),
                     "mean_newton_its": float(np.mean([x["newton_its"] for x in st])),
                     "ok_paths": int(np.sum(ok)),
                     "stages_per_s": float(sum(x["n_corr"] for x in st) / dt),
                     "paths_per_s": len(systems) / dt}
    return out


def regular_family(seed: int, count: int, nlo=10, nhi=64):
    """The uneven-path shape with a pure power and a constant per polynomial (paths end
    at regular roots)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(nlo, nhi + 1))
        out.append((synth.regular_system(rng, n, (20, 200), (2, 8), (1, 3), lead=1),
                    synth.unit_complex(rng)))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--records", type=int, default=1_000_000)
    ap.add_argument("--eval-paths", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--out", default="proposer_result.json")
    ap.add_argument("--weights", default="proposer_weights.npy")
    ap.add_argument("--uneven-eval-paths", type=int, default=512)
    ap.add_argument("--margins", default="0.5")
    ap.add_argument("--explore", type=float, default=1.5,
                    help="log2 range of the random step perturbation while collecting")
    ap.add_argument("--eval-only", default=None,
                    help="skip collection and training: evaluate these saved weights")
    args = ap.parse_args()
    import torch
    hc.load(build_if_missing=False)
    if args.eval_only:
        params = torch.from_numpy(np.load(args.eval_only).astype(np.float32)).cuda()
        res = {"weights": os.path.basename(args.eval_only)}
        res.update(evaluate_families(torch, params, args))
        with open(args.out, "w") as fh:
            json.dump(res, fh, indent=1)
        print(json.dumps(res))
        return
    # the plain controller with its steps perturbed by 2^u, u uniform in
    # [-explore, explore], so that the logs hold accepted and rejected steps over a range
    # of ratios around the plain choice
    plain = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, explore=args.explore)
    t0 = time.perf_counter()
    Xs, rs, as_ = [], [], []
    total, j = 0, 0
    # logs of the plain tracker, seeds 10..19: the uneven-path family and its regular
    # variant in equal parts (the family as drawn has no regular end points: every path
    # there ends at a singular root or at infinity, so its logs alone teach only the
    # approach to those)
    while total < args.records:
        systems, gammas = [], []
        for seed in range(10, 20):
            for k in range(16):
                s, g = synth.uneven_path_system(seed, j + k)
                systems.append(s)
                gammas.append(g)
            for s, g in regular_family(1000 * seed + j, 16):
                systems.append(s)
                gammas.append(g)
        plain.explore_seed = 1 + j
        j += 16
        X, r, a = collect(torch, systems, gammas, plain)
        Xs.append(X)
        rs.append(r)
        as_.append(a)
        total += X.shape[0]
    rng = np.random.default_rng(7)
    X, r, a = np.concatenate(Xs), np.concatenate(rs), np.concatenate(as_)
    keep = rng.permutation(X.shape[0])[:args.records]
    X, r, a = X[keep], r[keep], a[keep]
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    params, losses = train(torch, X, r, a, steps=args.steps)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    np.save(args.weights, params.cpu().numpy())
    res = {"records": int(X.shape[0]), "explore": args.explore, "accept_rate": float(a.mean()),
           "collect_s": t_collect,
           "train_s": t_train, "train_steps": args.steps, "loss_first": losses[0],
           "loss_last": losses[-1]}
    res.update(evaluate_families(torch, params, args))
    with open(args.out, "w") as fh:
        json.dump(res, fh, indent=1)
    print(json.dumps(res))


def evaluate_families(torch, params, args) -> dict:
    """The proposer against the plain controller on held-out seed-20 paths: the uneven
    family and its regular variant, at each margin."""
    res = {}
    margins = [float(v) for v in args.margins.split(",")]
    for fam_name, fam in (("uneven_seed20", [synth.uneven_path_system(20, k) for k in range(args.uneven_eval_paths)]),
                          ("uneven_regular_seed20", regular_family(20, args.eval_paths))):
        if not fam:
            continue
        systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
        res[fam_name] = {}
        for margin in margins:
            ev = evaluate(torch, systems, gammas, params, margin=margin)
            same = 0
            both = 0
            for p in range(len(systems)):
                if ev["plain"]["stats"][p]["status"] == 0 and ev["proposer"]["stats"][p]["status"] == 0:
                    both += 1
                    d = np.abs((ev["plain"]["ends"][p] - ev["proposer"]["ends"][p]).sum(-1)).max()
                    same += d <= 1e-28 * max(1.0, np.abs(ev["plain"]["ends"][p].sum(-1)).max())
            r = {k: {kk: vv for kk, vv in v.items() if kk not in ("stats", "ends")} for k, v in ev.items()}
            r["both_ok"] = both
            r["same_end_point_1e-28"] = int(same)
            r["status_plain"] = np.bincount([x["status"] for x in ev["plain"]["stats"]], minlength=7).tolist()
            r["status_proposer"] = np.bincount([x["status"] for x in ev["proposer"]["stats"]], minlength=7).tolist()
            res[fam_name][f"margin_{margin}"] = r
    return res


if __name__ == "__main__":
    main()
