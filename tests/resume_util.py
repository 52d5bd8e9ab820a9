"""Stage-level parity through hc_track_resume: the GPU saves a path's state at chosen
corrector stages; from each saved state the GPU and the oracle (or_track_resume, its own
predictor, corrector and step control) run the same stages, and the states they reach
must agree: status, phase, counts, t and step exactly, the points within the tolerance of
the precision.  This judges any stage of a long path without the oracle tracking it from
t = 0, and a rounding-level difference early on cannot steer the two apart."""
from __future__ import annotations

import ctypes as ct
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle
from helpers import TOL, rel_err_per_point
from paper_1109_0545_gb300 import hc, synth


def oracle_opts(o: "hc.TrackOpts"):
    return oracle.TrackOpts(lambda0=o.lambda0, lambda_min=o.lambda_min, lambda_max=o.lambda_max,
                            grow=o.grow, shrink=o.shrink, eps=o.eps, eps_x=o.eps_x,
                            eps_end=o.eps_end, eps_end_x=o.eps_end_x, div_bound=o.div_bound,
                            max_it=o.max_it, end_it=o.end_it, grow_after=o.grow_after,
                            max_steps=o.max_steps, predictor=o.predictor, lu_mode=o.lu_mode,
                            max_refine=o.max_refine)


def copy_states(st):
    out = hc.new_states(len(st))
    ct.memmove(out, st, ct.sizeof(st))
    return out


class GpuPath:
    """One path on the GPU, advanced by hc_track_resume; its state, point and history can
    be saved and restored."""

    def __init__(self, torch, s, gamma, L, opts):
        self.torch, self.s, self.L, self.opts = torch, s, L, opts
        self.h = hc.system_from(s, L, gamma)
        self.x = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(s.n), L)])).cuda()
        self.hist = torch.zeros(3 * self.x.numel(), dtype=torch.float64, device="cuda")
        self.st = hc.new_states(1)

    def advance(self, k, log_cap=0):
        log = None
        if log_cap:
            log = self.torch.zeros(log_cap * hc.STEP_RECORD_DTYPE.itemsize, dtype=self.torch.uint8, device="cuda")
        stats = hc.hc_track_resume([self.h], self.x, self.hist, self.st, k, self.opts, log, log_cap)
        self.torch.cuda.synchronize()
        if log_cap:
            return stats[0], log.cpu().numpy().view(hc.STEP_RECORD_DTYPE)
        return stats[0]

    def save(self):
        return copy_states(self.st), self.x.clone(), self.hist.clone()

    def restore(self, saved):
        st, x, hist = saved
        self.st = copy_states(st)
        self.x.copy_(x)
        self.hist.copy_(hist)

    def points(self):
        """(z, zp, zpp) as limbs [n][2][L]."""
        n, L = self.s.n, self.L
        z = hc.unpack_paths(self.x.cpu().numpy(), [n], L)[0]
        zp, zpp = hc.unpack_hist(self.hist.cpu().numpy(), [n], L)
        return z, zp[0], zpp[0]

    def free(self):
        self.h.free()


def to_oracle_state(g) -> "oracle.PathState":
    o = oracle.PathState()
    for a, b in (("t", "t"), ("tp", "tp"), ("tpp", "tpp"), ("lam", "lambda_"), ("min_step", "minstep"),
                 ("sum_step", "sumstep"), ("res_end", "res_end"), ("n_succ", "n_succ"), ("n_corr", "n_corr"),
                 ("newton_its", "nits"), ("nhist", "nhist"), ("consec", "consec"), ("status", "status"),
                 ("phase", "phase"), ("end_its", "end_its")):
        setattr(o, a, getattr(g, b))
    return o


EXACT = (("t", "t"), ("tp", "tp"), ("tpp", "tpp"), ("lam", "lambda_"), ("n_succ", "n_succ"),
         ("n_corr", "n_corr"), ("newton_its", "nits"), ("nhist", "nhist"), ("consec", "consec"),
         ("status", "status"), ("phase", "phase"), ("end_its", "end_its"), ("sum_step", "sumstep"))


def compare_states(gst, gpts, ost, opts_, L, where=""):
    """The GPU's state and points after some stages against the oracle's from the same
    saved state.  Returns the largest relative error of the points."""
    for a, b in EXACT:
        assert getattr(ost, a) == getattr(gst, b), (where, a, getattr(ost, a), getattr(gst, b))
    worst = 0.0
    nh = gst.nhist if gst.phase != 0 else 1
    for k, (g, o) in enumerate(zip(gpts, opts_)):
        if k >= nh:
            break
        e = rel_err_per_point(g[None], o[None])[0]
        assert e <= TOL[L], (where, k, e)
        worst = max(worst, e)
    return worst


def check_stages(torch, s, gamma, L, opts, checkpoints, k=2, tail=0, every=128, threads=None):
    """Advance one path through the stage numbers in `checkpoints` (and, with tail > 0,
    on to its end, to the stage `tail` stages before it); from each saved state run k
    stages on the GPU and in the oracle (in threads) and compare.  Returns a list of
    (checkpoint, phase after, largest point error, log10 condition estimate after)."""
    p = GpuPath(torch, s, gamma, L, opts)
    saved = []
    for c in sorted(set(checkpoints)):
        if c > p.st[0].n_corr:
            p.advance(c - p.st[0].n_corr)
        if p.st[0].phase == 3:
            break
        saved.append((c, p.save(), p.points()))
    if tail and p.st[0].phase != 3:
        keep = [(p.st[0].n_corr, p.save())]
        while p.st[0].phase != 3:
            p.advance(every)
            if p.st[0].phase != 3:
                keep.append((p.st[0].n_corr, p.save()))
        c = max(p.st[0].n_corr - tail, 0)
        at, sv = [x for x in keep if x[0] <= c][-1]
        p.restore(sv)
        if c > at:
            p.advance(c - at)
        # Near the end of a path that goes to infinity the Jacobian's entries can pass
        # 1e154, and the squared moduli of the pivot search overflow double range (the
        # condition estimate is +inf); accept or reject is then decided by overflow on
        # both sides.  The end check takes the last state from which the next k stages
        # still factor finite matrices.
        cands = [(c, p.save())] + [x for x in reversed(keep) if x[0] < c]
        for c, sv in cands:
            p.restore(sv)
            p.advance(k)
            if np.isfinite(p.st[0].cond):
                p.restore(sv)
                saved.append((c, p.save(), p.points()))
                break
    results = []
    for c, sv, _ in saved:
        p.restore(sv)
        p.advance(k)
        results.append((c, copy_states(p.st)[0], p.points()))
    p.free()
    g = np.array([gamma.real, gamma.imag])
    oo = oracle_opts(opts)

    def run(item):
        c, sv, (z, zp, zpp) = item
        st, oz, ozp, ozpp, _, _ = oracle.track_resume(s.as_dict(), s.coef_limbs(L), g, oo, to_oracle_state(sv[0][0]),
                                                      z, zp, zpp, k)
        return st, (oz, ozp, ozpp)

    with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
        orc = list(ex.map(run, saved))
    out = []
    for (c, gst, gpts), (ost, opts_) in zip(results, orc):
        out.append((c, gst.phase, compare_states(gst, gpts, ost, opts_, L, where=f"stage {c} (cond 1e{gst.cond:.1f})"),
                    round(gst.cond, 1)))
    return out
