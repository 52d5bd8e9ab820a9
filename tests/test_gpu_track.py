"""hc_track_path against the oracle tracker (Alg. 3.1 + Alg. 4.1, same readings, same
options): per path the status, the accepted/total corrector stages, and the end point
within the tolerance of the precision; batched (one launch for all paths) and one path
per launch agree bit for bit; the persistent kernel and the graph-stepped mode agree
bit for bit."""
import numpy as np
import pytest

from helpers import TOL, digits, rel_err_per_point
from gpu_util import torch_cuda
import oracle
from paper_1109_0545_gb300 import hc, synth

pytestmark = pytest.mark.gpu


def oracle_opts(o: "hc.TrackOpts"):
    return oracle.TrackOpts(lambda0=o.lambda0, lambda_min=o.lambda_min, lambda_max=o.lambda_max,
                            grow=o.grow, shrink=o.shrink, eps=o.eps, eps_x=o.eps_x,
                            eps_end=o.eps_end, eps_end_x=o.eps_end_x, div_bound=o.div_bound,
                            max_it=o.max_it, end_it=o.end_it, grow_after=o.grow_after,
                            max_steps=o.max_steps, predictor=o.predictor, lu_mode=o.lu_mode,
                            max_refine=o.max_refine)


def gpu_track(torch, systems, gammas, L, opts, starts=None, log_cap=0):
    handles = [hc.system_from(s, L, g) for s, g in zip(systems, gammas)]
    if starts is None:
        starts = [synth.limbs(np.ones(s.n), L) for s in systems]
    x0 = torch.from_numpy(hc.pack_paths(starts)).cuda()
    x1 = torch.zeros_like(x0)
    log = None
    if log_cap:
        log = torch.zeros(len(systems) * log_cap * hc.STEP_RECORD_DTYPE.itemsize, dtype=torch.uint8,
                          device="cuda")
    stats = hc.hc_track_path(handles, x0, x1, opts, log, log_cap)
    torch.cuda.synchronize()
    ends = hc.unpack_paths(x1.cpu().numpy(), [s.n for s in systems], L)
    recs = None
    if log_cap:
        recs = log.cpu().numpy().view(hc.STEP_RECORD_DTYPE).reshape(len(systems), log_cap)
    for h in handles:
        h.free()
    return stats, ends, recs


def regular_family(seed, count, n, L_lead=3):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        s = synth.regular_system(rng, n, 4, (1, min(2, n)), (1, 2), lead=L_lead)
        out.append((s, synth.unit_complex(rng)))
    return out


def compare_with_oracle(systems, gammas, L, opts, stats, ends, strict_counts=True):
    oo = oracle_opts(opts)
    n_ok = 0
    for s, g, st, x in zip(systems, gammas, stats, ends):
        r = oracle.track(s.as_dict(), s.coef_limbs(L), synth.limbs(np.ones(s.n), L),
                         np.array([g.real, g.imag]), oo)
        assert st["status"] == r.status, (st, oracle.STATUS[r.status])
        if strict_counts:
            assert (st["n_succ"], st["n_corr"]) == (r.n_succ, r.n_corr)
        if r.status == 0:
            e = rel_err_per_point(x[None], r.x[None])
            assert e[0] <= TOL[L], (e, digits(e))
            n_ok += 1
    return n_ok


@pytest.mark.parametrize("lu_mode", [hc.HC_LU_NATIVE, hc.HC_LU_FP64_REFINE])
def test_regular_systems_dd_match_oracle(lu_mode):
    torch = torch_cuda()
    fam = regular_family(400, 8, 3)
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    opts = hc.hc_track_opts_default(lu_mode=lu_mode)
    stats, ends, _ = gpu_track(torch, systems, gammas, 2, opts)
    n_ok = compare_with_oracle(systems, gammas, 2, opts, stats, ends)
    print(f"lu_mode={lu_mode}: {n_ok} of {len(systems)} paths end at a root; statuses "
          f"{[hc.STATUS_NAMES[s['status']] for s in stats]}")
    assert n_ok == len(systems)


@pytest.mark.parametrize("L", [1, 4])
def test_regular_systems_double_and_qd(L):
    torch = torch_cuda()
    fam = regular_family(410, 4, 2)
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    opts = hc.hc_track_opts_default()
    if L == 1:
        opts.eps, opts.eps_end, opts.eps_end_x = 1e-12, 1e-12, 1e-12
    else:
        opts.eps, opts.eps_end, opts.eps_end_x = 1e-58, 1e-58, 1e-58
    stats, ends, _ = gpu_track(torch, systems, gammas, L, opts)
    n_ok = compare_with_oracle(systems, gammas, L, opts, stats, ends)
    assert n_ok == len(systems)


def test_quadratic_predictor_matches_oracle():
    torch = torch_cuda()
    fam = regular_family(420, 6, 3)
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    opts = hc.hc_track_opts_default(predictor=hc.HC_PRED_QUADRATIC)
    stats, ends, _ = gpu_track(torch, systems, gammas, 2, opts)
    assert compare_with_oracle(systems, gammas, 2, opts, stats, ends) == len(systems)


def test_single_path_workload_matches_oracle():
    """n = 8, 12 monomials + constant, k = 3: the path from (1..1) goes to infinity;
    both trackers take the same stages and stop the same way."""
    torch = torch_cuda()
    s, g = synth.single_path_dd(1)
    opts = hc.hc_track_opts_default()
    stats, ends, _ = gpu_track(torch, [s], [g], 2, opts)
    r = oracle.track(s.as_dict(), s.coef_limbs(2), synth.limbs(np.ones(8), 2),
                     np.array([g.real, g.imag]), oracle_opts(opts))
    st = stats[0]
    print("gpu", st, "oracle", oracle.STATUS[r.status], r.n_succ, r.n_corr, r.t_end)
    assert st["status"] == r.status
    assert (st["n_succ"], st["n_corr"]) == (r.n_succ, r.n_corr)
    assert st["t_end"] == r.t_end


def test_graph_mode_and_one_path_per_launch_agree_bitwise():
    torch = torch_cuda()
    fam = regular_family(430, 5, 3)
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    opts = hc.hc_track_opts_default()
    a_stats, a_ends, a_log = gpu_track(torch, systems, gammas, 2, opts, log_cap=400)
    g_opts = hc.hc_track_opts_default(mode=hc.HC_TRACK_GRAPH, graph_steps=8)
    b_stats, b_ends, b_log = gpu_track(torch, systems, gammas, 2, g_opts, log_cap=400)
    assert a_stats == b_stats
    for x, y in zip(a_ends, b_ends):
        assert np.array_equal(x, y)
    assert np.array_equal(a_log, b_log)
    for p in range(len(systems)):
        st, ends, _ = gpu_track(torch, [systems[p]], [gammas[p]], 2, opts)
        assert st[0] == a_stats[p] and np.array_equal(ends[0], a_ends[p])
    # the log holds one record per corrector stage; accepted steps add up to t_end
    for p, st in enumerate(a_stats):
        recs = a_log[p, :st["n_corr"]]
        assert recs["accepted"].sum() == st["n_succ"]
        assert abs(recs["lam"][recs["accepted"] == 1].sum() - st["t_end"]) < 1e-12


# the smallest members of the batched uneven-path family (n = 10..11 of 10..64)
UNEVEN_SMALL = [4, 5, 85, 131, 145, 148, 169, 227]


def _oracle_tracks(jobs):
    import os
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        return list(ex.map(lambda a: oracle.track(*a), jobs))


@pytest.mark.parametrize("pred", [hc.HC_PRED_SECANT, hc.HC_PRED_QUADRATIC])
def test_uneven_family_matches_the_oracle_up_to_the_stage_cap(pred):
    """Members of the batched uneven-path family (n 10..64, 20..200 monomials per
    polynomial, k 2..8, exponents 1..3), the eight smallest of the first 240, tracked
    together (FP64 LU + DD refinement) with a cap of 48 corrector stages.  The paths of
    this family go to infinity (a random sparse system has far fewer roots than the
    Bezout number of the total-degree homotopy), so every path is compared whatever its
    status: status, accepted and total stages and t reached equal the oracle's, and the
    current point at the cap agrees within 1e-28."""
    torch = torch_cuda()
    fam = [synth.uneven_path_system(3, j) for j in UNEVEN_SMALL]
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=pred, max_steps=48)
    stats, ends, _ = gpu_track(torch, systems, gammas, 2, opts)
    oo = oracle_opts(opts)
    refs = _oracle_tracks([(s.as_dict(), s.coef_limbs(2), synth.limbs(np.ones(s.n), 2),
                            np.array([g.real, g.imag]), oo) for s, g in fam])
    worst = 0.0
    for s, st, x, r in zip(systems, stats, ends, refs):
        assert st["status"] == r.status, (s.n, st, oracle.STATUS[r.status])
        assert (st["n_succ"], st["n_corr"], st["newton_its"]) == (r.n_succ, r.n_corr, r.newton_its)
        assert st["t_end"] == r.t_end
        e = rel_err_per_point(x[None], r.x[None])[0]
        assert e <= TOL[2], (s.n, e)
        worst = max(worst, e)
    print(f"{len(systems)} paths compared: statuses {[hc.STATUS_NAMES[x['status']] for x in stats]}, "
          f"t reached {[round(x['t_end'], 4) for x in stats]}, worst point error {worst:.1e} "
          f"({digits(np.array([worst])):.1f} digits)")
    assert len(refs) == len(UNEVEN_SMALL)


def test_uneven_family_paths_to_their_end_agree_with_the_oracle_along_the_way():
    """Four small members of the uneven family tracked by the GPU until they stop (at most
    6,000 corrector stages): from saved states at the start, a third, two thirds and the
    last stages of each path, the GPU and the oracle take the same three stages, the
    stopping stage included."""
    from resume_util import check_stages
    torch = torch_cuda()
    fam = [synth.uneven_path_system(3, j) for j in UNEVEN_SMALL[:4]]
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_QUADRATIC, max_steps=6000)
    stats, _, _ = gpu_track(torch, systems, gammas, 2, opts)
    print([(s.n, hc.STATUS_NAMES[st["status"]], st["n_corr"], round(st["t_end"], 6)) for s, st in zip(systems, stats)])
    checks = 0
    for s, g, st in zip(systems, gammas, stats):
        n = int(st["n_corr"])
        out = check_stages(torch, s, g, 2, opts, [0, n // 3, 2 * n // 3, max(n - 3, 0)], k=3)
        print(s.n, out)
        assert out and out[-1][1] == 3      # the last check reaches the path's end
        checks += len(out)
    assert checks >= 12


def test_exploration_perturbs_steps_reproducibly_and_the_oracle_replays_them():
    """explore = 0 is the plain tracker bit for bit; explore > 0 draws step ratios off the
    plain controller's powers of two, the same ones for the same seed, and the oracle
    following the accepted t sequence reaches the same end points."""
    torch = torch_cuda()
    fam = regular_family(470, 4, 3)
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    base = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE)
    st0, ends0, _ = gpu_track(torch, systems, gammas, 2, base)
    off = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, explore=0.0, explore_seed=99)
    st1, ends1, _ = gpu_track(torch, systems, gammas, 2, off)
    for a, b, x, y in zip(st0, st1, ends0, ends1):
        assert (a["n_succ"], a["n_corr"], a["status"]) == (b["n_succ"], b["n_corr"], b["status"])
        assert np.array_equal(x, y)
    o = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, explore=1.5, explore_seed=7)
    st, ends, recs = gpu_track(torch, systems, gammas, 2, o, log_cap=4000)
    st2, ends2, recs2 = gpu_track(torch, systems, gammas, 2, o, log_cap=4000)
    oo = oracle_opts(o)
    off_lattice = 0
    for p, (s, g) in enumerate(fam):
        lg = recs[p][:st[p]["n_corr"]]
        assert np.array_equal(lg, recs2[p][:st2[p]["n_corr"]])
        ratios = np.log2(lg["lam"][1:-1] / lg["lam"][:-2])
        off_lattice += int(np.sum(np.abs(ratios - np.round(ratios)) > 1e-9))
        assert np.all(lg["lam"] <= o.lambda_max * (1 + 1e-15))
        if st[p]["status"] != hc.HC_OK:
            continue
        acc = np.nonzero(lg["accepted"] == 1)[0]
        tseq = [lg["t"][k + 1] if k + 1 < len(lg) else 1.0 for k in acc]
        x1, status, fail = oracle.track_replay(s.as_dict(), s.coef_limbs(2), synth.limbs(np.ones(s.n), 2),
                                               np.array([g.real, g.imag]), oo, tseq)
        assert fail == -1 and status == 0
        assert rel_err_per_point(ends[p][None], x1[None])[0] <= TOL[2]
    assert off_lattice > 0


def test_tangent_predictor_reaches_the_oracle_end_points():
    """The Euler (tangent) predictor: every path ends at the oracle's end point (the oracle
    tracks with the secant predictor; same gamma, same start root, so the same root), in
    fewer corrector stages than the secant predictor, and the persistent and graph-stepped
    modes agree bit for bit."""
    torch = torch_cuda()
    fam = regular_family(480, 6, 4)
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    sec = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE)
    tan = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_TANGENT)
    s_st, _, _ = gpu_track(torch, systems, gammas, 2, sec)
    t_st, t_end, _ = gpu_track(torch, systems, gammas, 2, tan)
    assert compare_with_oracle(systems, gammas, 2, sec, t_st, t_end, strict_counts=False) == len(systems)
    n_sec = np.mean([x["n_corr"] for x in s_st])
    n_tan = np.mean([x["n_corr"] for x in t_st])
    print(f"secant {n_sec:.1f}, tangent {n_tan:.1f} stages per path")
    assert n_tan < n_sec
    g_st, g_end, _ = gpu_track(torch, systems, gammas, 2,
                               hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_TANGENT,
                                                        mode=hc.HC_TRACK_GRAPH, graph_steps=3))
    for a, b, x, y in zip(t_st, g_st, t_end, g_end):
        assert (a["n_succ"], a["n_corr"], a["status"]) == (b["n_succ"], b["n_corr"], b["status"])
        assert np.array_equal(x, y)
