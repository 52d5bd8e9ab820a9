"""The whole-GPU engine for one large path (HC_TRACK_GRID): against the oracle tracker on
small systems, against the block-per-path engine, and on the large QD workload (n = 96,
96 x 1024 monomials, k = 12) with checks that hold at any size."""
import numpy as np
import pytest

from helpers import TOL, rel_err_per_point
from gpu_util import torch_cuda
from test_gpu_track import compare_with_oracle, gpu_track, regular_family
import oracle
from paper_1109_0545_gb300 import hc, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [2, 4])
def test_grid_engine_matches_oracle(L):
    torch = torch_cuda()
    fam = regular_family(440 + L, 4, 3)
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, mode=hc.HC_TRACK_GRID)
    if L == 4:
        opts.eps, opts.eps_end, opts.eps_end_x = 1e-58, 1e-58, 1e-58
    stats, ends, _ = gpu_track(torch, systems, gammas, L, opts)
    assert compare_with_oracle(systems, gammas, L, opts, stats, ends) == len(systems)


def test_grid_engine_agrees_with_block_engine():
    torch = torch_cuda()
    fam = regular_family(450, 5, 4)
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    block = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE)
    grid = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, mode=hc.HC_TRACK_GRID)
    a_st, a_ends, a_log = gpu_track(torch, systems, gammas, 2, block, log_cap=600)
    b_st, b_ends, b_log = gpu_track(torch, systems, gammas, 2, grid, log_cap=600)
    for p in range(len(systems)):
        assert a_st[p]["status"] == b_st[p]["status"]
        assert (a_st[p]["n_succ"], a_st[p]["n_corr"]) == (b_st[p]["n_succ"], b_st[p]["n_corr"])
        assert np.array_equal(a_log[p]["accepted"], b_log[p]["accepted"])
        assert rel_err_per_point(a_ends[p][None], b_ends[p][None])[0] <= TOL[2]


def test_large_qd_path_stages_match_the_qd_oracle():
    """The large single path (n = 96, 96 x 1024 monomials, k = 12, exponents 1..5, complex
    QD, FP64 LU with QD refinement) on the whole GPU, tracked until it stops: the path goes
    to infinity as t approaches 1, and the step falls below its minimum.  Saved states at
    stages 0, 1, 2, 40, 160, 1000 and near the end (two stages before it, or the last
    saved state before the Jacobian's entries grow past 1e154 and the pivot search's
    squared moduli overflow); from each, the GPU and the QD oracle (on the full system)
    take the same corrector stage: status, counts, t and step exactly, the corrected
    point (and the history) within 1e-58."""
    from resume_util import check_stages
    torch = torch_cuda()
    s, g = synth.large_path_qd(4)
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, mode=hc.HC_TRACK_GRID,
                                    eps=1e-58, eps_end=1e-58, eps_end_x=1e-58, max_refine=12)
    out = check_stages(torch, s, g, 4, opts, [0, 1, 2, 40, 160, 1000], k=1, tail=2, every=256)
    print("large QD path, (stage, phase, worst relative error, log10 cond):", out)
    assert [c for c, _, _, _ in out][:6] == [0, 1, 2, 40, 160, 1000] and len(out) == 7


def test_large_qd_path_log_is_consistent():
    """300 corrector stages of the large QD path: one log record per stage, the accepted
    ones adding up to the t reached, and the same statistics through hc_track_resume in
    chunks of 100 stages."""
    from resume_util import GpuPath
    torch = torch_cuda()
    s, g = synth.large_path_qd(4)
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, mode=hc.HC_TRACK_GRID,
                                    max_steps=300, eps=1e-58, eps_end=1e-58, eps_end_x=1e-58)
    import time
    t0 = time.perf_counter()
    st, ends, recs = gpu_track(torch, [s], [g], 4, opts, log_cap=400)
    dt = time.perf_counter() - t0
    st, x, lg = st[0], ends[0], recs[0][:st[0]["n_corr"]]
    print(f"large QD path: {hc.STATUS_NAMES[st['status']]}, {st['n_succ']} of {st['n_corr']} stages "
          f"accepted, t = {st['t_end']:.6f}, {st['newton_its']} Newton iterations, {dt:.1f} s "
          f"({st['n_corr'] / dt:.1f} stages/s)")
    assert st["n_corr"] == len(lg) and lg["accepted"].sum() == st["n_succ"]
    assert abs(lg["lam"][lg["accepted"] == 1].sum() - st["t_end"]) < 1e-12
    gp = GpuPath(torch, s, g, 4, opts)
    for _ in range(10):
        stats = gp.advance(100)
        if gp.st[0].phase == 3:
            break
    assert stats == st
    assert np.array_equal(gp.points()[0], x)
    gp.free()
