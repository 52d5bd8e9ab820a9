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


def test_large_qd_path_on_the_whole_gpu():
    """n = 96, 96 x 1024 monomials, k = 12, exponents 1..5, complex QD, FP64 LU with QD
    refinement, from (1..1), at most 300 corrector stages.  Too large for the oracle to
    track; checked: every logged stage is consistent with the statistics, accepted steps
    add up to t_end, and the residual of the oracle at the current point of a stage the
    GPU accepted (sampled rows, QD) is at the corrector's tolerance."""
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
    assert st["status"] in (hc.HC_OK, hc.HC_MAX_STEPS, hc.HC_MIN_STEP, hc.HC_DIVERGED)
    # the current point solves h(., t_end) to the corrector's tolerance on sampled rows
    if st["n_succ"] > 0 and st["t_end"] < 1.0:
        from test_gpu_eval import _rows_subsystem
        rows = [0, 50, 95]
        sub = _rows_subsystem(s, rows)
        f, _, _ = oracle.evaluate(sub.as_dict(), sub.coef_limbs(4), x[None], -1.0, np.array([g.real, g.imag]),
                                  jac=False)
        deg = oracle.degrees(s.as_dict())
        t = st["t_end"]
        # h_i = gamma (1-t) (x_i^d_i - 1) + t f_i, in double from the leading limbs
        z = x[:, 0, 0] + 1j * x[:, 1, 0]
        h = [g * (1 - t) * (z[i] ** int(deg[i]) - 1) + t * (f[0, k, 0, 0] + 1j * f[0, k, 1, 0])
             for k, i in enumerate(rows)]
        scale = max(1.0, np.abs(z).max()) ** int(deg.max()) * 1024
        assert max(abs(v) for v in h) <= 1e-10 * scale
