"""hc_track_resume (checkpoint / resume of the tracker, Alg. 3.1): a path advanced in
chunks of stages is the path of one hc_track_path call, bit for bit, in every mode; and
from saved states at stages along a path the GPU and the oracle take the same stages
(status, counts, t and step exactly; points at 1e-28 / 1e-58), including the code paths
of full-size systems: FP64 factors in global memory (n > 57 in double-double), QD at
three blocks per SM with n = 40 (the shapes of Table 4)."""
import numpy as np
import pytest

from gpu_util import torch_cuda
from resume_util import GpuPath, check_stages, copy_states
from test_gpu_track import gpu_track, regular_family
from paper_1109_0545_gb300 import hc, synth

pytestmark = pytest.mark.gpu


# Refinement sweeps of the stage checks: enough for the FP64-LU solve to reach the working
# precision at condition numbers up to about 1e8 (each sweep gains about 16 - log10(cond)
# digits); with fewer sweeps an ill-conditioned stage stops short of it, and the GPU's
# and the oracle's FP64 factorisations (FMA against split products) leave different
# remainders
REFINE = {1: 4, 2: 6, 4: 12}

MODES = [("persistent", dict()), ("graph", dict(mode=hc.HC_TRACK_GRAPH, graph_steps=4)),
         ("grid", dict(mode=hc.HC_TRACK_GRID))]


@pytest.mark.parametrize("mode", [m[0] for m in MODES])
@pytest.mark.parametrize("pred", [hc.HC_PRED_SECANT, hc.HC_PRED_QUADRATIC])
def test_resume_in_chunks_equals_one_call(mode, pred):
    torch = torch_cuda()
    fam = regular_family(700 + pred, 4, 3)
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=pred, **dict(MODES)[mode])
    ref_st, ref_end, ref_log = gpu_track(torch, systems, gammas, 2, opts, log_cap=600)
    handles = [hc.system_from(s, 2, g) for s, g in fam]
    x = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(s.n), 2) for s in systems])).cuda()
    hist = torch.zeros(3 * x.numel(), dtype=torch.float64, device="cuda")
    states = hc.new_states(len(systems))
    logs = [[] for _ in systems]
    chunk = 9
    for call in range(200):
        before = [states[p].n_corr for p in range(len(systems))]
        log = torch.zeros(len(systems) * chunk * hc.STEP_RECORD_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        stats = hc.hc_track_resume(handles, x, hist, states, chunk, opts, log, chunk)
        recs = log.cpu().numpy().view(hc.STEP_RECORD_DTYPE).reshape(len(systems), chunk)
        for p in range(len(systems)):
            took = states[p].n_corr - before[p]
            assert 0 <= took <= chunk
            logs[p].append(recs[p, :took])
        if all(states[p].phase == 3 for p in range(len(systems))):
            break
    assert stats == ref_st
    ends = hc.unpack_paths(x.cpu().numpy(), [s.n for s in systems], 2)
    for p in range(len(systems)):
        assert np.array_equal(ends[p], ref_end[p])
        assert np.array_equal(np.concatenate(logs[p]), ref_log[p, :ref_st[p]["n_corr"]])
    for h in handles:
        h.free()


def test_resume_with_the_tangent_predictor_equals_one_call():
    """The tangent rides in the third history vector between calls."""
    torch = torch_cuda()
    fam = regular_family(710, 3, 3)
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_TANGENT)
    ref_st, ref_end, _ = gpu_track(torch, systems, gammas, 2, opts)
    for p, (s, g) in enumerate(fam):
        gp = GpuPath(torch, s, g, 2, opts)
        for _ in range(500):
            stats = gp.advance(5)
            if gp.st[0].phase == 3:
                break
        assert stats == ref_st[p]
        assert np.array_equal(gp.points()[0], ref_end[p])
        gp.free()


def test_a_stopped_path_continues_after_raising_the_stage_cap():
    """A path stopped at HC_MAX_STEPS resumes (phase 1, status OK, a larger cap) and ends
    as the uncapped path does."""
    torch = torch_cuda()
    (s, g), = regular_family(720, 1, 3)
    full = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE)
    ref_st, ref_end, _ = gpu_track(torch, [s], [g], 2, full)
    capped = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, max_steps=10)
    gp = GpuPath(torch, s, g, 2, capped)
    gp.advance(1000)
    assert gp.st[0].status == hc.HC_MAX_STEPS and gp.st[0].phase == 3 and gp.st[0].n_corr == 10
    gp.st[0].status, gp.st[0].phase = hc.HC_OK, 1
    gp.opts = full
    stats = gp.advance(100000)
    assert stats == ref_st[0]
    assert np.array_equal(gp.points()[0], ref_end[0])
    gp.free()


@pytest.mark.parametrize("L", [1, 2, 4])
def test_stages_from_saved_states_match_the_oracle(L):
    torch = torch_cuda()
    eps = {1: 1e-12, 2: 1e-26, 4: 1e-58}[L]
    for pred in (hc.HC_PRED_SECANT, hc.HC_PRED_QUADRATIC):
        (s, g), = regular_family(730 + L + pred, 1, 4)
        opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=pred, eps=eps, eps_end=eps,
                                        eps_end_x=eps, max_refine=REFINE[L])
        out = check_stages(torch, s, g, L, opts, [0, 1, 2, 5, 17, 40], k=3, tail=3)
        print(L, pred, out)
        assert len(out) >= 4


def test_full_size_dd_path_with_global_memory_factors():
    """n = 62 regular-variant system (20..200 monomials per polynomial, k 2..8): with four
    blocks per SM its FP64 factors do not fit in shared memory (n > 57), so the solves
    read them from global memory; both LU modes, stages 0..3 and 9..11 vs the oracle."""
    torch = torch_cuda()
    rng = np.random.default_rng(740)
    s = synth.regular_system(rng, 62, (20, 200), (2, 8), (1, 3), lead=1)
    g = synth.unit_complex(rng)
    for lu in (hc.HC_LU_FP64_REFINE, hc.HC_LU_NATIVE):
        opts = hc.hc_track_opts_default(lu_mode=lu, predictor=hc.HC_PRED_QUADRATIC, max_refine=REFINE[2])
        out = check_stages(torch, s, g, 2, opts, [0, 2, 9], k=3)
        print("n = 62", lu, out)
        assert [c for c, _, _, _ in out] == [0, 2, 9]


@pytest.mark.parametrize("deg", [2, 20])
def test_table4_shape_qd_stages_match_the_oracle(deg):
    """Table 4's shape in complex QD (n = 40, 40 monomials of degree `deg` per polynomial,
    regular variant), three blocks per SM: stages 0..2, three stages from each of two
    later saved states, and the last three stages with the end game, vs the QD oracle at
    1e-58; the same on the whole-GPU engine."""
    torch = torch_cuda()
    s, g = synth.paper_dim_degree(40, 40, 40, deg)
    for mode in (hc.HC_TRACK_PERSISTENT, hc.HC_TRACK_GRID):
        opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_QUADRATIC, mode=mode,
                                        eps=1e-58, eps_end=1e-58, eps_end_x=1e-58, max_refine=REFINE[4])
        out = check_stages(torch, s, g, 4, opts, [0, 30, 90], k=3, tail=3)
        print("table 4", deg, mode, out)
        assert len(out) == 4 and out[-1][1] == 3


def test_table4_degree20_end_point_is_a_root_and_engines_agree():
    """Table 4, degree 20, QD: the path tracked to its end on one block and on the whole
    GPU: the same statuses, stage counts and accept sequence, end points equal within
    1e-58, and the QD oracle's Newton step from the end point moves it by less than 1e-58
    relative with a residual at QD rounding."""
    import oracle
    from helpers import TOL, rel_err_per_point
    torch = torch_cuda()
    s, g = synth.paper_dim_degree(40, 40, 40, 20)
    runs = []
    for mode in (hc.HC_TRACK_PERSISTENT, hc.HC_TRACK_GRID):
        opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_QUADRATIC, mode=mode,
                                        eps=1e-58, eps_end=1e-58, eps_end_x=1e-58)
        runs.append(gpu_track(torch, [s], [g], 4, opts, log_cap=2000))
    (a_st, a_end, a_log), (b_st, b_end, b_log) = runs
    assert a_st[0]["status"] == hc.HC_OK == b_st[0]["status"]
    assert (a_st[0]["n_succ"], a_st[0]["n_corr"]) == (b_st[0]["n_succ"], b_st[0]["n_corr"])
    n = a_st[0]["n_corr"]
    assert np.array_equal(a_log[0, :n]["accepted"], b_log[0, :n]["accepted"])
    assert rel_err_per_point(a_end[0][None], b_end[0][None])[0] <= TOL[4]
    ga = np.array([g.real, g.imag])
    xn, res, stn, _ = oracle.newton_step(s.as_dict(), s.coef_limbs(4), a_end[0][None], -1.0, ga, 1, 6)
    assert stn[0] == 0
    move = rel_err_per_point(xn, a_end[0][None])[0]
    print(f"degree 20: {n} stages, oracle Newton moves the end point by {move:.2e}, residual {res[0]:.2e}")
    assert move <= TOL[4]
