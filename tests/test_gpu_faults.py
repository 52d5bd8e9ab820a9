"""Failure detection of the tracker, injected from the host (no fault on the device): a
stage cap, an unreachable end tolerance, a non-finite start point, a divergence bound
below the path's norm, and a tiny minimum step.  Each path ends with the status the
oracle tracker gives, in every execution mode."""
import numpy as np
import pytest

from gpu_util import torch_cuda
from test_gpu_track import gpu_track, oracle_opts, regular_family
import oracle
from paper_1109_0545_gb300 import hc, synth

pytestmark = pytest.mark.gpu

CASES = {
    "MAX_STEPS": dict(max_steps=5),
    "NOCONV": dict(end_it=1, eps_end=1e-300, eps_end_x=1e-300),
    "DIVERGED": dict(div_bound=0.5),
    "MIN_STEP": dict(lambda_min=0.004, max_it=1, eps=1e-300, eps_x=1e-30),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("mode", [hc.HC_TRACK_PERSISTENT, hc.HC_TRACK_GRAPH, hc.HC_TRACK_GRID])
def test_injected_failures_give_the_oracle_status(name, mode):
    torch = torch_cuda()
    fam = regular_family(460, 2, 3)
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, mode=mode, **CASES[name])
    stats, _, _ = gpu_track(torch, systems, gammas, 2, opts)
    for s, g, st in zip(systems, gammas, stats):
        r = oracle.track(s.as_dict(), s.coef_limbs(2), synth.limbs(np.ones(s.n), 2),
                         np.array([g.real, g.imag]), oracle_opts(opts))
        assert hc.STATUS_NAMES[st["status"]] == name == oracle.STATUS[r.status]
        assert (st["n_succ"], st["n_corr"]) == (r.n_succ, r.n_corr)


def test_nonfinite_start_point():
    torch = torch_cuda()
    fam = regular_family(461, 1, 3)
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    start = synth.limbs(np.ones(3), 2)
    start[1, 0, 0] = np.nan
    stats, ends, _ = gpu_track(torch, systems, gammas, 2, hc.hc_track_opts_default(max_steps=50),
                               starts=[start])
    # every corrector stage fails on a non-finite residual; the step shrinks to the cap
    assert stats[0]["status"] in (hc.HC_MAX_STEPS, hc.HC_MIN_STEP)
    assert stats[0]["n_succ"] == 0


def test_invalid_options_are_rejected_before_any_launch():
    torch = torch_cuda()
    fam = regular_family(462, 1, 3)
    handles = [hc.system_from(s, 2, g) for s, g in fam]
    x0 = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(3), 2)])).cuda()
    x1 = torch.zeros_like(x0)
    for bad in (dict(lambda0=-1.0), dict(shrink=1.5), dict(max_it=0), dict(predictor=7),
                dict(mode=9), dict(mode=hc.HC_TRACK_GRID, lu_mode=hc.HC_LU_NATIVE),
                dict(predictor=hc.HC_PRED_TANGENT, lu_mode=hc.HC_LU_NATIVE),
                dict(predictor=hc.HC_PRED_TANGENT, lu_mode=hc.HC_LU_FP64_REFINE, mode=hc.HC_TRACK_GRID),
                dict(explore=-1.0)):
        with pytest.raises(hc.HCError) as e:
            hc.hc_track_path(handles, x0, x1, hc.hc_track_opts_default(**bad))
        assert e.value.code == hc.HC_EINVAL
    for h in handles:
        h.free()
