"""A path of the shape of Table 4 (n = 40, 40 monomials of degree 2 per polynomial, complex
QD, quadratic predictor; regular variant): the block engine and the whole-GPU engine take
the same decisions and reach the same end point, a root of f to QD accuracy (checked by the
oracle's evaluation of f at the end point)."""
import numpy as np
import pytest

from helpers import TOL, rel_err_per_point
from gpu_util import torch_cuda
from test_gpu_track import gpu_track
import oracle
from paper_1109_0545_gb300 import hc, synth

pytestmark = pytest.mark.gpu


def test_table4_shape_path_in_qd_on_both_engines():
    torch = torch_cuda()
    s, g = synth.paper_dim_degree(40, 40, 40, 2)
    kw = dict(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_QUADRATIC, eps=1e-58, eps_end=1e-58,
              eps_end_x=1e-58)
    a_st, a_end, a_log = gpu_track(torch, [s], [g], 4, hc.hc_track_opts_default(**kw), log_cap=2000)
    b_st, b_end, b_log = gpu_track(torch, [s], [g], 4, hc.hc_track_opts_default(mode=hc.HC_TRACK_GRID, **kw),
                                   log_cap=2000)
    a, b = a_st[0], b_st[0]
    print(f"n = 40, degree 2, QD: {hc.STATUS_NAMES[a['status']]}, {a['n_succ']} of {a['n_corr']} stages, "
          f"avg step {a['avg_step']:.3g}, min step {a['min_step']:.3g}")
    assert a["status"] == b["status"] == hc.HC_OK
    assert (a["n_succ"], a["n_corr"]) == (b["n_succ"], b["n_corr"])
    assert np.array_equal(a_log[0]["accepted"][:a["n_corr"]], b_log[0]["accepted"][:b["n_corr"]])
    assert rel_err_per_point(a_end[0][None], b_end[0][None])[0] <= TOL[4]
    x = a_end[0]
    f, _, _ = oracle.evaluate(s.as_dict(), s.coef_limbs(4), x[None], -1.0, np.array([g.real, g.imag]), jac=False)
    res = np.abs(f[0, :, 0, 0] + 1j * f[0, :, 1, 0]).max()
    z = np.abs(x[:, 0, 0] + 1j * x[:, 1, 0]).max()
    assert res <= 1e-55 * max(1.0, z) ** 3 * 42
