"""Host logic of the step proposer: the feature records built from a tracker log follow
the definition in include/hc.h (the same one the tracker kernel evaluates)."""
import math

import numpy as np

from paper_1109_0545_gb300 import hc, learn


def _log(rows):
    recs = np.zeros(len(rows), dtype=hc.STEP_RECORD_DTYPE)
    for k, (t, lam, res, pcd, cond, it, acc) in enumerate(rows):
        recs[k] = (t, lam, 1.0, res, pcd, cond, it, acc)
    return recs


def test_features_follow_the_definition():
    lam0 = 0.01
    rows = [(0.0, 0.01, 1e-20, 3e-4, 1.5, 2, 1),
            (0.01, 0.01, 1e-9, -1.0, 2.0, 3, 0),
            (0.01, 0.005, 1e-30, 1e-6, 2.5, 1, 1),
            (0.015, 0.005, 0.0, 2e-7, 3.0, 2, 1)]
    X, r, a = learn.features(_log(rows), 4, lam0)
    assert X.shape == (3, 12) and r.shape == (3,) and a.tolist() == [0, 1, 1]
    # stage 1: history = stage 0, then missing (lambda0, 0 iterations, residual -4)
    f = X[0]
    assert f[0] == np.float32(0.01)
    assert f[1] == 0.0 and f[2] == 0.0 and f[3] == 0.0
    assert f[4] == np.float32(0.5) and f[5] == 0.0 and f[6] == 0.0
    assert f[7] == np.float32(-2.0) and f[8] == -4.0 and f[9] == -4.0
    assert abs(f[10] - math.log10(3e-4) / 10) < 1e-6
    assert f[11] == np.float32(1.5 / 4)
    # stage 3: history stages 2, 1, 0; stage 2 was after a rejection (pc distance -1)
    f = X[2]
    assert abs(f[1] - math.log2(0.5) / 8) < 1e-7 and f[2] == 0.0 and f[3] == 0.0
    assert f[4] == np.float32(0.25) and f[5] == np.float32(0.75) and f[6] == np.float32(0.5)
    assert f[7] == np.float32(-3.0) and f[8] == np.float32(-0.9) and f[9] == np.float32(-2.0)
    assert abs(f[10] - (-0.6)) < 1e-6
    # targets: log2 of the step ratio to the previous attempt
    assert r.tolist() == [0.0, -1.0, 0.0]
    # the residual clip at -40 and the -4 for a rejection's distance
    X2, _, _ = learn.features(_log([(0.0, 0.01, 1e-300, -1.0, 0.0, 3, 0), (0.0, 0.005, 1e-3, -1.0, 0.0, 3, 0)]), 2, lam0)
    assert X2[0][7] == -4.0 and X2[0][10] == -4.0


def test_initial_parameters():
    p = learn.init_params(0)
    assert p.shape == (hc.HC_MLP_NPARAM,) and p.dtype == np.float32
    assert np.all(p[768:832] == 0) and np.all(p[4928:4992] == 0) and p[5056] == 0
