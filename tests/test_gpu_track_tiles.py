"""The tracker's execution shape (hc_set_track_tiles; the tracker autotuner's knobs):
threads per path block (64 / 128 / 256 / 512; quad double runs 512 as 256), path blocks
per SM and the FP64 factors in
shared or global memory change nothing in the results, bit for bit -- statuses,
statistics, end points and step logs -- in the persistent and the graph-stepped modes;
the whole-GPU engine's chunk length changes only the order of an entry's additions
(statuses and stage counts equal, end points within the tolerance); and the autotuner
picks one of its candidates and caches it."""
import numpy as np
import pytest

from gpu_util import torch_cuda
from helpers import TOL, rel_err_per_point
from test_gpu_track import gpu_track, regular_family, UNEVEN_SMALL
from paper_1109_0545_gb300 import autotune, hc, synth

pytestmark = pytest.mark.gpu


def _families():
    fam2 = regular_family(760, 5, 3) + [synth.uneven_path_system(3, j) for j in UNEVEN_SMALL[:3]]
    fam4 = regular_family(761, 3, 2) + [synth.paper_dim_degree(20, 20, 20, 10)]
    return {2: fam2, 4: fam4}


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("mode", [hc.HC_TRACK_PERSISTENT, hc.HC_TRACK_GRAPH])
def test_block_engine_shapes_give_identical_results(L, mode):
    torch = torch_cuda()
    fam = _families()[L]
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    eps = {2: 1e-26, 4: 1e-58}[L]
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_QUADRATIC, mode=mode,
                                    graph_steps=8, max_steps=150, eps=eps, eps_end=eps, eps_end_x=eps)
    try:
        hc.hc_set_track_tiles(0, 0, 0, 0)
        ref = gpu_track(torch, systems, gammas, L, opts, log_cap=160)
        for tb in (64, 128, 256, 512):
            for bps in (0, 2):
                for factors in (0, 2):
                    hc.hc_set_track_tiles(tb, bps, factors, 0)
                    st, ends, log = gpu_track(torch, systems, gammas, L, opts, log_cap=160)
                    assert st == ref[0], (tb, bps, factors)
                    for a, b in zip(ends, ref[1]):
                        assert np.array_equal(a, b), (tb, bps, factors)
                    assert np.array_equal(log, ref[2]), (tb, bps, factors)
    finally:
        hc.hc_set_track_tiles(0, 0, 0, 0)


def test_grid_chunk_changes_only_the_rounding():
    torch = torch_cuda()
    fam = regular_family(762, 3, 3) + [synth.paper_dim_degree(40, 40, 40, 2)]
    systems, gammas = [f[0] for f in fam], [f[1] for f in fam]
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_QUADRATIC,
                                    mode=hc.HC_TRACK_GRID, eps=1e-58, eps_end=1e-58, eps_end_x=1e-58)
    try:
        hc.hc_set_track_tiles(0, 0, 0, 0)
        ref_st, ref_end, _ = gpu_track(torch, systems, gammas, 4, opts)
        for chunk in (16, 32, 64, 128):
            hc.hc_set_track_tiles(0, 0, 0, chunk)
            st, ends, _ = gpu_track(torch, systems, gammas, 4, opts)
            for a, b, x, y in zip(st, ref_st, ends, ref_end):
                assert (a["status"], a["n_succ"], a["n_corr"]) == (b["status"], b["n_succ"], b["n_corr"]), chunk
                assert rel_err_per_point(x[None], y[None])[0] <= TOL[4], chunk
                if chunk == 32:
                    assert np.array_equal(x, y)
    finally:
        hc.hc_set_track_tiles(0, 0, 0, 0)


def test_tracker_autotuner_picks_and_caches_a_shape(tmp_path, monkeypatch):
    torch = torch_cuda()
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "cache.json"))
    fam = [synth.uneven_path_system(3, j) for j in UNEVEN_SMALL[:4]]
    handles = [hc.system_from(s, 2, g) for s, g in fam]
    x0 = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(s.n), 2) for s, _ in fam])).cuda()
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, max_steps=20)
    cands = [(64, 0, 0), (128, 0, 2), (256, 2, 0)]
    try:
        got = autotune.tune_track(handles, x0, opts, candidates=cands)
        assert not got["cached"] and len(got["tried"]) == 3
        assert (got["threads_per_block"], got["blocks_per_sm"], got["factors"]) in cands
        tiles = hc.hc_get_track_tiles()
        assert (tiles["threads_per_block"], tiles["blocks_per_sm"], tiles["factors"]) == \
            (got["threads_per_block"], got["blocks_per_sm"], got["factors"])
        again = autotune.tune_track(handles, x0, opts, candidates=cands)
        assert again["cached"] and again["threads_per_block"] == got["threads_per_block"]
        (s, g) = synth.paper_dim_degree(40, 40, 40, 2)
        h = hc.system_from(s, 4, g)
        xq = torch.from_numpy(hc.pack_paths([synth.limbs(np.ones(s.n), 4)])).cuda()
        go = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, mode=hc.HC_TRACK_GRID, max_steps=6)
        ch = autotune.tune_grid_chunk(h, xq, go, candidates=(16, 64))
        assert ch["grid_chunk"] in (16, 64) and hc.hc_get_track_tiles()["grid_chunk"] == ch["grid_chunk"]
        h.free()
    finally:
        hc.hc_set_track_tiles(0, 0, 0, 0)
        for hh in handles:
            hh.free()
