"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own points,
combine nothing but the slowest time (the only collective), and the whole-job value is
the units of all ranks over that time; paths shard in blocks and their results gather
once, in order."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1109_0545_gb300 import synth
    s, pts, _ = synth.eval_throughput(2, npts=64)
    mine = bench.rank_points(rank, 64, s.n, pts)
    ms = 100.0 + 50.0 * rank               # this rank's own time
    tmax = bench.max_over_ranks(ms, dist)
    out[rank] = (float(np.abs(mine).sum()), float(mine[0, 0].real), tmax)
    dist.destroy_process_group()


def test_two_gloo_ranks_share_only_the_max_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    # both ranks see the slowest rank's time
    assert res[0][2] == res[1][2] == 150.0
    # the ranks work on different points of the same size (independent problems)
    assert res[0][1] != res[1][1]
    assert abs(res[0][0] - res[1][0]) < 1e-9 * res[0][0] + 1e-6  # |x| = 1 on the torus
    # whole-job value: units of every rank over the job's (max) time
    npts, steps = 64, 3
    value = npts * world * steps / (res[0][2] * steps * 1e-3)
    assert value == pytest.approx(npts * world / 0.150)


def _path_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    lo, hi = bench.shard_range(9, rank, world)
    # each rank "tracks" its own block of paths (here: records the path index it owns)
    mine = [{"path": p, "rank": rank} for p in range(lo, hi)]
    out[rank] = bench.gather_stats(mine, dist)
    dist.destroy_process_group()


def test_paths_shard_in_blocks_and_gather_in_order():
    import bench
    for n in (0, 1, 7, 9, 8192):
        for world in (1, 2, 3, 8):
            blocks = [bench.shard_range(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(blocks[r][1] == blocks[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_path_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert [x["path"] for x in res[r]] == list(range(9))
        assert [x["rank"] for x in res[r]] == [0] * 5 + [1] * 4


def _track_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1109_0545_gb300 import hc, synth
    torch.cuda.set_device(0)
    fam = [synth.uneven_path_system(3, j) for j in range(11)]
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_QUADRATIC, max_steps=30)
    st, ends, dt = bench.sharded_tracker(torch, hc, synth, fam, opts, dist, rank, world)
    out[rank] = (st, [e.tolist() for e in ends])
    dist.destroy_process_group()


@pytest.mark.gpu
def test_two_ranks_track_their_blocks_and_gather_the_single_rank_result():
    """Two gloo ranks, each calling hc_track_path on its own block of 11 uneven-family
    paths (both on cuda:0 here; no kernel of one rank waits on the other), gather the
    per-path statistics and end points once: they equal, bit for bit, one rank tracking
    all 11 paths in one call."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    from paper_1109_0545_gb300 import hc, synth
    fam = [synth.uneven_path_system(3, j) for j in range(11)]
    opts = hc.hc_track_opts_default(lu_mode=hc.HC_LU_FP64_REFINE, predictor=hc.HC_PRED_QUADRATIC, max_steps=30)
    ref_st, ref_ends, _ = bench.sharded_tracker(torch, hc, synth, fam, opts)
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_track_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        st, ends = res[r]
        assert st == ref_st
        assert all(np.array_equal(np.array(a), b) for a, b in zip(ends, ref_ends))
