"""View-sharded scoring across ranks (``paper_2607_02721_b300.sharded``) with gloo ranks on
CPU.  Each rank scores its round-robin share of the views with the FP64 oracle and the
ranks combine their scores with the module's collective step; the result must be the
oracle's single-process score over all views:
  - per-pixel and per-image resolutions: a maximum over queries (Eq. sen), so bit for bit;
  - per-scene resolution: a ratio of sums over queries (Sec. 3.5), equal up to the
    rounding of the reordered sums.
Two ranks over three views (uneven shares) and three ranks over two views (a rank with
no views) are covered."""
import os
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _scene():
    from paper_2607_02721_b300 import synth

    return synth.uniform_cube_scene(400, seed=11), synth.cube_corner_cameras(3.0, 32, 32)


def _rank(rank, world, port, n_views, out):
    sys.path.insert(0, ROOT)
    import torch

    import oracle
    from paper_2607_02721_b300 import sharded

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc, cams = _scene()
    cams = cams[:n_views]
    views = sharded.shard_views(n_views, rank, world)
    res = {}
    for name, res_id in (("pixel", oracle.RES_PIXEL), ("image", oracle.RES_IMAGE), ("scene", oracle.RES_SCENE)):
        if len(views):
            r = oracle.score(sc, cams[views], oracle.Opts(resolution=res_id))
            s_local, A_local = torch.tensor(r["s"], dtype=torch.float64), float(r["sumA"])
        else:
            s_local, A_local = torch.zeros(sc.n, dtype=torch.float64), 0.0
        s = sharded.combine_shards(s_local, A_local, res_id, dist, lambda t, f: t.mul_(f))
        res[name] = s.numpy().copy()
    out[rank] = (views.tolist(), res)
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n_views", [(2, 3), (3, 2)])
def test_sharded_scores_equal_single_process(world, n_views):
    import socket

    import oracle

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, n_views, out), nprocs=world, join=True, start_method="spawn")
    sc, cams = _scene()
    cams = cams[:n_views]
    # every view on exactly one rank
    assert sorted(v for r in range(world) for v in out[r][0]) == list(range(n_views))
    ref = {name: oracle.score(sc, cams, oracle.Opts(resolution=res_id))["s"]
           for name, res_id in (("pixel", oracle.RES_PIXEL), ("image", oracle.RES_IMAGE),
                                ("scene", oracle.RES_SCENE))}
    for r in range(world):
        got = out[r][1]
        np.testing.assert_array_equal(got["pixel"], ref["pixel"])
        np.testing.assert_array_equal(got["image"], ref["image"])
        np.testing.assert_allclose(got["scene"], ref["scene"], rtol=1e-12, atol=1e-300)
        assert abs(got["scene"].sum() - 1.0) < 1e-12


def test_shard_views_partition():
    from paper_2607_02721_b300 import sharded

    for nv in (1, 7, 200):
        for world in (1, 2, 3, 8):
            parts = [sharded.shard_views(nv, r, world) for r in range(world)]
            assert sorted(np.concatenate(parts).tolist()) == list(range(nv))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        sharded.shard_views(4, 2, 2)
