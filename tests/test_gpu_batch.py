"""Multi-scene scoring in one submission (eager, captured as a CUDA graph, replayed)
and the view-batch / sort-grid / tile-shape autotuner: every path returns the scores csgs_score
returns scene by scene, and the replayed graph's scores match the FP64 oracle."""
import numpy as np
import pytest

import oracle
import paper_2607_02721_b300 as csgs
from paper_2607_02721_b300 import build, synth
from parity_helpers import check_scores

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    if not t.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    build.build()
    c = csgs.Context(0)
    yield c
    c.close()


SPEC = [(3000, 5, 96, 80, 1), (12000, 9, 128, 128, 2), (6000, 3, 200, 120, 3)]


def make_scene(k):
    n, v, W, H, seed = SPEC[k]
    return synth.mixture_scene(n, 16, 3, seed, half_extent=2.0), synth.hemisphere_cameras(v, W, H, radius=7.0, seed=seed)


@pytest.fixture(scope="module")
def scenes(ctx):
    """Three scenes of uneven size, each with its own views (count and resolution)."""
    sids = []
    for k in range(len(SPEC)):
        sc, cams = make_scene(k)
        sid = ctx.load_scene(sc)
        ctx.set_queries(sid, cams)
        sids.append(sid)
    return sids


@pytest.mark.parametrize("res", [("pixel", csgs.RES_PIXEL, oracle.RES_PIXEL), ("scene", csgs.RES_SCENE, oracle.RES_SCENE)],
                         ids=["pixel", "scene"])
def test_replayed_graph_matches_oracle(ctx, res):
    """Scenes 0 and 2 of a captured submission, after a replay, against the oracle
    scene by scene (its own context, so no earlier test changed the query sets)."""
    c = csgs.Context(0)
    try:
        data = [make_scene(k) for k in range(len(SPEC))]
        sids = []
        for sc, cams in data:
            sid = c.load_scene(sc)
            c.set_queries(sid, cams)
            sids.append(sid)
        opts = csgs.default_opts(resolution=res[1])
        outs, _ = c.score_batch(sids, opts, use_graph=True)       # eager pass + capture
        for o in outs:
            o.fill_(-1.0)
        outs, S = c.score_batch(sids, opts, outs=outs, use_graph=True)  # replay
        for k in (0, 2):
            sc, cams = data[k]
            ref = oracle.score(oracle.SceneArrays(sc), cams, oracle.Opts(resolution=res[2]))
            s = outs[k].cpu().numpy()
            if res[0] == "pixel":
                check_scores(s, S[k], ref)
            else:
                big = ref["s"] > 1e-6
                rel = np.abs(s[big].astype(np.float64) - ref["s"][big]) / ref["s"][big]
                assert np.quantile(rel, 0.999) <= 1e-3 and abs(S[k] - 1.0) < 1e-4
    finally:
        c.close()


def one_by_one(ctx, sids, opts):
    out = [ctx.score(k, opts) for k in sids]
    return [o[0].cpu().numpy() for o in out], [o[1] for o in out]


def test_batch_matches_single_scene_scoring(ctx, scenes):
    opts = csgs.default_opts()
    ref_s, ref_S = one_by_one(ctx, scenes, opts)
    for use_graph in (False, True):
        s, S = ctx.score_batch(scenes, opts, use_graph=use_graph)
        for k in range(len(scenes)):
            # pixel resolution: a max of per-pixel values, so any schedule gives the same bits
            np.testing.assert_array_equal(s[k].cpu().numpy(), ref_s[k])
            assert S[k] == ref_S[k]


def test_graph_replay_is_one_launch_and_repeats_results(ctx, scenes):
    opts = csgs.default_opts()
    outs, S0 = ctx.score_batch(scenes, opts, use_graph=True)  # eager pass + capture
    first = [o.cpu().numpy().copy() for o in outs]
    for o in outs:
        o.zero_()
    n0 = csgs.kernel_launch_count()
    outs2, S1 = ctx.score_batch(scenes, opts, outs=outs, use_graph=True)  # replay
    assert csgs.kernel_launch_count() == n0  # nothing launched one by one
    st = ctx.stats()
    assert st["kernel_launches"] > 3 * len(scenes)  # the graph's kernels
    assert st["views"] == 5 + 9 + 3
    for k in range(len(scenes)):
        np.testing.assert_array_equal(outs2[k].cpu().numpy(), first[k])
        assert S1[k] == S0[k]


def test_graph_follows_scene_and_view_changes(ctx, scenes, torch):
    """A replay reads the scene from device memory (in-place updates are seen); new
    query views change the captured launches, so they force a new capture."""
    opts = csgs.default_opts()
    outs, _ = ctx.score_batch(scenes, opts, use_graph=True)
    outs, _ = ctx.score_batch(scenes, opts, outs=outs, use_graph=True)
    cams = synth.hemisphere_cameras(4, 112, 96, radius=6.5, seed=11)
    ctx.set_queries(scenes[1], cams)
    ref_s, ref_S = one_by_one(ctx, scenes, opts)
    outs, S = ctx.score_batch(scenes, opts, outs=outs, use_graph=True)
    for k in range(len(scenes)):
        np.testing.assert_array_equal(outs[k].cpu().numpy(), ref_s[k])
        assert S[k] == ref_S[k]


def test_batch_scene_resolution(ctx, scenes):
    """Per-scene resolution sums in FP32 atomics: same values up to summation order."""
    opts = csgs.default_opts(resolution=csgs.RES_SCENE)
    ref_s, ref_S = one_by_one(ctx, scenes, opts)
    s, S = ctx.score_batch(scenes, opts, use_graph=True)
    s, S = ctx.score_batch(scenes, opts, outs=s, use_graph=True)
    for k in range(len(scenes)):
        np.testing.assert_allclose(s[k].cpu().numpy(), ref_s[k], rtol=1e-4, atol=1e-9)
        assert abs(S[k] - 1.0) < 1e-4


def test_autotune_keeps_scores(ctx, scenes):
    """The view batch and the sort grid leave the scores bit for bit; the tuned tile shape
    is what later CSGS_TILE_AUTO calls use."""
    fixed = csgs.default_opts(tile_shape=csgs.TILE_16X16)
    ref, Sref = ctx.score(scenes[1], fixed)
    ref = ref.cpu().numpy()
    tu = ctx.autotune(scenes[1], csgs.default_opts(), probe_views=4)
    assert tu["view_batch"] in (1, 2, 4) and tu["sort_blocks"] in (74, 148, 296, 592, 1184, 1776)
    assert tu["tile_shape"] in (csgs.TILE_16X16, csgs.TILE_32X8, csgs.TILE_16X8, csgs.TILE_8X8)
    assert tu["persist_ctas"] == 0 or tu["persist_ctas"] % 148 == 0 and tu["probe_ms"] > 0
    s, S = ctx.score(scenes[1], fixed)
    np.testing.assert_array_equal(s.cpu().numpy(), ref)
    assert S == Sref
    auto, Sa = ctx.score(scenes[1], csgs.default_opts())
    expl, Se = ctx.score(scenes[1], csgs.default_opts(tile_shape=tu["tile_shape"]))
    np.testing.assert_array_equal(auto.cpu().numpy(), expl.cpu().numpy())
    assert Sa == Se


@pytest.mark.parametrize("shape", [csgs.TILE_16X16, csgs.TILE_16X8, csgs.TILE_8X8], ids=["16x16", "16x8", "8x8"])
def test_persistent_compositing_matches_one_cta_per_tile(ctx, scenes, shape):
    """The persistent launch (few CTAs taking tiles from a queue, longest lists first) gives
    the per-tile launch's per-pixel scores bit for bit, for grids below, at and above the
    tile count, in a single call and in a replayed batch graph."""
    base = csgs.default_opts(tile_shape=shape, persist_ctas=-1)
    ref_s, ref_S = one_by_one(ctx, scenes, base)
    for grid in (1, 37, 148, 100000):
        opts = csgs.default_opts(tile_shape=shape, persist_ctas=grid)
        s, S = one_by_one(ctx, scenes, opts)
        for k in range(len(scenes)):
            np.testing.assert_array_equal(s[k], ref_s[k])
            assert S[k] == ref_S[k]
    opts = csgs.default_opts(tile_shape=shape, persist_ctas=37)
    outs, _ = ctx.score_batch(scenes, opts, use_graph=True)
    outs, S = ctx.score_batch(scenes, opts, outs=outs, use_graph=True)
    for k in range(len(scenes)):
        np.testing.assert_array_equal(outs[k].cpu().numpy(), ref_s[k])
        assert S[k] == ref_S[k]


@pytest.mark.parametrize("shape", [csgs.TILE_32X8, csgs.TILE_16X8, csgs.TILE_8X8], ids=["32x8", "16x8", "8x8"])
def test_batch_tile_shapes_match_single_scene_and_oracle(ctx, scenes, shape):
    """A captured batch in another tile shape returns csgs_score's scores scene by scene,
    and the ragged 200x120 scene matches the oracle."""
    opts = csgs.default_opts(tile_shape=shape)
    ref_s, ref_S = one_by_one(ctx, scenes, opts)
    outs, _ = ctx.score_batch(scenes, opts, use_graph=True)
    outs, S = ctx.score_batch(scenes, opts, outs=outs, use_graph=True)
    for k in range(len(scenes)):
        np.testing.assert_array_equal(outs[k].cpu().numpy(), ref_s[k])
        assert S[k] == ref_S[k]
    c = csgs.Context(0)
    try:
        sc, cams = make_scene(2)
        sid = c.load_scene(sc)
        c.set_queries(sid, cams)
        s, S2 = c.score(sid, opts)
        check_scores(s.cpu().numpy(), S2, oracle.score(oracle.SceneArrays(sc), cams))
    finally:
        c.close()


def test_batch_rejects_bad_arguments(ctx, scenes):
    with pytest.raises(csgs.CsgsError):
        ctx.score_batch([scenes[0], 12345])
    with pytest.raises(csgs.CsgsError):
        ctx.score_batch([])
