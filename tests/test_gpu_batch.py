"""Batched multi-view rendering (gs_render_batch): every view equals the
single-view render of the same camera bit for bit (same kernels, same
per-tile order), with the captured graph or direct launches, and across
camera changes between graph replays."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15951_gb300 as gs  # noqa: E402
from paper_2607_15951_gb300 import scenes  # noqa: E402
from paper_2607_15951_gb300 import _native as N  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15951_gb300 import build
    build.build()
    c = gs.Context(0)
    yield c
    c.close()


def per_view(ctx, g, deg, cams, **kw):
    outs = []
    for c in cams:
        o = gs.render(ctx, g, deg, c, **kw)
        torch.cuda.synchronize()
        outs.append({k: v.clone() for k, v in o.items()})
    return outs


@pytest.mark.parametrize("direct", [False, True], ids=["graph", "direct"])
@pytest.mark.parametrize("dtype", [N.GS_RECORD_F32, N.GS_RECORD_F16], ids=["f32", "f16"])
def test_batch_equals_single_view_renders(ctx, direct, dtype):
    scene = scenes.clustered(100_000, 21, box=6.0)
    cams = scenes.trajectory(6, 1021, radius=3.0, sizes=((320, 180), (160, 120)))
    g = gs.scene_to_device(scene)
    ref = per_view(ctx, g, scene.sh_degree, cams, record_dtype=dtype)
    outs = gs.alloc_outputs(cams, aux=True)
    gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs, record_dtype=dtype, direct=direct)
    torch.cuda.synchronize()
    for v, (a, b) in enumerate(zip(outs, ref)):
        for k in ("rgb", "final_T", "n_contrib", "n_eval"):
            assert torch.equal(a[k], b[k]), (v, k)


def test_graph_replay_follows_new_cameras(ctx):
    scene = scenes.clustered(50_000, 22, box=5.0)
    g = gs.scene_to_device(scene)
    outs = gs.alloc_outputs(scenes.trajectory(4, 1022, radius=2.0, sizes=((200, 150),)), aux=True)
    for seed in (1022, 1023, 1024):   # same sizes, new poses: the graph is replayed
        cams = scenes.trajectory(4, seed, radius=2.0, sizes=((200, 150),))
        gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs)
        torch.cuda.synchronize()
        ref = per_view(ctx, g, scene.sh_degree, cams)
        for a, b in zip(outs, ref):
            assert torch.equal(a["rgb"], b["rgb"])


def test_batch_tile_shapes_and_autotune(ctx, tmp_path):
    scene = scenes.uniform_box(5_000, 23)
    cams = [scenes.pinhole(96, 64), scenes.pinhole(130, 70)]
    g = gs.scene_to_device(scene)
    for tile in ((16, 16), (16, 8), (8, 8)):
        outs = gs.alloc_outputs(cams, aux=True)
        gs.gs_render_batch(ctx, g, 0, cams, outs, tile=tile)
        ref = per_view(ctx, g, 0, cams, tile=tile)
        for a, b in zip(outs, ref):
            assert torch.equal(a["rgb"], b["rgb"]), tile
    cache = str(tmp_path / "tune.json")
    tile, ms, depth, cluster, lists = gs.gs_autotune_batch(ctx, g, 0, cams, gs.alloc_outputs(cams),
                                                           cache_path=cache)
    assert tile in ((16, 16), (16, 8), (8, 8)) and len(ms) == 9 and all(m > 0 for m in ms)
    assert depth in (64, 128, 256) and cluster in (0, 2, 4) and lists in (0, 2, 4, 16, 64)
    assert (cluster == 0 and lists == 0) or (tile == (16, 16) and min(cluster, lists) == 0)
    again = gs.gs_autotune_batch(ctx, g, 0, cams, gs.alloc_outputs(cams), cache_path=cache)
    assert (again[0], again[2], again[3], again[4]) == (tile, depth, cluster, lists)
    for d in (64, 128, 256):  # every staging depth renders the same image
        outs = gs.alloc_outputs(cams, aux=True)
        gs.gs_render_batch(ctx, g, 0, cams, outs, tile=tile, batch_depth=d, batch_mode=N.GS_BATCH_JOINT)
        ref = per_view(ctx, g, 0, cams, tile=tile)
        for a, b in zip(outs, ref):
            for k in ("rgb", "final_T", "n_contrib", "n_eval"):
                assert torch.equal(a[k], b[k]), (d, k)


def test_batch_matches_oracle(ctx, oracle_mod):
    scene = scenes.uniform_box(3_000, 24)
    cams = scenes.random_poses(3, 1024, radius=0.5, sizes=((128, 96), (96, 96)))
    g = gs.scene_to_device(scene)
    outs = gs.alloc_outputs(cams, aux=True)
    gs.gs_render_batch(ctx, g, 0, cams, outs)
    torch.cuda.synchronize()
    for o, c in zip(outs, cams):
        _, _, img = oracle_mod.render(scene, c)
        keep = ~img.flag.astype(bool)
        err = np.abs(o["rgb"].cpu().numpy().astype(np.float64) - img.rgb)[keep].max()
        assert err <= 1e-3, err


@pytest.mark.parametrize("mode", [N.GS_BATCH_JOINT, N.GS_BATCH_PER_VIEW], ids=["joint", "per_view"])
def test_batch_schedules_agree(ctx, mode):
    scene = scenes.clustered(60_000, 25, box=5.0)
    cams = scenes.trajectory(5, 1025, radius=2.0, sizes=((256, 144), (200, 120)))
    g = gs.scene_to_device(scene)
    ref = per_view(ctx, g, scene.sh_degree, cams, record_dtype=N.GS_RECORD_BF16)
    outs = gs.alloc_outputs(cams, aux=True)
    gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs, record_dtype=N.GS_RECORD_BF16, batch_mode=mode)
    torch.cuda.synchronize()
    for a, b in zip(outs, ref):
        for k in ("rgb", "final_T", "n_contrib", "n_eval"):
            assert torch.equal(a[k], b[k]), k
