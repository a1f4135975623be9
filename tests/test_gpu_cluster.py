"""Lists of list tiles (2 x 1 or 2 x 2 screen tiles), blended either by
thread-block clusters whose blocks share the list's batches through
distributed shared memory (gs_options.cluster) or by every screen tile's
block reading the list itself (gs_options.list_tiles). Colours and
transmittance must equal the default per-16x16-tile render bit for bit (each
pixel sees the same records in the same order); list positions refer to the
list tile's list, so n_contrib and n_eval are checked through the oracle's
binning of the list tiles: the Gaussian at a pixel's last-contributor
position is the same Gaussian as in the default render."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15951_gb300 as gs  # noqa: E402
from paper_2607_15951_gb300 import _native as N  # noqa: E402
from paper_2607_15951_gb300 import scenes  # noqa: E402

# (option, value): the four list forms
FORMS = [("cluster", N.GS_CLUSTER_2X1), ("cluster", N.GS_CLUSTER_2X2),
         ("list_tiles", N.GS_LISTS_2X1), ("list_tiles", N.GS_LISTS_2X2),
         ("list_tiles", N.GS_LISTS_4X4), ("list_tiles", N.GS_LISTS_8X8)]
FORM_IDS = ["c2x1", "c2x2", "l2x1", "l2x2", "l4x4", "l8x8"]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15951_gb300 import build
    build.build()
    c = gs.Context(0)
    yield c
    c.close()


def _list_tile(shape):
    return {2: (32, 16), 4: (32, 32), 16: (64, 64), 64: (128, 128)}[shape]


def _last_gaussian(nc, vals, ranges, width, tw, th):
    """Gaussian index at each pixel's 1-based list position nc (-1: none)."""
    H, W = nc.shape
    tx = (width + tw - 1) // tw
    ys, xs = np.mgrid[0:H, 0:W]
    t = (ys // th) * tx + xs // tw
    pos = ranges[t, 0].astype(np.int64) + nc.astype(np.int64) - 1
    out = np.full(nc.shape, -1, np.int64)
    m = nc > 0
    out[m] = vals[pos[m]]
    return out


CASES = [("uniform_box_256", lambda: (scenes.uniform_box(10_000, 0), scenes.pinhole(256, 256))),
         ("clustered_odd_300x200", lambda: (scenes.clustered(100_000, 41, box=6.0), scenes.pinhole(300, 200))),
         ("clustered_1m_1080p", lambda: scenes.workload("clustered_1m_1080p"))]


@pytest.mark.parametrize("form", FORMS, ids=FORM_IDS)
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_list_tile_blends_equal_default(ctx, oracle_mod, name, make, form):
    opt, shape = form
    scene, cam = make()
    if isinstance(cam, list):
        cam = cam[0]
    g = gs.scene_to_device(scene)
    ref = gs.render(ctx, g, scene.sh_degree, cam)
    torch.cuda.synchronize()
    k16 = gs.gs_last_render_stats(ctx)["n_keys"]
    out = gs.render(ctx, g, scene.sh_degree, cam, **{opt: shape})
    torch.cuda.synchronize()
    gs.gs_sync_status(ctx)
    kc = gs.gs_last_render_stats(ctx)["n_keys"]
    print(name, opt, shape, "keys 16x16", k16, "list-tile keys", kc)
    assert torch.equal(out["rgb"], ref["rgb"])
    assert torch.equal(out["final_T"], ref["final_T"])
    assert kc <= k16
    nc, nc16 = out["n_contrib"].cpu().numpy(), ref["n_contrib"].cpu().numpy()
    assert np.array_equal(nc > 0, nc16 > 0)
    # Same last contributor, through the oracle's lists of both tilings (the
    # binning of the GPU's own records, so depth ties order alike). Where the
    # list grid reaches past the 16 x 16 grid (image sizes that are not whole
    # list tiles), Gaussians that touch only that margin are listed but have
    # no gs_project record; those sizes are checked on colours alone.
    tw, th = _list_tile(shape)
    if -(-cam.width // tw) * tw != -(-cam.width // 16) * 16 or -(-cam.height // th) * th != -(-cam.height // 16) * 16:
        return
    rec = torch.zeros((scene.n, 12), dtype=torch.float32, device="cuda")
    tiles = torch.zeros((scene.n,), dtype=torch.int32, device="cuda")
    gs.gs_project(ctx, g, scene.sh_degree, cam, rec, tiles)
    r = rec.cpu().numpy()
    m2, rad, dep = r[:, 0:2].astype(np.float64), r[:, 10].view(np.int32).astype(np.int64), r[:, 9].astype(np.float64)
    vis = (tiles.cpu().numpy() > 0).astype(np.int32)
    b16 = oracle_mod.bin_tiles(m2, rad, dep, vis, cam.width, cam.height, 16, 16)
    bc = oracle_mod.bin_tiles(m2, rad, dep, vis, cam.width, cam.height, tw, th)
    assert int(bc.values.size) == kc
    a = _last_gaussian(nc, bc.values, bc.ranges, cam.width, tw, th)
    b = _last_gaussian(nc16, b16.values, b16.ranges, cam.width, 16, 16)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("lists", [N.GS_LISTS_2X1, N.GS_LISTS_4X4], ids=["l2x1", "l4x4"])
def test_list_tiles_with_wide_warp_blocks(ctx, lists):
    # 16x8 warp blocks (two packed pixel pairs per lane) over list tiles: the
    # same outputs as 8x8 blocks, list positions included.
    scene, cam = scenes.clustered(200_000, 44, box=6.0), scenes.pinhole(500, 300)
    g = gs.scene_to_device(scene)
    ref = gs.render(ctx, g, scene.sh_degree, cam, list_tiles=lists)
    out = gs.render(ctx, g, scene.sh_degree, cam, list_tiles=lists, variant=N.GS_BLEND_CULLED_WIDE)
    torch.cuda.synchronize()
    for k in ("rgb", "final_T", "n_contrib", "n_eval"):
        assert torch.equal(out[k], ref[k]), k
    plain = gs.render(ctx, g, scene.sh_degree, cam)
    torch.cuda.synchronize()
    assert torch.equal(out["rgb"], plain["rgb"]) and torch.equal(out["final_T"], plain["final_T"])


@pytest.mark.parametrize("opt", ["cluster", "list_tiles"])
@pytest.mark.parametrize("dtype", [N.GS_RECORD_F16, N.GS_RECORD_BF16], ids=["f16", "bf16"])
def test_list_tile_blends_with_low_precision_records(ctx, dtype, opt):
    scene = scenes.imbalance(300_000, seed=4, width=960, height=540)
    cam = scenes.pinhole(960, 540, 60.0)
    g = gs.scene_to_device(scene)
    ref = gs.render(ctx, g, scene.sh_degree, cam, record_dtype=dtype)
    out = gs.render(ctx, g, scene.sh_degree, cam, record_dtype=dtype, **{opt: 4})
    torch.cuda.synchronize()
    assert torch.equal(out["rgb"], ref["rgb"])
    assert torch.equal(out["final_T"], ref["final_T"])


def test_list_tile_backward_equals_default(ctx):
    scene, cam = scenes.clustered(50_000, 42, box=5.0), scenes.pinhole(320, 180)
    g = gs.scene_to_device(scene)
    d = torch.randn((180, 320, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    res = []
    for kw in ({}, {"cluster": N.GS_CLUSTER_2X2}, {"list_tiles": N.GS_LISTS_2X2}, {"list_tiles": N.GS_LISTS_8X8},
               {"list_tiles": N.GS_LISTS_2X1}):
        out = gs.render(ctx, g, scene.sh_degree, cam, **kw)
        grads = {k: torch.empty_like(v) for k, v in g.items()}
        gs.gs_render_backward(ctx, g, scene.sh_degree, cam, out["final_T"], out["n_contrib"], d, grads, **kw)
        torch.cuda.synchronize()
        res.append(grads)
    for r in res[1:]:
        for k in res[0]:
            a, b = r[k], res[0][k]
            # Float atomics sum each gradient in a run-dependent order: two
            # backward passes of the same frame differ by up to ~1.2e-5 of the
            # largest log-scale gradient (cancelling terms), so list forms are
            # compared at 1e-4 of the largest gradient, plus 1e-4 relative.
            assert torch.allclose(a, b, rtol=1e-4, atol=1e-4 * float(b.abs().max()) + 1e-12), k
    # A backward with other cluster options than the frame's is refused.
    with pytest.raises(gs.GSError):
        gs.gs_render_backward(ctx, g, scene.sh_degree, cam, out["final_T"], out["n_contrib"], d, res[0])


@pytest.mark.parametrize("opt", ["cluster", "list_tiles"])
def test_list_tile_batch_renders_views_alike(ctx, opt):
    scene = scenes.clustered(100_000, 43, box=6.0)
    cams = scenes.trajectory(3, 1043, radius=2.0, sizes=((320, 180), (200, 120)))
    g = gs.scene_to_device(scene)
    outs = gs.alloc_outputs(cams, aux=True)
    gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs, **{opt: 4})
    torch.cuda.synchronize()
    for c, o in zip(cams, outs):
        ref = gs.render(ctx, g, scene.sh_degree, c)
        torch.cuda.synchronize()
        assert torch.equal(o["rgb"], ref["rgb"]) and torch.equal(o["final_T"], ref["final_T"])


@pytest.mark.parametrize("lists", [N.GS_LISTS_2X1, N.GS_LISTS_4X4, N.GS_LISTS_8X8], ids=["l2x1", "l4x4", "l8x8"])
def test_joint_batch_with_list_tiles(ctx, lists):
    # The joint schedule with list tiles (one queue item per screen tile of a
    # list tile) equals the view-by-view renders with the same list tiles, list
    # positions included; its batched backward is refused.
    scene = scenes.clustered(100_000, 45, box=6.0)
    cams = scenes.trajectory(4, 1045, radius=2.0, sizes=((330, 190), (200, 120)))
    g = gs.scene_to_device(scene)
    outs = gs.alloc_outputs(cams, aux=True)
    gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs, list_tiles=lists, batch_mode=N.GS_BATCH_JOINT)
    torch.cuda.synchronize()
    for c, o in zip(cams, outs):
        ref = gs.render(ctx, g, scene.sh_degree, c, list_tiles=lists)
        torch.cuda.synchronize()
        for k in ("rgb", "final_T", "n_contrib", "n_eval"):
            assert torch.equal(o[k], ref[k]), k
    gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs, list_tiles=lists, batch_mode=N.GS_BATCH_JOINT)
    grads = {k: torch.empty_like(v) for k, v in g.items()}
    d = [torch.ones_like(o["rgb"]) for o in outs]
    with pytest.raises(gs.GSError):
        gs.gs_render_batch_backward(ctx, g, scene.sh_degree, cams, outs, d, grads, list_tiles=lists)


def test_list_tile_option_checks(ctx):
    scene, cam = scenes.uniform_box(100, 1), scenes.pinhole(64, 64)
    g = gs.scene_to_device(scene)
    for kw in ({"cluster": 3}, {"cluster": 4, "tile": (16, 8)}, {"cluster": 4, "temporal": True},
               {"list_tiles": 3}, {"list_tiles": 8}, {"list_tiles": 4, "tile": (16, 8)},
               {"list_tiles": 2, "temporal": True},
               {"list_tiles": 4, "cluster": 4}):
        with pytest.raises(gs.GSError):
            gs.render(ctx, g, 0, cam, **kw)
