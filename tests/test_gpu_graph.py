"""gs_render's CUDA graph: a frame's launches are captured once and replayed
with each frame's camera while the scene arrays, image size, options,
framebuffer and buffers stay the same. Every replayed frame must equal a
frame launched directly (direct_launch = 1) bit for bit, whatever changes
between frames: the camera (pose and intrinsics), the sync mode, the
framebuffer, the options, the scene arrays, the key capacity."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15951_gb300 as gs  # noqa: E402
from paper_2607_15951_gb300 import _native as N  # noqa: E402
from paper_2607_15951_gb300 import scenes  # noqa: E402

KEYS = ("rgb", "final_T", "n_contrib", "n_eval")


@pytest.fixture(scope="module")
def ctxs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15951_gb300 import build
    build.build()
    a, b = gs.Context(0), gs.Context(0)
    yield a, b
    a.close()
    b.close()


def _equal(x, y):
    torch.cuda.synchronize()
    for k in KEYS:
        assert torch.equal(x[k], y[k]), k


@pytest.mark.parametrize("opts", [{}, {"list_tiles": N.GS_LISTS_4X4}, {"tile": (16, 8)},
                                  {"variant": N.GS_BLEND_CULLED}, {"cluster": N.GS_CLUSTER_2X2},
                                  {"record_dtype": N.GS_RECORD_BF16}, {"tile_order": N.GS_ORDER_GRID}],
                         ids=["default", "l4x4", "t16x8", "culled", "c2x2", "bf16", "grid_order"])
def test_replayed_frames_equal_direct_frames(ctxs, opts):
    graph_ctx, direct_ctx = ctxs
    scene = scenes.clustered(60_000, 51, box=6.0)
    g = gs.scene_to_device(scene)
    cams = scenes.trajectory(6, 1051, radius=2.5, sizes=((320, 200),))
    out = gs.render(graph_ctx, g, scene.sh_degree, cams[0], **opts)  # the framebuffer the graph writes
    for i, cam in enumerate(cams):
        gs.gs_render(graph_ctx, g, scene.sh_degree, cam, out["rgb"], out["final_T"], out["n_contrib"],
                     out["n_eval"], deferred=bool(i % 2), **opts)
        ref = gs.render(direct_ctx, g, scene.sh_degree, cam, direct=True, **opts)
        gs.gs_sync_status(graph_ctx)
        _equal(out, ref)


def test_replay_follows_intrinsics_framebuffers_and_scene(ctxs):
    graph_ctx, direct_ctx = ctxs
    scene = scenes.clustered(40_000, 52, box=6.0)
    g = gs.scene_to_device(scene)
    cam = scenes.trajectory(1, 1052, radius=2.5, sizes=((256, 160),))[0]
    outs = [gs.render(graph_ctx, g, scene.sh_degree, cam) for _ in range(2)]
    for i in range(6):
        c = scenes.trajectory(1, 1052, radius=2.5, sizes=((256, 160),))[0]
        c.fx *= 1.0 + 0.1 * i      # intrinsics change from frame to frame
        c.cx += 3.0 * i
        c.near_z = 0.2 + 0.3 * (i % 2)
        o = outs[i % 2]            # two framebuffers in turn
        if i == 4:                 # new scene arrays (same count)
            g = {k: v.clone() for k, v in g.items()}
            g["opacity_logits"] += 0.5
        gs.gs_render(graph_ctx, g, scene.sh_degree, c, o["rgb"], o["final_T"], o["n_contrib"], o["n_eval"])
        ref = gs.render(direct_ctx, g, scene.sh_degree, c, direct=True)
        _equal(o, ref)


def test_replay_after_the_key_buffers_grow(ctxs):
    _, direct_ctx = ctxs
    scene = scenes.clustered(80_000, 53, box=6.0)
    g = gs.scene_to_device(scene)
    cams = scenes.trajectory(3, 1053, radius=2.5, sizes=((320, 200),))
    c = gs.Context(0)
    gs.gs_reserve_keys(c, 1000)  # the first frame overflows and is rendered again in larger buffers
    for cam in cams:
        out = gs.render(c, g, scene.sh_degree, cam)
        ref = gs.render(direct_ctx, g, scene.sh_degree, cam, direct=True)
        _equal(out, ref)
    assert gs.gs_last_render_stats(c)["n_keys"] > 1000
    c.close()


def test_backward_of_a_replayed_frame(ctxs):
    graph_ctx, direct_ctx = ctxs
    scene = scenes.clustered(30_000, 54, box=5.0)
    g = gs.scene_to_device(scene)
    cams = scenes.trajectory(2, 1054, radius=2.0, sizes=((320, 180),))
    d = torch.randn((180, 320, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(6))
    res = []
    for ctx, direct in ((graph_ctx, False), (direct_ctx, True)):
        gs.render(ctx, g, scene.sh_degree, cams[0], direct=direct)
        out = gs.render(ctx, g, scene.sh_degree, cams[1], direct=direct)  # a replay on the graph context
        grads = {k: torch.empty_like(v) for k, v in g.items()}
        gs.gs_render_backward(ctx, g, scene.sh_degree, cams[1], out["final_T"], out["n_contrib"], d, grads)
        torch.cuda.synchronize()
        res.append(grads)
    for k in res[0]:
        a, b = res[0][k], res[1][k]
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-4 * float(b.abs().max()) + 1e-12), k


def test_frames_cycling_over_more_framebuffers_than_graphs(ctxs):
    """Twelve framebuffers in turn (more than the context keeps graphs for):
    captures miss, the context switches to direct launches for a while, tries
    again; every frame still equals a directly launched one."""
    _, direct_ctx = ctxs
    scene = scenes.clustered(20_000, 55, box=5.0)
    g = gs.scene_to_device(scene)
    cams = scenes.trajectory(12, 1055, radius=2.0, sizes=((160, 96),))
    c = gs.Context(0)
    outs = gs.alloc_outputs(cams, aux=True)
    refs = [gs.render(direct_ctx, g, scene.sh_degree, cam, direct=True) for cam in cams]
    for i in range(60):
        v = i % len(cams)
        o = outs[v]
        gs.gs_render(c, g, scene.sh_degree, cams[v], o["rgb"], o["final_T"], o["n_contrib"], o["n_eval"],
                     deferred=bool(i % 3))
        gs.gs_sync_status(c)
        _equal(o, refs[v])
    c.close()
