"""GS_SYNC_DEFERRED: gs_render without a host synchronisation per frame.

The images must equal those of the synchronised mode bit for bit (the same
kernels run); an overflow of the key buffers must be reported by the next
call on the context, after which the buffers have grown and a new render is
exact; a backward after an overflowed deferred forward must fail instead of
differentiating an incomplete frame."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15951_gb300 as gs  # noqa: E402
from paper_2607_15951_gb300 import scenes  # noqa: E402


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15951_gb300 import build
    build.build()


def _poses(n):
    return [scenes.pinhole(200 + 16 * i, 150 + 8 * i, 50.0 + 3 * i) for i in range(n)]


def test_deferred_frames_equal_synchronised_frames(built):
    scene = scenes.uniform_box(20_000, 21)
    g = gs.scene_to_device(scene)
    cams = _poses(7)  # more frames than the ring of frames in flight
    ref_ctx, ctx = gs.Context(0), gs.Context(0)
    refs = [gs.render(ref_ctx, g, scene.sh_degree, c) for c in cams]
    outs = [gs.render(ctx, g, scene.sh_degree, c, deferred=True) for c in cams]
    gs.gs_sync_status(ctx)
    torch.cuda.synchronize()
    for r, o in zip(refs, outs):
        for k in r:
            assert torch.equal(r[k], o[k]), k
    st = gs.gs_last_render_stats(ctx)
    assert st == gs.gs_last_render_stats(ref_ctx)


def test_deferred_overflow_is_reported_then_regrown(built):
    scene, cams = scenes.workload("uniform_box_256")
    g = gs.scene_to_device(scene)
    ref = gs.render(gs.Context(0), g, scene.sh_degree, cams[0])
    ctx = gs.Context(0)
    gs.gs_reserve_keys(ctx, 1000)
    gs.render(ctx, g, scene.sh_degree, cams[0], deferred=True)
    with pytest.raises(gs.GSError) as e:
        gs.gs_sync_status(ctx)
    assert e.value.status == 4  # GS_ERR_CAPACITY
    gs.gs_sync_status(ctx)      # reported once
    out = gs.render(ctx, g, scene.sh_degree, cams[0], deferred=True)
    gs.gs_sync_status(ctx)
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(ref[k], out[k]), k
    # The next call (here a render) also reports a pending overflow.
    gs.gs_reserve_keys(ctx, 1000)
    gs.render(ctx, g, scene.sh_degree, cams[0], deferred=True)
    torch.cuda.synchronize()
    with pytest.raises(gs.GSError) as e:
        gs.render(ctx, g, scene.sh_degree, cams[0], deferred=True)
    assert e.value.status == 4
    gs.gs_sync_status(ctx)


def _grads(ctx, scene, cam, target, deferred):
    g = gs.scene_to_device(scene)
    params = [g[k].clone().requires_grad_(True) for k in ("means", "log_scales", "quats",
                                                          "opacity_logits", "sh")]
    rgb, _ = gs.RasterizeGaussians(*params, ctx, cam, scene.sh_degree, deferred=deferred)
    (rgb - target).abs().mean().backward()
    torch.cuda.synchronize()
    return [p.grad.clone() for p in params]


def test_backward_after_overflowed_deferred_forward_fails(built):
    scene = scenes.uniform_box(5_000, 23)
    cam = scenes.pinhole(128, 96)
    target = torch.from_numpy(scenes.l1_target(cam.height, cam.width, 1023)).cuda()
    ref = _grads(gs.Context(0), scene, cam, target, deferred=False)
    ctx = gs.Context(0)
    gs.gs_reserve_keys(ctx, 100)
    with pytest.raises(gs.GSError) as e:
        _grads(ctx, scene, cam, target, deferred=True)
    assert e.value.status == 4
    got = _grads(ctx, scene, cam, target, deferred=True)  # buffers have grown
    for a, b in zip(ref, got):  # float atomics: equal up to summation order
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * float(a.abs().max()) + 1e-12)


def test_frames_in_flight_on_several_contexts_and_streams(built):
    """Consecutive frames on four contexts, each on its own stream, deferred
    (how a renderer keeps several frames in flight): every frame equals the
    same camera rendered alone and synchronously, for both blend schedules."""
    scene = scenes.clustered(200_000, 41)
    g = gs.scene_to_device(scene)
    rng = np.random.default_rng(41)
    cams = [scenes.pinhole(640, 360, 60.0, world_to_cam=scenes.look_at(rng.uniform(-1, 1, 3),
                                                                        [0.0, 0.0, 1.0] + rng.normal(0, 0.2, 3)))
            for _ in range(8)]
    ref_ctx = gs.Context(0)
    for variant in (0, 4):
        refs = [gs.render(ref_ctx, g, scene.sh_degree, c, variant=variant) for c in cams]
        torch.cuda.synchronize()
        ctxs = [gs.Context(0) for _ in range(4)]
        streams = [torch.cuda.Stream() for _ in range(4)]
        outs = [{"rgb": torch.empty((c.height, c.width, 3), device="cuda"),
                 "final_T": torch.empty((c.height, c.width), device="cuda"),
                 "n_contrib": torch.empty((c.height, c.width), dtype=torch.int32, device="cuda")} for c in cams]
        start = torch.cuda.Event()
        start.record()
        for s in streams:
            s.wait_event(start)
        for i, (c, o) in enumerate(zip(cams, outs)):
            k = i % 4
            with torch.cuda.stream(streams[k]):
                gs.gs_render(ctxs[k], g, scene.sh_degree, c, o["rgb"], o["final_T"], o["n_contrib"],
                             variant=variant, deferred=True, stream=streams[k])
        torch.cuda.synchronize()
        for c in ctxs:
            gs.gs_sync_status(c)
            c.close()
        for r, o in zip(refs, outs):
            for key in ("rgb", "final_T", "n_contrib"):
                assert torch.equal(r[key], o[key]), key
    ref_ctx.close()


def test_frames_in_flight_full_size_as_benchmarked(built):
    """The throughput configuration at full size: the 1M-Gaussian 1080p frame
    rendered deferred on sixteen contexts, each on its own stream, with 4x4
    list tiles in grid tile order and the inputs rotating over copies of the
    scene (and, with eight contexts, the 8x8-block blend with a list per
    tile); every frame equals the synchronous default render of the same
    frame bit for bit (and that render is checked against the FP64 oracle
    elsewhere)."""
    scene, cams = scenes.workload("clustered_1m_1080p")
    cam = cams[0]
    g = gs.scene_to_device(scene)
    copies = [g] + [{k: v.clone() for k, v in g.items()} for _ in range(2)]
    ref_ctx = gs.Context(0)
    ref = gs.render(ref_ctx, g, scene.sh_degree, cam)
    torch.cuda.synchronize()
    gs.gs_sync_status(ref_ctx)
    for F, frames, opt in ((16, 32, dict(list_tiles=16, tile_order=1)), (8, 16, dict(variant=4))):
        ctxs = [gs.Context(0) for _ in range(F)]
        streams = [torch.cuda.Stream() for _ in range(F)]
        for c in ctxs:  # warm-up frame per context, as the benchmark does
            gs.render(c, g, scene.sh_degree, cam, aux=False, **opt)
        torch.cuda.synchronize()
        H, W = cam.height, cam.width
        outs = [{"rgb": torch.empty((H, W, 3), device="cuda"),
                 "final_T": torch.empty((H, W), device="cuda"),
                 "n_contrib": torch.empty((H, W), dtype=torch.int32, device="cuda")} for _ in range(frames)]
        start = torch.cuda.Event()
        start.record()
        for s in streams:
            s.wait_event(start)
        for i, o in enumerate(outs):
            k = i % F
            with torch.cuda.stream(streams[k]):
                gs.gs_render(ctxs[k], copies[i % len(copies)], scene.sh_degree, cam, o["rgb"], o["final_T"],
                             o["n_contrib"], deferred=True, stream=streams[k], **opt)
        torch.cuda.synchronize()
        for c in ctxs:
            gs.gs_sync_status(c)
            c.close()
        for o in outs:
            assert torch.equal(ref["rgb"], o["rgb"]) and torch.equal(ref["final_T"], o["final_T"]), (F, opt)
            if "list_tiles" not in opt:  # list-tile frames count list-tile positions
                assert torch.equal(ref["n_contrib"], o["n_contrib"]), (F, opt)
        del outs
    ref_ctx.close()
