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
