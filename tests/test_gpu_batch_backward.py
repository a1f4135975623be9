"""Batched backward (gs_render_batch_backward, RasterizeGaussiansBatch): the
gradients of a joint multi-view batch equal the sum of the single-view
backward passes (up to the summation order of float atomics), for FP32 and
BF16 records; a backward without a preceding joint batch is rejected."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15951_gb300 as gs  # noqa: E402
from paper_2607_15951_gb300 import _native as N  # noqa: E402
from paper_2607_15951_gb300 import scenes  # noqa: E402

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15951_gb300 import build
    build.build()
    scene = scenes.clustered(40_000, 26, box=5.0)
    cams = scenes.trajectory(4, 1026, radius=2.0, sizes=((192, 108), (160, 120)))
    return scene, cams, gs.scene_to_device(scene), gs.Context(0)


def _close(a, b):
    for k in GROUPS:
        scale = float(b[k].abs().max()) + 1e-12
        assert torch.allclose(a[k], b[k], rtol=1e-3, atol=1e-5 * scale), (k, float((a[k] - b[k]).abs().max()), scale)


@pytest.mark.parametrize("dtype", [N.GS_RECORD_F32, N.GS_RECORD_BF16], ids=["f32", "bf16"])
def test_batch_backward_equals_sum_of_views(setup, dtype):
    scene, cams, g, ctx = setup
    gen = torch.Generator(device="cuda").manual_seed(7)
    ds = [torch.randn((c.height, c.width, 3), device="cuda", generator=gen) for c in cams]
    ref = {k: torch.zeros_like(v) for k, v in g.items()}
    for c, d in zip(cams, ds):
        out = gs.render(ctx, g, scene.sh_degree, c, record_dtype=dtype)
        gr = {k: torch.empty_like(v) for k, v in g.items()}
        gs.gs_render_backward(ctx, g, scene.sh_degree, c, out["final_T"], out["n_contrib"], d, gr,
                              record_dtype=dtype)
        for k in ref:
            ref[k] += gr[k]
    outs = gs.alloc_outputs(cams, aux=True)
    gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs, record_dtype=dtype, batch_mode=N.GS_BATCH_JOINT)
    got = {k: torch.empty_like(v) for k, v in g.items()}
    gs.gs_render_batch_backward(ctx, g, scene.sh_degree, cams, outs, ds, got, record_dtype=dtype)
    torch.cuda.synchronize()
    _close(got, ref)


def test_batch_autograd_matches_per_view_autograd(setup):
    scene, cams, g, ctx = setup
    targets = [torch.from_numpy(scenes.l1_target(c.height, c.width, 1030 + i)).cuda() for i, c in enumerate(cams)]

    def params():
        return [g[k].clone().requires_grad_(True) for k in GROUPS]

    p_batch = params()
    rgbs = gs.RasterizeGaussiansBatch(*p_batch, ctx, cams, scene.sh_degree)
    sum((r - t).abs().mean() for r, t in zip(rgbs, targets)).backward()
    p_view = params()
    for c, t in zip(cams, targets):
        rgb, _ = gs.RasterizeGaussians(*p_view, ctx, c, scene.sh_degree)
        (rgb - t).abs().mean().backward()
    torch.cuda.synchronize()
    _close({k: p.grad for k, p in zip(GROUPS, p_batch)}, {k: p.grad for k, p in zip(GROUPS, p_view)})


def test_batch_backward_needs_a_joint_batch(setup):
    scene, cams, g, ctx = setup
    outs = gs.alloc_outputs(cams, aux=True)
    gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs, batch_mode=N.GS_BATCH_PER_VIEW)
    got = {k: torch.empty_like(v) for k, v in g.items()}
    ds = [torch.zeros((c.height, c.width, 3), device="cuda") for c in cams]
    with pytest.raises(gs.GSError) as e:
        gs.gs_render_batch_backward(ctx, g, scene.sh_degree, cams, outs, ds, got)
    assert e.value.status == 1
