"""Temporal re-binning (gs_options.temporal): the per-tile lists of a frame
are rebuilt from the previous frame's. Every frame must equal the frame the
full binning renders, bit for bit (the per-tile order (depth bits, index) is
unique), for slow and abrupt camera motions, across the fall-back cases
(too many moved Gaussians, a tile list above the per-tile limit, key buffers
too small) and when other calls on the context intervene."""
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


def _equal(a, b):
    for k in a:
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("kind,step", [("static", None), ("orbit", 0.1), ("orbit", 2.0), ("translate", 0.01),
                                       ("rotate", 1.0), ("teleport", None)])
def test_rebinned_frames_equal_full_binning(built, kind, step):
    scene = scenes.clustered(200_000, 31, box=8.0)
    g = gs.scene_to_device(scene)
    cams = scenes.motion(kind, 6, 480, 272, step=step)
    full, temp = gs.Context(0), gs.Context(0)
    rebinned, moved = [], []
    for c in cams:
        ref = gs.render(full, g, scene.sh_degree, c)
        out = gs.render(temp, g, scene.sh_degree, c, temporal=2)
        torch.cuda.synchronize()
        _equal(ref, out)
        st = gs.gs_last_render_stats(temp)
        assert st["n_keys"] == gs.gs_last_render_stats(full)["n_keys"]
        rebinned.append(st["rebinned"])
        moved.append(st["n_moved"])
    assert not rebinned[0]
    if kind == "static":
        assert all(rebinned[1:]) and moved[1:] == [0] * 5
    if (kind, step) == ("orbit", 0.1):  # a slow motion (low churn) stays incremental
        assert all(rebinned[1:]), (rebinned, moved)
    if kind != "static":  # the churn is measured whichever way a frame was binned
        assert all(m > 0 for m in moved[1:]), moved
    print(kind, step, "rebinned", rebinned, "moved", moved)


def test_rebinned_moved_frames_match_oracle(built, oracle_mod):
    """Re-binned frames of a moving camera against the FP64 oracle's render of
    the same camera (not only against the full binning): a mistake shared by
    both binnings of this library cannot pass."""
    from parity_util import RGB_TOL, compare_image
    scene = scenes.clustered(200_000, 31, box=8.0)
    g = gs.scene_to_device(scene)
    cams = scenes.motion("orbit", 4, 480, 272, step=0.1)
    ctx = gs.Context(0)
    for i, c in enumerate(cams):
        out = gs.render(ctx, g, scene.sh_degree, c, temporal=2)
        torch.cuda.synchronize()
        st = gs.gs_last_render_stats(ctx)
        if i == 0:
            continue
        assert st["rebinned"] and st["n_moved"] > 0, st
        _, _, img = oracle_mod.render(scene, c)
        cmp = compare_image(out["rgb"].cpu().numpy(), out["final_T"].cpu().numpy(), img)
        cmp.pop("keep")
        print("re-binned frame", i, "moved", st["n_moved"], "vs FP64:", cmp)
        assert cmp["max_rgb_err"] <= RGB_TOL and cmp["max_T_err"] <= RGB_TOL, cmp


def test_adaptive_gate_keeps_frames_exact(built):
    """temporal = 1: the context times re-binned and full frames and picks
    the faster, re-trying re-binning now and then; every frame still equals
    the full binning's, and the first frame after the churn was measured is
    re-binned (to measure it)."""
    scene = scenes.clustered(200_000, 37, box=8.0)
    g = gs.scene_to_device(scene)
    cams = scenes.motion("static", 40, 480, 272)
    full, temp = gs.Context(0), gs.Context(0)
    rebinned = []
    for c in cams:
        ref = gs.render(full, g, scene.sh_degree, c)
        out = gs.render(temp, g, scene.sh_degree, c, temporal=1)
        torch.cuda.synchronize()
        _equal(ref, out)
        rebinned.append(gs.gs_last_render_stats(temp)["rebinned"])
    # The first frame with rects to compare (frame 1) bins in full and
    # measures the churn; frame 2 is re-binned.
    assert not rebinned[0] and not rebinned[1] and rebinned[2], rebinned
    print("adaptive gate, static camera: re-binned frames", sum(rebinned), "of", len(rebinned))


def test_adaptive_gate_cools_down_on_high_churn(built):
    """temporal = 1 with a fast camera (churn far above the limit): after a
    frame that measured the churn too high, six frames skip the rect tracking
    (n_moved = 0), then one frame writes rects and the next bins in full and
    measures the churn; every frame equals the full binning's."""
    scene = scenes.clustered(200_000, 38, box=8.0)
    g = gs.scene_to_device(scene)
    cams = scenes.motion("rotate", 34, 480, 272, step=1.0)
    full, temp = gs.Context(0), gs.Context(0)
    moved = []
    for c in cams:
        ref = gs.render(full, g, scene.sh_degree, c)
        out = gs.render(temp, g, scene.sh_degree, c, temporal=1)
        torch.cuda.synchronize()
        _equal(ref, out)
        moved.append(gs.gs_last_render_stats(temp)["n_moved"])
    tracked = [i for i, m in enumerate(moved) if m > 0]
    print("adaptive gate, rotating camera: frames that measured the churn", tracked)
    # Frame 1 bins in full and measures the churn; then one frame in eight:
    # 9, 17, 25, 33.
    assert tracked == list(range(1, len(cams), 8)), moved


def test_rebinning_falls_back_and_recovers(built):
    # One tile holds more than the per-tile limit: every frame is binned in
    # full, with identical results.
    s = scenes.uniform_box(6_000, 32)
    s.means[:, 0] = 0.01 * s.means[:, 0]
    s.means[:, 1] = 0.01 * s.means[:, 1]
    s.log_scales[:] = -6.0
    g = gs.scene_to_device(s)
    cams = scenes.motion("translate", 3, 256, 256, step=0.001)
    full, temp = gs.Context(0), gs.Context(0)
    for c in cams:
        _equal(gs.render(full, g, 0, c), gs.render(temp, g, 0, c, temporal=2))
        assert not gs.gs_last_render_stats(temp)["rebinned"]
    # Key buffers too small for the re-binned frame: it is binned again.
    scene = scenes.clustered(100_000, 33, box=8.0)
    g = gs.scene_to_device(scene)
    cams = scenes.motion("orbit", 4, 320, 240, step=0.5)
    full, temp = gs.Context(0), gs.Context(0)
    gs.gs_reserve_keys(temp, 2000)
    for c in cams:
        _equal(gs.render(full, g, scene.sh_degree, c), gs.render(temp, g, scene.sh_degree, c, temporal=2))


def test_intervening_calls_drop_the_state(built):
    scene = scenes.clustered(100_000, 34, box=8.0)
    g = gs.scene_to_device(scene)
    cams = scenes.motion("orbit", 5, 320, 240, step=0.2)
    other = scenes.pinhole(200, 120)
    full, temp = gs.Context(0), gs.Context(0)
    for i, c in enumerate(cams):
        if i == 2:  # a non-temporal frame of another size on the same context
            gs.render(temp, g, scene.sh_degree, other)
        if i == 3:  # a stage call that reuses the context's key buffers
            k = torch.arange(1000, 0, -1, dtype=torch.int64, device="cuda")
            v = torch.arange(1000, dtype=torch.int32, device="cuda")
            gs.gs_sort_pairs(temp, k, v, 1000, 16)
        _equal(gs.render(full, g, scene.sh_degree, c), gs.render(temp, g, scene.sh_degree, c, temporal=2))


def test_backward_after_rebinned_frame(built):
    scene = scenes.clustered(50_000, 35, box=6.0)
    cams = scenes.motion("orbit", 3, 256, 192, step=0.3)
    target = torch.from_numpy(scenes.l1_target(192, 256, 1035)).cuda()

    def grads(ctx, temporal):
        g = gs.scene_to_device(scene)
        out = None
        for c in cams:
            out = gs.render(ctx, g, scene.sh_degree, c, temporal=2 if temporal else 0)
        d_rgb = torch.sign(out["rgb"] - target) / target.numel()
        gr = {k: torch.empty_like(v) for k, v in g.items()}
        gs.gs_render_backward(ctx, g, scene.sh_degree, cams[-1], out["final_T"], out["n_contrib"],
                              d_rgb.contiguous(), gr)
        torch.cuda.synchronize()
        return gr

    t_ctx = gs.Context(0)
    a, b = grads(gs.Context(0), False), grads(t_ctx, True)
    assert gs.gs_last_render_stats(t_ctx)["rebinned"]
    for k in a:  # float atomics: equal up to summation order (cancellation in sums of many terms)
        assert torch.allclose(a[k], b[k], rtol=1e-3, atol=1e-5 * float(a[k].abs().max()) + 1e-12), k


def test_rejects_deferred_temporal(built):
    s = scenes.uniform_box(100, 36)
    with pytest.raises(gs.GSError) as e:
        gs.render(gs.Context(0), gs.scene_to_device(s), 0, scenes.pinhole(64, 64), temporal=True, deferred=True)
    assert e.value.status == 1
