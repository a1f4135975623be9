"""GPU backward (gs_render_backward) against the FP64 oracle gradient, which
is itself pinned by finite differences (tests/test_oracle_grad_pins.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15951_gb300 as gs  # noqa: E402
from paper_2607_15951_gb300 import scenes  # noqa: E402

from test_oracle_grad_pins import fd_scene  # noqa: E402

GROUPS = ["means", "log_scales", "quats", "opacity_logits", "sh"]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15951_gb300 import build
    build.build()
    c = gs.Context(0)
    yield c
    c.close()


def gpu_grads(ctx, scene, cam, dL_dC, bg=(0.0, 0.0, 0.0), tile=(16, 16)):
    g = gs.scene_to_device(scene)
    out = gs.render(ctx, g, scene.sh_degree, cam, bg=bg, tile=tile)
    grads = {k: torch.full_like(v, float("nan")) for k, v in g.items()}
    grads["records"] = torch.zeros((scene.n, 9), dtype=torch.float32, device="cuda")
    d = torch.from_numpy(np.ascontiguousarray(dL_dC, dtype=np.float32)).cuda()
    gs.gs_render_backward(ctx, g, scene.sh_degree, cam, out["final_T"], out["n_contrib"], d, grads,
                          bg=bg, tile=tile)
    torch.cuda.synchronize()
    gs.gs_sync_status(ctx)
    return {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}, out


def compare(gpu, ora, rtol=1e-3):
    """Element error normalised by |oracle| + 1e-3 max|oracle| of the group;
    returns (max error, fraction of elements above rtol, Gaussian index of
    every element above rtol)."""
    a = gpu.reshape(gpu.shape[0], -1)
    b = ora.reshape(a.shape)
    scale = np.abs(b) + 1e-3 * max(np.abs(b).max(), 1e-30)
    err = np.abs(a - b) / scale
    return float(err.max()), float((err > rtol).mean()), np.nonzero((err > rtol).any(axis=1))[0]


def flagged_gaussians(bn, img, width, tile=16):
    """Gaussians listed in a tile that holds a pixel whose alpha or T decision
    lies within 1e-6 of its cutoff (the oracle's flag): the only Gaussians
    whose FP32 gradient may legitimately differ from the FP64 one by more
    than rounding, because FP32 may take that decision the other way."""
    tiles_x = (width + tile - 1) // tile
    ys, xs = np.nonzero(img.flag)
    out = set()
    for t in set((ys // tile * tiles_x + xs // tile).tolist()):
        out.update(bn.values[bn.ranges[t, 0]:bn.ranges[t, 1]].tolist())
    return out


# Elements of a parameter group allowed above 1e-3 relative error: at most
# one in 10^4, and each must belong to a Gaussian of a tile with a flagged
# pixel.
MAX_EXCESS_FRACTION = 1e-4


def check_groups(gpu, ora, bn, img, width, name):
    tied = flagged_gaussians(bn, img, width)
    report = {}
    for grp in GROUPS + ["records"]:
        g = gpu[grp]
        o = ora.record if grp == "records" else getattr(ora, grp).reshape(g.shape)
        assert np.isfinite(g).all(), grp
        mx, frac, idx = compare(g, o)
        untied = [int(i) for i in idx if int(i) not in tied]
        report[grp] = (mx, frac, len(idx), len(untied))
    print(name, "flagged pixels", int(img.flag.sum()), report)
    for grp, (mx, frac, n_ex, n_untied) in report.items():
        assert frac <= MAX_EXCESS_FRACTION, (grp, mx, frac)
        assert n_untied == 0, (grp, n_untied)


CASES = [
    ("fd_scene_sh3_bg", lambda: (fd_scene(3, 3), scenes.pinhole(32, 32)), (0.1, 0.2, 0.3)),
    ("fd_scene_sh0", lambda: (fd_scene(4, 0), scenes.pinhole(32, 32)), (0.0, 0.0, 0.0)),
    ("uniform_box_2k_128x96", lambda: (scenes.uniform_box(2_000, 5), scenes.pinhole(128, 96)), (0.0, 0.0, 0.0)),
    ("clustered_30k_320x180_sh3", lambda: (scenes.clustered(30_000, 9, box=4.0), scenes.pinhole(320, 180)), (0.0, 0.0, 0.0)),
]


@pytest.mark.parametrize("name,make,bg", CASES, ids=[c[0] for c in CASES])
def test_backward_matches_oracle(ctx, oracle_mod, name, make, bg):
    scene, cam = make()
    rng = np.random.default_rng(11)
    dL = rng.normal(0.0, 1.0, (cam.height, cam.width, 3))
    gpu, out = gpu_grads(ctx, scene, cam, dL, bg=bg)
    ora = oracle_mod.render_backward(scene, cam, dL, bg=bg)
    _, bn, img = oracle_mod.render(scene, cam, bg=bg)
    # Pixels at an alpha/T cutoff can move one contribution between FP32 and
    # FP64; everywhere else the gradient agrees to 1e-3 relative.
    check_groups(gpu, ora, bn, img, cam.width, name)


def test_backward_at_500k_1080p_l1_loss(ctx, oracle_mod):
    """The forward+backward workload at full size: 500k clustered Gaussians,
    SH3, 1920x1080, L1 loss against a seeded target, dL/dC = sign(C - target)
    / (3 P); all five parameter groups against the FP64 oracle gradient."""
    scene, cams = scenes.workload("clustered_500k_1080p")
    cam = cams[0]
    g = gs.scene_to_device(scene)
    out = gs.render(ctx, g, scene.sh_degree, cam)
    target = torch.from_numpy(scenes.l1_target(cam.height, cam.width, 1002)).cuda()
    dL = (torch.sign(out["rgb"] - target) / out["rgb"].numel()).cpu().numpy().astype(np.float64)
    gpu, _ = gpu_grads(ctx, scene, cam, dL)
    ora = oracle_mod.render_backward(scene, cam, dL)
    _, bn, img = oracle_mod.render(scene, cam)
    check_groups(gpu, ora, bn, img, cam.width, "clustered_500k_1080p")


def test_backward_of_an_earlier_frame(ctx, oracle_mod):
    """Two views rendered before the first view's backward (multi-view
    training): the C call refuses the stale frame instead of differentiating
    the second view's lists, and the autograd function renders the first view
    again, giving its own gradients."""
    scene = scenes.clustered(20_000, 12, box=4.0)
    cams = scenes.trajectory(2, 1012, radius=1.0, sizes=((160, 120),))
    g = gs.scene_to_device(scene)
    first = gs.render(ctx, g, scene.sh_degree, cams[0])
    gs.render(ctx, g, scene.sh_degree, cams[1])
    grads = {k: torch.empty_like(v) for k, v in g.items()}
    d = torch.ones((120, 160, 3), device="cuda")
    with pytest.raises(gs.GSError):
        gs.gs_render_backward(ctx, g, scene.sh_degree, cams[0], first["final_T"], first["n_contrib"], d, grads)

    target = [torch.from_numpy(scenes.l1_target(120, 160, 1012 + v)).cuda() for v in range(2)]
    params = [g[k].clone().requires_grad_(True) for k in GROUPS]
    rgb0, _ = gs.RasterizeGaussians(*params, ctx, cams[0], scene.sh_degree)
    rgb1, _ = gs.RasterizeGaussians(*params, ctx, cams[1], scene.sh_degree)
    (rgb0 - target[0]).abs().sum().backward(retain_graph=True)
    both = [p.grad.clone() for p in params]
    ((rgb0 - target[0]).abs().sum() + (rgb1 - target[1]).abs().sum()).backward()
    total = [p.grad.clone() for p in params]
    torch.cuda.synchronize()
    # Each view's gradient alone, with nothing rendered in between, and from the oracle.
    for v in range(2):
        sub = [g[k].clone().requires_grad_(True) for k in GROUPS]
        rgb, _ = gs.RasterizeGaussians(*sub, ctx, cams[v], scene.sh_degree)
        (rgb - target[v]).abs().sum().backward()
        alone = [p.grad for p in sub]
        if v == 0:
            for a, b in zip(both, alone):
                _close(a, b)
            dL = torch.sign(rgb.detach() - target[0]).cpu().numpy().astype(np.float64)
            ora = oracle_mod.render_backward(scene, cams[0], dL)
            for grp, a in zip(GROUPS, alone):
                mx, frac, _ = compare(a.cpu().numpy().astype(np.float64), getattr(ora, grp))
                assert frac <= MAX_EXCESS_FRACTION, (grp, mx, frac)
        else:
            for a, t, b0 in zip(alone, total, both):
                _close(b0 * 2 + a, t)


def _close(a, b):
    """Equal up to the FP32 summation order of the gradient atomics."""
    tol = 1e-4 * b.abs() + 1e-5 * float(b.abs().max())
    assert bool(((a - b).abs() <= tol).all()), float((a - b).abs().max())


def _fd_render(ctx, g, deg, cam):
    out = gs.render(ctx, g, deg, cam)
    return out["rgb"].double(), out["n_contrib"], out["n_eval"], gs.gs_last_render_stats(ctx)["n_keys"]


@pytest.mark.parametrize("seed,deg", [(3, 3), (4, 0)])
def test_gpu_gradient_matches_gpu_central_differences(ctx, seed, deg):
    """The GPU gradient against central differences of the GPU's own FP32
    forward at 64 Gaussians / 32x32 (L = sum w . C). A finite step can carry a
    discrete decision across it (a pixel's alpha crossing 1/255, a rect
    gaining a tile), which adds a jump to the difference quotient; such steps
    are found per pixel, where jumps cannot cancel: the image differences at h
    and h/2 must agree pixel by pixel (and the lists and stop positions must
    not change), otherwise the parameter is skipped. FP32 rounding of the
    image bounds the error of an accepted quotient by about 1e-4 at h = 2e-3."""
    from test_oracle_grad_pins import fd_scene
    scene = fd_scene(seed, deg)
    cam = scenes.pinhole(32, 32, 60.0)
    w_np = np.random.default_rng(seed + 100).normal(0.0, 1.0, (32, 32, 3))
    w = torch.from_numpy(w_np).cuda()
    an, _ = gpu_grads(ctx, scene, cam, w_np)
    g = gs.scene_to_device(scene)
    rng = np.random.default_rng(seed + 300)
    checked = skipped = 0
    for grp in GROUPS:
        arr = g[grp]
        flat = arr.view(-1)
        scale = np.abs(an[grp]).max()
        for fi in rng.permutation(flat.numel())[:40]:
            old = float(flat[fi])
            h = 2e-3 * max(1.0, abs(old))

            def diff(step):
                flat[fi] = old + step
                cp, ncp, nep, kp = _fd_render(ctx, g, deg, cam)
                flat[fi] = old - step
                cm, ncm, nem, km = _fd_render(ctx, g, deg, cam)
                flat[fi] = old
                same = kp == km and torch.equal(ncp, ncm) and torch.equal(nep, nem)
                return cp - cm, same

            d1, same1 = diff(h)
            d2, same2 = diff(h / 2)
            smooth = bool(((d1 - 2 * d2).abs() <= 2e-6 + 2e-2 * d1.abs()).all())
            a = float(an[grp].reshape(-1)[fi])
            if not (same1 and same2 and smooth):
                skipped += 1
                continue
            fd = float((d1 * w).sum()) / (2 * h)
            tol = 1e-2 * abs(a) + 1e-3 * scale + 2e-4
            assert abs(fd - a) <= tol, (grp, int(fi), fd, a)
            checked += 1
    print("GPU central differences: checked", checked, "skipped", skipped)
    assert checked >= 120, (checked, skipped)


@pytest.mark.parametrize("form", [{}, {"tile": (16, 8)}, {"list_tiles": 4}, {"list_tiles": 64}],
                         ids=["t16", "t16x8", "l2x2", "l8x8"])
def test_backward_after_either_tile_order(ctx, form):
    """A forward whose blend took its tiles longest list first leaves the
    same frame to differentiate as a grid-order forward: the same gradients.
    Float atomics add in a run-dependent order, so the comparison allows 1e-4
    of the largest gradient (the run-to-run spread is ~1e-5)."""
    scene, cam = scenes.clustered(50_000, 42, box=5.0), scenes.pinhole(320, 180)
    g = gs.scene_to_device(scene)
    d = torch.randn((180, 320, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    res = []
    for order in (gs._native.GS_ORDER_LONGEST_FIRST, gs._native.GS_ORDER_GRID):
        out = gs.render(ctx, g, scene.sh_degree, cam, tile_order=order, **form)
        grads = {k: torch.empty_like(v) for k, v in g.items()}
        bw = {k: v for k, v in form.items()}
        gs.gs_render_backward(ctx, g, scene.sh_degree, cam, out["final_T"], out["n_contrib"], d, grads, **bw)
        torch.cuda.synchronize()
        res.append(grads)
    for k in GROUPS:
        a, b = res[0][k], res[1][k]
        assert torch.isfinite(a).all(), k
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-4 * float(b.abs().max()) + 1e-12), k


def test_autograd_function_matches_direct_call(ctx):
    scene, cam = scenes.uniform_box(1_000, 6), scenes.pinhole(96, 64)
    g = gs.scene_to_device(scene)
    params = [g[k].clone().requires_grad_(True) for k in GROUPS]
    target = torch.rand((cam.height, cam.width, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    rgb, T = gs.RasterizeGaussians(*params, ctx, cam, scene.sh_degree)
    loss = (rgb - target).abs().mean()
    loss.backward()
    d = torch.sign(rgb.detach() - target) / rgb.numel()
    direct, _ = gpu_grads(ctx, scene, cam, d.cpu().numpy())
    for p, grp in zip(params, GROUPS):
        np.testing.assert_allclose(p.grad.cpu().numpy(), direct[grp], rtol=1e-5, atol=1e-9)


def test_backward_requires_preceding_render(ctx):
    scene, cam = scenes.uniform_box(100, 1), scenes.pinhole(64, 64)
    g = gs.scene_to_device(scene)
    gs.render(ctx, g, 0, cam)
    other = scenes.pinhole(32, 32)
    grads = {k: torch.empty_like(v) for k, v in g.items()}
    T = torch.ones((32, 32), device="cuda")
    nc = torch.zeros((32, 32), dtype=torch.int32, device="cuda")
    with pytest.raises(gs.GSError):
        gs.gs_render_backward(ctx, g, 0, other, T, nc, torch.zeros((32, 32, 3), device="cuda"), grads)
