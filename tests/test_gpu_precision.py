"""Reduced-precision blend records (16-bit opacity and colour; FP32 2D mean,
conic and alpha threshold; FP32 compositing) against the FP64 oracle: max
abs error per channel on pixels whose alpha / T decisions are not at a
cutoff, against the bound stated for every precision (4e-3); the gradients
element by element against the oracle's; the measured errors are printed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15951_gb300 as gs  # noqa: E402
from paper_2607_15951_gb300 import scenes  # noqa: E402
from paper_2607_15951_gb300 import _native as N  # noqa: E402

from parity_util import compare_render  # noqa: E402

# Stated bound per record precision (max abs per channel, non-cutoff pixels).
# Derivation: the alpha decisions use the FP32 threshold, so only the values
# move: a colour error |dc| <= 2^-11 c (FP16; c < 2: 9.8e-4) or 2^-9 (BF16
# stores c - 1) weighted by sum alpha T <= 1, plus an opacity error
# (FP16 in both) |d alpha| <= 2^-11 alpha times |c_k - (later light)/(1 -
# alpha_k)| <= max c < 2 (<= 9.8e-4): at most 3e-3 with FP32 rounding.
BOUND = {N.GS_RECORD_F16: 4e-3, N.GS_RECORD_BF16: 4e-3}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15951_gb300 import build
    build.build()
    c = gs.Context(0)
    yield c
    c.close()


CASES = [("uniform_box_256", "uniform_box_256"), ("clustered_1m_1080p", "clustered_1m_1080p")]


@pytest.mark.parametrize("dtype", [N.GS_RECORD_F16, N.GS_RECORD_BF16], ids=["f16", "bf16"])
@pytest.mark.parametrize("name,workload", CASES, ids=[c[0] for c in CASES])
def test_low_precision_records_within_bound(ctx, oracle_mod, name, workload, dtype):
    scene, cams = scenes.workload(workload)
    cam = cams[0]
    g = gs.scene_to_device(scene)
    out = gs.render(ctx, g, scene.sh_degree, cam, record_dtype=dtype)
    ref = gs.render(ctx, g, scene.sh_degree, cam)
    torch.cuda.synchronize()
    gs.gs_sync_status(ctx)
    pr, bn, img = oracle_mod.render(scene, cam)
    st = compare_render(out["rgb"].cpu().numpy(), out["final_T"].cpu().numpy(), pr, bn, img, cam.width, cam.height)
    st.pop("keep")
    diff32 = float((out["rgb"] - ref["rgb"]).abs().max())
    print(name, "f16" if dtype == 1 else "bf16", "vs FP64:", st, "vs FP32 records:", diff32)
    assert np.isfinite(out["rgb"].cpu().numpy()).all()
    assert st["max_rgb_err"] <= BOUND[dtype], st


# Gradient bound for 16-bit records. The backward differentiates the image
# the forward made from the rounded opacity and colours, so each gradient
# element carries that rounding through sums of many terms of both signs:
# its error is measured against the typical size of the group's elements,
# |g - g64| / (|g64| + rms(g64)), and bounded by eight times the unit
# roundoff of the stored colours (FP16 2^-11; BF16 2^-9 on colour - 1);
# at most one element in 10^3 may exceed it.
GRAD_RHO = {N.GS_RECORD_F16: 8 * 2.0 ** -11, N.GS_RECORD_BF16: 8 * 2.0 ** -9}
GRAD_EXCESS = 1e-3


@pytest.mark.parametrize("dtype", [N.GS_RECORD_F16, N.GS_RECORD_BF16], ids=["f16", "bf16"])
@pytest.mark.parametrize("name", ["uniform_box_2k_128x96", "clustered_30k_320x180_sh3"])
def test_low_precision_backward_matches_oracle(ctx, oracle_mod, dtype, name):
    from test_gpu_backward import GROUPS
    scene, cam = {"uniform_box_2k_128x96": lambda: (scenes.uniform_box(2_000, 5), scenes.pinhole(128, 96)),
                  "clustered_30k_320x180_sh3": lambda: (scenes.clustered(30_000, 9, box=4.0),
                                                        scenes.pinhole(320, 180))}[name]()
    g = gs.scene_to_device(scene)
    dL = np.random.default_rng(11).normal(0.0, 1.0, (cam.height, cam.width, 3))
    out = gs.render(ctx, g, scene.sh_degree, cam, record_dtype=dtype)
    grads = {k: torch.empty_like(v) for k, v in g.items()}
    d = torch.from_numpy(dL.astype(np.float32)).cuda()
    gs.gs_render_backward(ctx, g, scene.sh_degree, cam, out["final_T"], out["n_contrib"], d, grads,
                          record_dtype=dtype)
    torch.cuda.synchronize()
    ora = oracle_mod.render_backward(scene, cam, dL)
    report = {}
    for grp in GROUPS:
        a = grads[grp].cpu().numpy().astype(np.float64).reshape(-1)
        o = getattr(ora, grp).reshape(-1)
        assert np.isfinite(a).all(), grp
        err = np.abs(a - o) / (np.abs(o) + np.sqrt(np.mean(o ** 2)))
        report[grp] = (float(err.max()), float(np.quantile(err, 0.999)), float((err > GRAD_RHO[dtype]).mean()))
    print(name, "f16" if dtype == 1 else "bf16", "gradient vs FP64 (max, 99.9 %, above bound):", report)
    for grp, (mx, q, frac) in report.items():
        assert frac <= GRAD_EXCESS, (grp, mx, q, frac)


@pytest.mark.parametrize("dtype", [N.GS_RECORD_F16, N.GS_RECORD_BF16], ids=["f16", "bf16"])
def test_low_precision_backward_runs_and_tracks_fp32(ctx, dtype):
    scene, cam = scenes.uniform_box(2_000, 5), scenes.pinhole(128, 96)
    g = gs.scene_to_device(scene)
    d = torch.randn((96, 128, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    res = {}
    for dt in (N.GS_RECORD_F32, dtype):
        out = gs.render(ctx, g, 0, cam, record_dtype=dt)
        grads = {k: torch.empty_like(v) for k, v in g.items()}
        gs.gs_render_backward(ctx, g, 0, cam, out["final_T"], out["n_contrib"], d, grads, record_dtype=dt)
        torch.cuda.synchronize()
        res[dt] = grads
    for k in res[dtype]:
        a, b = res[dtype][k], res[N.GS_RECORD_F32][k]
        assert torch.isfinite(a).all()
        rel = float((a - b).norm() / (b.norm() + 1e-30))
        print(k, "relative L2 difference to FP32 records", rel)
        assert rel < 0.05, (k, rel)
