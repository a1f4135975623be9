"""Reduced-precision projected records (16-bit opacity and colour; FP32 2D
mean and conic; FP32 compositing) against the FP64 oracle: max abs error per
channel on pixels whose alpha / T decisions are not at a cutoff, against the
bound stated for each precision; the measured error is printed."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15951_gb300 as gs  # noqa: E402
from paper_2607_15951_gb300 import scenes  # noqa: E402
from paper_2607_15951_gb300 import _native as N  # noqa: E402

from parity_util import compare_image  # noqa: E402

# Stated bound per record precision (max abs per channel, non-cutoff pixels).
# FP16 opacity/colour meet the 4e-3 target; BF16's 2^-9 rounding of opacity
# and colour alone reaches ~5e-3 on the dense 1080p scene, so its stated bound
# is 6e-3.
BOUND = {N.GS_RECORD_F16: 4e-3, N.GS_RECORD_BF16: 6e-3}


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
    _, _, img = oracle_mod.render(scene, cam)
    st = compare_image(out["rgb"].cpu().numpy(), out["final_T"].cpu().numpy(), img)
    st.pop("keep")
    diff32 = float((out["rgb"] - ref["rgb"]).abs().max())
    print(name, "f16" if dtype == 1 else "bf16", "vs FP64:", st, "vs FP32 records:", diff32)
    assert np.isfinite(out["rgb"].cpu().numpy()).all()
    assert st["max_rgb_err"] <= BOUND[dtype], st


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
