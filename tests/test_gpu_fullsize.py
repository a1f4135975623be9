"""The full-size paths that only long key lists reach, in the launch
configuration the benchmark times:

* the reduce-then-scan sort passes used from 8M pairs on (per-partition
  digit counts, a scan per digit, a scatter with known offsets), against
  numpy's stable argsort at 9M and 33M pairs with 16-, 32- and 64-bit keys;
* the 64-view trajectory batch (1M Gaussians, views alternating 1280x720 and
  640x480, FP16 records, 16x16 tiles, staging depth 128): a joint batch of
  about 25M keys whose global tile sort runs three reduce-then-scan passes
  over 32-bit tile ids; every view equals its single-view render
  bit for bit, and one view of each size is within the FP16 bound of the
  FP64 oracle;
* the automatic switch of gs_render_batch to view-by-view rendering after a
  batch averaging more than 8M keys per view (an imbalance scene at 4K): the
  switched batch equals the joint batch and the single-view renders bit for
  bit, and its first view is within the BF16 bound of the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15951_gb300 as gs  # noqa: E402
from paper_2607_15951_gb300 import _native as N  # noqa: E402
from paper_2607_15951_gb300 import scenes  # noqa: E402

from parity_util import compare_render  # noqa: E402

# Stated bound for 16-bit records (max abs per channel on non-cutoff pixels).
LOW_PRECISION_BOUND = 4e-3


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15951_gb300 import build
    build.build()
    c = gs.Context(0)
    yield c
    c.close()


def _sort_case(rng, n, bits):
    hi = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    keys = rng.integers(0, 2 ** 63 - 1, n, dtype=np.int64).view(np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, n, dtype=np.int64).view(np.uint64)
    keys &= hi
    # A quarter of the keys repeat a few values, so the order of equal keys
    # (stability) is exercised across partitions.
    keys[: n // 4] &= np.uint64(0xFF)
    return keys


@pytest.mark.parametrize("n", [9_000_001, 33_554_467], ids=["9M", "33M"])
@pytest.mark.parametrize("bits", [16, 32, 64])
def test_long_list_sort_matches_stable_sort(ctx, n, bits):
    rng = np.random.default_rng(n + bits)
    keys = _sort_case(rng, n, bits)
    vals = np.arange(n, dtype=np.uint32)
    k = torch.from_numpy(keys.view(np.int64)).cuda()
    v = torch.from_numpy(vals.view(np.int32)).cuda()
    gs.gs_sort_pairs(ctx, k, v, n, bits)
    torch.cuda.synchronize()
    gs.gs_sync_status(ctx)
    order = np.argsort(keys, kind="stable")
    # Integer results: exact equality (the values are the input positions, so
    # equal keys must keep their input order).
    assert np.array_equal(v.cpu().numpy().view(np.uint32), order.astype(np.uint32))
    assert np.array_equal(k.cpu().numpy().view(np.uint64), keys[order])
    del k, v
    torch.cuda.empty_cache()


def _oracle_view(oracle_mod, scene, cam, rgb, T):
    pr, bn, img = oracle_mod.render(scene, cam)
    st = compare_render(rgb.cpu().numpy(), T.cpu().numpy(), pr, bn, img, cam.width, cam.height)
    st.pop("keep")
    return st


def test_trajectory_64_views_fp16_as_benchmarked(ctx, oracle_mod):
    scene, cams = scenes.workload("clustered_1m_traj64")
    g = gs.scene_to_device(scene)
    outs = gs.alloc_outputs(cams, aux=True)
    gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs, tile=(16, 16), record_dtype=N.GS_RECORD_F16,
                       batch_depth=128)
    torch.cuda.synchronize()
    st = gs.gs_last_render_stats(ctx)
    print("64-view batch: keys", st["n_keys"], "records", st["n_visible"])
    assert st["n_keys"] > (8 << 20)  # the long-list sort shape
    for v, c in enumerate(cams):
        ref = gs.render(ctx, g, scene.sh_degree, c, record_dtype=N.GS_RECORD_F16)
        torch.cuda.synchronize()
        for k in ("rgb", "final_T", "n_contrib", "n_eval"):
            assert torch.equal(outs[v][k], ref[k]), (v, k)
    for v in (0, 1):  # 1280x720 and 640x480
        cmp = _oracle_view(oracle_mod, scene, cams[v], outs[v]["rgb"], outs[v]["final_T"])
        print("view", v, cams[v].width, "x", cams[v].height, "FP16 vs FP64:", cmp)
        assert cmp["max_rgb_err"] <= LOW_PRECISION_BOUND, cmp


def test_batch_switches_to_per_view_on_long_lists(ctx, oracle_mod):
    scene = scenes.imbalance(1_000_000, seed=4)
    cams = scenes.random_poses(2, 1004)  # 3840x2160, the first at the identity pose
    g = gs.scene_to_device(scene)
    outs = [gs.alloc_outputs(cams, aux=True) for _ in range(2)]
    dt = N.GS_RECORD_BF16
    # The first batch runs jointly and measures its keys per view ...
    f0 = gs.gs_last_frame_id(ctx)
    gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs[0], record_dtype=dt)
    torch.cuda.synchronize()
    keys = gs.gs_last_render_stats(ctx)["n_keys"]
    assert gs.gs_last_frame_id(ctx) == f0  # the joint schedule renders no single frame
    assert keys / len(cams) > (8 << 20), keys
    # ... then the automatic schedule renders view by view (one gs_render frame each).
    gs.gs_render_batch(ctx, g, scene.sh_degree, cams, outs[1], record_dtype=dt)
    torch.cuda.synchronize()
    assert gs.gs_last_frame_id(ctx) == f0 + len(cams)
    assert gs.gs_last_render_stats(ctx)["n_keys"] == keys
    for v, c in enumerate(cams):
        ref = gs.render(ctx, g, scene.sh_degree, c, record_dtype=dt)
        torch.cuda.synchronize()
        for k in ("rgb", "final_T", "n_contrib", "n_eval"):
            assert torch.equal(outs[0][v][k], ref[k]), ("joint", v, k)
            assert torch.equal(outs[1][v][k], ref[k]), ("per view", v, k)
    cmp = _oracle_view(oracle_mod, scene, cams[0], outs[1][0]["rgb"], outs[1][0]["final_T"])
    print("imbalance 1M 4K view 0, BF16 vs FP64:", cmp, "keys per view", keys / len(cams))
    assert cmp["max_rgb_err"] <= LOW_PRECISION_BOUND, cmp
