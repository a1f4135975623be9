"""GPU parity: every stage of libgs against the FP64 oracle, through the C ABI.

* projection: continuous fields to FP32 accuracy, discrete decisions exact
  except at FP64 decision boundaries (adjudicated, counted);
* binning: bit-exact keys, values and ranges for identical FP32 records;
* sort: bit-exact against a stable library sort;
* blending: max abs error <= 1e-3 per channel, pixels whose alpha or T
  decision lies within 1e-6 of its cutoff counted separately;
* end to end (scene -> image) on the 10k-Gaussian 256x256 scene and the
  1M-Gaussian 1080p clustered scene at full size.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2607_15951_gb300 as gs  # noqa: E402
from paper_2607_15951_gb300 import scenes  # noqa: E402

from parity_util import (RGB_TOL, T_TOL, adjudicate_lists, adjudicate_projection,  # noqa: E402
                         compare_image, records_from_oracle, tile_mask, unpack_records)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15951_gb300 import build
    build.build()
    c = gs.Context(0)
    yield c
    c.close()


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def gpu_project(ctx, scene, cam, tile=(16, 16)):
    g = gs.scene_to_device(scene)
    n = scene.n
    rec = torch.zeros((max(n, 1), 12), dtype=torch.float32, device="cuda")
    tiles = torch.full((max(n, 1),), 0x7fffffff, dtype=torch.int32, device="cuda")
    gs.gs_project(ctx, g, scene.sh_degree, cam, rec, tiles, tile=tile)
    torch.cuda.synchronize()
    r = rec[:n].cpu().numpy()
    t = tiles[:n].cpu().numpy().view(np.uint32)
    out = unpack_records(r)
    out["tiles"] = t
    out["rec"] = r
    return out


def gpu_bin(ctx, rec, tiles, n, cam, tile=(16, 16), capacity=None):
    rec_d = dev(rec if n else np.zeros((1, 12), np.float32))
    tiles_d = dev(tiles.view(np.int32) if n else np.zeros(1, np.int32))
    tw, th = tile
    n_tiles = ((cam.width + tw - 1) // tw) * ((cam.height + th - 1) // th)
    ranges = torch.full((n_tiles, 2), -1, dtype=torch.int32, device="cuda")
    if capacity is None:
        capacity = int(tiles.astype(np.int64).sum()) if n else 0
    keys = torch.empty(max(capacity, 1), dtype=torch.int64, device="cuda")
    vals = torch.empty(max(capacity, 1), dtype=torch.int32, device="cuda")
    K = gs.gs_bin(ctx, rec_d, tiles_d, n, cam, keys if capacity else None,
                  vals if capacity else None, ranges, tile=tile)
    torch.cuda.synchronize()
    gs.gs_sync_status(ctx)
    return (K, keys[:K].cpu().numpy().view(np.uint64), vals[:K].cpu().numpy().view(np.uint32),
            ranges.cpu().numpy().view(np.uint32), rec_d, vals, ranges)


def gpu_blend(ctx, rec_d, vals_d, ranges_d, cam, tile=(16, 16), bg=(0.0, 0.0, 0.0)):
    H, W = cam.height, cam.width
    rgb = torch.full((H, W, 3), float("nan"), dtype=torch.float32, device="cuda")
    T = torch.full((H, W), float("nan"), dtype=torch.float32, device="cuda")
    nc = torch.full((H, W), -1, dtype=torch.int32, device="cuda")
    ne = torch.full((H, W), -1, dtype=torch.int32, device="cuda")
    gs.gs_blend(ctx, rec_d, vals_d, ranges_d, cam, rgb, T, nc, ne, tile=tile, bg=bg)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), T.cpu().numpy(), nc.cpu().numpy(), ne.cpu().numpy()


# ---------------------------------------------------------------------------
# Projection
# ---------------------------------------------------------------------------

PROJ_CASES = [
    ("uniform_box_256", lambda: (scenes.uniform_box(10_000, 0), scenes.pinhole(256, 256))),
    ("clustered_200k_1080p_sh3", lambda: (scenes.clustered(200_000, 7), scenes.pinhole(1920, 1080))),
    ("clustered_50k_traj_view", lambda: (scenes.clustered(50_000, 8), scenes.trajectory(4, 1008)[1])),
]


@pytest.mark.parametrize("name,make", PROJ_CASES, ids=[c[0] for c in PROJ_CASES])
def test_projection_parity(ctx, oracle_mod, name, make):
    scene, cam = make()
    gpu = gpu_project(ctx, scene, cam)
    ora = oracle_mod.project(scene, cam)
    ties, st, _ = adjudicate_projection(gpu, ora, cam.width, cam.height, 16, 16, cam.near_z)
    print(name, st)
    assert st["unexplained"] == 0, st
    assert st["ties"] <= max(3, 1e-4 * scene.n), st
    assert st["mean2d_max_abs"] < 2e-3, st
    assert st["conic_max_rel"] < 2e-4, st
    assert st["opacity_max_abs"] < 1e-6, st
    assert st["rgb_max_abs"] < 2e-6, st
    assert st["depth_max_rel"] < 2e-6, st


def test_projection_culls_behind_and_degenerate(ctx, oracle_mod):
    s = scenes.uniform_box(64, 3)
    s.means[:16, 2] = -1.0          # behind the camera
    s.means[16:20, 2] = 0.2         # exactly on the near plane
    s.quats[20:24] = 0.0            # degenerate rotation -> NaN -> culled
    s.means[24:28, 0] = 1e6         # far off screen
    cam = scenes.pinhole(64, 48)
    gpu = gpu_project(ctx, s, cam)
    ora = oracle_mod.project(s, cam)
    assert (gpu["tiles"][:28] == 0).all()
    assert ((gpu["tiles"] > 0) == ora.visible.astype(bool)).all()


# ---------------------------------------------------------------------------
# Binning and sort
# ---------------------------------------------------------------------------

BIN_CASES = [
    ("uniform_box_256_t16", lambda: (scenes.uniform_box(10_000, 0), scenes.pinhole(256, 256)), (16, 16)),
    ("ragged_257x131_t16x8", lambda: (scenes.uniform_box(3_000, 5), scenes.pinhole(257, 131)), (16, 8)),
    ("ragged_257x131_t8", lambda: (scenes.uniform_box(3_000, 6), scenes.pinhole(257, 131)), (8, 8)),
    ("clustered_1m_1080p", lambda: (scenes.clustered(1_000_000, 1), scenes.pinhole(1920, 1080)), (16, 16)),
]


@pytest.mark.parametrize("name,make,tile", BIN_CASES, ids=[c[0] for c in BIN_CASES])
def test_binning_bit_exact(ctx, oracle_mod, name, make, tile):
    scene, cam = make()
    pr = oracle_mod.project(scene, cam, *tile)
    R = records_from_oracle(pr, oracle_mod, cam.width, cam.height, *tile)
    K, keys, vals, ranges, *_ = gpu_bin(ctx, R["rec"], R["tiles"], scene.n, cam, tile)
    b = R["binned"]
    assert K == len(b.keys)
    assert np.array_equal(keys, b.keys)
    assert np.array_equal(vals, b.values)
    assert np.array_equal(ranges, b.ranges)


def test_binning_equal_depths_break_by_index(ctx, oracle_mod):
    scene = scenes.uniform_box(2_000, 11)
    scene.means[:, 2] = 5.0  # every depth identical
    cam = scenes.pinhole(128, 96)
    pr = oracle_mod.project(scene, cam)
    R = records_from_oracle(pr, oracle_mod, cam.width, cam.height)
    K, keys, vals, ranges, *_ = gpu_bin(ctx, R["rec"], R["tiles"], scene.n, cam)
    assert np.array_equal(vals, R["binned"].values)
    for t in range(ranges.shape[0]):
        v = vals[ranges[t, 0]:ranges[t, 1]]
        assert (np.diff(v.astype(np.int64)) > 0).all()


def test_binning_empty_and_single(ctx, oracle_mod):
    cam = scenes.pinhole(100, 60)
    K, keys, vals, ranges, *_ = gpu_bin(ctx, np.zeros((0, 12), np.float32), np.zeros(0, np.uint32), 0, cam)
    assert K == 0 and (ranges == 0).all()
    s = scenes.uniform_box(1, 1)
    s.means[0] = [0.0, 0.0, 4.0]
    pr = oracle_mod.project(s, cam)
    R = records_from_oracle(pr, oracle_mod, cam.width, cam.height)
    K, keys, vals, ranges, *_ = gpu_bin(ctx, R["rec"], R["tiles"], 1, cam)
    assert K == len(R["binned"].keys) and np.array_equal(ranges, R["binned"].ranges)


def test_binning_whole_screen_splat(ctx, oracle_mod):
    # One Gaussian near the camera covering every tile (warp-cooperative emit),
    # plus small ones.
    s = scenes.uniform_box(500, 12)
    s.means[0] = [0.0, 0.0, 0.5]
    s.log_scales[0] = np.log(0.5)
    cam = scenes.pinhole(640, 360)
    pr = oracle_mod.project(s, cam)
    R = records_from_oracle(pr, oracle_mod, cam.width, cam.height)
    assert R["tiles"][0] == 40 * 23
    K, keys, vals, ranges, *_ = gpu_bin(ctx, R["rec"], R["tiles"], s.n, cam)
    assert np.array_equal(keys, R["binned"].keys) and np.array_equal(vals, R["binned"].values)


def test_binning_capacity_error(ctx, oracle_mod):
    s, cam = scenes.uniform_box(1_000, 13), scenes.pinhole(128, 128)
    pr = oracle_mod.project(s, cam)
    R = records_from_oracle(pr, oracle_mod, cam.width, cam.height)
    need = int(R["tiles"].astype(np.int64).sum())
    with pytest.raises(gs.GSError) as e:
        gpu_bin(ctx, R["rec"], R["tiles"], s.n, cam, capacity=need - 1)
    assert e.value.status == 4 and e.value.n_keys == need


@pytest.mark.parametrize("n,bits", [(2, 13), (4095, 45), (4096, 45), (4097, 45), (100_003, 32),
                                    (1_000_000, 45), (300_001, 64), (65_536, 8), (50_000, 1)])
def test_sort_pairs_matches_stable_sort(ctx, n, bits):
    rng = np.random.default_rng(n + bits)
    mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    keys = rng.integers(0, 2 ** 63, n, dtype=np.int64).view(np.uint64)
    keys ^= rng.integers(0, 2, n, dtype=np.int64).view(np.uint64) << np.uint64(63)
    keys &= mask
    keys[: n // 3] &= np.uint64(0xFF)  # many duplicates -> stability matters
    vals = np.arange(n, dtype=np.uint32)
    kd, vd = dev(keys.view(np.int64)), dev(vals.view(np.int32))
    gs.gs_sort_pairs(ctx, kd, vd, n, bits)
    torch.cuda.synchronize()
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(kd.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(vd.cpu().numpy().view(np.uint32), vals[order])
    gs.gs_sync_status(ctx)


def test_tile_ranges(ctx):
    rng = np.random.default_rng(3)
    n_tiles = 700
    tiles = np.sort(rng.integers(0, n_tiles, 50_000)).astype(np.uint64)
    keys = (tiles << np.uint64(32)) | rng.integers(0, 2 ** 32, 50_000).astype(np.uint64)
    ranges = torch.full((n_tiles, 2), -1, dtype=torch.int32, device="cuda")
    gs.gs_tile_ranges(ctx, dev(keys.view(np.int64)), len(keys), n_tiles, ranges)
    r = ranges.cpu().numpy().view(np.uint32)
    for t in range(n_tiles):
        idx = np.nonzero(tiles == t)[0]
        assert tuple(r[t]) == ((idx[0], idx[-1] + 1) if len(idx) else (0, 0))


# ---------------------------------------------------------------------------
# Blending on identical FP32 records
# ---------------------------------------------------------------------------

BLEND_CASES = BIN_CASES + [
    ("uniform_box_256_bg", lambda: (scenes.uniform_box(10_000, 0), scenes.pinhole(256, 256)), (16, 16)),
]


@pytest.mark.parametrize("name,make,tile", BLEND_CASES, ids=[c[0] for c in BLEND_CASES])
def test_blend_parity(ctx, oracle_mod, name, make, tile):
    scene, cam = make()
    bg = (0.1, 0.2, 0.3) if name.endswith("_bg") else (0.0, 0.0, 0.0)
    pr = oracle_mod.project(scene, cam, *tile)
    R = records_from_oracle(pr, oracle_mod, cam.width, cam.height, *tile)
    K, keys, vals, ranges, rec_d, vals_d, ranges_d = gpu_bin(ctx, R["rec"], R["tiles"], scene.n, cam, tile)
    rgb, T, nc, ne = gpu_blend(ctx, rec_d, vals_d, ranges_d, cam, tile, bg)
    b = R["binned"]
    img = oracle_mod.blend(R["mean2d"], R["conic"], R["opacity"], R["rgb"], b.values, b.ranges,
                           cam.width, cam.height, *tile, bg=bg)
    st = compare_image(rgb, T, img)
    keep = st.pop("keep")
    print(name, st)
    assert np.isfinite(rgb).all() and np.isfinite(T).all()
    assert st["max_rgb_err"] <= RGB_TOL, st
    assert st["max_T_err"] <= T_TOL, st
    assert st["flagged"] <= 0.05 * cam.width * cam.height
    assert (nc[keep] == img.last[keep]).mean() > 0.999
    assert (ne[keep] == img.neval[keep]).mean() > 0.999


@pytest.mark.parametrize("case", ["three_cocentred", "transmittance_stop", "faint_front_skipped",
                                  "opaque_front_clamped", "off_centre_falloff", "anisotropic_cross_term",
                                  "depth_order_not_index_order"])
def test_blend_hand_examples_on_gpu(ctx, case):
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")))
    c = next(x for x in g["blend_cases"] if x["name"] == case)
    W, H = g["image"]["width"], g["image"]["height"]
    n = len(c["records"])
    rec = np.zeros((n, 12), np.float32)
    tiles = np.zeros(n, np.uint32)
    for i, r in enumerate(c["records"]):
        rec[i, 0:2], rec[i, 2:5], rec[i, 5] = r["mean2d"], r["conic"], r["opacity"]
        rec[i, 6:9], rec[i, 9] = r["rgb"], r["depth"]
        rec[i, 10] = np.array([r["radius"]], np.int32).view(np.float32)[0]
        x0 = max(0, int(np.floor((np.floor(r["mean2d"][0]) - r["radius"]) / 16)))
        x1 = min(W // 16, int(np.floor((np.floor(r["mean2d"][0]) + r["radius"] + 15) / 16)))
        y0 = max(0, int(np.floor((np.floor(r["mean2d"][1]) - r["radius"]) / 16)))
        y1 = min(H // 16, int(np.floor((np.floor(r["mean2d"][1]) + r["radius"] + 15) / 16)))
        tiles[i] = (x1 - x0) * (y1 - y0)
        rec[i, 11] = np.array([tiles[i]], np.uint32).view(np.float32)[0]
    cam = scenes.pinhole(W, H)
    K, keys, vals, ranges, rec_d, vals_d, ranges_d = gpu_bin(ctx, rec, tiles, n, cam)
    rgb, T, nc, ne = gpu_blend(ctx, rec_d, vals_d, ranges_d, cam)
    x, y = c["pixel"]
    np.testing.assert_allclose(rgb[y, x], c["rgb"], atol=1e-6)
    assert abs(T[y, x] - c["T"]) < 1e-6
    assert nc[y, x] == c["last"] and ne[y, x] == c["neval"]


# ---------------------------------------------------------------------------
# End to end: scene -> image
# ---------------------------------------------------------------------------

E2E_CASES = [
    ("uniform_box_256", lambda: scenes.workload("uniform_box_256"), (16, 16)),
    ("uniform_box_256_t8", lambda: scenes.workload("uniform_box_256"), (8, 8)),
    ("clustered_1m_1080p", lambda: scenes.workload("clustered_1m_1080p"), (16, 16)),
]


@pytest.mark.parametrize("name,make,tile", E2E_CASES, ids=[c[0] for c in E2E_CASES])
def test_render_end_to_end(ctx, oracle_mod, name, make, tile):
    scene, cams = make()
    cam = cams[0]
    g = gs.scene_to_device(scene)
    out = gs.render(ctx, g, scene.sh_degree, cam, tile=tile)
    torch.cuda.synchronize()
    gs.gs_sync_status(ctx)
    stats = gs.gs_last_render_stats(ctx)
    rgb, T = out["rgb"].cpu().numpy(), out["final_T"].cpu().numpy()
    pr, b, img = oracle_mod.render(scene, cam, *tile)
    # GPU intermediate state for adjudication, through the stage entry points.
    gpu = gpu_project(ctx, scene, cam, tile)
    ties, pst, tiles_x = adjudicate_projection(gpu, pr, cam.width, cam.height, *tile, cam.near_z)
    assert pst["unexplained"] == 0, pst
    K, keys, vals, ranges, *_ = gpu_bin(ctx, gpu["rec"], gpu["tiles"], scene.n, cam, tile)
    assert K == stats["n_keys"]
    n_tiles = ranges.shape[0]
    amb, invalid = adjudicate_lists(vals, ranges, b, ties, pr.depth, n_tiles)
    assert invalid == 0
    excl = tile_mask(amb, cam.width, cam.height, *tile)
    st = compare_image(rgb, T, img, excl)
    st.pop("keep")
    print(name, pst, "ambiguous tiles", len(amb), st)
    assert len(amb) <= max(2, 0.01 * n_tiles)
    assert st["max_rgb_err"] <= RGB_TOL, st
    assert st["max_T_err"] <= T_TOL, st


def test_render_empty_scene(ctx):
    s = scenes.uniform_box(10, 1)
    s.means[:, 2] = -5.0
    cam = scenes.pinhole(33, 17)
    out = gs.render(ctx, gs.scene_to_device(s), 0, cam, bg=(0.25, 0.5, 0.75))
    torch.cuda.synchronize()
    assert np.allclose(out["rgb"].cpu().numpy(), [0.25, 0.5, 0.75])
    assert (out["final_T"].cpu().numpy() == 1).all()
    assert (out["n_contrib"].cpu().numpy() == 0).all()


def test_render_one_pixel_image(ctx, oracle_mod):
    s = scenes.uniform_box(200, 2)
    cam = scenes.pinhole(1, 1, 60.0)
    out = gs.render(ctx, gs.scene_to_device(s), 0, cam)
    torch.cuda.synchronize()
    _, _, img = oracle_mod.render(s, cam)
    assert np.abs(out["rgb"].cpu().numpy() - img.rgb).max() <= RGB_TOL or img.flag.any()


def test_invalid_arguments_rejected(ctx):
    s = scenes.uniform_box(10, 1)
    g = gs.scene_to_device(s)
    cam = scenes.pinhole(64, 64)
    rgb = torch.empty((64, 64, 3), device="cuda")
    with pytest.raises(gs.GSError) as e:
        gs.gs_render(ctx, g, 5, cam, rgb)            # sh_degree out of range
    assert e.value.status == 1
    with pytest.raises(gs.GSError) as e:
        gs.gs_render(ctx, g, 0, cam, rgb, tile=(32, 32))
    assert e.value.status == 1
    bad = scenes.pinhole(64, 64)
    bad.near_z = 0.0
    with pytest.raises(gs.GSError):
        gs.gs_render(ctx, g, 0, bad, rgb)


# ---------------------------------------------------------------------------
# Blend schedules: the culled schedule must equal the basic one bit for bit
# ---------------------------------------------------------------------------

def _needles(n=4000, seed=21):
    s = scenes.uniform_box(n, seed)
    s.log_scales[:, 0] += 3.5     # ~33x longer along one local axis
    s.log_scales[:, 1:] -= 1.5
    s.opacity_logits[:] = np.abs(s.opacity_logits) + 1.0
    return s


VARIANT_CASES = [
    ("uniform_box_256_t16", lambda: (scenes.uniform_box(10_000, 0), scenes.pinhole(256, 256)), (16, 16)),
    ("uniform_box_257x131_t16x8", lambda: (scenes.uniform_box(5_000, 3), scenes.pinhole(257, 131)), (16, 8)),
    ("uniform_box_257x131_t8", lambda: (scenes.uniform_box(5_000, 4), scenes.pinhole(257, 131)), (8, 8)),
    ("needles_320x200", lambda: (_needles(), scenes.pinhole(320, 200)), (16, 16)),
    ("clustered_1m_1080p", lambda: scenes.workload("clustered_1m_1080p")[0:1] + (scenes.pinhole(1920, 1080),), (16, 16)),
]


@pytest.mark.parametrize("name,make,tile", VARIANT_CASES, ids=[c[0] for c in VARIANT_CASES])
def test_blend_variants_identical(ctx, name, make, tile):
    scene, cam = make()
    g = gs.scene_to_device(scene)
    outs = []
    N_ = gs._native
    for variant in (N_.GS_BLEND_BASIC, N_.GS_BLEND_CULLED, N_.GS_BLEND_CULLED_WIDE, N_.GS_BLEND_CULLED_TILE,
                    N_.GS_BLEND_CULLED_8X8, N_.GS_BLEND_TMA):
        out = gs.render(ctx, g, scene.sh_degree, cam, tile=tile, variant=variant)
        torch.cuda.synchronize()
        outs.append({k: v.cpu().numpy() for k, v in out.items()})
    gs.gs_sync_status(ctx)
    for o in outs[1:]:
        for k in ("rgb", "final_T", "n_contrib", "n_eval"):
            assert np.array_equal(outs[0][k], o[k]), k


@pytest.mark.parametrize("name,make,tile", VARIANT_CASES, ids=[c[0] for c in VARIANT_CASES])
def test_tile_order_does_not_change_the_image(ctx, name, make, tile):
    """The blend blocks take the tiles longest list first (default) or in
    grid order: every output is the same bit for bit, for each culled
    schedule and, on 16x16 tiles, each list-tile form."""
    scene, cam = make()
    g = gs.scene_to_device(scene)
    N_ = gs._native
    forms = [dict(variant=v) for v in (N_.GS_BLEND_CULLED, N_.GS_BLEND_CULLED_WIDE, N_.GS_BLEND_CULLED_TILE,
                                       N_.GS_BLEND_CULLED_8X8)]
    if tile == (16, 16):
        forms += [dict(list_tiles=c) for c in (N_.GS_LISTS_2X1, N_.GS_LISTS_2X2, N_.GS_LISTS_4X4, N_.GS_LISTS_8X8)]
    for f in forms:
        a = gs.render(ctx, g, scene.sh_degree, cam, tile=tile, tile_order=N_.GS_ORDER_LONGEST_FIRST, **f)
        b = gs.render(ctx, g, scene.sh_degree, cam, tile=tile, tile_order=N_.GS_ORDER_GRID, **f)
        torch.cuda.synchronize()
        for k in ("rgb", "final_T", "n_contrib", "n_eval"):
            assert torch.equal(a[k], b[k]), (f, k)
    with pytest.raises(RuntimeError, match="tile_order"):
        gs.render(ctx, g, scene.sh_degree, cam, tile=tile, tile_order=2)


def test_render_regrows_key_buffers(oracle_mod):
    """A context whose key buffers are far too small still returns the exact
    frame: the overflow is detected and the frame rendered again."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    scene, cams = scenes.workload("uniform_box_256")
    g = gs.scene_to_device(scene)
    c = gs.Context(0)
    gs.gs_reserve_keys(c, 1000)
    out = gs.render(c, g, scene.sh_degree, cams[0])
    torch.cuda.synchronize()
    st = gs.gs_last_render_stats(c)
    assert st["n_keys"] > 1000
    ref = gs.Context(0)
    out2 = gs.render(ref, g, scene.sh_degree, cams[0])
    torch.cuda.synchronize()
    for k in out:
        assert torch.equal(out[k], out2[k]), k
    c.close()
    ref.close()


def test_render_equal_depths_follow_index_order(ctx, oracle_mod):
    """Many Gaussians at exactly the same depth overlap: the rendered order
    within each tile must be Gaussian-index order, as the oracle's."""
    s = scenes.uniform_box(3_000, 17)
    s.means[:, 2] = 4.0
    s.opacity_logits[:] = 1.5
    cam = scenes.pinhole(160, 120)
    out = gs.render(ctx, gs.scene_to_device(s), 0, cam)
    torch.cuda.synchronize()
    _, _, img = oracle_mod.render(s, cam)
    st = compare_image(out["rgb"].cpu().numpy(), out["final_T"].cpu().numpy(), img)
    st.pop("keep")
    assert st["max_rgb_err"] <= RGB_TOL, st
    assert np.array_equal(out["n_contrib"].cpu().numpy()[~img.flag.astype(bool)],
                          img.last[~img.flag.astype(bool)])


@pytest.mark.parametrize("n", [20_000, 90_000])
def test_render_depth_ties_short_and_long_lists(ctx, oracle_mod, n):
    """Depths drawn from eight values, so most Gaussians tie with thousands of
    others, in lists of 18k and 82k visible Gaussians (9 and 41 depth-sort
    partitions): every tile's list must be in (depth, index) order, as the
    oracle's."""
    s = scenes.uniform_box(n, 29)
    rng = np.random.default_rng(29)
    s.means[:, 2] = rng.choice(np.arange(3.0, 7.0, 0.5, dtype=np.float32), n)
    s.log_scales[:] = s.log_scales - 1.0
    cam = scenes.pinhole(320, 240)
    out = gs.render(ctx, gs.scene_to_device(s), 0, cam)
    torch.cuda.synchronize()
    _, _, img = oracle_mod.render(s, cam)
    st = compare_image(out["rgb"].cpu().numpy(), out["final_T"].cpu().numpy(), img)
    st.pop("keep")
    assert st["max_rgb_err"] <= RGB_TOL, st
    keep = ~img.flag.astype(bool)
    assert np.array_equal(out["n_contrib"].cpu().numpy()[keep], img.last[keep])


@pytest.mark.parametrize("shape", ["wide", "tall"])
def test_render_extreme_aspect_grids(ctx, oracle_mod, shape):
    """Grids wider than 256 tiles use tile-id keys with histograms counted
    by the emission; grids taller than 256 tiles use (row << 8 | column) keys
    of 17 bits (32-bit keys, a third tile pass over the row's high byte).
    Both must match the oracle."""
    s = scenes.uniform_box(40_000, 31)
    if shape == "wide":
        cam = scenes.pinhole(4200, 48, 90.0)        # 263 x 3 tiles
        s.means[:, 1] *= 0.01
    else:
        cam = scenes.pinhole(48, 4200, 1.0)         # 3 x 263 tiles
        s.means[:, 0] *= 0.004
    s.log_scales[:] = s.log_scales - 1.0
    out = gs.render(ctx, gs.scene_to_device(s), 0, cam)
    torch.cuda.synchronize()
    assert gs.gs_last_render_stats(ctx)["n_visible"] > 500
    _, _, img = oracle_mod.render(s, cam)
    st = compare_image(out["rgb"].cpu().numpy(), out["final_T"].cpu().numpy(), img)
    st.pop("keep")
    assert st["max_rgb_err"] <= RGB_TOL, st
    keep = ~img.flag.astype(bool)
    assert np.array_equal(out["n_contrib"].cpu().numpy()[keep], img.last[keep])


@pytest.mark.parametrize("case", ["clustered_rotated", "large_anisotropic", "skewed_camera"])
def test_frame_visible_set_equals_full_projection(ctx, case):
    """A frame skips the full projection of Gaussians that a screen bound
    built from the mean and the largest scale rules out. That bound must be
    conservative: the frame's visible Gaussians and key count equal those of
    projecting every Gaussian in full (gs_project), on scenes that stress it
    (rotated cameras, large anisotropic splats around the borders, a camera
    matrix with scaled rows)."""
    rng = np.random.default_rng(71)
    if case == "clustered_rotated":
        s = scenes.clustered(200_000, 71)
        cams = [scenes.pinhole(1280, 720, 70.0, world_to_cam=scenes.look_at(rng.uniform(-3, 3, 3),
                                                                              rng.normal(size=3)))
                for _ in range(3)]
    elif case == "large_anisotropic":
        s = scenes.uniform_box(50_000, 72)
        s.means[:, 0:2] *= 2.5
        s.log_scales[:] = rng.normal(-1.5, 1.0, s.log_scales.shape).astype(np.float32)
        s.log_scales[:, 0] += 1.5
        cams = [scenes.pinhole(640, 480, 60.0), scenes.pinhole(300, 900, 40.0)]
    else:
        s = scenes.uniform_box(50_000, 73)
        w2c = scenes.look_at([0.3, -0.2, -1.0], [0.1, 0.05, 1.0])
        w2c[0, :3] *= 1.7
        w2c[1, :3] *= 0.6
        cams = [scenes.pinhole(512, 384, 60.0, world_to_cam=w2c)]
    g = gs.scene_to_device(s)
    for cam in cams:
        rec = torch.zeros((s.n, 12), dtype=torch.float32, device="cuda")
        tiles = torch.zeros(s.n, dtype=torch.int32, device="cuda")
        gs.gs_project(ctx, g, s.sh_degree, cam, rec, tiles)
        gs.render(ctx, g, s.sh_degree, cam, aux=False)
        torch.cuda.synchronize()
        st = gs.gs_last_render_stats(ctx)
        t = tiles.to(torch.int64)
        assert st["n_visible"] == int((t > 0).sum())
        assert st["n_keys"] == int(t.sum())


def test_render_is_deterministic(ctx):
    scene, cams = scenes.workload("clustered_1m_1080p")
    g = gs.scene_to_device(scene)
    a = gs.render(ctx, g, scene.sh_degree, cams[0])
    b = gs.render(ctx, g, scene.sh_degree, cams[0])
    torch.cuda.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k]), k
