"""Helpers shared by the GPU parity tests: packing oracle records into the
gs_record layout, unpacking GPU records, and adjudicating the few places
where FP32 and FP64 may legitimately take different discrete decisions."""
from __future__ import annotations

import numpy as np

# Per-channel colour tolerance for the FP32 image against the FP64 oracle.
RGB_TOL = 1e-3
# Transmittance tolerance (same scale as colour).
T_TOL = 1e-3


def f32(a):
    return np.asarray(a, dtype=np.float32)


def records_from_oracle(pr, oracle_mod, width, height, tile_w=16, tile_h=16):
    """FP32 gs_record words (n, 12) built from an oracle projection, plus the
    FP64 copies of exactly those FP32 values and the per-record tile counts of
    the oracle's binning of them. Culled records are zero with tiles = 0."""
    n = pr.n
    m = f32(pr.mean2d).astype(np.float64)
    c = f32(pr.conic).astype(np.float64)
    o = f32(pr.opacity).astype(np.float64)
    col = f32(pr.rgb).astype(np.float64)
    d = f32(pr.depth).astype(np.float64)
    rad = pr.radius.astype(np.int64)
    vis = pr.visible.astype(np.int32)
    b = oracle_mod.bin_tiles(m, rad, d, vis, width, height, tile_w, tile_h)
    tiles = np.bincount(b.values.astype(np.int64), minlength=n).astype(np.uint32)
    vis = (tiles > 0).astype(np.int32)
    rec = np.zeros((n, 12), np.float32)
    rec[:, 0:2] = m
    rec[:, 2:5] = c
    rec[:, 5] = o
    rec[:, 6:9] = col
    rec[:, 9] = d
    rec[:, 10] = rad.astype(np.int32).view(np.float32)
    rec[:, 11] = tiles.view(np.float32)
    rec[vis == 0] = 0
    return dict(rec=rec, tiles=tiles, mean2d=m, conic=c, opacity=o, rgb=col, depth=d, radius=rad,
                visible=vis, binned=b)


def unpack_records(rec: np.ndarray):
    rec = np.ascontiguousarray(rec, dtype=np.float32)
    return dict(mean2d=rec[:, 0:2].astype(np.float64), conic=rec[:, 2:5].astype(np.float64),
                opacity=rec[:, 5].astype(np.float64), rgb=rec[:, 6:9].astype(np.float64),
                depth=rec[:, 9].astype(np.float64), radius=rec[:, 10].view(np.int32).astype(np.int64),
                tiles=rec[:, 11].view(np.uint32))


def compare_image(gpu_rgb, gpu_T, ora_img, exclude_mask=None):
    """Max abs error on pixels that are neither flagged by the oracle (an alpha
    or T decision within 1e-6 of its cutoff) nor excluded. Returns a dict of
    statistics; the caller asserts."""
    flag = ora_img.flag.astype(bool)
    keep = ~flag
    if exclude_mask is not None:
        keep &= ~exclude_mask
    err = np.abs(gpu_rgb.astype(np.float64) - ora_img.rgb)
    terr = np.abs(gpu_T.astype(np.float64) - ora_img.T)
    return dict(
        max_rgb_err=float(err[keep].max()) if keep.any() else 0.0,
        max_T_err=float(terr[keep].max()) if keep.any() else 0.0,
        flagged=int(flag.sum()),
        flagged_max_err=float(err[flag].max()) if flag.any() else 0.0,
        excluded=int(exclude_mask.sum()) if exclude_mask is not None else 0,
        compared=int(keep.sum()),
        keep=keep,
    )


def tile_mask(tiles, width, height, tile_w, tile_h):
    """Pixel mask of a set of tile ids."""
    tiles_x = (width + tile_w - 1) // tile_w
    m = np.zeros((height, width), bool)
    for t in tiles:
        tx, ty = t % tiles_x, t // tiles_x
        m[ty * tile_h:(ty + 1) * tile_h, tx * tile_w:(tx + 1) * tile_w] = True
    return m


def rect_tiles(rect, tiles_x):
    x0, y0, x1, y1 = [int(v) for v in rect]
    return {ty * tiles_x + tx for ty in range(y0, y1) for tx in range(x0, x1)}


def near_integer(x, tol):
    return np.abs(x - np.round(x)) <= tol


def adjudicate_projection(gpu, ora, width, height, tile_w, tile_h, near_z=0.2):
    """Compare GPU records with the FP64 projection. Continuous fields must
    agree to FP32 accuracy; the discrete decisions (visibility, radius, tile
    rect) must agree except for Gaussians whose FP64 value sits at a decision
    boundary, where either side is a correct rounding. Returns (tie indices,
    statistics)."""
    g_vis = gpu["tiles"] > 0
    o_vis = ora.visible.astype(bool)
    both = g_vis & o_vis
    stats = {}
    # Continuous fields on Gaussians both sides keep.
    dm = np.abs(gpu["mean2d"][both] - ora.mean2d[both])
    stats["mean2d_max_abs"] = float(dm.max()) if dm.size else 0.0
    scale = np.sqrt(np.abs(ora.conic[both, 0] * ora.conic[both, 2]))[:, None]
    dq = np.abs(gpu["conic"][both] - ora.conic[both]) / np.maximum(scale, 1e-30)
    stats["conic_max_rel"] = float(dq.max()) if dq.size else 0.0
    stats["opacity_max_abs"] = float(np.abs(gpu["opacity"][both] - ora.opacity[both]).max()) if both.any() else 0.0
    stats["rgb_max_abs"] = float(np.abs(gpu["rgb"][both] - ora.rgb[both]).max()) if both.any() else 0.0
    dd = np.abs(gpu["depth"][both] - ora.depth[both]) / ora.depth[both]
    stats["depth_max_rel"] = float(dd.max()) if dd.size else 0.0
    # Discrete decisions.
    tiles_x = (width + tile_w - 1) // tile_w
    ext = ora.extent
    r_tie = near_integer(ext, 2e-4 * np.maximum(1.0, ext))
    u, v = ora.mean2d[:, 0], ora.mean2d[:, 1]
    u_tie = near_integer(u, 2e-3 + 1e-6 * np.abs(u)) | near_integer(v, 2e-3 + 1e-6 * np.abs(v))
    z_tie = np.abs(ora.depth - near_z) <= 1e-5
    vis_diff = g_vis != o_vis
    rad_diff = both & (gpu["radius"] != ora.radius)
    tiles_diff = both & (gpu["tiles"].astype(np.int64) != (ora.rect[:, 2] - ora.rect[:, 0]) * (ora.rect[:, 3] - ora.rect[:, 1]))
    bad = (vis_diff | rad_diff | tiles_diff) & ~(r_tie | u_tie | z_tie)
    stats["unexplained"] = int(bad.sum())
    ties = np.nonzero(vis_diff | rad_diff | tiles_diff)[0]
    stats["ties"] = int(len(ties))
    return ties, stats, tiles_x


def adjudicate_lists(gvals, granges, ora_bin, ties, depth_ref, n_tiles):
    """Tiles whose GPU list differs from the oracle's. A difference is valid
    when (a) the symmetric difference of the two lists contains only tie
    Gaussians and (b) the GPU order of the common Gaussians is a depth order
    up to FP32 rounding. Returns (ambiguous tile ids, number of invalid tiles)."""
    tie_set = set(int(t) for t in ties)
    amb, invalid = [], 0
    ov, orng = ora_bin.values, ora_bin.ranges
    for t in range(n_tiles):
        g = gvals[granges[t, 0]:granges[t, 1]]
        o = ov[orng[t, 0]:orng[t, 1]]
        if len(g) == len(o) and np.array_equal(g, o):
            continue
        sg, so = set(g.tolist()), set(o.tolist())
        if (sg ^ so) - tie_set:
            invalid += 1
            continue
        common = [x for x in g.tolist() if x in so]
        d = depth_ref[np.asarray(common, dtype=np.int64)] if common else np.zeros(0)
        tol = 8 * np.spacing(d.astype(np.float32)).astype(np.float64)
        if d.size > 1 and np.any(d[1:] < d[:-1] - tol[1:]):
            invalid += 1
            continue
        amb.append(t)
    return amb, invalid


def depth_tie_mask(pr, bn, width, height, tile_w=16, tile_h=16, ulps=3):
    """Pixels where two Gaussians of the pixel's tile list have depths closer
    than FP32 can order them and both reach alpha >= 1/255 (FP64 values).
    The GPU computes camera-space depth in FP32 to within 1.3 ulps (measured
    on the 1M-Gaussian scenes), so two Gaussians whose FP64 depths differ by
    less than ulps FP32 ulps may come out in either order, or tie and fall
    back to index order. Both orders are correct at FP32 precision; they give
    the same transmittance but different colours where both Gaussians
    contribute. Returns (mask, number of such pairs)."""
    vals = bn.values.astype(np.int64)
    mask = np.zeros((height, width), bool)
    if vals.size < 2:
        return mask, 0
    lengths = (bn.ranges[:, 1] - bn.ranges[:, 0]).astype(np.int64)
    tile_of = np.repeat(np.arange(len(lengths)), lengths)
    d = pr.depth[vals]
    tol = ulps * np.spacing(np.abs(d[:-1]).astype(np.float32)).astype(np.float64)
    tie = np.nonzero((np.diff(d) <= tol) & (tile_of[1:] == tile_of[:-1]))[0]
    tiles_x = (width + tile_w - 1) // tile_w
    for k in tie:
        t = int(tile_of[k])
        x0, y0 = (t % tiles_x) * tile_w, (t // tiles_x) * tile_h
        xs = np.arange(x0, min(x0 + tile_w, width)) + 0.5
        ys = np.arange(y0, min(y0 + tile_h, height)) + 0.5
        X, Y = np.meshgrid(xs, ys)
        both = np.ones(X.shape, bool)
        for gi in (vals[k], vals[k + 1]):
            dx, dy = X - pr.mean2d[gi, 0], Y - pr.mean2d[gi, 1]
            q = pr.conic[gi]
            power = -0.5 * (q[0] * dx * dx + q[2] * dy * dy) - q[1] * dx * dy
            both &= np.minimum(0.99, pr.opacity[gi] * np.exp(power)) >= 1.0 / 255.0
        mask[y0:y0 + X.shape[0], x0:x0 + X.shape[1]] |= both
    return mask, int(tie.size)


def compare_render(gpu_rgb, gpu_T, pr, bn, img, width, height, tile_w=16, tile_h=16):
    """compare_image with the depth-tie pixels excluded (and counted)."""
    mask, n_tie = depth_tie_mask(pr, bn, width, height, tile_w, tile_h)
    st = compare_image(gpu_rgb, gpu_T, img, exclude_mask=mask)
    st["depth_tie_pairs"] = n_tie
    return st
