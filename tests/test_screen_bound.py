"""The projection skips the full covariance of Gaussians that a screen bound
built from the mean and the largest scale rules out (its derivation: the
rows of T = J W are (fx/tz)(W0 - rx W2) and (fy/tz)(W1 - ry W2), so
|A0|^2 + |A1|^2 <= s_max^2 (|T0|^2 + |T1|^2), and lambda_max as computed is
at most the trace + sqrt(0.1)). Here that bound, written out in FP64 with
the kernel's slack, must keep every Gaussian the FP64 oracle finds visible,
on random anisotropic scenes and cameras with rotated, skewed and scaled
rows; the GPU test checks the kernel against the full projection."""
import math

import numpy as np
import pytest

from paper_2607_15951_gb300 import scenes


def screen_bound_keeps(scene, cam, tile=16):
    w2c = np.asarray(cam.world_to_cam, np.float64).reshape(3, 4)
    R, t = w2c[:, :3], w2c[:, 3]
    m = scene.means.astype(np.float64)
    tc = m @ R.T + t
    tx, ty, tz = tc[:, 0], tc[:, 1], tc[:, 2]
    front = tz > cam.near_z
    tzs = np.where(front, tz, 1.0)
    lim_x = 1.3 * (0.5 * cam.width / cam.fx)
    lim_y = 1.3 * (0.5 * cam.height / cam.fy)
    rx = np.clip(tx / tzs, -lim_x, lim_x)
    ry = np.clip(ty / tzs, -lim_y, lim_y)
    n = np.linalg.norm(R, axis=1)
    t0 = cam.fx / tzs * (np.abs(rx) * n[2] + n[0])
    t1 = cam.fy / tzs * (np.abs(ry) * n[2] + n[1])
    B = np.exp(2.0 * scene.log_scales.astype(np.float64).max(axis=1)) * (t0 ** 2 + t1 ** 2)
    rb = 3.0 * np.sqrt(1.01 * B + 0.92) + 2.0
    u = cam.fx * tx / tzs + cam.cx
    v = cam.fy * ty / tzs + cam.cy
    tiles_x = (cam.width + tile - 1) // tile
    tiles_y = (cam.height + tile - 1) // tile
    out = (u + rb < 0) | (u - rb > tiles_x * tile) | (v + rb < 0) | (v - rb > tiles_y * tile)
    return front & ~out


def _cameras(rng):
    cams = [scenes.pinhole(640, 480, 60.0), scenes.pinhole(320, 900, 35.0)]
    for _ in range(4):
        w2c = scenes.look_at(rng.uniform(-2, 2, 3), [0.0, 0.0, 1.0] + rng.normal(0, 0.5, 3))
        cams.append(scenes.pinhole(int(rng.integers(64, 1024)), int(rng.integers(64, 1024)),
                                   float(rng.uniform(20, 110)), world_to_cam=w2c))
    w2c = scenes.look_at([0.2, -0.1, -1.0], [0.1, 0.05, 1.0])
    w2c[0, :3] *= 1.7   # scaled and skewed rows: the bound uses the actual row norms
    w2c[1, :3] = 0.6 * w2c[1, :3] + 0.3 * w2c[0, :3]
    cams.append(scenes.pinhole(512, 384, 60.0, world_to_cam=w2c))
    return cams


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_screen_bound_never_drops_a_visible_gaussian(oracle_mod, seed):
    rng = np.random.default_rng(500 + seed)
    s = scenes.uniform_box(20_000, 500 + seed)
    s.means[:] = rng.uniform(-6, 6, s.means.shape).astype(np.float32)
    s.log_scales[:] = rng.normal(-2.5, 1.2, s.log_scales.shape).astype(np.float32)
    kept_total = visible_total = 0
    for cam in _cameras(rng):
        pr = oracle_mod.project(s, cam)
        vis = pr.visible > 0
        keep = screen_bound_keeps(s, cam)
        assert not np.any(vis & ~keep), np.nonzero(vis & ~keep)[0][:10]
        kept_total += int(keep.sum())
        visible_total += int(vis.sum())
    # The bound does cull: far fewer kept than in front of the cameras.
    assert kept_total < 0.8 * 8 * s.n
    assert visible_total > 0


def test_screen_bound_uses_the_camera_rows_as_given(oracle_mod):
    """Large Gaussians just outside the image of a camera whose first row is
    scaled by 3: only their stretched footprint reaches the image, which the
    bound must see through the actual row norm."""
    rng = np.random.default_rng(77)
    w2c = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1).astype(np.float32)
    w2c[0, :3] *= 3.0
    cam = scenes.pinhole(400, 300, 60.0, world_to_cam=w2c)
    n = 20_000
    s = scenes.uniform_box(n, 77)
    z = rng.uniform(2.0, 8.0, n)
    half = 0.5 * cam.width / cam.fx  # image half-width in x / z before the row scale
    side = rng.choice([-1.0, 1.0], n)
    x = side * z * (half / 3.0) * rng.uniform(1.02, 1.6, n)  # just outside, horizontally
    s.means[:] = np.stack([x, rng.uniform(-1, 1, n), z], axis=1).astype(np.float32)
    s.log_scales[:] = (np.log(rng.uniform(0.05, 0.6, (n, 1))) + rng.normal(0, 0.3, (n, 3))).astype(np.float32)
    pr = oracle_mod.project(s, cam)
    vis = pr.visible > 0
    assert vis.sum() > 200   # many reach the image only through their footprint
    keep = screen_bound_keeps(s, cam)
    assert not np.any(vis & ~keep)


def test_screen_bound_keeps_tiny_gaussians_at_the_border(oracle_mod):
    """Point-like Gaussians whose means sit up to two pixels outside the tile
    grid: their footprint is the +0.3 dilation alone (radius 2 px), so only
    the bound's constant slack keeps them."""
    rng = np.random.default_rng(91)
    cam = scenes.pinhole(333, 250, 50.0)
    tile = 16
    gw = ((cam.width + tile - 1) // tile) * tile
    gh = ((cam.height + tile - 1) // tile) * tile
    n = 4000
    z = rng.uniform(1.0, 10.0, n)
    edge = rng.integers(0, 4, n)
    off = rng.uniform(0.05, 1.95, n)
    along_u = rng.uniform(0, gw, n)
    along_v = rng.uniform(0, gh, n)
    u = np.where(edge == 0, -off, np.where(edge == 1, gw + off, along_u))
    v = np.where(edge == 2, -off, np.where(edge == 3, gh + off, along_v))
    s = scenes.uniform_box(n, 91)
    x = (u - cam.cx) / cam.fx * z
    y = (v - cam.cy) / cam.fy * z
    s.means[:] = np.stack([x, y, z], axis=1).astype(np.float32)
    s.log_scales[:] = np.float32(np.log(1e-5))
    pr = oracle_mod.project(s, cam)
    vis = pr.visible > 0
    assert vis.sum() > n // 2
    keep = screen_bound_keeps(s, cam, tile)
    assert not np.any(vis & ~keep)


def test_screen_bound_uses_the_guard_band_of_the_jacobian(oracle_mod):
    """Means past the guard band (view ratio 1.3-1.7 x the half field of view)
    of a camera whose z row is scaled by 10, Gaussians long along world z: the
    footprint reaching into the image comes from the |r| n2 term at the
    clamped ratio, so the bound must clamp where the Jacobian does (1.3)."""
    rng = np.random.default_rng(5)
    n = 20_000
    w2c = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1).astype(np.float32)
    w2c[2, :3] *= 10.0
    cam = scenes.pinhole(400, 300, 60.0, world_to_cam=w2c)
    half_x = 0.5 * cam.width / cam.fx
    half_y = 0.5 * cam.height / cam.fy
    z = rng.uniform(2.0, 6.0, n)                      # camera depth is 10 z
    rx = rng.choice([-1.0, 1.0], n) * half_x * rng.uniform(1.3, 1.7, n)
    ry = rng.uniform(-0.3, 0.3, n) * half_y
    s = scenes.uniform_box(n, 5)
    s.means[:] = np.stack([rx * 10 * z, ry * 10 * z, z], axis=1).astype(np.float32)
    ls = np.full((n, 3), math.log(1e-3))
    ls[:, 2] = np.log(rng.uniform(0.05, 3.0, n))
    s.log_scales[:] = ls.astype(np.float32)
    s.quats[:] = np.array([1.0, 0.0, 0.0, 0.0], np.float32)
    pr = oracle_mod.project(s, cam)
    vis = pr.visible > 0
    assert vis.sum() > 1000
    keep = screen_bound_keeps(s, cam)
    assert not np.any(vis & ~keep)
