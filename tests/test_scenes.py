"""The seeded synthetic inputs follow their stated recipes: value ranges and
distributions, the density structure of the clustered and imbalance scenes,
camera intrinsics and paths, determinism per seed. They stand in for the
paper's GS-SLAM maps (Sec. 5.1), so their shape is what the measurements
rest on."""
import math

import numpy as np
import pytest

from paper_2607_15951_gb300 import scenes

Y00 = 0.5 / math.sqrt(math.pi)


def _soa_ok(s, sh_coeffs):
    n = s.n
    for a, shape in [(s.means, (n, 3)), (s.log_scales, (n, 3)), (s.quats, (n, 4)),
                     (s.opacity_logits, (n,)), (s.sh, (n, sh_coeffs, 3))]:
        assert a.shape == shape and a.dtype == np.float32 and a.flags.c_contiguous
    assert np.allclose(np.linalg.norm(s.quats.astype(np.float64), axis=1), 1.0, atol=1e-6)


def test_uniform_box_recipe():
    s = scenes.uniform_box(10_000, 0)
    _soa_ok(s, 1)
    assert s.sh_degree == 0
    m = s.means
    assert m[:, :2].min() >= -2 and m[:, :2].max() <= 2 and m[:, 2].min() >= 2 and m[:, 2].max() <= 8
    ls = s.log_scales.astype(np.float64)
    assert abs(ls.mean() + 3.0) < 0.02 and abs(ls.std() - 0.5) < 0.02
    lg = s.opacity_logits.astype(np.float64)
    assert abs(lg.mean()) < 0.05 and abs(lg.std() - 1.0) < 0.05
    rgb = Y00 * s.sh[:, 0, :].astype(np.float64) + 0.5     # degree-0 colour
    assert rgb.min() >= -1e-6 and rgb.max() <= 1 + 1e-6
    assert abs(rgb.mean() - 0.5) < 0.01 and abs(rgb.var() - 1 / 12) < 0.005   # U[0, 1]


def test_clustered_recipe_and_density():
    n = 200_000
    s = scenes.clustered(n, 1)
    _soa_ok(s, 16)
    assert s.sh_degree == 3
    ls = s.log_scales.astype(np.float64)
    assert abs(ls.mean() + 4.0) < 0.01 and abs(ls.std() - 0.7) < 0.01
    sh = s.sh.astype(np.float64)
    assert abs(sh.mean()) < 0.002 and abs(sh.std() - 0.2) < 0.002
    # 10 % uniform over the 20 m box, 90 % in 200 clusters of sigma <= 1 m:
    # on a 1 m grid of the box, the fullest 10 % of the cells hold most of the
    # Gaussians (about 10 % if the scene were uniform).
    m = s.means.astype(np.float64)
    inside = np.all(np.abs(m) < 10, axis=1)
    cells = np.floor(m[inside] + 10).astype(int)
    counts = np.bincount(cells[:, 0] * 400 + cells[:, 1] * 20 + cells[:, 2], minlength=8000)
    top = np.sort(counts)[::-1][:800].sum() / inside.sum()
    assert top > 0.7
    # The emptiest half of the cells holds about half of the 10 % background.
    low = np.sort(counts)[:4000].sum() / n
    assert 0.02 < low < 0.08


def test_same_seed_same_scene_other_seed_other_scene():
    a, b, c = scenes.clustered(5000, 7), scenes.clustered(5000, 7), scenes.clustered(5000, 8)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
        assert not np.array_equal(getattr(a, k), getattr(c, k))


def test_pinhole_intrinsics():
    cam = scenes.pinhole(1920, 1080, 60.0)
    assert cam.fx == pytest.approx(960 / math.tan(math.radians(30)), rel=1e-6)
    assert cam.fy == cam.fx and cam.cx == 960 and cam.cy == 540
    assert np.array_equal(cam.world_to_cam, np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1))
    # look_at: a rotation, and the camera centre maps to the origin.
    w2c = scenes.look_at([1.0, -2.0, 0.5], [0.3, 0.1, 1.0]).astype(np.float64)
    R, t = w2c[:, :3], w2c[:, 3]
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-6) and np.linalg.det(R) == pytest.approx(1, abs=1e-6)
    assert np.allclose(R @ np.array([1.0, -2.0, 0.5]) + t, 0, atol=1e-5)


def test_trajectory_recipe():
    cams = scenes.trajectory(64, 1003)
    assert len(cams) == 64
    assert all((c.width, c.height) == ((1280, 720) if i % 2 == 0 else (640, 480)) for i, c in enumerate(cams))
    centres = []
    for c in cams:
        w2c = c.world_to_cam.astype(np.float64)
        centres.append(-w2c[:, :3].T @ w2c[:, 3])
    centres = np.array(centres)
    assert np.linalg.norm(centres, axis=1).max() <= 4.0 * 1.3     # spline near the waypoints' 4 m ball
    steps = np.linalg.norm(np.diff(centres, axis=0), axis=1)
    assert steps.max() < 4 * np.median(steps)                    # smooth: no jumps between views


def test_imbalance_recipe():
    n, W, H = 100_000, 3840, 2160
    s = scenes.imbalance(n, 4, W, H)
    f = (W / 2) / math.tan(math.radians(30))
    m = s.means.astype(np.float64)
    front = m[:, 2] > 0.2
    u = np.where(front, f * m[:, 0] / np.where(front, m[:, 2], 1) + W / 2, -1e9)
    v = np.where(front, f * m[:, 1] / np.where(front, m[:, 2], 1) + H / 2, -1e9)
    # 20 % packed into a disc of 2 % of the image area around the centre.
    r_disc = math.sqrt(0.02 * W * H / math.pi)
    in_disc = (u - W / 2) ** 2 + (v - H / 2) ** 2 <= r_disc ** 2
    assert in_disc.sum() >= 0.2 * n
    # 1 % large splats: projected 3-sigma radius above 256 px at their depth.
    sig = np.exp(s.log_scales.astype(np.float64).max(axis=1))
    big = front & (3 * sig * f / np.where(front, m[:, 2], 1) > 256)
    assert big.sum() >= 0.005 * n
