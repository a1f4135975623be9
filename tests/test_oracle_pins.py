"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test ties one part of the oracle to something independent of it: an
independent library routine (scipy's complex spherical harmonics, scipy's
quaternion rotations, numpy's eigen-solver and inverse, scipy's multivariate
normal density), a finite-difference Jacobian, a geometric restatement of the
tile rule, a closed form, a hand-computed example (tests/golden), or an
invariant of Eq. 1. A plausible slip in the oracle (a sign, an index, a
transposed matrix, a dropped term) changes one of these.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import expit, sph_harm_y
from scipy.stats import multivariate_normal

from paper_2607_15951_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

class Cam:
    def __init__(self, w2c, fx, fy, cx, cy, width, height, near_z=0.2):
        self.world_to_cam = np.asarray(w2c, np.float64).reshape(3, 4)
        self.fx, self.fy, self.cx, self.cy = fx, fy, cx, cy
        self.width, self.height, self.near_z = width, height, near_z


def ident_cam(fx=100.0, cx=32.0, w=64, h=64, fy=None, cy=None):
    return Cam(np.concatenate([np.eye(3), np.zeros((3, 1))], 1), fx, fy or fx, cx,
               cy if cy is not None else cx, w, h)


def one_gaussian(mean, scales, quat, logit=0.0, sh=None, deg=0):
    k = (deg + 1) ** 2
    if sh is None:
        sh = np.zeros((1, k, 3))
    return scenes.Scene(np.array([mean], np.float64), np.log(np.array([scales], np.float64)),
                        np.array([quat], np.float64), np.array([logit], np.float64),
                        np.asarray(sh, np.float64).reshape(1, k, 3), deg)


def records_scene(recs):
    m = np.array([r["mean2d"] for r in recs], np.float64)
    c = np.array([r["conic"] for r in recs], np.float64)
    o = np.array([r["opacity"] for r in recs], np.float64)
    col = np.array([r["rgb"] for r in recs], np.float64)
    d = np.array([r["depth"] for r in recs], np.float64)
    rad = np.array([r["radius"] for r in recs], np.int64)
    return m, c, o, col, d, rad


def real_sh_scipy(l, m, d):
    """Real SH with the Condon-Shortley phase from scipy's complex Y_l^m."""
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    y = sph_harm_y(l, abs(m), theta, phi)
    if m == 0:
        return y.real
    if m > 0:
        return math.sqrt(2) * y.real
    return math.sqrt(2) * y.imag


def random_dirs(rng, n):
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


# ---------------------------------------------------------------------------
# Spherical harmonics (view-dependent colour, Sec. 3.1)
# ---------------------------------------------------------------------------

def test_sh_matches_scipy_complex_harmonics(oracle_mod):
    rng = np.random.default_rng(11)
    d = random_dirs(rng, 64)
    Y = oracle_mod.sh_basis(3, d)
    for l in range(4):
        for m in range(-l, l + 1):
            np.testing.assert_allclose(Y[:, l * l + l + m], real_sh_scipy(l, m, d),
                                       rtol=0, atol=1e-12, err_msg=f"l={l} m={m}")


def test_sh_addition_theorem(oracle_mod):
    # sum_m Y_lm(d)^2 = (2l+1) / (4 pi) for every unit direction.
    rng = np.random.default_rng(12)
    Y = oracle_mod.sh_basis(3, random_dirs(rng, 100))
    for l in range(4):
        s = (Y[:, l * l:(l + 1) ** 2] ** 2).sum(1)
        np.testing.assert_allclose(s, (2 * l + 1) / (4 * math.pi), rtol=1e-12)


def test_sh_orthonormal_by_quadrature(oracle_mod):
    # Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6 exactly.
    x, w = np.polynomial.legendre.leggauss(8)
    nphi = 16
    phi = 2 * math.pi * np.arange(nphi) / nphi
    ct = np.repeat(x, nphi)
    ww = np.repeat(w, nphi) * (2 * math.pi / nphi)
    st = np.sqrt(1 - ct ** 2)
    ph = np.tile(phi, len(x))
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], 1)
    Y = oracle_mod.sh_basis(3, d)
    G = (Y * ww[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_axis_values_and_sign_convention(oracle_mod):
    c1 = math.sqrt(3 / (4 * math.pi))
    Y = oracle_mod.sh_basis(1, np.eye(3))
    # rows: +x, +y, +z; columns: (l,m) = (0,0), (1,-1), (1,0), (1,1)
    np.testing.assert_allclose(Y[:, 0], 1 / (2 * math.sqrt(math.pi)), rtol=1e-14)
    np.testing.assert_allclose(Y[0, 1:], [0, 0, -c1], atol=1e-14)   # Y_11 = -c1 x
    np.testing.assert_allclose(Y[1, 1:], [-c1, 0, 0], atol=1e-14)   # Y_1-1 = -c1 y
    np.testing.assert_allclose(Y[2, 1:], [0, c1, 0], atol=1e-14)    # Y_10 = c1 z


def test_colour_uses_camera_to_mean_direction(oracle_mod):
    # Degree 1, only the (1,0) coefficient of red set: red = c * Y_10(d) + 0.5
    # with d from the camera centre C = -R^T t to the mean.
    rng = np.random.default_rng(13)
    R = Rotation.from_rotvec([0.1, -0.2, 0.05]).as_matrix()
    C = np.array([0.3, -0.4, -1.0])
    t = -R @ C
    cam = Cam(np.concatenate([R, t[:, None]], 1), 100.0, 100.0, 32.0, 32.0, 64, 64)
    for _ in range(5):
        mu = C + R.T @ np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(3, 6)])
        sh = np.zeros((4, 3))
        sh[2, 0] = 0.7
        sh[0, 1] = 0.3
        g = one_gaussian(mu, [0.05] * 3, [1, 0, 0, 0], sh=sh, deg=1)
        pr = oracle_mod.project(g, cam)
        assert pr.visible[0] == 1
        d = (mu - C) / np.linalg.norm(mu - C)
        assert abs(pr.rgb[0, 0] - max(0.0, 0.7 * real_sh_scipy(1, 0, d[None])[0] + 0.5)) < 1e-12
        assert abs(pr.rgb[0, 1] - (0.3 / (2 * math.sqrt(math.pi)) + 0.5)) < 1e-12
        assert abs(pr.rgb[0, 2] - 0.5) < 1e-12


def test_degree3_colour_against_scipy_basis(oracle_mod):
    # Every SH coefficient set: rgb = max(0, sum_k c_k Y_k(d) + 0.5) with the
    # basis from scipy and k = l^2 + l + m.
    rng = np.random.default_rng(14)
    cam = ident_cam()
    for _ in range(6):
        mu = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(3, 6)])
        sh = rng.normal(0, 0.3, (16, 3))
        pr = oracle_mod.project(one_gaussian(mu, [0.05] * 3, [1, 0, 0, 0], sh=sh, deg=3), cam)
        d = (mu / np.linalg.norm(mu))[None]
        Y = np.array([real_sh_scipy(l, m, d)[0] for l in range(4) for m in range(-l, l + 1)])
        np.testing.assert_allclose(pr.rgb[0], np.maximum(0.0, Y @ sh + 0.5), atol=1e-12)


def test_sh_degree0_colour_is_rgb(oracle_mod):
    s = scenes.uniform_box(200, 3)
    cam = scenes.pinhole(256, 256, 60.0)
    pr = oracle_mod.project(s, cam)
    vis = pr.visible == 1
    rgb = s.sh[:, 0, :].astype(np.float64) / (2 * math.sqrt(math.pi)) + 0.5
    np.testing.assert_allclose(pr.rgb[vis], rgb[vis], atol=1e-12)


def test_colour_clamped_at_zero(oracle_mod):
    sh = np.zeros((1, 3))
    sh[0] = [-5.0, 0.0, 1.0]
    g = one_gaussian([0, 0, 5], [0.1] * 3, [1, 0, 0, 0], sh=sh, deg=0)
    pr = oracle_mod.project(g, ident_cam())
    np.testing.assert_allclose(pr.rgb[0], [0.0, 0.5, 0.5 + 1 / (2 * math.sqrt(math.pi))], atol=1e-14)


# ---------------------------------------------------------------------------
# Projection (Sec. 3.1 stage 2, Sec. 4.4, Sec. 4.5 step 1)
# ---------------------------------------------------------------------------

def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("case", _golden()["projection_cases"], ids=lambda c: c["name"])
def test_projection_hand_examples(oracle_mod, case):
    c = case["cam"]
    cam = ident_cam(c["fx"], c["cx"], c["width"], c["height"], c["fy"], c["cy"])
    g = one_gaussian(case["mean"], case["scales"], case["quat"])
    pr = oracle_mod.project(g, cam)
    assert pr.visible[0] == 1
    np.testing.assert_allclose(pr.mean2d[0], case["mean2d"], atol=1e-12)
    np.testing.assert_allclose(pr.conic[0], case["conic"], atol=1e-9)
    assert abs(pr.extent[0] - case["extent"]) < 1e-6
    assert pr.radius[0] == case["radius"]
    assert list(pr.rect[0]) == case["rect"]


def _cov2d_independent(mu, scales, quat_wxyz, R_cam, t_cam, fx, fy, cx, cy):
    """Covariance from scipy's rotation and a finite-difference Jacobian of the
    pinhole map, plus the 0.3 px^2 dilation."""
    Rq = Rotation.from_quat([quat_wxyz[1], quat_wxyz[2], quat_wxyz[3], quat_wxyz[0]]).as_matrix()
    Sigma = Rq @ np.diag(np.asarray(scales) ** 2) @ Rq.T

    def pi(p_world):
        p = R_cam @ p_world + t_cam
        return np.array([fx * p[0] / p[2] + cx, fy * p[1] / p[2] + cy])

    h = 1e-6
    Jw = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        Jw[:, k] = (pi(mu + e) - pi(mu - e)) / (2 * h)
    return Jw @ Sigma @ Jw.T + 0.3 * np.eye(2), pi(mu)


def test_projection_matches_independent_covariance(oracle_mod):
    rng = np.random.default_rng(21)
    Rc = Rotation.from_rotvec([0.2, -0.3, 0.1]).as_matrix()
    Ccen = np.array([0.5, 0.2, -2.0])
    tc = -Rc @ Ccen
    fx, fy, cx, cy, W, H = 300.0, 280.0, 160.0, 120.0, 320, 240
    cam = Cam(np.concatenate([Rc, tc[:, None]], 1), fx, fy, cx, cy, W, H)
    checked = 0
    for _ in range(40):
        pc = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.25, 0.25), 1]) * rng.uniform(2, 8)
        mu = Rc.T @ (pc - tc)
        scales = np.exp(rng.normal(-3, 0.5, 3))
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        g = one_gaussian(mu, scales, q)
        pr = oracle_mod.project(g, cam)
        cov, uv = _cov2d_independent(mu, scales, q, Rc, tc, fx, fy, cx, cy)
        np.testing.assert_allclose(pr.mean2d[0], uv, rtol=1e-12)
        Qref = np.linalg.inv(cov)
        np.testing.assert_allclose(pr.conic[0], [Qref[0, 0], Qref[0, 1], Qref[1, 1]], rtol=1e-6)
        lam = np.linalg.eigvalsh(cov).max()
        mid = 0.5 * np.trace(cov)
        # The eigenvalue used for the bound is floored at mid + sqrt(0.1).
        lam_b = max(lam, mid + math.sqrt(0.1))
        np.testing.assert_allclose(pr.extent[0], 3 * math.sqrt(lam_b), rtol=1e-6)
        assert pr.depth[0] == pytest.approx(pc[2], rel=1e-12)
        checked += pr.visible[0]
    assert checked > 20


def test_isotropic_gaussian_rotation_invariant(oracle_mod):
    rng = np.random.default_rng(22)
    cam = ident_cam()
    base = oracle_mod.project(one_gaussian([0.2, 0.1, 4.0], [0.07] * 3, [1, 0, 0, 0]), cam)
    for _ in range(5):
        q = rng.standard_normal(4)
        pr = oracle_mod.project(one_gaussian([0.2, 0.1, 4.0], [0.07] * 3, q), cam)
        np.testing.assert_allclose(pr.conic, base.conic, rtol=1e-12)


def test_quaternion_sign_and_scale_invariance(oracle_mod):
    # q and -q, and q scaled by any positive factor, give the same rotation.
    cam = ident_cam()
    q = np.array([0.3, -0.5, 0.7, 0.2])
    a = oracle_mod.project(one_gaussian([0.1, 0.0, 3.0], [0.02, 0.05, 0.1], q), cam)
    b = oracle_mod.project(one_gaussian([0.1, 0.0, 3.0], [0.02, 0.05, 0.1], -2.5 * q), cam)
    np.testing.assert_allclose(a.conic, b.conic, rtol=1e-12)


def test_camera_and_world_moved_together(oracle_mod):
    # Rendering world points with camera [R|t] equals rendering the points
    # already expressed in camera space with the identity camera.
    rng = np.random.default_rng(23)
    s = scenes.uniform_box(300, 5)
    Rc = Rotation.from_rotvec([0.05, 0.1, -0.2]).as_matrix()
    tc = np.array([0.1, -0.2, 0.3])
    camA = Cam(np.concatenate([Rc, tc[:, None]], 1), 221.7, 221.7, 128, 128, 256, 256)
    # world -> camera for the means, and rotate each orientation by Rc.
    m2 = (Rc @ s.means.astype(np.float64).T).T + tc
    rq = Rotation.from_quat(s.quats.astype(np.float64)[:, [1, 2, 3, 0]])
    q2 = (Rotation.from_matrix(Rc) * rq).as_quat()[:, [3, 0, 1, 2]]
    s2 = scenes.Scene(m2, s.log_scales.astype(np.float64), q2, s.opacity_logits.astype(np.float64),
                      s.sh.astype(np.float64), 0)
    a = oracle_mod.project(s, camA)
    b = oracle_mod.project(s2, ident_cam(221.7, 128, 256, 256))
    assert (a.visible == b.visible).all()
    np.testing.assert_allclose(a.mean2d, b.mean2d, rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(a.conic, b.conic, rtol=1e-8, atol=1e-12)
    assert (a.radius == b.radius).all()
    del rng


def test_jacobian_guard_band(oracle_mod):
    # Far off-axis (x/z = 1.0 > 1.3 * tan_x = 0.416): the Jacobian is taken at
    # the clamped ratio, i.e. at the point (0.416 z, y, z).
    cam = ident_cam()   # tan_x = 0.5 * 64 / 100 = 0.32
    mu = np.array([5.0, 0.0, 5.0])
    pr = oracle_mod.project(one_gaussian(mu, [0.1] * 3, [1, 0, 0, 0]), cam)
    lim = 1.3 * 0.32
    cov, _ = _cov2d_independent(np.array([lim * 5.0, 0.0, 5.0]), [0.1] * 3, [1, 0, 0, 0],
                                np.eye(3), np.zeros(3), 100.0, 100.0, 32.0, 32.0)
    Q = np.linalg.inv(cov)
    np.testing.assert_allclose(pr.conic[0], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-6)
    assert pr.mean2d[0, 0] == pytest.approx(100.0 * 1.0 + 32.0)


def test_near_plane_cull(oracle_mod):
    cam = ident_cam()
    for z, vis in [(0.19, 0), (0.2, 0), (0.2000001, 1), (-3.0, 0)]:
        pr = oracle_mod.project(one_gaussian([0, 0, z], [0.001] * 3, [1, 0, 0, 0]), cam)
        assert pr.visible[0] == vis, z


def test_opacity_is_sigmoid_of_logit(oracle_mod):
    rng = np.random.default_rng(24)
    s = scenes.uniform_box(100, 9)
    pr = oracle_mod.project(s, scenes.pinhole(256, 256))
    vis = pr.visible == 1
    np.testing.assert_allclose(pr.opacity[vis], expit(s.opacity_logits.astype(np.float64))[vis],
                               rtol=1e-14)
    del rng


def test_offscreen_gaussians_invisible(oracle_mod):
    cam = ident_cam()
    # Projects to u = 100*2/1 + 32 = 232 >> 64 with a small radius.
    pr = oracle_mod.project(one_gaussian([2.0, 0.0, 1.0], [0.001] * 3, [1, 0, 0, 0]), cam)
    assert pr.visible[0] == 0


# ---------------------------------------------------------------------------
# Binning (Sec. 3.1 stage 3, Sec. 4.4, Sec. 4.5 step 2)
# ---------------------------------------------------------------------------

def _geometric_tiles(u, r, tile, ntiles):
    """Tiles overlapped by the closed interval [u - r, u + r - 1]: a geometric
    restatement of the rect rule floor((u-r)/t) .. floor((u+r+t-1)/t)."""
    out = []
    for t in range(ntiles):
        if u - r < (t + 1) * tile and u + r - 1 >= t * tile:
            out.append(t)
    return out


def test_binning_bruteforce_tiny(oracle_mod):
    rng = np.random.default_rng(31)
    W, H, T = 100, 70, 16
    tx, ty = (W + T - 1) // T, (H + T - 1) // T
    n = 60
    mean2d = np.stack([rng.uniform(-40, W + 40, n), rng.uniform(-40, H + 40, n)], 1)
    mean2d = mean2d.astype(np.float32).astype(np.float64)
    radius = rng.integers(1, 40, n).astype(np.int64)
    depth = rng.uniform(0.5, 3, n).astype(np.float32).astype(np.float64)
    depth[5] = depth[7]  # an exact tie, broken by index
    visible = (rng.uniform(size=n) > 0.1).astype(np.int32)
    b = oracle_mod.bin_tiles(mean2d, radius, depth, visible, W, H, T, T)
    expect = []
    for i in range(n):
        if not visible[i]:
            continue
        xs = _geometric_tiles(mean2d[i, 0], radius[i], T, tx)
        ys = _geometric_tiles(mean2d[i, 1], radius[i], T, ty)
        for yy in ys:
            for xx in xs:
                expect.append((yy * tx + xx, float(np.float32(depth[i])), i))
    expect.sort()
    assert len(b.values) == len(expect)
    assert [int(v) for v in b.values] == [e[2] for e in expect]
    assert [int(k >> np.uint64(32)) for k in b.keys] == [e[0] for e in expect]
    bits = [int(np.array([e[1]], np.float32).view(np.uint32)[0]) for e in expect]
    assert [int(k & np.uint64(0xffffffff)) for k in b.keys] == bits
    for t in range(tx * ty):
        idx = [k for k, e in enumerate(expect) if e[0] == t]
        if idx:
            assert tuple(b.ranges[t]) == (idx[0], idx[-1] + 1)
        else:
            assert tuple(b.ranges[t]) == (0, 0)


def test_rect_rule_edges(oracle_mod):
    # u + r in [16k, 16k+1) does not reach tile k; in [16k+1, 16k+2) it does.
    for u, r, expect in [(20.0, 12, [0, 1]), (20.0, 11, [0, 1]), (19.5, 12, [0, 1]),
                         (20.5, 12, [0, 1]), (21.0, 12, [0, 1, 2]), (16.0, 1, [0, 1]),
                         (15.9, 1, [0])]:
        b = oracle_mod.bin_tiles(np.array([[u, 8.0]]), np.array([r]), np.array([1.0]),
                                 np.array([1]), 64, 16, 16, 16)
        got = sorted(int(k >> np.uint64(32)) for k in b.keys)
        assert got == _geometric_tiles(u, r, 16, 4) == expect, (u, r, got)


# ---------------------------------------------------------------------------
# Blending, Eq. 1 (Sec. 3.1; Sec. 4.5 step 3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", _golden()["blend_cases"], ids=lambda c: c["name"])
def test_blend_hand_examples(oracle_mod, case):
    g = _golden()["image"]
    m, c, o, col, d, rad = records_scene(case["records"])
    vis = np.ones(len(o), np.int32)
    b = oracle_mod.bin_tiles(m, rad, d, vis, g["width"], g["height"], g["tile"], g["tile"])
    img = oracle_mod.blend(m, c, o, col, b.values, b.ranges, g["width"], g["height"],
                           g["tile"], g["tile"])
    x, y = case["pixel"]
    np.testing.assert_allclose(img.rgb[y, x], case["rgb"], atol=1e-9)
    assert img.T[y, x] == pytest.approx(case["T"], abs=1e-9)
    assert img.last[y, x] == case["last"]
    assert img.neval[y, x] == case["neval"]


def test_single_gaussian_closed_form(oracle_mod):
    # C(p) = rgb * alpha(p), alpha = min(0.99, o * N(p; mu, S) / N(mu; mu, S))
    # where it is >= 1/255, else 0; the density ratio from scipy.
    rng = np.random.default_rng(41)
    W = H = 64
    for trial in range(4):
        A = rng.normal(size=(2, 2)) * 3
        S = A @ A.T + 0.3 * np.eye(2)
        Q = np.linalg.inv(S)
        mu = rng.uniform(20, 44, 2)
        o = rng.uniform(0.2, 1.0)
        rgb = rng.uniform(0, 1, 3)
        lam = np.linalg.eigvalsh(S).max()
        r = int(math.ceil(3 * math.sqrt(lam)))
        m = mu[None]
        c = np.array([[Q[0, 0], Q[0, 1], Q[1, 1]]])
        b = oracle_mod.bin_tiles(m, [r], [1.0], [1], W, H)
        img = oracle_mod.blend(m, c, [o], rgb[None], b.values, b.ranges, W, H)
        mvn = multivariate_normal(mean=mu, cov=S)
        ys, xs = np.mgrid[0:H, 0:W]
        P = np.stack([xs + 0.5, ys + 0.5], -1)
        a = np.minimum(0.99, o * mvn.pdf(P) / mvn.pdf(mu))
        a[a < 1 / 255] = 0
        covered = np.zeros((H, W), bool)
        for t in range(16):
            lo, hi = b.ranges[t]
            if hi > lo:
                covered[(t // 4) * 16:(t // 4) * 16 + 16, (t % 4) * 16:(t % 4) * 16 + 16] = True
        a[~covered] = 0
        np.testing.assert_allclose(img.rgb, a[..., None] * rgb, atol=1e-12)
        np.testing.assert_allclose(img.T, 1 - a, atol=1e-12)


def _small_scene_records(oracle_mod, n=400, seed=51, W=96, H=80):
    s = scenes.uniform_box(n, seed)
    cam = scenes.pinhole(W, H, 60.0)
    return oracle_mod.project(s, cam), W, H


def test_bruteforce_global_sort_equals_tile_lists(oracle_mod):
    pr, W, H = _small_scene_records(oracle_mod)
    b = oracle_mod.bin_tiles(pr.mean2d, pr.radius, pr.depth, pr.visible, W, H)
    a = oracle_mod.blend(pr.mean2d, pr.conic, pr.opacity, pr.rgb, b.values, b.ranges, W, H)
    c = oracle_mod.blend_bruteforce(pr.mean2d, pr.conic, pr.opacity, pr.rgb, pr.depth, pr.radius,
                                    pr.visible, W, H)
    assert np.array_equal(a.rgb, c.rgb)
    assert np.array_equal(a.T, c.T)
    assert np.array_equal(a.last, c.last)
    assert np.array_equal(a.neval, c.neval)


def test_blend_invariants(oracle_mod):
    pr, W, H = _small_scene_records(oracle_mod, n=600, seed=52)
    b = oracle_mod.bin_tiles(pr.mean2d, pr.radius, pr.depth, pr.visible, W, H)
    img = oracle_mod.blend(pr.mean2d, pr.conic, pr.opacity, pr.rgb, b.values, b.ranges, W, H)
    assert (img.T >= 0).all() and (img.T <= 1).all()
    # Colour is a convex combination: sum of weights = 1 - T, colours in [0, max rgb].
    assert (img.rgb >= 0).all()
    assert (img.rgb <= pr.rgb.max() * (1 - img.T[..., None]) + 1e-12).all()
    # A pixel that stopped has T >= 1e-4 (the stopping Gaussian was not added).
    assert (img.T[img.neval > 0] >= 1e-4 - 1e-15).all()
    assert (img.last <= img.neval).all()


def test_permuting_input_order_leaves_image_unchanged(oracle_mod):
    s = scenes.uniform_box(500, 53)
    cam = scenes.pinhole(80, 64, 60.0)
    _, _, a = oracle_mod.render(s, cam)
    perm = np.random.default_rng(54).permutation(s.n)
    _, _, b = oracle_mod.render(s.subset(perm), cam)
    np.testing.assert_allclose(a.rgb, b.rgb, atol=1e-13)
    np.testing.assert_allclose(a.T, b.T, atol=1e-13)


def test_transmittance_is_product_of_one_minus_alpha(oracle_mod):
    # Final T equals the product of (1 - alpha) over the blended Gaussians,
    # recomputed here pixel by pixel from the closed-form alphas.
    pr, W, H = _small_scene_records(oracle_mod, n=200, seed=55)
    b = oracle_mod.bin_tiles(pr.mean2d, pr.radius, pr.depth, pr.visible, W, H)
    img = oracle_mod.blend(pr.mean2d, pr.conic, pr.opacity, pr.rgb, b.values, b.ranges, W, H)
    tiles_x = (W + 15) // 16
    rng = np.random.default_rng(56)
    for _ in range(50):
        x, y = int(rng.integers(0, W)), int(rng.integers(0, H))
        t = (y // 16) * tiles_x + x // 16
        lo, hi = b.ranges[t]
        T = 1.0
        for k in range(lo, lo + img.last[y, x]):
            g = b.values[k]
            d = np.array([x + 0.5, y + 0.5]) - pr.mean2d[g]
            Q = np.array([[pr.conic[g, 0], pr.conic[g, 1]], [pr.conic[g, 1], pr.conic[g, 2]]])
            a = min(0.99, pr.opacity[g] * math.exp(-0.5 * d @ Q @ d))
            if a >= 1 / 255:
                T *= 1 - a
        assert img.T[y, x] == pytest.approx(T, rel=1e-12, abs=1e-15)
        del hi
