"""Pins of the oracle's FP64 gradient against central finite differences of
the oracle's own forward render (64 Gaussians, 32x32, the size at which the
gradient is checked by finite differences), for every parameter group:
means, log-scales, quaternions, opacity logits and SH coefficients."""
import numpy as np
import pytest

from paper_2607_15951_gb300 import scenes


def fd_scene(seed, sh_degree=3, n=64):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1.5, 1.5, n), rng.uniform(-1.5, 1.5, n), rng.uniform(3, 6, n)], 1)
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    k = (sh_degree + 1) ** 2
    return scenes.Scene(means, rng.normal(-1.2, 0.4, (n, 3)), q, rng.normal(0.0, 1.0, n),
                        rng.normal(0.0, 0.3, (n, k, 3)), sh_degree, f"fd_{seed}")


def loss(oracle_mod, scene, cam, w, bg):
    _, _, img = oracle_mod.render(scene, cam, bg=bg)
    return float((img.rgb * w).sum()), img


PARAMS = ["means", "log_scales", "quats", "opacity_logits", "sh"]


@pytest.mark.parametrize("seed,deg", [(3, 3), (4, 0)])
def test_gradient_matches_central_differences(oracle_mod, seed, deg):
    scene = fd_scene(seed, deg)
    cam = scenes.pinhole(32, 32, 60.0)
    bg = (0.1, 0.2, 0.3)
    w = np.random.default_rng(seed + 100).normal(0.0, 1.0, (32, 32, 3))
    gr = oracle_mod.render_backward(scene, cam, w, bg=bg)
    pr0 = oracle_mod.project(scene, cam)
    rng = np.random.default_rng(seed + 200)
    checked = 0
    worst = 0.0
    for name in PARAMS:
        arr = getattr(scene, name)
        an = getattr(gr, name)
        flat_idx = rng.permutation(arr.size)[:120]
        for fi in flat_idx:
            idx = np.unravel_index(fi, arr.shape)
            g = idx[0]
            if not pr0.visible[g]:
                assert an[idx] == 0.0
                continue
            h = 1e-6 * max(1.0, abs(arr[idx]))
            old = arr[idx]
            arr[idx] = old + h
            lp, ip = loss(oracle_mod, scene, cam, w, bg)
            prp = oracle_mod.project(scene, cam)
            arr[idx] = old - h
            lm, im = loss(oracle_mod, scene, cam, w, bg)
            prm = oracle_mod.project(scene, cam)
            arr[idx] = old
            # Skip steps across a discrete decision (rect, radius, contributor set).
            if (not np.array_equal(prp.rect, prm.rect) or not np.array_equal(ip.last, im.last)
                    or not np.array_equal(ip.neval, im.neval)):
                continue
            fd = (lp - lm) / (2 * h)
            err = abs(fd - an[idx]) / (abs(an[idx]) + 1e-4)
            worst = max(worst, err)
            assert abs(fd - an[idx]) <= 1e-5 * (abs(an[idx]) + 1e-3), (name, idx, fd, an[idx])
            checked += 1
    assert checked > 300, checked
    print("checked", checked, "worst relative", worst)


def test_record_gradient_of_single_gaussian_closed_form(oracle_mod):
    # One Gaussian, alpha below the clamp everywhere: L = sum_p w_p . rgb alpha_p
    # so dL/dr = sum_p w_p,r alpha_p and dL/do = sum_p (w_p . rgb) G_p.
    s = fd_scene(7, 0, n=1)
    s.means[0] = [0.1, -0.05, 4.0]
    s.log_scales[0] = np.log([0.3, 0.2, 0.25])
    s.opacity_logits[0] = -0.5
    cam = scenes.pinhole(32, 32, 60.0)
    w = np.random.default_rng(8).normal(size=(32, 32, 3))
    gr = oracle_mod.render_backward(s, cam, w)
    pr, _, img = oracle_mod.render(s, cam)
    alpha = 1.0 - img.T
    assert alpha.max() < 0.99
    np.testing.assert_allclose(gr.record[0, 6:9], (w * alpha[..., None]).sum((0, 1)), rtol=1e-12)
    G = alpha / pr.opacity[0]
    np.testing.assert_allclose(gr.record[0, 5], ((w * pr.rgb[0]).sum(-1) * G).sum(), rtol=1e-12)
