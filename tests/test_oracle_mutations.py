"""Planted mistakes: each mutation below is applied to a copy of the oracle
source, compiled, and a pin suite is run against it: the forward pins
(tests/test_oracle_pins.py) for mistakes in the projection, binning and
blend, the finite-difference gradient pins (tests/test_oracle_grad_pins.py)
for mistakes in the gradient. Every mutation must make at least one pin
fail, which shows the pins are not blind to that class of slip. The real
oracle is never modified."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gs_oracle.cpp")

MUTATIONS = {
    "no_dilation": ("const double kDilation = 0.3;", "const double kDilation = 0.0;"),
    "conic_offdiag_sign": ("P.q[1] = -cov[0][1] / det", "P.q[1] = cov[0][1] / det"),
    "quat_sign": ("R[0][1] = 2 * (x * y - w * z);", "R[0][1] = 2 * (x * y + w * z);"),
    "camera_rotation_transposed": ("matmul3(cam.R, Sigma, tmp);\n    matmul3(tmp, Wt, Sc);",
                                   "matmul3(Wt, Sigma, tmp);\n    matmul3(tmp, cam.R, Sc);"),
    "alpha_clamp": ("const double kAlphaMax = 0.99;", "const double kAlphaMax = 1.0;"),
    "no_alpha_skip": ("o.flag = 1;\n        if (alpha < kAlphaMin) continue;",
                      "o.flag = 1;\n        if (alpha <= 0.0) continue;"),
    "stop_after_adding": ("if (Tn < kTMin) break;\n        for (int ch = 0; ch < 3; ++ch) o.c[ch] += rgb[3 * g + ch] * alpha * T;",
                          "for (int ch = 0; ch < 3; ++ch) o.c[ch] += rgb[3 * g + ch] * alpha * T;\n        if (Tn < kTMin) break;"),
    "rect_off_by_one": ("rect[2] = tile_coord(u + (double)r + (tw - 1), tw, tiles_x);",
                        "rect[2] = tile_coord(u + (double)r + tw, tw, tiles_x);"),
    "sh_sin_cos_swapped": ("if (m > 0) return std::sqrt(2.0) * K * cos(am * phi) * P;",
                           "if (m > 0) return std::sqrt(2.0) * K * sin(am * phi) * P;"),
    "sh_index": ("s = s + coef[(l * l + l + m) * 3 + ch]", "s = s + coef[(l * l + l - m) * 3 + ch]"),
    "sort_ignores_depth": ("items.emplace_back(ty * tiles_x + tx, f32_bits(depth[i]), i);",
                           "items.emplace_back(ty * tiles_x + tx, 0u, i);"),
    "guard_band": ("const double kGuard = 1.3;", "const double kGuard = 1.6;"),
    "eigen_floor": ("std::max(0.1, mid * mid - val(det))", "std::max(0.0, mid * mid - val(det))"),
    "near_inclusive": ("if (!(val(t[2]) > cam.near_z)) return false;", "if (!(val(t[2]) >= cam.near_z)) return false;"),
    "jacobian_sign": ("{T(0.0), cam.fy / t[2], -cam.fy * ry / t[2]}", "{T(0.0), cam.fy / t[2], cam.fy * ry / t[2]}"),
    "pixel_centre": ("x + 0.5, y + 0.5, last - first", "x, y, last - first"),
    "opacity_not_sigmoid": ("P.o = 1.0 / (1.0 + exp(-logit));", "P.o = 1.0 / (1.0 + exp(logit));"),
    "colour_no_offset": ("P.rgb[ch] = vmax(s + 0.5, 0.0);", "P.rgb[ch] = vmax(s, 0.0);"),
}


# Mistakes in the gradient (Eq. 1 differentiated per pixel, then the
# projection in forward mode), caught by the finite-difference pins.
GRAD_MUTATIONS = {
    "grad_no_background_term": ("(S[ch] + bg[ch] * T_N) / (1.0 - c.alpha)", "(S[ch]) / (1.0 - c.alpha)"),
    "grad_suffix_sign": ("ck[ch] * c.T - (S[ch] + bg[ch] * T_N)", "ck[ch] * c.T + (S[ch] + bg[ch] * T_N)"),
    "grad_no_one_minus_alpha": ("(S[ch] + bg[ch] * T_N) / (1.0 - c.alpha);", "(S[ch] + bg[ch] * T_N);"),
    "grad_mean_sign": ("const double du = dL_dpower * (q[0] * c.dx + q[1] * c.dy);",
                       "const double du = -dL_dpower * (q[0] * c.dx + q[1] * c.dy);"),
    "grad_cross_term_factor": ("const double dq01 = dL_dpower * (-c.dx * c.dy);",
                               "const double dq01 = dL_dpower * (-0.5 * c.dx * c.dy);"),
    "grad_opacity_without_G": ("const double dL_do = dL_dalpha * c.G;", "const double dL_do = dL_dalpha;"),
    "grad_log_scale_seed": ("ls[a] = Dual(log_scales[3 * i + a], j == 3 + a ? 1.0 : 0.0);",
                            "ls[a] = Dual(log_scales[3 * i + a], j == 4 + a ? 1.0 : 0.0);"),
    "grad_colour_weight": ("dr[6 + ch] += gp[ch] * c.alpha * c.T;", "dr[6 + ch] += gp[ch] * c.alpha;"),
}

CASES = [(n, "test_oracle_pins.py") for n in sorted(MUTATIONS)] + \
        [(n, "test_oracle_grad_pins.py") for n in sorted(GRAD_MUTATIONS)]


@pytest.mark.slow
@pytest.mark.parametrize("name,pins", CASES, ids=[c[0] for c in CASES])
def test_pins_catch_planted_mistake(name, pins, tmp_path):
    src = open(SRC).read()
    old, new = {**MUTATIONS, **GRAD_MUTATIONS}[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutated = tmp_path / "mut.cpp"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                           "-o", str(lib), str(mutated)])
    env = dict(os.environ, GS_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"no pin caught mutation {name}:\n{r.stdout[-2000:]}"
