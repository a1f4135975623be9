"""FP64 CPU oracle of the 3D Gaussian Splatting forward rasterizer.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package. It shares no code with
the CUDA library and imports nothing from it.

The arithmetic lives in ``gs_oracle.cpp`` (double precision, plain loops);
this module compiles it with the host C++ compiler and marshals numpy arrays
through ctypes. Each function cites the passage of the paper it follows:

* ``sh_basis``            — real SH basis Y_lm from the Legendre definition
                            (view-dependent colour, Sec. 3.1).
* ``project``             — Sec. 3.1 stages 1-2 and the 3-sigma square bound
                            of Sec. 4.4; near-plane cull of Sec. 4.5 step 1.
* ``bin_tiles``           — per-tile depth order (Sec. 3.1 stage 3, Sec. 4.5
                            step 2) as sorted (tile, depth) keys and ranges.
* ``blend``               — Eq. 1 per pixel over each tile's ordered list
                            (Sec. 4.5 step 3).
* ``blend_bruteforce``    — Eq. 1 over one global depth order, filtered per
                            pixel by tile coverage; equals ``blend``.
* ``render``              — project -> bin -> blend.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.cpp")
_LIB = os.path.join(_HERE, "libgs_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``libgs_oracle.so`` (g++, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        # GS_ORACLE_LIB points the tests at a deliberately mutated copy of the
        # oracle (tests/test_oracle_mutations.py); normally unset.
        path = os.environ.get("GS_ORACLE_LIB") or build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        L.gso_num_threads.argtypes = [ctypes.c_int]
        L.gso_num_threads.restype = ctypes.c_int
        L.gso_sh_basis.argtypes = [i32, i64, P, P]
        L.gso_sh_basis.restype = None
        L.gso_project.argtypes = [i64, P, P, P, P, P, i32, P, i32, i32, i32, i32] + [P] * 9
        L.gso_project.restype = i64
        L.gso_bin_count.argtypes = [i64, P, P, P, i32, i32, i32, i32]
        L.gso_bin_count.restype = i64
        L.gso_bin.argtypes = [i64, P, P, P, P, i32, i32, i32, i32, P, P, P]
        L.gso_bin.restype = None
        L.gso_blend.argtypes = [i64, P, P, P, P, P, P, i32, i32, i32, i32, P, P, P, P, P, P]
        L.gso_blend.restype = None
        L.gso_blend_bruteforce.argtypes = [i64, P, P, P, P, P, P, P, i32, i32, i32, i32,
                                           P, P, P, P, P, P]
        L.gso_blend_bruteforce.restype = None
        L.gso_render_backward.argtypes = [i64, P, P, P, P, P, i32, P, i32, i32, i32, i32, P, P,
                                          P, P, P, P, P, P]
        L.gso_render_backward.restype = None
        _lib = L
    return _lib


def num_threads(set_to: int = 0) -> int:
    """OpenMP threads the oracle uses (``set_to`` > 0 changes it)."""
    return int(lib().gso_num_threads(int(set_to)))


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def camera_flat(world_to_cam, fx, fy, cx, cy, near_z) -> np.ndarray:
    w2c = _f64(world_to_cam).reshape(12)
    return _f64(np.concatenate([w2c, [fx, fy, cx, cy, near_z]]))


def _cam(cam) -> tuple[np.ndarray, int, int]:
    """Accept any object with world_to_cam/fx/fy/cx/cy/width/height/near_z."""
    return (camera_flat(cam.world_to_cam, cam.fx, cam.fy, cam.cx, cam.cy, cam.near_z),
            int(cam.width), int(cam.height))


# ---------------------------------------------------------------------------
# Spherical harmonics
# ---------------------------------------------------------------------------

def sh_basis(degree: int, dirs) -> np.ndarray:
    """Y_k(d) for k < (degree+1)^2; ``dirs`` (n,3) unit vectors."""
    d = _f64(dirs).reshape(-1, 3)
    out = np.zeros((d.shape[0], (degree + 1) ** 2), np.float64)
    lib().gso_sh_basis(int(degree), d.shape[0], _p(d), _p(out))
    return out


# ---------------------------------------------------------------------------
# Projection
# ---------------------------------------------------------------------------

@dataclass
class Projected:
    mean2d: np.ndarray    # (n,2) pixel coordinates, pixel centres at +0.5
    conic: np.ndarray     # (n,3) (Q00, Q01, Q11) of the inverse 2D covariance
    opacity: np.ndarray   # (n,)
    rgb: np.ndarray       # (n,3)
    depth: np.ndarray     # (n,) camera-space z
    extent: np.ndarray    # (n,) 3 sqrt(lambda_max) before rounding up
    radius: np.ndarray    # (n,) int64
    rect: np.ndarray      # (n,4) int64 tile rect (x0, y0, x1, y1), half-open
    visible: np.ndarray   # (n,) int32

    @property
    def n(self):
        return int(self.depth.shape[0])


def project(scene, cam, tile_w: int = 16, tile_h: int = 16) -> Projected:
    """Sec. 3.1 stages 1-2, Sec. 4.4 bound, Sec. 4.5 near cull, in FP64."""
    n = int(np.asarray(scene.means).shape[0])
    means = _f64(scene.means)
    ls = _f64(scene.log_scales)
    q = _f64(scene.quats)
    lo = _f64(scene.opacity_logits)
    sh = _f64(scene.sh)
    cf, w, h = _cam(cam)
    out = Projected(np.zeros((n, 2)), np.zeros((n, 3)), np.zeros(n), np.zeros((n, 3)),
                    np.zeros(n), np.zeros(n), np.zeros(n, np.int64),
                    np.zeros((n, 4), np.int64), np.zeros(n, np.int32))
    lib().gso_project(n, _p(means), _p(ls), _p(q), _p(lo), _p(sh), int(scene.sh_degree),
                      _p(cf), w, h, tile_w, tile_h, _p(out.mean2d), _p(out.conic),
                      _p(out.opacity), _p(out.rgb), _p(out.depth), _p(out.extent),
                      _p(out.radius), _p(out.rect), _p(out.visible))
    return out


# ---------------------------------------------------------------------------
# Binning
# ---------------------------------------------------------------------------

@dataclass
class Binned:
    keys: np.ndarray     # (K,) uint64: tile << 32 | FP32 bits of depth
    values: np.ndarray   # (K,) uint32 Gaussian index
    ranges: np.ndarray   # (tiles, 2) uint32 [first, last+1)


def bin_tiles(mean2d, radius, depth, visible, width, height, tile_w=16, tile_h=16) -> Binned:
    """Per-tile ordered lists (Sec. 3.1 stage 3; Sec. 4.5 step 2)."""
    m = _f64(mean2d).reshape(-1, 2)
    n = m.shape[0]
    r = np.ascontiguousarray(np.asarray(radius, dtype=np.int64))
    d = _f64(depth)
    v = np.ascontiguousarray(np.asarray(visible, dtype=np.int32))
    K = int(lib().gso_bin_count(n, _p(m), _p(r), _p(v), width, height, tile_w, tile_h))
    tiles = ((width + tile_w - 1) // tile_w) * ((height + tile_h - 1) // tile_h)
    keys = np.zeros(max(K, 1), np.uint64)
    vals = np.zeros(max(K, 1), np.uint32)
    ranges = np.zeros((tiles, 2), np.uint32)
    lib().gso_bin(n, _p(m), _p(r), _p(d), _p(v), width, height, tile_w, tile_h,
                  _p(keys), _p(vals), _p(ranges))
    return Binned(keys[:K], vals[:K], ranges)


# ---------------------------------------------------------------------------
# Blending
# ---------------------------------------------------------------------------

@dataclass
class Image:
    rgb: np.ndarray      # (H,W,3) float64
    T: np.ndarray        # (H,W) final transmittance
    last: np.ndarray     # (H,W) int32 1-based list position of the last blended Gaussian
    neval: np.ndarray    # (H,W) int32 list entries evaluated
    flag: np.ndarray     # (H,W) uint8 alpha or T decision within 1e-6 of its cutoff


def _image(h, w):
    return Image(np.zeros((h, w, 3)), np.zeros((h, w)), np.zeros((h, w), np.int32),
                 np.zeros((h, w), np.int32), np.zeros((h, w), np.uint8))


def blend(mean2d, conic, opacity, rgb, values, ranges, width, height, tile_w=16, tile_h=16,
          bg=(0.0, 0.0, 0.0)) -> Image:
    """Eq. 1 per pixel over each tile's ordered list (Sec. 4.5 step 3)."""
    m, c, o, col = _f64(mean2d), _f64(conic), _f64(opacity), _f64(rgb)
    vals = np.ascontiguousarray(np.asarray(values, dtype=np.uint32))
    if vals.size == 0:
        vals = np.zeros(1, np.uint32)
    rg = np.ascontiguousarray(np.asarray(ranges, dtype=np.uint32))
    b = _f64(bg)
    img = _image(height, width)
    lib().gso_blend(m.shape[0], _p(m), _p(c), _p(o), _p(col), _p(vals), _p(rg), width, height,
                    tile_w, tile_h, _p(b), _p(img.rgb), _p(img.T), _p(img.last), _p(img.neval),
                    _p(img.flag))
    return img


def blend_bruteforce(mean2d, conic, opacity, rgb, depth, radius, visible, width, height,
                     tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0)) -> Image:
    """Eq. 1 per pixel over one global depth order filtered by tile coverage."""
    m, c, o, col, d = _f64(mean2d), _f64(conic), _f64(opacity), _f64(rgb), _f64(depth)
    r = np.ascontiguousarray(np.asarray(radius, dtype=np.int64))
    v = np.ascontiguousarray(np.asarray(visible, dtype=np.int32))
    b = _f64(bg)
    img = _image(height, width)
    lib().gso_blend_bruteforce(m.shape[0], _p(m), _p(c), _p(o), _p(col), _p(d), _p(r), _p(v),
                               width, height, tile_w, tile_h, _p(b), _p(img.rgb), _p(img.T),
                               _p(img.last), _p(img.neval), _p(img.flag))
    return img


def render(scene, cam, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0)):
    """Full FP64 forward render: project -> bin -> blend."""
    pr = project(scene, cam, tile_w, tile_h)
    bn = bin_tiles(pr.mean2d, pr.radius, pr.depth, pr.visible, cam.width, cam.height,
                   tile_w, tile_h)
    img = blend(pr.mean2d, pr.conic, pr.opacity, pr.rgb, bn.values, bn.ranges,
                cam.width, cam.height, tile_w, tile_h, bg)
    return pr, bn, img


# ---------------------------------------------------------------------------
# Gradients
# ---------------------------------------------------------------------------

@dataclass
class Grads:
    means: np.ndarray          # (n,3)
    log_scales: np.ndarray     # (n,3)
    quats: np.ndarray          # (n,4)
    opacity_logits: np.ndarray # (n,)
    sh: np.ndarray             # (n,K,3)
    record: np.ndarray         # (n,9) dL/d(u, v, Q00, Q01, Q11, opacity, r, g, b)


def render_backward(scene, cam, dL_dC, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0)) -> Grads:
    """FP64 gradient of L = sum dL_dC * C with respect to every parameter:
    Eq. 1 differentiated per pixel over its contributors, the projection
    differentiated with dual numbers."""
    n = int(np.asarray(scene.means).shape[0])
    K = (int(scene.sh_degree) + 1) ** 2
    cf, w, h = _cam(cam)
    g = _f64(dL_dC).reshape(h, w, 3)
    out = Grads(np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 4)), np.zeros(n),
                np.zeros((n, K, 3)), np.zeros((n, 9)))
    arrs = [_f64(scene.means), _f64(scene.log_scales), _f64(scene.quats),
            _f64(scene.opacity_logits), _f64(scene.sh)]
    b = _f64(bg)
    lib().gso_render_backward(n, *[_p(a) for a in arrs], int(scene.sh_degree), _p(cf), w, h,
                              tile_w, tile_h, _p(b), _p(g), _p(out.means), _p(out.log_scales),
                              _p(out.quats), _p(out.opacity_logits), _p(out.sh), _p(out.record))
    return out
