// gs_project.cu — per-Gaussian projection (Sec. 3.1 stages 1-2; the square
// 3-sigma bound of Sec. 4.4; the near-plane cull of Sec. 4.5 step 1).
//
// One thread per Gaussian. Every thread reads the 12-byte mean; only
// Gaussians in front of the near plane go on to read scale, rotation,
// opacity and SH, so the HBM traffic of a mostly-culled scene is ~16 B per
// Gaussian (mean in, tile count out) plus ~250 B per visible one.
//
// Numerics, all FP32:
//  * 2D covariance as (T M)(T M)^T with T = J W (2x3) and M = R(q) S, so the
//    result is positive semi-definite by construction;
//  * det = |A0 x A1|^2 + 0.3 (a0 + c0) + 0.09 (Lagrange's identity for
//    a0 c0 - b^2), which avoids the cancellation of a c - b^2;
//  * lambda_max = mid + sqrt(max(0.1, ((a - c)/2)^2 + b^2)), the same value as
//    mid + sqrt(max(0.1, mid^2 - det)) without its cancellation.
#include "gs_internal.cuh"

namespace {

using namespace gs;

// Real SH basis with the Condon-Shortley phase written as polynomials in the
// unit direction (x, y, z); coefficient k = l^2 + l + m. Each constant is
// the closed form of sqrt(2) K_l^|m| times the leading factor of P_l^|m|:
constexpr float kY00 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;    // sqrt(3 / (4 pi))
constexpr float kY2a = 1.0925484305920792f;    // sqrt(15 / (4 pi))
constexpr float kY2b = 0.31539156525252005f;   // sqrt(5 / (16 pi))
constexpr float kY2c = 0.54627421529603959f;   // sqrt(15 / (16 pi))
constexpr float kY3a = 0.59004358992664352f;   // sqrt(35 / (32 pi))
constexpr float kY3b = 2.8906114426405538f;    // sqrt(105 / (4 pi))
constexpr float kY3c = 0.45704579946446572f;   // sqrt(21 / (32 pi))
constexpr float kY3d = 0.37317633259011540f;   // sqrt(7 / (16 pi))
constexpr float kY3e = 1.4453057213202769f;    // sqrt(105 / (16 pi))

template <int DEG>
__device__ __forceinline__ float3 sh_colour(const float *__restrict__ c, float x, float y, float z) {
    // c points at this Gaussian's (DEG+1)^2 x 3 coefficients.
    auto C = [&](int k, float w, float3 acc) {
        acc.x = fmaf(w, __ldg(c + 3 * k + 0), acc.x);
        acc.y = fmaf(w, __ldg(c + 3 * k + 1), acc.y);
        acc.z = fmaf(w, __ldg(c + 3 * k + 2), acc.z);
        return acc;
    };
    float3 s = make_float3(0.f, 0.f, 0.f);
    s = C(0, kY00, s);
    if (DEG >= 1) {
        s = C(1, -kY1 * y, s);
        s = C(2, kY1 * z, s);
        s = C(3, -kY1 * x, s);
    }
    if (DEG >= 2) {
        float xx = x * x, yy = y * y, zz = z * z;
        s = C(4, kY2a * x * y, s);
        s = C(5, -kY2a * y * z, s);
        s = C(6, kY2b * (2.f * zz - xx - yy), s);
        s = C(7, -kY2a * x * z, s);
        s = C(8, kY2c * (xx - yy), s);
        if (DEG >= 3) {
            s = C(9, -kY3a * y * (3.f * xx - yy), s);
            s = C(10, kY3b * x * y * z, s);
            s = C(11, -kY3c * y * (4.f * zz - xx - yy), s);
            s = C(12, kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy), s);
            s = C(13, -kY3c * x * (4.f * zz - xx - yy), s);
            s = C(14, kY3e * z * (xx - yy), s);
            s = C(15, -kY3a * x * (xx - 3.f * yy), s);
        }
    }
    return make_float3(fmaxf(s.x + 0.5f, 0.f), fmaxf(s.y + 0.5f, 0.f), fmaxf(s.z + 0.5f, 0.f));
}

struct ProjectArgs {
    const float *means, *log_scales, *quats, *logits, *sh;
    int64_t n;
    GsCameraDev cam;
    GsGrid grid;
    float4 *records;
    uint32_t *tiles;
};

template <int DEG>
__global__ void __launch_bounds__(256) project_kernel(const ProjectArgs P) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const GsCameraDev &K = P.cam;
    const float mx = __ldg(P.means + 3 * i), my = __ldg(P.means + 3 * i + 1),
                mz = __ldg(P.means + 3 * i + 2);
    const float tx = fmaf(K.R[0], mx, fmaf(K.R[1], my, fmaf(K.R[2], mz, K.t[0])));
    const float ty = fmaf(K.R[3], mx, fmaf(K.R[4], my, fmaf(K.R[5], mz, K.t[1])));
    const float tz = fmaf(K.R[6], mx, fmaf(K.R[7], my, fmaf(K.R[8], mz, K.t[2])));
    if (!(tz > K.near_z)) {
        P.tiles[i] = 0;
        return;
    }

    // Rotation of the normalised quaternion (w, x, y, z), scaled columns M = R S.
    float qw = __ldg(P.quats + 4 * i), qx = __ldg(P.quats + 4 * i + 1),
          qy = __ldg(P.quats + 4 * i + 2), qz = __ldg(P.quats + 4 * i + 3);
    const float qinv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= qinv; qx *= qinv; qy *= qinv; qz *= qinv;
    const float sx = expf(__ldg(P.log_scales + 3 * i)), sy = expf(__ldg(P.log_scales + 3 * i + 1)),
                sz = expf(__ldg(P.log_scales + 3 * i + 2));
    float M[3][3];
    M[0][0] = (1.f - 2.f * (qy * qy + qz * qz)) * sx;
    M[0][1] = 2.f * (qx * qy - qw * qz) * sy;
    M[0][2] = 2.f * (qx * qz + qw * qy) * sz;
    M[1][0] = 2.f * (qx * qy + qw * qz) * sx;
    M[1][1] = (1.f - 2.f * (qx * qx + qz * qz)) * sy;
    M[1][2] = 2.f * (qy * qz - qw * qx) * sz;
    M[2][0] = 2.f * (qx * qz - qw * qy) * sx;
    M[2][1] = 2.f * (qy * qz + qw * qx) * sy;
    M[2][2] = (1.f - 2.f * (qx * qx + qy * qy)) * sz;

    // T = J W: rows (fx/tz)(W0 - rx W2), (fy/tz)(W1 - ry W2) with the view
    // ratios clamped to the guard band when forming J.
    const float iz = 1.f / tz;
    const float rx = fminf(K.lim_x, fmaxf(-K.lim_x, tx * iz));
    const float ry = fminf(K.lim_y, fmaxf(-K.lim_y, ty * iz));
    const float fxz = K.fx * iz, fyz = K.fy * iz;
    float T0[3], T1[3];
    for (int c = 0; c < 3; ++c) {
        T0[c] = fxz * fmaf(-rx, K.R[6 + c], K.R[c]);
        T1[c] = fyz * fmaf(-ry, K.R[6 + c], K.R[3 + c]);
    }
    // A = T M (2x3); cov2d = A A^T + 0.3 I.
    float A0[3], A1[3];
    for (int c = 0; c < 3; ++c) {
        A0[c] = fmaf(T0[0], M[0][c], fmaf(T0[1], M[1][c], T0[2] * M[2][c]));
        A1[c] = fmaf(T1[0], M[0][c], fmaf(T1[1], M[1][c], T1[2] * M[2][c]));
    }
    const float a0 = fmaf(A0[0], A0[0], fmaf(A0[1], A0[1], A0[2] * A0[2]));
    const float c0 = fmaf(A1[0], A1[0], fmaf(A1[1], A1[1], A1[2] * A1[2]));
    const float b = fmaf(A0[0], A1[0], fmaf(A0[1], A1[1], A0[2] * A1[2]));
    const float cr0 = A0[1] * A1[2] - A0[2] * A1[1];
    const float cr1 = A0[2] * A1[0] - A0[0] * A1[2];
    const float cr2 = A0[0] * A1[1] - A0[1] * A1[0];
    const float a = a0 + kDilation, c = c0 + kDilation;
    const float det = fmaf(cr0, cr0, fmaf(cr1, cr1, cr2 * cr2)) + kDilation * (a0 + c0) +
                      kDilation * kDilation;
    const float u = fmaf(K.fx * tx, iz, K.cx);
    const float v = fmaf(K.fy * ty, iz, K.cy);
    const float half_diff = 0.5f * (a - c);
    const float lam = 0.5f * (a + c) + sqrtf(fmaxf(0.1f, fmaf(half_diff, half_diff, b * b)));
    const float ext = 3.f * sqrtf(lam);
    if (!(det > 0.f) || !isfinite(u) || !isfinite(v) || !isfinite(ext)) {
        P.tiles[i] = 0;
        return;
    }
    const int r = ext >= (float)kMaxRadius ? kMaxRadius : (int)ceilf(ext);
    const Rect R = tile_rect(u, v, r, P.grid.tile_w, P.grid.tile_h, P.grid.tiles_x, P.grid.tiles_y);
    const uint32_t ntiles = (uint32_t)((R.x1 - R.x0) * (R.y1 - R.y0));
    P.tiles[i] = r > 0 ? ntiles : 0u;
    if (ntiles == 0 || r <= 0) return;
    const float idet = 1.f / det;

    // View direction from the camera centre to the mean.
    float dx = mx - K.C[0], dy = my - K.C[1], dz = mz - K.C[2];
    const float dinv = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= dinv; dy *= dinv; dz *= dinv;
    const float3 rgb = sh_colour<DEG>(P.sh + (size_t)i * (DEG + 1) * (DEG + 1) * 3, dx, dy, dz);
    const float opacity = 1.f / (1.f + expf(-__ldg(P.logits + i)));

    float4 *out = P.records + 3 * i;
    out[0] = make_float4(u, v, c * idet, -b * idet);
    out[1] = make_float4(a * idet, opacity, rgb.x, rgb.y);
    out[2] = make_float4(rgb.z, tz, __int_as_float(r), __uint_as_float(ntiles));
}

}  // namespace

cudaError_t gs_launch_project(const gs_gaussians &g, const GsCameraDev &cam, const GsGrid &grid,
                              gs_record *records, uint32_t *tiles, cudaStream_t s) {
    if (g.n == 0) return cudaSuccess;
    ProjectArgs a{g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, g.n, cam, grid,
                  reinterpret_cast<float4 *>(records), tiles};
    const int threads = 256;
    const unsigned blocks = (unsigned)((g.n + threads - 1) / threads);
    switch (g.sh_degree) {
        case 0: project_kernel<0><<<blocks, threads, 0, s>>>(a); break;
        case 1: project_kernel<1><<<blocks, threads, 0, s>>>(a); break;
        case 2: project_kernel<2><<<blocks, threads, 0, s>>>(a); break;
        default: project_kernel<3><<<blocks, threads, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}
