// gs_oracle.cpp — plain FP64 CPU reference of the 3D Gaussian Splatting
// forward rasterizer (and, further down, its analytic gradients).
//
// TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU
// baseline leg of the benchmark may load this library. The product path (the
// CUDA library) shares no code, header, table or constant with it.
//
// What it computes, with the passage each step follows:
//   * Gaussian model: mean, covariance Sigma = R S S^T R^T with R from a unit
//     quaternion and S diagonal, opacity, SH colour (Sec. 3.1).
//   * Projection to a 2D mean, conic Q (inverse 2D covariance) and a square
//     bound of three standard deviations of the larger eigenvalue of the 2D
//     covariance (Sec. 3.1 stage 2; Sec. 4.4).
//   * Culling of Gaussians behind the near plane (Sec. 4.5, step 1).
//   * Depth ordering per screen tile (Sec. 3.1 stage 3; Sec. 4.5 step 2).
//   * Front-to-back alpha compositing, Eq. 1 (Sec. 3.1; Sec. 4.5 step 3).
// The paper gives no numeric constants; the readings used here are the ones of
// the standard 3DGS formulation it cites: +0.3 on the 2D covariance diagonal,
// alpha = min(0.99, o * exp(power)), skip alpha < 1/255, stop before a
// Gaussian that would take transmittance below 1e-4, near plane at the
// camera's near_z, Jacobian formed at view ratios clamped to 1.3 tan(fov/2).
//
// Everything is double precision and written for clarity, not speed: loops
// over Gaussians, tiles and pixels, a library sort for the depth order, and
// OpenMP only to spread independent tiles / Gaussians over cores.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <tuple>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------------------
// Camera: world_to_cam = [R | t] (3x4, row-major), pinhole intrinsics.
// Layout of the flat array: the 3x4 matrix row by row, then fx, fy, cx, cy,
// near_z.
// ---------------------------------------------------------------------------
struct Cam {
    double R[3][3];
    double t[3];
    double fx, fy, cx, cy, near_z;
    int width, height;
};

Cam make_cam(const double *c, int width, int height) {
    Cam k;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) k.R[i][j] = c[4 * i + j];
        k.t[i] = c[4 * i + 3];
    }
    k.fx = c[12];
    k.fy = c[13];
    k.cx = c[14];
    k.cy = c[15];
    k.near_z = c[16];
    k.width = width;
    k.height = height;
    return k;
}

// ---------------------------------------------------------------------------
// Real spherical harmonics from their definition.
//   P_l(x)      = 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l) x^(l-2k)      (explicit)
//   P_l^m(x)    = (-1)^m (1-x^2)^(m/2) d^m/dx^m P_l(x)  (Condon-Shortley phase)
//   K_l^m       = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
//   Y_l^0       = K_l^0 P_l(cos theta)
//   Y_l^m  (m>0)= sqrt(2) K_l^m cos(m phi) P_l^m(cos theta)
//   Y_l^-m (m>0)= sqrt(2) K_l^m sin(m phi) P_l^m(cos theta)
// with cos theta = z, phi = atan2(y, x), coefficient index k = l^2 + l + m.
// ---------------------------------------------------------------------------
double factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

double binomial(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    return factorial(n) / (factorial(k) * factorial(n - k));
}

// Coefficients c[p] of P_l(x) = sum_p c[p] x^p.
std::vector<double> legendre_poly(int l) {
    std::vector<double> c(l + 1, 0.0);
    for (int k = 0; 2 * k <= l; ++k) {
        double v = std::pow(-1.0, k) * binomial(l, k) * binomial(2 * l - 2 * k, l) / std::pow(2.0, l);
        c[l - 2 * k] += v;
    }
    return c;
}

double assoc_legendre(int l, int m, double x) {
    std::vector<double> c = legendre_poly(l);
    // m-th derivative of the polynomial.
    for (int d = 0; d < m; ++d) {
        std::vector<double> dc(std::max<size_t>(1, c.size() - 1), 0.0);
        for (size_t p = 1; p < c.size(); ++p) dc[p - 1] = p * c[p];
        c = dc;
    }
    double poly = 0.0;
    for (size_t p = 0; p < c.size(); ++p) poly += c[p] * std::pow(x, (double)p);
    double s = std::pow(std::max(0.0, 1.0 - x * x), 0.5 * m);
    return std::pow(-1.0, m) * s * poly;
}

double real_sh(int l, int m, const double d[3]) {
    int am = m < 0 ? -m : m;
    double ct = d[2];
    double phi = std::atan2(d[1], d[0]);
    double K = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * factorial(l - am) / factorial(l + am));
    double P = assoc_legendre(l, am, ct);
    if (m == 0) return K * P;
    if (m > 0) return std::sqrt(2.0) * K * std::cos(am * phi) * P;
    return std::sqrt(2.0) * K * std::sin(am * phi) * P;
}

// ---------------------------------------------------------------------------
// Small dense helpers.
// ---------------------------------------------------------------------------
void matmul3(const double A[3][3], const double B[3][3], double C[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
            C[i][j] = s;
        }
}

void transpose3(const double A[3][3], double B[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B[i][j] = A[j][i];
}

// Rotation matrix of the unit quaternion (w, x, y, z) (normalised here).
void quat_to_rot(const double q_in[4], double R[3][3]) {
    double n = std::sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0][0] = 1 - 2 * (y * y + z * z);
    R[0][1] = 2 * (x * y - w * z);
    R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);
    R[1][1] = 1 - 2 * (x * x + z * z);
    R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);
    R[2][1] = 2 * (y * z + w * x);
    R[2][2] = 1 - 2 * (x * x + y * y);
}

// Floor division of a real by the tile size, clamped to [0, limit].
int64_t tile_coord(double v, int tile, int64_t limit) {
    double f = std::floor(v / tile);
    if (f < 0) return 0;
    if (f > (double)limit) return limit;
    return (int64_t)f;
}

// Tile rectangle of a Gaussian with pixel-coordinate mean (u, v) and integer
// radius r: columns [floor((u-r)/tw), floor((u+r+tw-1)/tw)), rows likewise,
// clamped to the tile grid (the square 3-sigma bound of Sec. 4.4, in tiles).
void tile_rect(double u, double v, int64_t r, int tw, int th, int64_t tiles_x, int64_t tiles_y,
               int64_t rect[4]) {
    rect[0] = tile_coord(u - (double)r, tw, tiles_x);
    rect[1] = tile_coord(v - (double)r, th, tiles_y);
    rect[2] = tile_coord(u + (double)r + (tw - 1), tw, tiles_x);
    rect[3] = tile_coord(v + (double)r + (th - 1), th, tiles_y);
}

uint32_t f32_bits(double d) {
    float f = (float)d;
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return b;
}

const double kDilation = 0.3;        // added to the 2D covariance diagonal
const double kAlphaMax = 0.99;       // opacity clamp
const double kAlphaMin = 1.0 / 255;  // contributions below are skipped
const double kTMin = 1e-4;           // transmittance at which a pixel stops
const double kGuard = 1.3;           // Jacobian view-ratio clamp, x tan(fov/2)

// Front-to-back compositing of one pixel over an ordered candidate list
// (Eq. 1 with the standard clamp / skip / stop rules). pix = pixel centre.
// Returns the final transmittance; writes colour, the 1-based list position
// of the last Gaussian blended (0 if none), the number of list entries
// evaluated (up to and including the one that stopped the pixel), and a flag
// set when an alpha or a transmittance decision fell within 1e-6 of its cutoff.
struct PixelOut {
    double c[3];
    double T;
    int32_t last;
    int32_t neval;
    uint8_t flag;
};

template <class GetIdx>
PixelOut blend_pixel(double px, double py, int64_t count, GetIdx idx, const double *mean2d,
                     const double *conic, const double *opacity, const double *rgb) {
    PixelOut o = {{0, 0, 0}, 1.0, 0, 0, 0};
    double T = 1.0;
    for (int64_t k = 0; k < count; ++k) {
        int64_t g = idx(k);
        o.neval = (int32_t)(k + 1);
        double dx = px - mean2d[2 * g], dy = py - mean2d[2 * g + 1];
        double power = -0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) - conic[3 * g + 1] * dx * dy;
        if (power > 0.0) continue;
        double alpha = std::min(kAlphaMax, opacity[g] * std::exp(power));
        if (std::fabs(alpha - kAlphaMin) < 1e-6) o.flag = 1;
        if (alpha < kAlphaMin) continue;
        double Tn = T * (1.0 - alpha);
        if (std::fabs(Tn - kTMin) < 1e-6) o.flag = 1;
        if (Tn < kTMin) break;
        for (int ch = 0; ch < 3; ++ch) o.c[ch] += rgb[3 * g + ch] * alpha * T;
        T = Tn;
        o.last = (int32_t)(k + 1);
    }
    o.T = T;
    return o;
}

}  // namespace

extern "C" {

int gso_num_threads(int set) {
#ifdef _OPENMP
    if (set > 0) omp_set_num_threads(set);
    return omp_get_max_threads();
#else
    (void)set;
    return 1;
#endif
}

// Y_k(d) for every coefficient k < (deg+1)^2 and each unit direction.
void gso_sh_basis(int32_t deg, int64_t n, const double *dirs, double *out) {
    int K = (deg + 1) * (deg + 1);
    for (int64_t i = 0; i < n; ++i)
        for (int l = 0; l <= deg; ++l)
            for (int m = -l; m <= l; ++m) out[i * K + l * l + l + m] = real_sh(l, m, dirs + 3 * i);
}

// Projection of every Gaussian (Sec. 3.1 stage 2, Sec. 4.4, Sec. 4.5 step 1).
// Outputs per Gaussian: mean2d (u,v) in pixels with pixel centres at +0.5,
// conic (Q00, Q01, Q11), opacity, rgb, depth (camera z), extent = 3 sqrt(lambda_max)
// before rounding, radius = ceil(extent), rect (x0, y0, x1, y1) in tiles,
// visible. Returns the number of visible Gaussians.
int64_t gso_project(int64_t n, const double *means, const double *log_scales, const double *quats,
                    const double *opacity_logits, const double *sh, int32_t sh_degree,
                    const double *cam_flat, int32_t width, int32_t height, int32_t tile_w,
                    int32_t tile_h, double *mean2d, double *conic, double *opacity, double *rgb,
                    double *depth, double *extent, int64_t *radius, int64_t *rect,
                    int32_t *visible) {
    const Cam cam = make_cam(cam_flat, width, height);
    const int64_t tiles_x = (width + tile_w - 1) / tile_w;
    const int64_t tiles_y = (height + tile_h - 1) / tile_h;
    const int K = (sh_degree + 1) * (sh_degree + 1);
    // Camera centre C = -R^T t.
    double C[3];
    for (int i = 0; i < 3; ++i) C[i] = -(cam.R[0][i] * cam.t[0] + cam.R[1][i] * cam.t[1] + cam.R[2][i] * cam.t[2]);
    const double tan_x = 0.5 * width / cam.fx, tan_y = 0.5 * height / cam.fy;
    int64_t count = 0;
#pragma omp parallel for schedule(static) reduction(+ : count)
    for (int64_t i = 0; i < n; ++i) {
        visible[i] = 0;
        radius[i] = 0;
        for (int j = 0; j < 4; ++j) rect[4 * i + j] = 0;
        mean2d[2 * i] = mean2d[2 * i + 1] = 0;
        conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0;
        opacity[i] = 0;
        rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = 0;
        extent[i] = 0;
        const double *mu = means + 3 * i;
        double t[3];
        for (int r = 0; r < 3; ++r) t[r] = cam.R[r][0] * mu[0] + cam.R[r][1] * mu[1] + cam.R[r][2] * mu[2] + cam.t[r];
        depth[i] = t[2];
        if (!(t[2] > cam.near_z)) continue;  // behind the near plane

        // 3D covariance Sigma = (R S)(R S)^T.
        double Rq[3][3], M[3][3], Mt[3][3], Sigma[3][3];
        quat_to_rot(quats + 4 * i, Rq);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) M[r][c] = Rq[r][c] * std::exp(log_scales[3 * i + c]);
        transpose3(M, Mt);
        matmul3(M, Mt, Sigma);

        // Camera-space covariance W Sigma W^T, W the world-to-camera rotation.
        double Wt[3][3], tmp[3][3], Sc[3][3];
        transpose3(cam.R, Wt);
        matmul3(cam.R, Sigma, tmp);
        matmul3(tmp, Wt, Sc);

        // Jacobian of the perspective map at the (guard-band clamped) point.
        double rx = std::min(kGuard * tan_x, std::max(-kGuard * tan_x, t[0] / t[2]));
        double ry = std::min(kGuard * tan_y, std::max(-kGuard * tan_y, t[1] / t[2]));
        double J[2][3] = {{cam.fx / t[2], 0.0, -cam.fx * rx / t[2]},
                          {0.0, cam.fy / t[2], -cam.fy * ry / t[2]}};
        double cov[2][2];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) s += J[a][k] * Sc[k][l] * J[b][l];
                cov[a][b] = s;
            }
        cov[0][0] += kDilation;
        cov[1][1] += kDilation;

        double det = cov[0][0] * cov[1][1] - cov[0][1] * cov[1][0];
        if (!(det > 0.0)) continue;
        double Q00 = cov[1][1] / det, Q01 = -cov[0][1] / det, Q11 = cov[0][0] / det;

        // Larger eigenvalue; radius = ceil(3 sqrt(lambda_max)) (Sec. 4.4).
        double mid = 0.5 * (cov[0][0] + cov[1][1]);
        double lam = mid + std::sqrt(std::max(0.1, mid * mid - det));
        double ext = 3.0 * std::sqrt(lam);
        int64_t r = (int64_t)std::ceil(ext);

        double u = cam.fx * t[0] / t[2] + cam.cx;
        double v = cam.fy * t[1] / t[2] + cam.cy;
        int64_t rc[4];
        tile_rect(u, v, r, tile_w, tile_h, tiles_x, tiles_y, rc);
        extent[i] = ext;
        mean2d[2 * i] = u;
        mean2d[2 * i + 1] = v;
        conic[3 * i] = Q00;
        conic[3 * i + 1] = Q01;
        conic[3 * i + 2] = Q11;
        if (r <= 0 || (rc[2] - rc[0]) * (rc[3] - rc[1]) <= 0) continue;

        // View-dependent colour from SH along the camera-to-mean direction.
        double d[3] = {mu[0] - C[0], mu[1] - C[1], mu[2] - C[2]};
        double dn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int k = 0; k < 3; ++k) d[k] /= dn;
        for (int ch = 0; ch < 3; ++ch) {
            double s = 0.0;
            for (int l = 0; l <= sh_degree; ++l)
                for (int m = -l; m <= l; ++m) s += sh[(i * K + l * l + l + m) * 3 + ch] * real_sh(l, m, d);
            rgb[3 * i + ch] = std::max(0.0, s + 0.5);
        }
        opacity[i] = 1.0 / (1.0 + std::exp(-opacity_logits[i]));
        radius[i] = r;
        for (int j = 0; j < 4; ++j) rect[4 * i + j] = rc[j];
        visible[i] = 1;
        count += 1;
    }
    return count;
}

// Number of (tile, Gaussian) pairs: the sum of the visible rect areas.
int64_t gso_bin_count(int64_t n, const double *mean2d, const int64_t *radius, const int32_t *visible,
                      int32_t width, int32_t height, int32_t tile_w, int32_t tile_h) {
    const int64_t tiles_x = (width + tile_w - 1) / tile_w;
    const int64_t tiles_y = (height + tile_h - 1) / tile_h;
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!visible[i]) continue;
        int64_t rc[4];
        tile_rect(mean2d[2 * i], mean2d[2 * i + 1], radius[i], tile_w, tile_h, tiles_x, tiles_y, rc);
        k += (rc[2] - rc[0]) * (rc[3] - rc[1]);
    }
    return k;
}

// Per-tile depth-ordered lists. Every visible Gaussian is listed once in each
// tile of its rect; the list is ordered by (tile id, FP32 bits of depth,
// Gaussian index). keys[k] = tile << 32 | bits(depth), values[k] = index;
// ranges[2t], ranges[2t+1] = [first, last+1) of tile t, [0, 0) when empty.
void gso_bin(int64_t n, const double *mean2d, const int64_t *radius, const double *depth,
             const int32_t *visible, int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
             uint64_t *keys, uint32_t *values, uint32_t *ranges) {
    const int64_t tiles_x = (width + tile_w - 1) / tile_w;
    const int64_t tiles_y = (height + tile_h - 1) / tile_h;
    std::vector<std::tuple<int64_t, uint32_t, int64_t>> items;
    for (int64_t i = 0; i < n; ++i) {
        if (!visible[i]) continue;
        int64_t rc[4];
        tile_rect(mean2d[2 * i], mean2d[2 * i + 1], radius[i], tile_w, tile_h, tiles_x, tiles_y, rc);
        for (int64_t ty = rc[1]; ty < rc[3]; ++ty)
            for (int64_t tx = rc[0]; tx < rc[2]; ++tx)
                items.emplace_back(ty * tiles_x + tx, f32_bits(depth[i]), i);
    }
    std::sort(items.begin(), items.end());
    for (int64_t t = 0; t < tiles_x * tiles_y; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
    for (size_t k = 0; k < items.size(); ++k) {
        int64_t tile = std::get<0>(items[k]);
        keys[k] = ((uint64_t)tile << 32) | std::get<1>(items[k]);
        values[k] = (uint32_t)std::get<2>(items[k]);
        if (k == 0 || std::get<0>(items[k - 1]) != tile) ranges[2 * tile] = (uint32_t)k;
        ranges[2 * tile + 1] = (uint32_t)(k + 1);
    }
}

// Tile-ordered blend (Sec. 4.5 step 3): every pixel of tile t walks the
// tile's list values[ranges[2t] .. ranges[2t+1]). Output images are HWC.
void gso_blend(int64_t n, const double *mean2d, const double *conic, const double *opacity,
               const double *rgb, const uint32_t *values, const uint32_t *ranges, int32_t width,
               int32_t height, int32_t tile_w, int32_t tile_h, const double *bg, double *out_rgb,
               double *out_T, int32_t *out_last, int32_t *out_neval, uint8_t *out_flag) {
    (void)n;
    const int64_t tiles_x = (width + tile_w - 1) / tile_w;
    const int64_t tiles_y = (height + tile_h - 1) / tile_h;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < tiles_x * tiles_y; ++t) {
        int64_t tx = t % tiles_x, ty = t / tiles_x;
        int64_t first = ranges[2 * t], last = ranges[2 * t + 1];
        for (int64_t y = ty * tile_h; y < std::min<int64_t>(height, (ty + 1) * tile_h); ++y)
            for (int64_t x = tx * tile_w; x < std::min<int64_t>(width, (tx + 1) * tile_w); ++x) {
                PixelOut o = blend_pixel(
                    x + 0.5, y + 0.5, last - first, [&](int64_t k) { return (int64_t)values[first + k]; },
                    mean2d, conic, opacity, rgb);
                int64_t p = y * width + x;
                for (int ch = 0; ch < 3; ++ch) out_rgb[3 * p + ch] = o.c[ch] + o.T * bg[ch];
                out_T[p] = o.T;
                out_last[p] = o.last;
                out_neval[p] = o.neval;
                out_flag[p] = o.flag;
            }
    }
}

// Brute force: one global order of all visible Gaussians by (FP32 depth bits,
// index); every pixel walks that order keeping only Gaussians whose rect
// contains the pixel's tile. Must equal gso_blend on gso_bin's lists.
void gso_blend_bruteforce(int64_t n, const double *mean2d, const double *conic, const double *opacity,
                          const double *rgb, const double *depth, const int64_t *radius,
                          const int32_t *visible, int32_t width, int32_t height, int32_t tile_w,
                          int32_t tile_h, const double *bg, double *out_rgb, double *out_T,
                          int32_t *out_last, int32_t *out_neval, uint8_t *out_flag) {
    const int64_t tiles_x = (width + tile_w - 1) / tile_w;
    const int64_t tiles_y = (height + tile_h - 1) / tile_h;
    std::vector<std::pair<uint32_t, int64_t>> order;
    for (int64_t i = 0; i < n; ++i)
        if (visible[i]) order.emplace_back(f32_bits(depth[i]), i);
    std::sort(order.begin(), order.end());
    std::vector<int64_t> rects(4 * order.size());
    for (size_t k = 0; k < order.size(); ++k) {
        int64_t i = order[k].second;
        tile_rect(mean2d[2 * i], mean2d[2 * i + 1], radius[i], tile_w, tile_h, tiles_x, tiles_y, &rects[4 * k]);
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t p = 0; p < (int64_t)width * height; ++p) {
        int64_t x = p % width, y = p / width;
        int64_t tx = x / tile_w, ty = y / tile_h;
        std::vector<int64_t> cand;
        for (size_t k = 0; k < order.size(); ++k) {
            const int64_t *rc = &rects[4 * k];
            if (tx >= rc[0] && tx < rc[2] && ty >= rc[1] && ty < rc[3]) cand.push_back(order[k].second);
        }
        PixelOut o = blend_pixel(x + 0.5, y + 0.5, (int64_t)cand.size(), [&](int64_t k) { return cand[k]; },
                                 mean2d, conic, opacity, rgb);
        for (int ch = 0; ch < 3; ++ch) out_rgb[3 * p + ch] = o.c[ch] + o.T * bg[ch];
        out_T[p] = o.T;
        out_last[p] = o.last;
        out_neval[p] = o.neval;
        out_flag[p] = o.flag;
    }
}

}  // extern "C"
