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
// Forward-mode dual numbers v + d eps (eps^2 = 0): evaluating a function on
// Dual(x, 1) gives its value and its exact derivative along x. The gradient
// code below differentiates the very same projection routine this way.
// ---------------------------------------------------------------------------
struct Dual {
    double v, d;
    Dual(double v_ = 0.0, double d_ = 0.0) : v(v_), d(d_) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, Dual b) { return Dual(a / b.v, -a * b.d / (b.v * b.v)); }
inline Dual &operator+=(Dual &a, Dual b) { return a = a + b; }
inline Dual sqrt(Dual a) {
    const double s = std::sqrt(a.v);
    return Dual(s, a.d / (2.0 * s));
}
inline Dual exp(Dual a) {
    const double e = std::exp(a.v);
    return Dual(e, a.d * e);
}
inline Dual cos(Dual a) { return Dual(std::cos(a.v), -std::sin(a.v) * a.d); }
inline Dual sin(Dual a) { return Dual(std::sin(a.v), std::cos(a.v) * a.d); }
inline Dual atan2(Dual y, Dual x) {
    return Dual(std::atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / (x.v * x.v + y.v * y.v));
}
inline double val(double x) { return x; }
inline double val(Dual x) { return x.v; }
using std::atan2;
using std::cos;
using std::exp;
using std::sin;
using std::sqrt;

// min / max / clamp decided on the value; the derivative follows the branch.
template <class T> T vmin(T a, double b) { return val(a) < b ? a : T(b); }
template <class T> T vmax(T a, double b) { return val(a) > b ? a : T(b); }

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

template <class T>
T ipow(T x, int p) {
    T r(1.0);
    for (int i = 0; i < p; ++i) r = r * x;
    return r;
}

template <class T>
T assoc_legendre(int l, int m, T x) {
    std::vector<double> c = legendre_poly(l);
    // m-th derivative of the polynomial.
    for (int d = 0; d < m; ++d) {
        std::vector<double> dc(std::max<size_t>(1, c.size() - 1), 0.0);
        for (size_t p = 1; p < c.size(); ++p) dc[p - 1] = p * c[p];
        c = dc;
    }
    T poly(0.0);
    for (size_t p = 0; p < c.size(); ++p) poly = poly + c[p] * ipow(x, (int)p);
    // (1 - x^2)^(m/2) = sqrt(1 - x^2)^m
    T s = sqrt(vmax(1.0 - x * x, 0.0));
    return std::pow(-1.0, m) * ipow(s, m) * poly;
}

template <class T>
T real_sh(int l, int m, const T d[3]) {
    int am = m < 0 ? -m : m;
    T ct = d[2];
    T phi = atan2(d[1], d[0]);
    double K = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * factorial(l - am) / factorial(l + am));
    T P = assoc_legendre(l, am, ct);
    if (m == 0) return K * P;
    if (m > 0) return std::sqrt(2.0) * K * cos(am * phi) * P;
    return std::sqrt(2.0) * K * sin(am * phi) * P;
}

// ---------------------------------------------------------------------------
// Small dense helpers.
// ---------------------------------------------------------------------------
template <class T, class U, class V>
void matmul3(const T A[3][3], const U B[3][3], V C[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            V s(0.0);
            for (int k = 0; k < 3; ++k) s = s + A[i][k] * B[k][j];
            C[i][j] = s;
        }
}

template <class T>
void transpose3(const T A[3][3], T B[3][3]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B[i][j] = A[j][i];
}

// Rotation matrix of the unit quaternion (w, x, y, z) (normalised here).
template <class T>
void quat_to_rot(const T q_in[4], T R[3][3]) {
    T n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    T w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
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

// The differentiable part of the projection of one Gaussian, generic in the
// scalar type (double for the forward pass, Dual for derivatives). Returns
// false when the Gaussian is culled (behind the near plane or degenerate).
template <class T>
struct Proj {
    T u, v, q[3], o, rgb[3];
    double depth = 0.0, ext = 0.0;
};

template <class T>
bool project_core(const T *mu, const T *log_scale, const T *quat, T logit, const T *coef, int sh_degree,
                  const Cam &cam, Proj<T> &P) {
    const int K = (sh_degree + 1) * (sh_degree + 1);
    // Camera centre C = -R^T t.
    double C[3];
    for (int i = 0; i < 3; ++i) C[i] = -(cam.R[0][i] * cam.t[0] + cam.R[1][i] * cam.t[1] + cam.R[2][i] * cam.t[2]);
    const double tan_x = 0.5 * cam.width / cam.fx, tan_y = 0.5 * cam.height / cam.fy;
    T t[3];
    for (int r = 0; r < 3; ++r) t[r] = cam.R[r][0] * mu[0] + cam.R[r][1] * mu[1] + cam.R[r][2] * mu[2] + cam.t[r];
    P.depth = val(t[2]);
    if (!(val(t[2]) > cam.near_z)) return false;  // behind the near plane

    // 3D covariance Sigma = (R S)(R S)^T.
    T Rq[3][3], M[3][3], Mt[3][3], Sigma[3][3];
    quat_to_rot(quat, Rq);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[r][c] = Rq[r][c] * exp(log_scale[c]);
    transpose3(M, Mt);
    matmul3(M, Mt, Sigma);

    // Camera-space covariance W Sigma W^T, W the world-to-camera rotation.
    double Wt[3][3];
    T tmp[3][3], Sc[3][3];
    transpose3(cam.R, Wt);
    matmul3(cam.R, Sigma, tmp);
    matmul3(tmp, Wt, Sc);

    // Jacobian of the perspective map at the (guard-band clamped) point.
    T rx = vmin(vmax(t[0] / t[2], -kGuard * tan_x), kGuard * tan_x);
    T ry = vmin(vmax(t[1] / t[2], -kGuard * tan_y), kGuard * tan_y);
    T J[2][3] = {{cam.fx / t[2], T(0.0), -cam.fx * rx / t[2]},
                 {T(0.0), cam.fy / t[2], -cam.fy * ry / t[2]}};
    T cov[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            T s(0.0);
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) s = s + J[a][k] * Sc[k][l] * J[b][l];
            cov[a][b] = s;
        }
    cov[0][0] = cov[0][0] + kDilation;
    cov[1][1] = cov[1][1] + kDilation;

    T det = cov[0][0] * cov[1][1] - cov[0][1] * cov[1][0];
    if (!(val(det) > 0.0)) return false;
    P.q[0] = cov[1][1] / det;
    P.q[1] = -cov[0][1] / det;
    P.q[2] = cov[0][0] / det;

    // Larger eigenvalue; radius = ceil(3 sqrt(lambda_max)) (Sec. 4.4).
    double mid = 0.5 * (val(cov[0][0]) + val(cov[1][1]));
    double lam = mid + std::sqrt(std::max(0.1, mid * mid - val(det)));
    P.ext = 3.0 * std::sqrt(lam);

    P.u = cam.fx * t[0] / t[2] + cam.cx;
    P.v = cam.fy * t[1] / t[2] + cam.cy;

    // View-dependent colour from SH along the camera-to-mean direction.
    T d[3] = {mu[0] - C[0], mu[1] - C[1], mu[2] - C[2]};
    T dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; ++k) d[k] = d[k] / dn;
    for (int ch = 0; ch < 3; ++ch) {
        T s(0.0);
        for (int l = 0; l <= sh_degree; ++l)
            for (int m = -l; m <= l; ++m) s = s + coef[(l * l + l + m) * 3 + ch] * real_sh(l, m, d);
        P.rgb[ch] = vmax(s + 0.5, 0.0);
    }
    (void)K;
    P.o = 1.0 / (1.0 + exp(-logit));
    return true;
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
        Proj<double> P;
        const bool ok = project_core<double>(means + 3 * i, log_scales + 3 * i, quats + 4 * i,
                                             opacity_logits[i], sh + (size_t)i * K * 3, sh_degree, cam, P);
        depth[i] = P.depth;
        if (!ok) continue;
        int64_t r = (int64_t)std::ceil(P.ext);
        int64_t rc[4];
        tile_rect(P.u, P.v, r, tile_w, tile_h, tiles_x, tiles_y, rc);
        extent[i] = P.ext;
        mean2d[2 * i] = P.u;
        mean2d[2 * i + 1] = P.v;
        conic[3 * i] = P.q[0];
        conic[3 * i + 1] = P.q[1];
        conic[3 * i + 2] = P.q[2];
        if (r <= 0 || (rc[2] - rc[0]) * (rc[3] - rc[1]) <= 0) continue;
        for (int ch = 0; ch < 3; ++ch) rgb[3 * i + ch] = P.rgb[ch];
        opacity[i] = P.o;
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

// Gradient of L = sum_p dL_dC[p] . C[p] with respect to every Gaussian
// parameter, where C is the image of project -> bin -> blend above (any loss
// enters through its image gradient dL/dC). Two plain steps:
//  1. Eq. 1 per pixel written out over its contributors i_1..i_m (alpha_k,
//     T_k = prod_{l<k} (1 - alpha_l), T_N the final transmittance):
//       dC/dc_k     = alpha_k T_k
//       dC/dalpha_k = c_k T_k - (sum_{l>k} c_l alpha_l T_l + bg T_N) / (1 - alpha_k)
//     with alpha = min(0.99, o G) (no derivative where clamped), G = exp(power),
//     power = -(Q00 dx^2 + Q11 dy^2)/2 - Q01 dx dy, d = pixel centre - mean2d;
//     this gives dL/d(record) = dL/d(u, v, Q00, Q01, Q11, o, r, g, b).
//  2. The projection differentiated in forward mode: project_core is run on
//     dual numbers seeded along each parameter and its record derivatives are
//     contracted with dL/d(record).
// Parameters per Gaussian: means 3, log_scales 3, quats 4, logit 1, SH K x 3.
// d_rec (n x 9) also returns dL/d(record). Culled Gaussians get zeros.
void gso_render_backward(int64_t n, const double *means, const double *log_scales, const double *quats,
                         const double *opacity_logits, const double *sh, int32_t sh_degree,
                         const double *cam_flat, int32_t width, int32_t height, int32_t tile_w,
                         int32_t tile_h, const double *bg, const double *dL_dC, double *d_means,
                         double *d_log_scales, double *d_quats, double *d_logits, double *d_sh,
                         double *d_rec) {
    const int K = (sh_degree + 1) * (sh_degree + 1);
    std::vector<double> m2(2 * n), con(3 * n), op(n), col(3 * n), dep(n), ext(n);
    std::vector<int64_t> rad(n), rect(4 * n);
    std::vector<int32_t> vis(n);
    gso_project(n, means, log_scales, quats, opacity_logits, sh, sh_degree, cam_flat, width, height, tile_w,
                tile_h, m2.data(), con.data(), op.data(), col.data(), dep.data(), ext.data(), rad.data(),
                rect.data(), vis.data());
    const int64_t K_pairs = gso_bin_count(n, m2.data(), rad.data(), vis.data(), width, height, tile_w, tile_h);
    const int64_t tiles_x = (width + tile_w - 1) / tile_w;
    const int64_t tiles_y = (height + tile_h - 1) / tile_h;
    std::vector<uint64_t> keys(std::max<int64_t>(K_pairs, 1));
    std::vector<uint32_t> values(std::max<int64_t>(K_pairs, 1)), ranges(2 * tiles_x * tiles_y);
    gso_bin(n, m2.data(), rad.data(), dep.data(), vis.data(), width, height, tile_w, tile_h, keys.data(),
            values.data(), ranges.data());
    for (int64_t i = 0; i < 9 * n; ++i) d_rec[i] = 0.0;

    // Step 1: dL/d(record), pixel by pixel.
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t t = 0; t < tiles_x * tiles_y; ++t) {
        const int64_t tx = t % tiles_x, ty = t / tiles_x;
        const int64_t first = ranges[2 * t], last = ranges[2 * t + 1];
        struct Contrib { int64_t g; double alpha, T, G, dx, dy; bool clamped; };
        std::vector<Contrib> cs;
        for (int64_t y = ty * tile_h; y < std::min<int64_t>(height, (ty + 1) * tile_h); ++y)
            for (int64_t x = tx * tile_w; x < std::min<int64_t>(width, (tx + 1) * tile_w); ++x) {
                const double px = x + 0.5, py = y + 0.5;
                cs.clear();
                double T = 1.0;
                for (int64_t k = first; k < last; ++k) {
                    const int64_t g = values[k];
                    const double dx = px - m2[2 * g], dy = py - m2[2 * g + 1];
                    const double power = -0.5 * (con[3 * g] * dx * dx + con[3 * g + 2] * dy * dy) -
                                         con[3 * g + 1] * dx * dy;
                    if (power > 0.0) continue;
                    const double G = std::exp(power);
                    const double raw = op[g] * G;
                    const double alpha = std::min(kAlphaMax, raw);
                    if (alpha < kAlphaMin) continue;
                    const double Tn = T * (1.0 - alpha);
                    if (Tn < kTMin) break;
                    cs.push_back({g, alpha, T, G, dx, dy, raw >= kAlphaMax});
                    T = Tn;
                }
                const double T_N = T;
                const double *gp = dL_dC + 3 * (y * width + x);
                double S[3] = {0.0, 0.0, 0.0};
                for (int64_t k = (int64_t)cs.size() - 1; k >= 0; --k) {
                    const Contrib &c = cs[k];
                    const double *ck = &col[3 * c.g];
                    double dL_dalpha = 0.0;
                    for (int ch = 0; ch < 3; ++ch) {
                        const double dC_dalpha = ck[ch] * c.T - (S[ch] + bg[ch] * T_N) / (1.0 - c.alpha);
                        dL_dalpha += gp[ch] * dC_dalpha;
                    }
                    double *dr = d_rec + 9 * c.g;
                    for (int ch = 0; ch < 3; ++ch) {
#pragma omp atomic
                        dr[6 + ch] += gp[ch] * c.alpha * c.T;
                        S[ch] += ck[ch] * c.alpha * c.T;
                    }
                    if (c.clamped) continue;
                    const double dL_do = dL_dalpha * c.G;
                    const double dL_dpower = dL_dalpha * op[c.g] * c.G;
                    const double *q = &con[3 * c.g];
                    const double du = dL_dpower * (q[0] * c.dx + q[1] * c.dy);
                    const double dv = dL_dpower * (q[1] * c.dx + q[2] * c.dy);
                    const double dq00 = dL_dpower * (-0.5 * c.dx * c.dx);
                    const double dq01 = dL_dpower * (-c.dx * c.dy);
                    const double dq11 = dL_dpower * (-0.5 * c.dy * c.dy);
#pragma omp atomic
                    dr[0] += du;
#pragma omp atomic
                    dr[1] += dv;
#pragma omp atomic
                    dr[2] += dq00;
#pragma omp atomic
                    dr[3] += dq01;
#pragma omp atomic
                    dr[4] += dq11;
#pragma omp atomic
                    dr[5] += dL_do;
                }
            }
    }

    // Step 2: chain through the projection with dual numbers.
    const Cam cam = make_cam(cam_flat, width, height);
    const int n_par = 11 + 3 * K;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double grad[11 + 48];
        for (int j = 0; j < n_par; ++j) grad[j] = 0.0;
        if (vis[i]) {
            const double *dr = d_rec + 9 * i;
            std::vector<Dual> coef(3 * K);
            for (int j = 0; j < n_par; ++j) {
                Dual mu[3], ls[3], q[4], lo;
                for (int a = 0; a < 3; ++a) mu[a] = Dual(means[3 * i + a], j == a ? 1.0 : 0.0);
                for (int a = 0; a < 3; ++a) ls[a] = Dual(log_scales[3 * i + a], j == 3 + a ? 1.0 : 0.0);
                for (int a = 0; a < 4; ++a) q[a] = Dual(quats[4 * i + a], j == 6 + a ? 1.0 : 0.0);
                lo = Dual(opacity_logits[i], j == 10 ? 1.0 : 0.0);
                for (int a = 0; a < 3 * K; ++a) coef[a] = Dual(sh[(size_t)i * K * 3 + a], j == 11 + a ? 1.0 : 0.0);
                Proj<Dual> P;
                project_core<Dual>(mu, ls, q, lo, coef.data(), sh_degree, cam, P);
                grad[j] = dr[0] * P.u.d + dr[1] * P.v.d + dr[2] * P.q[0].d + dr[3] * P.q[1].d +
                          dr[4] * P.q[2].d + dr[5] * P.o.d + dr[6] * P.rgb[0].d + dr[7] * P.rgb[1].d +
                          dr[8] * P.rgb[2].d;
            }
        }
        for (int a = 0; a < 3; ++a) d_means[3 * i + a] = grad[a];
        for (int a = 0; a < 3; ++a) d_log_scales[3 * i + a] = grad[3 + a];
        for (int a = 0; a < 4; ++a) d_quats[4 * i + a] = grad[6 + a];
        d_logits[i] = grad[10];
        for (int a = 0; a < 3 * K; ++a) d_sh[(size_t)i * K * 3 + a] = grad[11 + a];
    }
}

}  // extern "C"
