// gs_project.cu — per-Gaussian projection (Sec. 3.1 stages 1-2; the square
// 3-sigma bound of Sec. 4.4; the near-plane cull of Sec. 4.5 step 1).
//
// Two kernels share the per-Gaussian arithmetic (project_one):
//  * project_kernel, the gs_project stage entry point: one thread per
//    Gaussian; every thread reads the 12-byte mean, only Gaussians in front
//    of the near plane go on to read scale, rotation, opacity and SH (~16 B
//    per culled Gaussian, ~250 B per visible one), and every Gaussian gets a
//    record slot and a tile count.
//  * project_list_kernel, the first launch of gs_render: 1024 Gaussians per
//    block; a conservative screen bound from the mean and the largest scale
//    (24 B per Gaussian) picks the candidates, which alone get the full
//    projection; the visible ones get a record and an entry of the compact
//    list, the depth digits and the tile sort's digit histograms are counted
//    on the way, and SH colours are evaluated after the block's last barrier.
//    The batched variant (project_list_batch_kernel) does the same per view.
//
// Numerics, all FP32:
//  * 2D covariance as (T M)(T M)^T with T = J W (2x3) and M = R(q) S, so the
//    result is positive semi-definite by construction;
//  * det = |A0 x A1|^2 + 0.3 (a0 + c0) + 0.09 (Lagrange's identity for
//    a0 c0 - b^2), which avoids the cancellation of a c - b^2;
//  * lambda_max = mid + sqrt(max(0.1, ((a - c)/2)^2 + b^2)), the same value as
//    mid + sqrt(max(0.1, mid^2 - det)) without its cancellation.
#include <algorithm>

#include "gs_internal.cuh"
#include "gs_onesweep.cuh"

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

struct ProjectArgs {
    const float *means, *log_scales, *quats, *logits, *sh;
    int64_t n;
    GsCameraDev cam;
    GsGrid grid;
    float4 *records;
    uint32_t *tiles;
    bool sh_vec;    // SH rows 16-byte aligned: load them as float4
    bool quat_vec;  // quaternion array 16-byte aligned
};

// SH colour of one Gaussian: the basis values along (x, y, z) first, then
// the coefficients streamed in (as float4 when the rows are 16-byte aligned)
// and accumulated per channel.
template <int DEG>
__device__ __forceinline__ float3 sh_colour(const float *__restrict__ src, bool vec, float x,
                                            float y, float z) {
    constexpr int kK = (DEG + 1) * (DEG + 1);
    constexpr int kN = kK * 3;
    float Y[kK];
    Y[0] = kY00;
    if (DEG >= 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;
        Y[5] = -kY2a * y * z;
        Y[6] = kY2b * (2.f * zz - xx - yy);
        Y[7] = -kY2a * x * z;
        Y[8] = kY2c * (xx - yy);
        if (DEG >= 3) {
            Y[9] = -kY3a * y * (3.f * xx - yy);
            Y[10] = kY3b * x * y * z;
            Y[11] = -kY3c * y * (4.f * zz - xx - yy);
            Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kY3c * x * (4.f * zz - xx - yy);
            Y[14] = kY3e * z * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.f * yy);
        }
    }
    float acc[3] = {0.f, 0.f, 0.f};
    if (kN % 4 == 0 && vec) {
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
        for (int j = 0; j < kN / 4; ++j) {
            const float4 v = __ldg(s4 + j);
            const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                acc[(4 * j + q) % 3] = fmaf(Y[(4 * j + q) / 3], e[q], acc[(4 * j + q) % 3]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < kN; ++j) acc[j % 3] = fmaf(Y[j / 3], __ldg(src + j), acc[j % 3]);
    }
    return make_float3(fmaxf(acc[0] + 0.5f, 0.f), fmaxf(acc[1] + 0.5f, 0.f), fmaxf(acc[2] + 0.5f, 0.f));
}

// Result of projecting one Gaussian.
struct Projected {
    float4 r0, r1, r2;  // gs_record words
    Rect rect;
    uint32_t tiles;     // 0 when culled
    float3 dir;         // unit view direction (for a deferred colour)
};

// COLOUR = false leaves the colour words (r1.z, r1.w, r2.x) unset and
// returns the view direction instead, for a colour evaluated later (the list
// projections evaluate the SH colours of a block's visible Gaussians after
// its last barrier, by consecutive threads: visible Gaussians are a few
// percent of a frame's, and evaluated by their own threads they would hold
// whole warps, and through the barriers whole blocks, for one lane).
template <int DEG, bool COLOUR = true>
__device__ __forceinline__ Projected project_one(const ProjectArgs &P, const GsCameraDev &K, const GsGrid &G,
                                                 int64_t i) {
    Projected out;
    out.tiles = 0;
    const float mx = __ldg(P.means + 3 * i), my = __ldg(P.means + 3 * i + 1),
                mz = __ldg(P.means + 3 * i + 2);
    const float tx = fmaf(K.R[0], mx, fmaf(K.R[1], my, fmaf(K.R[2], mz, K.t[0])));
    const float ty = fmaf(K.R[3], mx, fmaf(K.R[4], my, fmaf(K.R[5], mz, K.t[1])));
    // The other per-Gaussian inputs are loaded before the near-plane test so
    // that all of them are in flight together (one memory round trip).
    const float4 q = P.quat_vec ? __ldg(reinterpret_cast<const float4 *>(P.quats) + i)
                                : make_float4(__ldg(P.quats + 4 * i), __ldg(P.quats + 4 * i + 1),
                                              __ldg(P.quats + 4 * i + 2), __ldg(P.quats + 4 * i + 3));
    const float ls0 = __ldg(P.log_scales + 3 * i), ls1 = __ldg(P.log_scales + 3 * i + 1),
                ls2 = __ldg(P.log_scales + 3 * i + 2);
    const float logit = __ldg(P.logits + i);
    const float tz = fmaf(K.R[6], mx, fmaf(K.R[7], my, fmaf(K.R[8], mz, K.t[2])));
    if (!(tz > K.near_z)) return out;

    // Rotation of the normalised quaternion (w, x, y, z), scaled columns M = R S.
    const float qinv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float qw = q.x * qinv, qx = q.y * qinv, qy = q.z * qinv, qz = q.w * qinv;
    const float sx = expf(ls0), sy = expf(ls1), sz = expf(ls2);
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
    if (!(det > 0.f) || !isfinite(u) || !isfinite(v) || !isfinite(ext)) return out;
    const int r = ext >= (float)kMaxRadius ? kMaxRadius : (int)ceilf(ext);
    if (r <= 0) return out;
    const Rect R = tile_rect(u, v, r, G.tile_w, G.tile_h, G.tiles_x, G.tiles_y);
    const uint32_t ntiles = (uint32_t)((R.x1 - R.x0) * (R.y1 - R.y0));
    if (ntiles == 0) return out;
    const float idet = 1.f / det;

    // View direction from the camera centre to the mean.
    float dx = mx - K.C[0], dy = my - K.C[1], dz = mz - K.C[2];
    const float dinv = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= dinv; dy *= dinv; dz *= dinv;
    const float3 rgb = COLOUR ? sh_colour<DEG>(P.sh + (size_t)i * (DEG + 1) * (DEG + 1) * 3, P.sh_vec, dx, dy, dz)
                              : make_float3(0.f, 0.f, 0.f);
    out.dir = make_float3(dx, dy, dz);
    const float opacity = 1.f / (1.f + expf(-logit));

    out.r0 = make_float4(u, v, c * idet, -b * idet);
    out.r1 = make_float4(a * idet, opacity, rgb.x, rgb.y);
    out.r2 = make_float4(rgb.z, tz, __int_as_float(r), __uint_as_float(ntiles));
    out.rect = R;
    out.tiles = ntiles;
    return out;
}

// Conservative screen test from the mean and the largest scale only: false
// only for Gaussians the full projection culls (behind the near plane, or a
// tile rect that misses the grid). The rows of T = J W are
// (fx/tz)(W0 - rx W2) and (fy/tz)(W1 - ry W2), so |T0| <= (fx/tz)(|W0| +
// |rx| |W2|) for any W; with s_max the largest scale, |A0|^2 + |A1|^2 <=
// s_max^2 (|T0|^2 + |T1|^2) =: B (R(q) is a rotation). lambda_max as the
// projection computes it is at most the trace + sqrt(0.1) = a0 + c0 + 0.6 +
// 0.317, so the pixel radius is at most 3 sqrt(B + 0.92); 1 % of B and 2
// pixels of slack cover FP32 rounding and the approximate reciprocal,
// exponential and square root used here (relative errors below 1e-6). The
// row norms come precomputed with the camera. A non-finite bound keeps the
// Gaussian (every comparison with NaN is false).
__device__ __forceinline__ bool maybe_visible(const ProjectArgs &P, const GsCameraDev &K, const GsGrid &G,
                                              int64_t i) {
    const float mx = __ldg(P.means + 3 * i), my = __ldg(P.means + 3 * i + 1), mz = __ldg(P.means + 3 * i + 2);
    const float ls = fmaxf(__ldg(P.log_scales + 3 * i), fmaxf(__ldg(P.log_scales + 3 * i + 1),
                                                              __ldg(P.log_scales + 3 * i + 2)));
    const float tz = fmaf(K.R[6], mx, fmaf(K.R[7], my, fmaf(K.R[8], mz, K.t[2])));
    if (!(tz > K.near_z)) return false;
    const float tx = fmaf(K.R[0], mx, fmaf(K.R[1], my, fmaf(K.R[2], mz, K.t[0])));
    const float ty = fmaf(K.R[3], mx, fmaf(K.R[4], my, fmaf(K.R[5], mz, K.t[1])));
    const float iz = __fdividef(1.f, tz);
    const float rx = fminf(K.lim_x, fmaxf(-K.lim_x, tx * iz));
    const float ry = fminf(K.lim_y, fmaxf(-K.lim_y, ty * iz));
    const float t0 = K.fx * iz * fmaf(fabsf(rx), K.rn[2], K.rn[0]), t1 = K.fy * iz * fmaf(fabsf(ry), K.rn[2], K.rn[1]);
    float s2;  // s_max^2 = 2^(2 ls log2 e)
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(s2) : "f"(2.f * 1.4426950408889634f * ls));
    const float B = s2 * fmaf(t0, t0, t1 * t1);
    float sq;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sq) : "f"(fmaf(B, 1.01f, 0.92f)));
    const float rb = fmaf(3.f, sq, 2.f);
    const float u = fmaf(K.fx * tx, iz, K.cx), v = fmaf(K.fy * ty, iz, K.cy);
    return !(u + rb < 0.f || u - rb > (float)(G.tiles_x * G.tile_w) || v + rb < 0.f ||
             v - rb > (float)(G.tiles_y * G.tile_h));
}

template <int DEG>
__global__ void __launch_bounds__(256) project_kernel(const ProjectArgs P) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const Projected pr = project_one<DEG>(P, P.cam, P.grid, i);
    P.tiles[i] = pr.tiles;
    if (pr.tiles) {
        float4 *out = P.records + 3 * i;
        out[0] = pr.r0;
        out[1] = pr.r1;
        out[2] = pr.r2;
    }
}

// ---------------------------------------------------------------------------
// Front end of a frame, depth first:
//  P. project_list_kernel: one thread per Gaussian projects it and writes the
//     record of a visible one; every block reserves, with one atomicAdd on a
//     packed 64-bit counter (visible count << 33 | key count), a segment of a
//     compact list of the visible Gaussians (tiles << 32 | depth bits, index),
//     notes the segment in a per-block table and counts the four depth
//     digits. The last block turns the counts into the depth sort's bucket
//     offsets and the table's counts, in block order, into the segments'
//     places in index order.
//  G. list_gather_kernel: one warp per segment copies it to its place, so
//     the list is in Gaussian index order.
//  D. the depth sort: four onesweep digit passes over the compact list.
//  S. entry_scan_kernel: exclusive scan of the tile counts in depth order
//     (decoupled look-back) giving each entry its first key slot, and the
//     entry that covers the first slot of every key block.
//  E. emit_keys_kernel: threads own runs of eight key slots, find their
//     entries (whose first slots ascend) and produce the keys — balanced
//     however large a single splat is — while counting the tile digits; the
//     block writes its keys and values out in coalesced 16-byte stores. A
//     key is the tile id alone (16 bits below 65536 tiles, else 32). The
//     last block turns the counts into the tile sort's bucket offsets and
//     publishes the key count it should use.
// The gathered list is in index order and the depth sort is stable, so
// entries are in (depth bits, index) order and the keys are emitted in it; the stable sort
// on the tile id then leaves every tile's list exactly in (depth bits, index)
// order, with no tie fix-up.
// ---------------------------------------------------------------------------
constexpr int kMaxTilePasses = 4;
constexpr unsigned long long kKeyMask = (1ull << 33) - 1;
constexpr int kKeyBlock = 1 << kKeyBlockLog2;
constexpr int kKeysPerThread = kKeyBlock / 256;
static_assert(kKeysPerThread == 8, "emission stages eight keys per thread");
constexpr int kDepthPasses = 4;                // the depth bits are the low word of a list key
constexpr int kDepthItems = 8;                 // short list: smaller sort partitions, shorter latency
constexpr int kEntryItems = 8;                 // list entries per thread of the entry scan
constexpr int kEntryTile = 256 * kEntryItems;
constexpr int kProjPer = 4;                       // Gaussians per thread of the list projection
constexpr int kProjBlock = 256 * kProjPer;        // ... and per block (one list segment)

struct ListArgs {
    ProjectArgs P;
    BlendRecordOut br;           // blend records of the visible Gaussians (geo null: none)
    unsigned long long *packed;  // visible << 33 | keys
    uint2 *seg;                  // per block: (first list slot, visible count)
    uint32_t *seg_dst;           // per block: first slot of its segment in index order
    uint64_t *lkeys;             // n: tiles << 32 | depth bits of visible entry j
    uint32_t *lvals;             // n: its Gaussian index
    GsSortScratch dsc;           // the depth sort's histograms, bucket offsets, ticket
    unsigned long long *counts;  // [0] K, [1] visible, [2] K if it fits, [3] visible (depth sort's count)
    bool xy_keys;                // keys (row << 8 | column): the tile sort's histograms are counted
    GsSortScratch tsc;           // here from the rects, for the emission fused with its first pass
    int tile_passes;             // at least 1
    int64_t key_capacity;
    uint32_t *d_err;
    uint2 *prect;                // optional, n: packed tile rect of every Gaussian (0 = none),
                                 // kept for temporal re-binning
    const uint2 *prev_rect;      // optional, n: the previous frame's; rects that differ
    unsigned long long *moved;   // are counted here (the churn)
};

// Tile rect packed in 2 words (x0 | x1 << 16, y0 | y1 << 16); 0 = no tiles.
__device__ __forceinline__ uint2 pack_rect(const Projected &pr) {
    return pr.tiles ? make_uint2((uint32_t)pr.rect.x0 | ((uint32_t)pr.rect.x1 << 16),
                                 (uint32_t)pr.rect.y0 | ((uint32_t)pr.rect.y1 << 16))
                    : make_uint2(0u, 0u);
}

// Digit histograms of a frame's tile keys, counted from the tile rects when
// the keys are (tile row << 8 | tile column) (grids at most 256 tiles wide):
// the low digit is the column, so a rect adds its height to each of its
// columns (a difference array: two updates), the next digit the low byte of
// the row (its width to each of its rows, a circular range), the third the
// row's high byte. Four updates per Gaussian, however large its rect.
struct TileDigitHist {
    int dx[257];       // column digit: difference array
    int dy[257];       // row low byte: difference array
    uint32_t turns;    // whole turns of the row range (256 rows or more) x width
    uint32_t hy[256];  // row high byte
};

__device__ __forceinline__ void count_rect_digits(TileDigitHist &H, const Rect &R, int passes) {
    const int w = R.x1 - R.x0, h = R.y1 - R.y0;
    atomicAdd(&H.dx[R.x0], h);
    atomicAdd(&H.dx[R.x1], -h);
    if (passes > 1) {
        const uint32_t t = (uint32_t)h >> 8, r = (uint32_t)h & 255u, st = (uint32_t)R.y0 & 255u;
        if (t) atomicAdd(&H.turns, t * (uint32_t)w);
        if (r) {
            atomicAdd(&H.dy[st], w);
            if (st + r <= 256u) {
                atomicAdd(&H.dy[st + r], -w);
            } else {
                atomicAdd(&H.dy[0], w);
                atomicAdd(&H.dy[st + r - 256u], -w);
            }
        }
    }
    if (passes > 2)
        for (int v = R.y0 >> 8; v <= (R.y1 - 1) >> 8; ++v) {
            const int lo = max(R.y0, v << 8), hi = min(R.y1, (v + 1) << 8);
            atomicAdd(&H.hy[v & 255], (uint32_t)((hi - lo) * w));
        }
}

// Adds a block's counts to the global histograms (passes x 256).
__device__ __forceinline__ void flush_tile_digits(TileDigitHist &H, uint32_t *hist, int passes, uint32_t *s_tmp) {
    const int tid = threadIdx.x;
    // Inclusive prefixes of the difference arrays give the counts.
    const int cx = H.dx[tid];
    const uint32_t nx = block_exclusive_scan_256((uint32_t)cx, s_tmp) + (uint32_t)cx;
    if (nx) atomicAdd(&hist[tid], nx);
    if (passes > 1) {
        const int cy = H.dy[tid];
        const uint32_t ny = block_exclusive_scan_256((uint32_t)cy, s_tmp) + (uint32_t)cy + H.turns;
        if (ny) atomicAdd(&hist[256 + tid], ny);
    }
    if (passes > 2 && H.hy[tid]) atomicAdd(&hist[512 + tid], H.hy[tid]);
}

// The last block of a list-building projection: the depth sort's bucket
// offsets, and the places of the n_seg list segments (one per projection
// block, in index order); counts[3] = the list's length, or 0 when it
// exceeds list_cap (nothing is then sorted).
__device__ void list_tail(const GsSortScratch &dsc, const uint2 *seg, uint32_t *seg_dst, int64_t n_seg,
                          const unsigned long long *packed, unsigned long long *counts, int64_t list_cap,
                          uint32_t *s_tmp, const GsSortScratch *tsc = nullptr, int tile_passes = 0,
                          int64_t key_cap = 0, uint32_t *d_err = nullptr) {
    const int tid = threadIdx.x;
    __threadfence();
    for (int d = 0; d < kDepthPasses; ++d) {
        const uint32_t c = __ldcg(&dsc.hist[d * 256 + tid]);
        dsc.bucket[d * 256 + tid] = block_exclusive_scan_256(c, s_tmp);
    }
    // With the tile histograms counted from the rects: the tile sort's bucket
    // offsets and the key count (which the emission would publish).
    if (tsc) {
        for (int d = 0; d < tile_passes; ++d) {
            const uint32_t c = __ldcg(&tsc->hist[d * 256 + tid]);
            tsc->bucket[d * 256 + tid] = block_exclusive_scan_256(c, s_tmp);
        }
        if (tid == 0) {
            const unsigned long long pk = __ldcg(packed);
            const unsigned long long K = pk & kKeyMask;
            counts[0] = K;
            counts[1] = pk >> 33;
            const bool fits = (int64_t)K <= key_cap;
            if (!fits) atomicOr(d_err, kErrCapacity);
            counts[2] = fits ? K : 0ull;
        }
    }
    // Segments in order, 4096 per round: thread tid takes 16 consecutive
    // table entries (eight 16-byte loads in flight).
    uint32_t carry = 0;
    for (int64_t r0 = 0; r0 < n_seg; r0 += 256 * 16) {
        const int64_t b0 = r0 + (int64_t)tid * 16;
        uint32_t cnt[16];
        if (b0 + 16 <= n_seg) {
            const uint4 *q = reinterpret_cast<const uint4 *>(seg + b0);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint4 x = __ldcg(q + k);
                cnt[2 * k] = x.y;
                cnt[2 * k + 1] = x.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) cnt[k] = b0 + k < n_seg ? __ldcg(&seg[b0 + k].y) : 0u;
        }
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) sum += cnt[k];
        const uint32_t ex = block_exclusive_scan_256(sum, s_tmp);
        uint32_t pre = carry + ex;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (b0 + k < n_seg) seg_dst[b0 + k] = pre;
            pre += cnt[k];
        }
        if (tid == 255) s_tmp[0] = ex + sum;  // the round's total (s_tmp is free again)
        __syncthreads();
        carry += s_tmp[0];
        __syncthreads();
    }
    if (tid == 0) {
        const unsigned long long nl = __ldcg(packed) >> 33;
        counts[3] = (int64_t)nl <= list_cap ? nl : 0ull;
    }
}

// A block of the list projection takes kProjBlock Gaussians (kProjPer per
// thread), so its chain of dependent steps (screen test, full projection of
// the candidates, reservation, list writes, ticket, colours) is paid once
// per 1024 Gaussians. Candidates and the colour inputs are staged in
// shared memory by candidate rank (index order).
struct ListStage {
    uint32_t cand[kProjBlock];   // candidate -> Gaussian offset in the block
    uint32_t tiles[kProjBlock];  // candidate -> tile count (0: culled)
    uint32_t dbits[kProjBlock];  // depth bits (record word r2.y)
    float qa[kProjBlock], op[kProjBlock];  // record words r1.x, r1.y
    float rad[kProjBlock];       // r2.z (radius bits)
    float dx[kProjBlock], dy[kProjBlock], dz[kProjBlock];  // view direction
};

template <int DEG>
__global__ void __launch_bounds__(256, 4) project_list_kernel(const ListArgs A) {
    __shared__ uint32_t s_cnt[kProjPer * 8];
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_hist[kDepthPasses * 256];
    __shared__ uint32_t s_tmp[8];
    __shared__ bool s_last;
    __shared__ ListStage S;
    __shared__ TileDigitHist s_th;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = tid; k < kDepthPasses * 256; k += 256) s_hist[k] = 0;
    for (int k = tid; k < 257; k += 256) {
        s_th.dx[k] = 0;
        s_th.dy[k] = 0;
    }
    s_th.hy[tid] = 0;
    if (tid == 0) s_th.turns = 0;
    const int64_t i0 = (int64_t)blockIdx.x * kProjBlock;
    // Screen test of Gaussians i0 + 256 q + tid; candidates keep index order,
    // which is (q, warp, lane) order.
    bool cand[kProjPer];
    uint32_t cm[kProjPer];
    uint32_t n_moved = 0;  // rects that changed (temporal re-binning's churn)
#pragma unroll
    for (int q = 0; q < kProjPer; ++q) {
        const int64_t i = i0 + q * 256 + tid;
        cand[q] = i < A.P.n && maybe_visible(A.P, A.P.cam, A.P.grid, i);
        if (A.prect && i < A.P.n && !cand[q]) {
            A.prect[i] = make_uint2(0u, 0u);
            if (A.prev_rect) {
                const uint2 orr = A.prev_rect[i];
                n_moved += (orr.x | orr.y) != 0u ? 1u : 0u;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kProjPer; ++q) {
        cm[q] = __ballot_sync(0xffffffffu, cand[q]);
        if (lane == 0) s_cnt[q * 8 + warp] = __popc(cm[q]);
    }
    __syncthreads();
    uint32_t nc = 0;
    uint32_t pre[kProjPer];
#pragma unroll
    for (int q = 0; q < kProjPer; ++q) pre[q] = 0;
    for (int k = 0; k < kProjPer * 8; ++k) {
        const uint32_t x = s_cnt[k];
#pragma unroll
        for (int q = 0; q < kProjPer; ++q)
            if (k < q * 8 + warp) pre[q] += x;
        nc += x;
    }
#pragma unroll
    for (int q = 0; q < kProjPer; ++q)
        if (cand[q]) S.cand[pre[q] + __popc(cm[q] & lanemask_lt())] = (uint32_t)(q * 256 + tid);
    __syncthreads();
    // Full projection of candidates tid, tid + 256, ...
    for (uint32_t c = tid; c < nc; c += 256) {
        const int64_t g = i0 + S.cand[c];
        const Projected pr = project_one<DEG, false>(A.P, A.P.cam, A.P.grid, g);
        S.tiles[c] = pr.tiles;
        if (pr.tiles) {
            A.P.records[3 * g] = pr.r0;
            if (A.xy_keys) count_rect_digits(s_th, pr.rect, A.tile_passes);
            S.dbits[c] = __float_as_uint(pr.r2.y);
            S.qa[c] = pr.r1.x;
            S.op[c] = pr.r1.y;
            S.rad[c] = pr.r2.z;
            S.dx[c] = pr.dir.x;
            S.dy[c] = pr.dir.y;
            S.dz[c] = pr.dir.z;
        }
        if (A.prect) {
            const uint2 nr = pack_rect(pr);
            A.prect[g] = nr;
            if (A.prev_rect) {
                const uint2 orr = A.prev_rect[g];
                n_moved += (nr.x != orr.x || nr.y != orr.y) ? 1u : 0u;
            }
        }
    }
    if (A.prev_rect) {
        const uint32_t wm = __reduce_add_sync(0xffffffffu, n_moved);
        if (lane == 0 && wm) atomicAdd(A.moved, (unsigned long long)wm);
    }
    __syncthreads();
    // List slots: thread tid owns candidates [4 tid, 4 tid + 4).
    uint32_t tsum = 0, vsum = 0;
#pragma unroll
    for (int q = 0; q < kProjPer; ++q) {
        const uint32_t c = kProjPer * tid + q;
        const uint32_t t = c < nc ? S.tiles[c] : 0u;
        tsum += t;
        vsum += t != 0u;
    }
    const uint32_t vpre = block_exclusive_scan_256(vsum, s_tmp);
    const uint32_t tpre = block_exclusive_scan_256(tsum, s_tmp);
    if (tid == 255) {
        const uint32_t bv = vpre + vsum, bt = tpre + tsum;
        s_base = bv ? atomicAdd(A.packed, ((unsigned long long)bv << 33) | bt) >> 33 : 0ull;
        A.seg[blockIdx.x] = make_uint2((uint32_t)s_base, bv);
        s_cnt[0] = bv;
    }
    __syncthreads();
    const uint32_t bv = s_cnt[0];
    uint64_t j = s_base + vpre;
#pragma unroll
    for (int q = 0; q < kProjPer; ++q) {
        const uint32_t c = kProjPer * tid + q;
        const uint32_t t = c < nc ? S.tiles[c] : 0u;
        if (t) {
            const uint32_t dbits = S.dbits[c];
            A.lkeys[j] = ((uint64_t)t << 32) | dbits;
            A.lvals[j] = (uint32_t)(i0 + S.cand[c]);
            for (int d = 0; d < kDepthPasses; ++d) atomicAdd(&s_hist[d * 256 + ((dbits >> (8 * d)) & 255u)], 1u);
            ++j;
        }
    }
    __syncthreads();
    if (bv) {
        for (int k = tid; k < kDepthPasses * 256; k += 256)
            if (s_hist[k]) atomicAdd(&A.dsc.hist[k], s_hist[k]);
        if (A.xy_keys) flush_tile_digits(s_th, A.tsc.hist, A.tile_passes, s_tmp);
    }
    // The barrier orders the block's counter updates before thread 0's fence,
    // which publishes them (cumulatively) before its ticket.
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(A.dsc.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    // Colours of the visible candidates, after the block's last barrier.
    for (uint32_t c = tid; c < nc; c += 256) {
        const uint32_t t = S.tiles[c];
        if (!t) continue;
        const size_t g = (size_t)(i0 + S.cand[c]);
        const float3 rgb = sh_colour<DEG>(A.P.sh + g * (DEG + 1) * (DEG + 1) * 3, A.P.sh_vec, S.dx[c], S.dy[c],
                                          S.dz[c]);
        const float4 r1 = make_float4(S.qa[c], S.op[c], rgb.x, rgb.y);
        const float4 r2 = make_float4(rgb.z, __uint_as_float(S.dbits[c]), S.rad[c], __uint_as_float(t));
        float4 *out = A.P.records + 3 * g;
        out[1] = r1;
        out[2] = r2;
        // Word r0 was written by this thread in the projection loop above
        // (same candidate-to-thread mapping).
        if (A.br.geo) A.br.write(g, out[0], r1.x, r1.y, rgb.x, rgb.y, rgb.z, __float_as_int(S.rad[c]));
    }
    if (!s_last) return;
    // Last block: every block's counts and list entries are in.
    list_tail(A.dsc, A.seg, A.seg_dst, gridDim.x, A.packed, A.counts, A.P.n, s_tmp, A.xy_keys ? &A.tsc : nullptr,
              A.tile_passes, A.key_capacity, A.d_err);
}

// Warp w of block b copies list segment 8 b + w (the visible Gaussians of
// one projection block, in index order) to its place in index order
// (segments of a batch are in (view, block) order).
__global__ void __launch_bounds__(256) list_gather_kernel(const uint2 *__restrict__ seg,
                                                         const uint32_t *__restrict__ seg_dst, int64_t n_seg,
                                                         const unsigned long long *count,
                                                         const uint64_t *__restrict__ lkeys,
                                                         const uint32_t *__restrict__ lvals, uint64_t *okeys,
                                                         uint32_t *ovals) {
    const int64_t b = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (b >= n_seg || *count == 0ull) return;  // nothing listed, or more than the list holds
    const uint2 sg = seg[b];
    const uint32_t dst = seg_dst[b];
    for (uint32_t k = threadIdx.x & 31; k < sg.y; k += 32) {
        okeys[dst + k] = lkeys[sg.x + k];
        ovals[dst + k] = lvals[sg.x + k];
    }
}

// ---------------------------------------------------------------------------
// Temporal re-binning, projection step: projects every Gaussian as above,
// writes its packed tile rect into `rect` and compares it with the previous
// frame's (`prev_rect`). A Gaussian whose rect changed (including becoming
// visible or culled) is "moved" and appended to the moved list; the per-tile
// bookkeeping of moved Gaussians runs in gs_temporal.cu, spread over warps.
// Counters: [0] visible << 33 | keys (as in project_list_kernel), [1] moved.
// ---------------------------------------------------------------------------
struct TemporalProjectArgs {
    ProjectArgs P;
    BlendRecordOut br;             // blend records (geo null: none)
    const uint2 *prev_rect;        // n: previous frame's packed rects
    uint2 *rect;                   // n: this frame's
    uint8_t *moved;                // n: 1 if the rect changed
    unsigned long long *items;     // work items of moved Gaussians: index << 32 | chunk
    int64_t item_capacity;
    unsigned long long *counters;  // zeroed
    uint32_t *d_err;
};

// Tiles of a rect handled by one work item of the moved-Gaussian kernels.
constexpr int kChunkTiles = 256;

template <int DEG>
__global__ void __launch_bounds__(256) project_temporal_kernel(const TemporalProjectArgs A) {
    __shared__ uint32_t s_t[8], s_v[8], s_m[8], s_c[8];
    __shared__ unsigned long long s_cbase;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = (int64_t)blockIdx.x * 256 + tid;
    Projected pr;
    pr.tiles = 0;
    if (i < A.P.n) pr = project_one<DEG>(A.P, A.P.cam, A.P.grid, i);
    if (pr.tiles) {
        float4 *out = A.P.records + 3 * i;
        out[0] = pr.r0;
        out[1] = pr.r1;
        out[2] = pr.r2;
        if (A.br.geo) A.br.write(i, pr.r0, pr.r1.x, pr.r1.y, pr.r1.z, pr.r1.w, pr.r2.x);
    }
    bool mv = false;
    uint32_t chunks = 0;  // work items: one per kChunkTiles tiles of the larger rect
    if (i < A.P.n) {
        const uint2 nr = pack_rect(pr), orr = A.prev_rect[i];
        mv = nr.x != orr.x || nr.y != orr.y;
        A.rect[i] = nr;
        A.moved[i] = mv ? 1 : 0;
        if (mv) {
            const uint32_t ow = (orr.x >> 16) - (orr.x & 0xffffu), oh = (orr.y >> 16) - (orr.y & 0xffffu);
            const uint32_t t_old = ow * oh, t_new = pr.tiles;
            const uint32_t t_max = t_old > t_new ? t_old : t_new;
            chunks = t_max ? (t_max + kChunkTiles - 1) / kChunkTiles : 1u;
        }
    }
    const uint32_t t = pr.tiles, v = t != 0u, m = mv;
    uint32_t it = t, iv = v, im = m, ic = chunks;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t a = __shfl_up_sync(0xffffffffu, it, o);
        const uint32_t b = __shfl_up_sync(0xffffffffu, iv, o);
        const uint32_t c = __shfl_up_sync(0xffffffffu, im, o);
        const uint32_t d = __shfl_up_sync(0xffffffffu, ic, o);
        if (lane >= o) { it += a; iv += b; im += c; ic += d; }
    }
    if (lane == 31) { s_t[warp] = it; s_v[warp] = iv; s_m[warp] = im; s_c[warp] = ic; }
    __syncthreads();
    uint32_t pc = 0, bt = 0, bv = 0, bm = 0, bc = 0;
    for (int w = 0; w < 8; ++w) {
        if (w < warp) pc += s_c[w];
        bt += s_t[w];
        bv += s_v[w];
        bm += s_m[w];
        bc += s_c[w];
    }
    if (tid == 0) {
        if (bv) atomicAdd(A.counters, ((unsigned long long)bv << 33) | bt);
        if (bm) atomicAdd(A.counters + 1, (unsigned long long)bm);
        s_cbase = bc ? atomicAdd(A.counters + 2, (unsigned long long)bc) : 0ull;
    }
    __syncthreads();
    const unsigned long long first = s_cbase + pc + ic - chunks;
    for (uint32_t c = 0; c < chunks; ++c) {
        if ((int64_t)(first + c) < A.item_capacity)
            A.items[first + c] = ((unsigned long long)i << 32) | c;
        else
            atomicOr(A.d_err, kErrTemporal);
    }
}

template <int DEG>
void launch_project_temporal(const TemporalProjectArgs &A, unsigned blocks, cudaStream_t s) {
    project_temporal_kernel<DEG><<<blocks, 256, 0, s>>>(A);
}

struct EntryScanArgs {
    const uint64_t *lkeys;             // depth-sorted list keys (tile count in the high word)
    const unsigned long long *count;   // list entries
    uint32_t *off;                     // out: first key slot of entry j
    uint32_t *block_entry;             // out: entry covering the first slot of each key block
    int64_t n_key_blocks;              // ceil(capacity / kKeyBlock)
    uint32_t *counter;                 // partition counter (zeroed)
    unsigned long long *status;        // one look-back word per partition (zeroed)
    uint32_t *d_err;
};

// Exclusive scan of the tile counts of the depth-sorted entries. Blocks take
// partitions of kEntryTile entries in launch order and resolve their prefix
// by decoupled look-back (bounded waits); partitions past the visible count
// return at once (no partition waits on a later one).
__global__ void __launch_bounds__(256) entry_scan_kernel(const EntryScanArgs A) {
    __shared__ uint32_t s_part;
    __shared__ unsigned long long s_warp[8];
    __shared__ unsigned long long s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_part = atomicAdd(A.counter, 1u);
    __syncthreads();
    const int64_t p = s_part;
    const int64_t nv = (int64_t)*A.count;
    if (p * kEntryTile >= nv) return;
    const int64_t base = p * kEntryTile + (int64_t)tid * kEntryItems;
    uint32_t t[kEntryItems];
    unsigned long long sum = 0;
#pragma unroll
    for (int j = 0; j < kEntryItems; ++j) {
        const int64_t idx = base + j;
        t[j] = idx < nv ? (uint32_t)(A.lkeys[idx] >> 32) : 0u;
        sum += t[j];
    }
    unsigned long long incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    unsigned long long warp_prefix = 0, block_total = 0;
    for (int w = 0; w < 8; ++w) {
        if (w < warp) warp_prefix += s_warp[w];
        block_total += s_warp[w];
    }
    if (warp == 0) {
        unsigned long long prefix = 0;
        if (p == 0) {
            if (lane == 0) st_relaxed_u64(A.status, kFlagIncl | block_total);
        } else {
            if (lane == 0) st_relaxed_u64(A.status + p, kFlagAgg | block_total);
            bool to;
            prefix = warp_lookback(A.status, p, A.d_err, &to);
            if (lane == 0) st_relaxed_u64(A.status + p, kFlagIncl | ((prefix + block_total) & kValueMask));
        }
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    unsigned long long run = s_prefix + warp_prefix + incl - sum;
#pragma unroll
    for (int j = 0; j < kEntryItems; ++j) {
        const int64_t idx = base + j;
        if (idx < nv) {
            A.off[idx] = (uint32_t)run;
            // Key blocks whose first slot falls in [run, run + t) start in this entry.
            const int64_t b0 = (int64_t)((run + kKeyBlock - 1) >> kKeyBlockLog2);
            const int64_t b1 = min((int64_t)((run + t[j] - 1) >> kKeyBlockLog2), A.n_key_blocks - 1);
            for (int64_t b = b0; b <= b1; ++b) A.block_entry[b] = (uint32_t)idx;
        }
        run += t[j];
    }
}

struct EmitArgs {
    const float4 *records;
    const unsigned long long *packed;
    const uint32_t *list_idx;     // record of entry j (depth order): Gaussian index, or compact slot
    const uint32_t *list_off;     // first key slot of entry j (ascending)
    const uint32_t *block_entry;
    GsGrid grid;                  // single view
    const uint2 *meta;            // batch: (view, Gaussian) of a compact slot
    const ViewDesc *views;        // batch: grids and first global tiles
    int64_t list_capacity;        // entries the list holds
    void *keys;                   // tile ids (KT)
    uint32_t *values;
    int64_t capacity;
    unsigned long long *counts;  // out: [0] K, [1] visible, [2] K if it fits else 0
    GsSortScratch sc;            // the tile sort (its digits are the tile id's)
    uint32_t *d_err;
};

// Block b covers key slots [2048 b, 2048 b + 2048), eight consecutive slots
// per thread. The list entries covering them (at most 2049, first slots
// ascending) are staged in shared memory; a thread finds the entry of its
// first slot by binary search and walks forward. Digit counts of a thread's
// run of keys are merged before they are added to the block's histogram.
// Keys and values are staged in shared memory and written with 16-byte
// stores (the key buffers are 256-byte aligned and blocks start at multiples
// of 2048 slots).
template <typename KT, bool BATCH>
__global__ void __launch_bounds__(256) emit_keys_kernel(const EmitArgs E) {
    __shared__ uint32_t s_hist[kMaxTilePasses * 256];
    __shared__ uint32_t s_off[kKeyBlock + 2], s_idx[kKeyBlock + 2];
    __shared__ __align__(16) KT s_key[kKeyBlock];
    __shared__ __align__(16) uint32_t s_val[kKeyBlock];
    __shared__ uint32_t s_tmp[8];
    __shared__ int s_j0, s_cnt;
    __shared__ bool s_last;
    const int tid = threadIdx.x;
    const int passes = E.sc.passes;
    const GsGrid &G = E.grid;
    for (int k = tid; k < kMaxTilePasses * 256; k += 256) s_hist[k] = 0;
    const unsigned long long packed = *E.packed;
    const int64_t K = (int64_t)(packed & kKeyMask);
    const int64_t nv = (int64_t)(packed >> 33);
    const int64_t k0 = (int64_t)blockIdx.x * kKeyBlock;
    const bool active = k0 < K && K <= E.capacity && nv <= E.list_capacity;
    if (tid == 0 && active) {
        // Entries from the one covering slot k0 to the one covering the next
        // block's first slot (at most 2049 of them; one for a large splat).
        const int64_t j0 = E.block_entry[blockIdx.x];
        const int64_t last = (K - 1) >> kKeyBlockLog2;
        int64_t j1 = (int64_t)blockIdx.x < last ? (int64_t)E.block_entry[blockIdx.x + 1] + 1 : nv;
        j1 = min(j1, min(nv, j0 + kKeyBlock + 2));
        s_j0 = (int)j0;
        s_cnt = (int)(j1 - j0);
    }
    __syncthreads();
    if (active) {
        for (int q = tid; q < s_cnt; q += 256) {
            s_off[q] = E.list_off[s_j0 + q];
            s_idx[q] = E.list_idx[s_j0 + q];
        }
    }
    __syncthreads();
    const int64_t kb = k0 + (int64_t)tid * kKeysPerThread;
    if (active && kb < K) {
        int lo = 0, hi = s_cnt - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int64_t)s_off[mid] <= kb) lo = mid; else hi = mid - 1;
        }
        int e = -1;
        uint32_t g = 0, w = 1, x0 = 0, y0 = 0, ebase = 0, eend = 0, tiles_x = (uint32_t)G.tiles_x, tbase = 0;
        uint32_t qy = 0, rx = 0;  // row and column of key k within its entry's rect
        uint32_t run_digit[kMaxTilePasses], run_count[kMaxTilePasses];
        uint32_t tk[kKeysPerThread], tv[kKeysPerThread];
        for (int d = 0; d < kMaxTilePasses; ++d) { run_digit[d] = 0xffffffffu; run_count[d] = 0; }
#pragma unroll
        for (int q = 0; q < kKeysPerThread; ++q) {
            const int64_t k = kb + q;
            tk[q] = 0u;
            tv[q] = 0u;
            if (k >= K) continue;
            if (e < 0 || (uint64_t)k >= eend) {
                if (e >= 0) ++lo;
                while (lo + 1 < s_cnt && (int64_t)s_off[lo + 1] <= k) ++lo;
                e = lo;
                g = s_idx[e];
                ebase = s_off[e];
                const float4 r0 = E.records[3 * (size_t)g];
                const float4 r2 = E.records[3 * (size_t)g + 2];
                GsGrid vg = G;
                if (BATCH) {
                    const ViewDesc &V = E.views[E.meta[g].x];
                    vg = V.grid;
                    tbase = V.tile_base;
                    tiles_x = (uint32_t)vg.tiles_x;
                }
                const Rect R = tile_rect(r0.x, r0.y, __float_as_int(r2.z), vg.tile_w, vg.tile_h, vg.tiles_x,
                                         vg.tiles_y);
                w = (uint32_t)(R.x1 - R.x0);
                x0 = (uint32_t)R.x0;
                y0 = (uint32_t)R.y0;
                eend = ebase + w * (uint32_t)(R.y1 - R.y0);
                // Only the thread's first key can start inside an entry.
                const uint32_t m = (uint32_t)(k - ebase);
                qy = m ? m / w : 0u;
                rx = m - qy * w;
            } else if (++rx == w) {  // the next key of the same rect, row-major
                rx = 0;
                ++qy;
            }
            const uint32_t tile = tbase + (y0 + qy) * tiles_x + x0 + rx;
            tk[q] = tile;
            tv[q] = g;
            for (int d = 0; d < passes; ++d) {
                const uint32_t dg = (tile >> (8 * d)) & 255u;
                if (dg != run_digit[d]) {
                    if (run_count[d]) atomicAdd(&s_hist[d * 256 + run_digit[d]], run_count[d]);
                    run_digit[d] = dg;
                    run_count[d] = 0;
                }
                ++run_count[d];
            }
        }
        for (int d = 0; d < passes; ++d)
            if (run_count[d]) atomicAdd(&s_hist[d * 256 + run_digit[d]], run_count[d]);
        // A thread's eight slots are contiguous: vector stores into the
        // staging arrays (entries past K are never written out).
        uint4 *sv4 = reinterpret_cast<uint4 *>(s_val + tid * kKeysPerThread);
        sv4[0] = make_uint4(tv[0], tv[1], tv[2], tv[3]);
        sv4[1] = make_uint4(tv[4], tv[5], tv[6], tv[7]);
        uint4 *sk4 = reinterpret_cast<uint4 *>(s_key + tid * kKeysPerThread);
        if (sizeof(KT) == 2) {
            sk4[0] = make_uint4(tk[0] | tk[1] << 16, tk[2] | tk[3] << 16, tk[4] | tk[5] << 16, tk[6] | tk[7] << 16);
        } else {
            sk4[0] = make_uint4(tk[0], tk[1], tk[2], tk[3]);
            sk4[1] = make_uint4(tk[4], tk[5], tk[6], tk[7]);
        }
    }
    __syncthreads();
    if (active) {
        // Slots [k0, k0 + nk) of this block, in 16-byte vectors (the ragged
        // end of the last block element by element).
        const int nk = (int)((K - k0) < kKeyBlock ? (K - k0) : kKeyBlock);
        constexpr int kPerVec = 16 / sizeof(KT);
        KT *gk = static_cast<KT *>(E.keys) + k0;
        uint32_t *gv = E.values + k0;
        for (int q = tid; q < nk / kPerVec; q += 256)
            reinterpret_cast<uint4 *>(gk)[q] = reinterpret_cast<const uint4 *>(s_key)[q];
        for (int q = (nk / kPerVec) * kPerVec + tid; q < nk; q += 256) gk[q] = s_key[q];
        for (int q = tid; q < nk / 4; q += 256)
            reinterpret_cast<uint4 *>(gv)[q] = reinterpret_cast<const uint4 *>(s_val)[q];
        for (int q = (nk / 4) * 4 + tid; q < nk; q += 256) gv[q] = s_val[q];
        for (int q = tid; q < passes * 256; q += 256)
            if (s_hist[q]) atomicAdd(&E.sc.hist[q], s_hist[q]);
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(E.sc.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // Last block: every histogram is complete.
    __threadfence();
    for (int d = 0; d < passes; ++d) {
        const uint32_t c = __ldcg(&E.sc.hist[d * 256 + tid]);
        E.sc.bucket[d * 256 + tid] = block_exclusive_scan_256(c, s_tmp);
    }
    if (tid == 0) {
        E.counts[0] = (unsigned long long)K;
        E.counts[1] = (unsigned long long)nv;
        const bool fits = K <= E.capacity && nv <= E.list_capacity;
        if (!fits) atomicOr(E.d_err, kErrCapacity);
        E.counts[2] = fits ? (unsigned long long)K : 0ull;
    }
}

// Key emission fused with the first (column) pass of the tile sort, for a
// single view at most 256 tiles wide whose keys are (row << 8 | column) and
// whose digit histograms were counted from the rects in the projection:
// block p (taken in ticket order) produces the keys of
// slots [2048 p, 2048 p + 2048) as emit_keys_kernel does, stages them in
// shared memory, reads them back warp-striped and runs one Onesweep
// partition on them, writing the pass's output. The keys never make a round
// trip through memory before their first pass.
struct EmitSortArgs {
    EmitArgs E;                     // entries and records; keys / values receive the pass's output
    const uint32_t *bucket;         // the pass's 256 exclusive digit offsets
    unsigned long long *status;     // the pass's look-back words (one row of 256 per key block, zeroed)
    uint32_t *ticket;               // key-block tickets (zeroed)
    unsigned long long timeout_ns;
};

template <typename KT>
__host__ __device__ constexpr int emit_sort_smem() {
    constexpr int emit = (kKeyBlock + 2) * 8 + kKeyBlock * (int)(sizeof(KT) + 4);
    constexpr int part = (int)onesweep_partition_smem<KT, kKeysPerThread>();
    return emit > part ? emit : part;
}

template <typename KT>
__global__ void __launch_bounds__(256, 3) emit_sort_kernel(const EmitSortArgs A) {
    const EmitArgs &E = A.E;
    __shared__ __align__(16) unsigned char s_raw[emit_sort_smem<KT>()];
    __shared__ int s_j0, s_cnt;
    __shared__ uint32_t s_part;
    uint32_t *s_off = reinterpret_cast<uint32_t *>(s_raw);
    uint32_t *s_idx = s_off + kKeyBlock + 2;
    KT *s_key = reinterpret_cast<KT *>(s_idx + kKeyBlock + 2);
    uint32_t *s_val = reinterpret_cast<uint32_t *>(s_key + kKeyBlock);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const GsGrid &G = E.grid;
    if (tid == 0) s_part = atomicAdd(A.ticket, 1u);
    __syncthreads();
    const int64_t p = s_part;
    const unsigned long long packed = *E.packed;
    const int64_t K = (int64_t)(packed & kKeyMask);
    const int64_t nv = (int64_t)(packed >> 33);
    const int64_t k0 = p * kKeyBlock;
    // Blocks past the keys (or every block, when the keys overflow the
    // buffers) have nothing to do; no block waits on a later one.
    if (!(k0 < K && K <= E.capacity && nv <= E.list_capacity)) return;
    if (tid == 0) {
        const int64_t j0 = E.block_entry[p];
        const int64_t last = (K - 1) >> kKeyBlockLog2;
        int64_t j1 = p < last ? (int64_t)E.block_entry[p + 1] + 1 : nv;
        j1 = min(j1, min(nv, j0 + kKeyBlock + 2));
        s_j0 = (int)j0;
        s_cnt = (int)(j1 - j0);
    }
    __syncthreads();
    for (int q = tid; q < s_cnt; q += 256) {
        s_off[q] = E.list_off[s_j0 + q];
        s_idx[q] = E.list_idx[s_j0 + q];
    }
    __syncthreads();
    const int64_t kb = k0 + (int64_t)tid * kKeysPerThread;
    if (kb < K) {
        int lo = 0, hi = s_cnt - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int64_t)s_off[mid] <= kb) lo = mid; else hi = mid - 1;
        }
        int e = -1;
        uint32_t g = 0, w = 1, x0 = 0, y0 = 0, ebase = 0, eend = 0;
        uint32_t qy = 0, rx = 0;  // row and column of key k within its entry's rect
        uint32_t tk[kKeysPerThread], tv[kKeysPerThread];
#pragma unroll
        for (int q = 0; q < kKeysPerThread; ++q) {
            const int64_t k = kb + q;
            tk[q] = 0u;
            tv[q] = 0u;
            if (k >= K) continue;
            if (e < 0 || (uint64_t)k >= eend) {
                if (e >= 0) ++lo;
                while (lo + 1 < s_cnt && (int64_t)s_off[lo + 1] <= k) ++lo;
                e = lo;
                g = s_idx[e];
                ebase = s_off[e];
                const float4 r0 = E.records[3 * (size_t)g];
                const float4 r2 = E.records[3 * (size_t)g + 2];
                const Rect R = tile_rect(r0.x, r0.y, __float_as_int(r2.z), G.tile_w, G.tile_h, G.tiles_x,
                                         G.tiles_y);
                w = (uint32_t)(R.x1 - R.x0);
                x0 = (uint32_t)R.x0;
                y0 = (uint32_t)R.y0;
                eend = ebase + w * (uint32_t)(R.y1 - R.y0);
                // Only the thread's first key can start inside an entry.
                const uint32_t m = (uint32_t)(k - ebase);
                qy = m ? m / w : 0u;
                rx = m - qy * w;
            } else if (++rx == w) {  // the next key of the same rect, row-major
                rx = 0;
                ++qy;
            }
            tk[q] = ((y0 + qy) << 8) | (x0 + rx);
            tv[q] = g;
        }
        uint4 *sv4 = reinterpret_cast<uint4 *>(s_val + tid * kKeysPerThread);
        sv4[0] = make_uint4(tv[0], tv[1], tv[2], tv[3]);
        sv4[1] = make_uint4(tv[4], tv[5], tv[6], tv[7]);
        uint4 *sk4 = reinterpret_cast<uint4 *>(s_key + tid * kKeysPerThread);
        if (sizeof(KT) == 2) {
            sk4[0] = make_uint4(tk[0] | tk[1] << 16, tk[2] | tk[3] << 16, tk[4] | tk[5] << 16, tk[6] | tk[7] << 16);
        } else {
            sk4[0] = make_uint4(tk[0], tk[1], tk[2], tk[3]);
            sk4[1] = make_uint4(tk[4], tk[5], tk[6], tk[7]);
        }
    }
    __syncthreads();
    // Slot order within the block is (thread, item); read back warp-striped
    // so that the partition's (item, lane) order within a warp is slot order.
    KT key[kKeysPerThread];
    uint32_t val[kKeysPerThread];
#pragma unroll
    for (int j = 0; j < kKeysPerThread; ++j) {
        const int i = warp * 32 * kKeysPerThread + j * 32 + lane;
        const bool ok = k0 + i < K;
        key[j] = ok ? s_key[i] : (KT)~(KT)0;
        val[j] = ok ? s_val[i] : 0u;
    }
    __syncthreads();  // the partition reuses the staging memory
    onesweep_partition<KT, kKeysPerThread>(key, val, k0, K, p, 0, A.status, A.bucket, static_cast<KT *>(E.keys),
                                           E.values, E.d_err, A.timeout_ns, true, s_raw);
}

// ---------------------------------------------------------------------------
// Batched front end (many views of one scene), depth first as a single view:
// block (b, v) projects Gaussians [2048 b, 2048 b + 2048) for view v and
// reserves compact record slots with the packed counter; slot j gets the
// record, meta[j] = (view, Gaussian index) and list entry j (tiles << 32 |
// depth bits, j). The list segments, placed in (view, block) order, give the
// list in (view, index) order; the stable depth sort, the entry scan and the
// emission follow, the keys being global tile ids (view's first tile + tile),
// so every global tile's list ends in (depth bits, index) order.
// ---------------------------------------------------------------------------
struct ListBatchArgs {
    ProjectArgs P;               // scene arrays (cam / grid unused; records compact)
    bool views_fast;             // grid (views, ranges) rather than (ranges, views)
    const ViewDesc *views;
    BlendRecordOut br;             // blend records (geo null: none)
    uint2 *meta;
    int64_t rec_capacity;
    unsigned long long *packed;  // records << 33 | keys
    uint2 *seg;                  // per (view, block): (first slot, records)
    uint32_t *seg_dst;
    uint64_t *lkeys;
    uint32_t *lvals;
    GsSortScratch dsc;
    unsigned long long *counts;
    uint32_t *d_err;
};

// Candidates of a batched block (kProjBlock Gaussians of one view) staged by
// rank: the records go to compact slots, known only after the block's
// reservation.
// A batched block takes kBatchBlock Gaussians of one view (kBatchPer per
// thread); its candidates are projected, reserved and written in rounds of
// up to kProjBlock (the stage's size), each round one list segment. The
// stage holds a round's candidates until their compact slots are known.
constexpr int kBatchPer = 8;
constexpr int kBatchBlock = 256 * kBatchPer;          // 2048
constexpr int kBatchRounds = kBatchBlock / kProjBlock;  // list segments per block

struct BatchStage {
    float4 r0[kProjBlock];
    uint32_t cand[kBatchBlock];  // every candidate of the block, in index order
    uint32_t tiles[kProjBlock];
    uint32_t dbits[kProjBlock];  // depth bits, then the record slot
    float qa[kProjBlock], op[kProjBlock], tz[kProjBlock], rad[kProjBlock];
    float dx[kProjBlock], dy[kProjBlock], dz[kProjBlock];
};

template <int DEG>
__global__ void __launch_bounds__(256, 3) project_list_batch_kernel(const ListBatchArgs A) {
    __shared__ uint32_t s_cnt[kBatchPer * 8];
    __shared__ uint32_t s_nc;
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_hist[kDepthPasses * 256];
    __shared__ uint32_t s_tmp[8];
    __shared__ bool s_last;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    BatchStage &S = *reinterpret_cast<BatchStage *>(s_dyn);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // With views_fast the views of one Gaussian range are neighbouring blocks,
    // so they read that range's parameters from L2 rather than each from DRAM
    // (grid.y holds the ranges, at most 65,535 of them).
    const int view = A.views_fast ? blockIdx.x : blockIdx.y;
    const int64_t rb = A.views_fast ? blockIdx.y : blockIdx.x;
    const int64_t nb = A.views_fast ? gridDim.y : gridDim.x;
    const ViewDesc &V = A.views[view];
    for (int k = tid; k < kDepthPasses * 256; k += 256) s_hist[k] = 0;
    const int64_t i0 = rb * kBatchBlock;
    // Screen test, candidates in index order ((q, warp, lane) order).
    bool cand[kBatchPer];
    uint32_t cm[kBatchPer];
#pragma unroll
    for (int q = 0; q < kBatchPer; ++q) {
        const int64_t i = i0 + q * 256 + tid;
        cand[q] = i < A.P.n && maybe_visible(A.P, V.cam, V.grid, i);
        cm[q] = __ballot_sync(0xffffffffu, cand[q]);
        if (lane == 0) s_cnt[q * 8 + warp] = __popc(cm[q]);
    }
    __syncthreads();
    {
        const uint32_t c = tid < kBatchPer * 8 ? s_cnt[tid] : 0u;
        const uint32_t ex = block_exclusive_scan_256(c, s_tmp);
        if (tid < kBatchPer * 8) s_cnt[tid] = ex;
        if (tid == kBatchPer * 8 - 1) s_nc = ex + c;
    }
    __syncthreads();
    const uint32_t nc = s_nc;
#pragma unroll
    for (int q = 0; q < kBatchPer; ++q)
        if (cand[q]) S.cand[s_cnt[q * 8 + warp] + __popc(cm[q] & lanemask_lt())] = (uint32_t)(q * 256 + tid);
    __syncthreads();
    uint32_t bv_all = 0;
    for (int r = 0; r < kBatchRounds; ++r) {
        const uint32_t c0 = (uint32_t)r * kProjBlock;
        const uint32_t cn = nc > c0 ? min(nc - c0, (uint32_t)kProjBlock) : 0u;
        if (cn == 0) {  // block-uniform
            if (tid == 0) A.seg[((int64_t)view * nb + rb) * kBatchRounds + r] = make_uint2(0u, 0u);
            continue;
        }
        for (uint32_t c = tid; c < cn; c += 256) {
            const Projected pr = project_one<DEG, false>(A.P, V.cam, V.grid, i0 + S.cand[c0 + c]);
            S.tiles[c] = pr.tiles;
            if (pr.tiles) {
                S.r0[c] = pr.r0;
                S.dbits[c] = __float_as_uint(pr.r2.y);
                S.qa[c] = pr.r1.x;
                S.op[c] = pr.r1.y;
                S.tz[c] = pr.r2.y;
                S.rad[c] = pr.r2.z;
                S.dx[c] = pr.dir.x;
                S.dy[c] = pr.dir.y;
                S.dz[c] = pr.dir.z;
            }
        }
        __syncthreads();
        // Compact slots: thread tid owns the round's candidates [4 tid, 4 tid + 4).
        uint32_t tsum = 0, vsum = 0;
#pragma unroll
        for (int q = 0; q < kProjPer; ++q) {
            const uint32_t c = kProjPer * tid + q;
            const uint32_t t = c < cn ? S.tiles[c] : 0u;
            tsum += t;
            vsum += t != 0u;
        }
        const uint32_t vpre = block_exclusive_scan_256(vsum, s_tmp);
        const uint32_t tpre = block_exclusive_scan_256(tsum, s_tmp);
        if (tid == 255) {
            const uint32_t bv = vpre + vsum, bt = tpre + tsum;
            s_base = bv ? atomicAdd(A.packed, ((unsigned long long)bv << 33) | bt) >> 33 : 0ull;
            A.seg[((int64_t)view * nb + rb) * kBatchRounds + r] = make_uint2((uint32_t)s_base, bv);
            s_cnt[0] = bv;
        }
        __syncthreads();
        bv_all += s_cnt[0];
        uint64_t j = s_base + vpre;
#pragma unroll
        for (int q = 0; q < kProjPer; ++q) {
            const uint32_t c = kProjPer * tid + q;
            const uint32_t t = c < cn ? S.tiles[c] : 0u;
            if (t) {
                const uint32_t dbits = S.dbits[c];
                const bool fits = (int64_t)j < A.rec_capacity;
                if (fits) {
                    A.P.records[3 * j] = S.r0[c];
                    A.meta[j] = make_uint2((uint32_t)view, (uint32_t)(i0 + S.cand[c0 + c]));
                    A.lkeys[j] = ((uint64_t)t << 32) | dbits;
                    A.lvals[j] = (uint32_t)j;
                    for (int d = 0; d < kDepthPasses; ++d)
                        atomicAdd(&s_hist[d * 256 + ((dbits >> (8 * d)) & 255u)], 1u);
                } else {
                    atomicOr(A.d_err, kErrCapacity);
                }
                S.dbits[c] = fits ? (uint32_t)j : 0xffffffffu;
                ++j;
            }
        }
        __syncthreads();
        // Colours of this round's visible candidates (the stage is reused by
        // the next round).
        for (uint32_t c = tid; c < cn; c += 256) {
            const uint32_t t = S.tiles[c], slot = S.dbits[c];
            if (!t || slot == 0xffffffffu) continue;
            const size_t g = (size_t)(i0 + S.cand[c0 + c]);
            const float3 rgb = sh_colour<DEG>(A.P.sh + g * (DEG + 1) * (DEG + 1) * 3, A.P.sh_vec, S.dx[c], S.dy[c],
                                              S.dz[c]);
            const float4 r1 = make_float4(S.qa[c], S.op[c], rgb.x, rgb.y);
            const float4 r2 = make_float4(rgb.z, S.tz[c], S.rad[c], __uint_as_float(t));
            float4 *out = A.P.records + 3 * (size_t)slot;
            out[1] = r1;
            out[2] = r2;
            if (A.br.geo) {
                // The 16 x 16 tile ranges (list tiles) are on this view's screen.
                BlendRecordOut br = A.br;
                br.t16x = (V.cam.width + 15) / 16;
                br.t16y = (V.cam.height + 15) / 16;
                br.write(slot, S.r0[c], r1.x, r1.y, rgb.x, rgb.y, rgb.z, __float_as_int(S.rad[c]));
            }
        }
        __syncthreads();
    }
    if (bv_all)
        for (int k = tid; k < kDepthPasses * 256; k += 256)
            if (s_hist[k]) atomicAdd(&A.dsc.hist[k], s_hist[k]);
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(A.dsc.ticket, 1u) == gridDim.x * gridDim.y - 1;
    }
    __syncthreads();
    if (!s_last) return;
    list_tail(A.dsc, A.seg, A.seg_dst, (int64_t)gridDim.x * gridDim.y * kBatchRounds, A.packed, A.counts,
              A.rec_capacity, s_tmp);
}

template <int DEG>
cudaError_t launch_project_list_batch(const ListBatchArgs &A, dim3 grid, cudaStream_t s) {
    const cudaError_t e = cudaFuncSetAttribute(project_list_batch_kernel<DEG>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BatchStage));
    if (e != cudaSuccess) return e;
    project_list_batch_kernel<DEG><<<grid, 256, sizeof(BatchStage), s>>>(A);
    return cudaGetLastError();
}

}  // namespace

namespace {

// Front-end scratch: the packed counter and the entry scan's partition
// counter, the depth sort's scratch and the entry scan's status words (all
// zeroed per frame), then the segment table, the compact list, its sort buffers, the entries'
// first slots and the key-block table.
struct FrontLayout {
    size_t dsort, scan_status, st0, zero, seg, seg_dst, lkeys, lvals, akeys, avals, off, block_entry, total;
};

// n_list: entries the list holds; n_seg: projection blocks (list segments);
// fused: emission fused with the first tile pass (single view).
FrontLayout front_layout(int64_t n_list, int64_t capacity, int64_t n_seg, bool fused) {
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const int64_t nn = n_list > 0 ? n_list : 1;
    const int64_t ns = n_seg > 0 ? n_seg : 1;
    FrontLayout L;
    size_t o = 256;
    L.dsort = o;
    o += al(gs_sort_scratch_bytes_digits(nn, kDepthPasses, kDepthItems));
    L.scan_status = o;
    o += al((size_t)((nn + kEntryTile - 1) / kEntryTile + 1) * 8);
    L.st0 = o;  // the fused emission pass: look-back words per key block, then its ticket
    if (fused) o += al((size_t)((capacity + kKeyBlock - 1) / kKeyBlock + 1) * kOsRadix * 8 + 16);
    L.zero = o;
    L.seg = o;
    o += al((size_t)ns * 8);
    L.seg_dst = o;
    o += al((size_t)ns * 4);
    L.lkeys = o;
    o += al((size_t)nn * 8);
    L.lvals = o;
    o += al((size_t)nn * 4);
    L.akeys = o;
    o += al((size_t)nn * 8);
    L.avals = o;
    o += al((size_t)nn * 4);
    L.off = o;
    o += al((size_t)nn * 4);
    L.block_entry = o;
    o += al(gs_key_block_bytes(capacity));
    L.total = o;
    return L;
}

// After the list-building projection: gather into index order (into the
// alternate buffers), depth sort (count counts[3]; the even number of passes
// leaves the list there), entry scan and key emission. E carries the
// record, grid and output fields; the list fields are filled here.
cudaError_t launch_list_stages(const FrontLayout &L, char *base, int64_t n_list, int64_t n_seg,
                               const GsSortScratch &dsc, EmitArgs E, int key_bytes, bool batch, bool xy_keys,
                               unsigned long long *counts, uint32_t *d_err, cudaStream_t s, const cudaEvent_t *marks) {
    const uint2 *seg = reinterpret_cast<const uint2 *>(base + L.seg);
    const uint32_t *seg_dst = reinterpret_cast<const uint32_t *>(base + L.seg_dst);
    uint64_t *lkeys = reinterpret_cast<uint64_t *>(base + L.lkeys);
    uint32_t *lvals = reinterpret_cast<uint32_t *>(base + L.lvals);
    uint64_t *gkeys = reinterpret_cast<uint64_t *>(base + L.akeys);
    uint32_t *gvals = reinterpret_cast<uint32_t *>(base + L.avals);
    list_gather_kernel<<<(unsigned)((n_seg + 7) / 8), 256, 0, s>>>(seg, seg_dst, n_seg, counts + 3, lkeys, lvals,
                                                                  gkeys, gvals);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bool in_alt = false;
    e = gs_launch_sort_passes(gkeys, gvals, lkeys, lvals, n_list, counts + 3, dsc, d_err, &in_alt, s);
    if (e != cudaSuccess) return e;
    if (marks && marks[1]) cudaEventRecord(marks[1], s);
    EntryScanArgs S;
    S.lkeys = in_alt ? lkeys : gkeys;
    S.count = counts + 3;
    S.off = reinterpret_cast<uint32_t *>(base + L.off);
    S.block_entry = reinterpret_cast<uint32_t *>(base + L.block_entry);
    S.n_key_blocks = (E.capacity + kKeyBlock - 1) / kKeyBlock;
    S.counter = reinterpret_cast<uint32_t *>(base + 8);
    S.status = reinterpret_cast<unsigned long long *>(base + L.scan_status);
    S.d_err = d_err;
    gs_carveout(entry_scan_kernel);
    entry_scan_kernel<<<(unsigned)((n_list + kEntryTile - 1) / kEntryTile), 256, 0, s>>>(S);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (marks && marks[2]) cudaEventRecord(marks[2], s);
    E.packed = reinterpret_cast<const unsigned long long *>(base);
    E.list_idx = in_alt ? lvals : gvals;
    E.list_off = S.off;
    E.block_entry = S.block_entry;
    E.list_capacity = n_list;
    E.counts = counts;
    E.d_err = d_err;
    // One block per 2048 key slots of the capacity (blocks past K only take
    // their ticket).
    const unsigned eblocks = (unsigned)((E.capacity + kKeyBlock - 1) / kKeyBlock);
    if (batch) {
        emit_keys_kernel<uint32_t, true><<<eblocks, 256, 0, s>>>(E);
        return cudaGetLastError();
    }
    if (!xy_keys) {  // wide grids: tile ids, histograms counted by the emission
        if (key_bytes == 2) {
            gs_carveout(emit_keys_kernel<uint16_t, false>);
            emit_keys_kernel<uint16_t, false><<<eblocks, 256, 0, s>>>(E);
        } else {
            gs_carveout(emit_keys_kernel<uint32_t, false>);
            emit_keys_kernel<uint32_t, false><<<eblocks, 256, 0, s>>>(E);
        }
        return cudaGetLastError();
    }
    // Single view: the histograms came from the projection; emission and the
    // first tile pass are one kernel writing that pass's output.
    EmitSortArgs F;
    F.E = E;
    F.bucket = E.sc.bucket;
    F.status = reinterpret_cast<unsigned long long *>(base + L.st0);
    F.ticket = reinterpret_cast<uint32_t *>(base + L.st0 + (size_t)(eblocks + 1) * kOsRadix * 8);
    F.timeout_ns = kSpinTimeoutNs;
    if (key_bytes == 2) {
        gs_carveout(emit_sort_kernel<uint16_t>);
        emit_sort_kernel<uint16_t><<<eblocks, 256, 0, s>>>(F);
    } else {
        gs_carveout(emit_sort_kernel<uint32_t>);
        emit_sort_kernel<uint32_t><<<eblocks, 256, 0, s>>>(F);
    }
    return cudaGetLastError();
}

}  // namespace

size_t gs_fused_scratch_bytes(int64_t n, int64_t capacity) {
    return front_layout(n, capacity, (n + kProjBlock - 1) / kProjBlock, true).total;
}

size_t gs_key_block_bytes(int64_t capacity) {
    return ((size_t)(capacity + kKeyBlock - 1) / kKeyBlock + 1) * 4;
}

cudaError_t gs_launch_project_bin(const gs_gaussians &g, const GsCameraDev &cam, const GsGrid &grid,
                                  gs_record *records, const gs::BlendRecordOut &br,
                                  void *keys, int key_bytes, bool xy_keys, uint32_t *values,
                                  int64_t capacity, unsigned long long *counts, void *scan_scratch,
                                  const GsSortScratch &sc, uint32_t *d_err, cudaStream_t s,
                                  const cudaEvent_t *marks, uint2 *prect, const uint2 *prev_rect,
                                  unsigned long long *moved) {
    // counts and the front-end counters start at zero; the tile sort's
    // scratch was zeroed by the caller.
    if (key_bytes != 2 && key_bytes != 4) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(counts, 0, 5 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (g.n + kProjBlock - 1) / kProjBlock;
    const FrontLayout L = front_layout(g.n, capacity, blocks, xy_keys);
    char *base = static_cast<char *>(scan_scratch);
    e = cudaMemsetAsync(base, 0, L.zero, s);
    if (e != cudaSuccess || g.n == 0) return e;
    ListArgs A;
    A.P = ProjectArgs{g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, g.n, cam, grid,
                      reinterpret_cast<float4 *>(records), nullptr,
                      reinterpret_cast<uintptr_t>(g.sh) % 16 == 0,
                      reinterpret_cast<uintptr_t>(g.quats) % 16 == 0};
    A.br = br;
    A.packed = reinterpret_cast<unsigned long long *>(base);
    A.seg = reinterpret_cast<uint2 *>(base + L.seg);
    A.seg_dst = reinterpret_cast<uint32_t *>(base + L.seg_dst);
    A.lkeys = reinterpret_cast<uint64_t *>(base + L.lkeys);
    A.lvals = reinterpret_cast<uint32_t *>(base + L.lvals);
    A.dsc = gs_sort_carve_digits(base + L.dsort, g.n, 0, kDepthPasses, kDepthItems);
    A.counts = counts;
    A.xy_keys = xy_keys;
    A.tsc = sc;
    A.tile_passes = sc.passes > 0 ? sc.passes : 1;
    A.key_capacity = capacity;
    A.d_err = d_err;
    A.prect = prect;
    A.prev_rect = prect ? prev_rect : nullptr;
    A.moved = moved;
    switch (g.sh_degree) {
        case 0: project_list_kernel<0><<<(unsigned)blocks, 256, 0, s>>>(A); break;
        case 1: project_list_kernel<1><<<(unsigned)blocks, 256, 0, s>>>(A); break;
        case 2: project_list_kernel<2><<<(unsigned)blocks, 256, 0, s>>>(A); break;
        default:
            gs_carveout(project_list_kernel<3>);
            project_list_kernel<3><<<(unsigned)blocks, 256, 0, s>>>(A);
            break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (marks && marks[0]) cudaEventRecord(marks[0], s);
    EmitArgs E{};
    E.records = reinterpret_cast<const float4 *>(records);
    E.grid = grid;
    E.keys = keys;
    E.values = values;
    E.capacity = capacity;
    E.sc = sc;
    return launch_list_stages(L, base, g.n, blocks, A.dsc, E, key_bytes, false, xy_keys, counts, d_err, s, marks);
}

namespace {
// 1: a launch of project_list_kernel, 2: of project_temporal_kernel, else 0.
int camera_node_kind(const cudaKernelNodeParams &p) {
    if (p.func == reinterpret_cast<void *>(project_list_kernel<0>) ||
        p.func == reinterpret_cast<void *>(project_list_kernel<1>) ||
        p.func == reinterpret_cast<void *>(project_list_kernel<2>) ||
        p.func == reinterpret_cast<void *>(project_list_kernel<3>))
        return 1;
    if (p.func == reinterpret_cast<void *>(project_temporal_kernel<0>) ||
        p.func == reinterpret_cast<void *>(project_temporal_kernel<1>) ||
        p.func == reinterpret_cast<void *>(project_temporal_kernel<2>) ||
        p.func == reinterpret_cast<void *>(project_temporal_kernel<3>))
        return 2;
    return 0;
}
}  // namespace

bool gs_is_camera_node(cudaGraphNode_t node) {
    cudaGraphNodeType type;
    if (cudaGraphNodeGetType(node, &type) != cudaSuccess || type != cudaGraphNodeTypeKernel) return false;
    cudaKernelNodeParams p{};
    if (cudaGraphKernelNodeGetParams(node, &p) != cudaSuccess) return false;
    return camera_node_kind(p) != 0;
}

cudaError_t gs_set_node_camera(cudaGraphExec_t exec, cudaGraphNode_t node, const GsCameraDev &cam) {
    cudaKernelNodeParams p{};
    cudaError_t e = cudaGraphKernelNodeGetParams(node, &p);
    if (e != cudaSuccess) return e;
    p.extra = nullptr;
    const int kind = camera_node_kind(p);
    if (kind == 1) {
        ListArgs A = *static_cast<const ListArgs *>(p.kernelParams[0]);
        A.P.cam = cam;
        void *args[1] = {&A};
        p.kernelParams = args;
        return cudaGraphExecKernelNodeSetParams(exec, node, &p);
    }
    if (kind == 2) {
        TemporalProjectArgs A = *static_cast<const TemporalProjectArgs *>(p.kernelParams[0]);
        A.P.cam = cam;
        void *args[1] = {&A};
        p.kernelParams = args;
        return cudaGraphExecKernelNodeSetParams(exec, node, &p);
    }
    return cudaErrorInvalidValue;
}

cudaError_t gs_launch_project_temporal(const gs_gaussians &g, const GsCameraDev &cam, const GsGrid &grid,
                                       gs_record *records, const gs::BlendRecordOut &br, const uint2 *prev_rect, uint2 *rect, uint8_t *moved,
                                       unsigned long long *items, int64_t item_capacity,
                                       unsigned long long *counters, uint32_t *d_err, cudaStream_t s) {
    if (g.n == 0) return cudaSuccess;
    TemporalProjectArgs A;
    A.P = ProjectArgs{g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, g.n, cam, grid,
                      reinterpret_cast<float4 *>(records), nullptr,
                      reinterpret_cast<uintptr_t>(g.sh) % 16 == 0,
                      reinterpret_cast<uintptr_t>(g.quats) % 16 == 0};
    A.br = br;
    A.prev_rect = prev_rect;
    A.rect = rect;
    A.moved = moved;
    A.items = items;
    A.item_capacity = item_capacity;
    A.counters = counters;
    A.d_err = d_err;
    const unsigned blocks = (unsigned)((g.n + 255) / 256);
    switch (g.sh_degree) {
        case 0: launch_project_temporal<0>(A, blocks, s); break;
        case 1: launch_project_temporal<1>(A, blocks, s); break;
        case 2: launch_project_temporal<2>(A, blocks, s); break;
        default: launch_project_temporal<3>(A, blocks, s); break;
    }
    return cudaGetLastError();
}

cudaError_t gs_launch_project(const gs_gaussians &g, const GsCameraDev &cam, const GsGrid &grid,
                              gs_record *records, uint32_t *tiles, cudaStream_t s) {
    if (g.n == 0) return cudaSuccess;
    ProjectArgs a{g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, g.n, cam, grid,
                  reinterpret_cast<float4 *>(records), tiles,
                  reinterpret_cast<uintptr_t>(g.sh) % 16 == 0,
                  reinterpret_cast<uintptr_t>(g.quats) % 16 == 0};
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

// ---------------------------------------------------------------------------
// Backward of the projection: from dL/d(u, v, Q00, Q01, Q11, opacity, r, g, b)
// of each record to the Gaussian's parameters, by the chain rule written out
// in reverse order of the forward computation (project_one).
// ---------------------------------------------------------------------------
namespace {

struct ProjectBwdArgs {
    ProjectArgs P;
    const float *d_rec;  // n rows of kRecGradStride
    float *d_means, *d_log_scales, *d_quats, *d_logits, *d_sh;
};

// Gradient of the SH colour with respect to the unit direction and the
// coefficients: rgb_c = max(0, sum_k Y_k(d) c_kc + 0.5).
template <int DEG>
__device__ __forceinline__ float3 sh_colour_bwd(const float *__restrict__ src, float *__restrict__ dsrc,
                                                float x, float y, float z, const float gr[3]) {
    constexpr int kK = (DEG + 1) * (DEG + 1);
    float Y[kK], Dx[kK], Dy[kK], Dz[kK];
    Y[0] = kY00; Dx[0] = Dy[0] = Dz[0] = 0.f;
    if (DEG >= 1) {
        Y[1] = -kY1 * y; Dx[1] = 0.f;   Dy[1] = -kY1; Dz[1] = 0.f;
        Y[2] = kY1 * z;  Dx[2] = 0.f;   Dy[2] = 0.f;  Dz[2] = kY1;
        Y[3] = -kY1 * x; Dx[3] = -kY1;  Dy[3] = 0.f;  Dz[3] = 0.f;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;                 Dx[4] = kY2a * y;          Dy[4] = kY2a * x;          Dz[4] = 0.f;
        Y[5] = -kY2a * y * z;                Dx[5] = 0.f;               Dy[5] = -kY2a * z;         Dz[5] = -kY2a * y;
        Y[6] = kY2b * (2.f * zz - xx - yy);  Dx[6] = -2.f * kY2b * x;   Dy[6] = -2.f * kY2b * y;   Dz[6] = 4.f * kY2b * z;
        Y[7] = -kY2a * x * z;                Dx[7] = -kY2a * z;         Dy[7] = 0.f;               Dz[7] = -kY2a * x;
        Y[8] = kY2c * (xx - yy);             Dx[8] = 2.f * kY2c * x;    Dy[8] = -2.f * kY2c * y;   Dz[8] = 0.f;
        if (DEG >= 3) {
            Y[9] = -kY3a * y * (3.f * xx - yy);
            Dx[9] = -6.f * kY3a * x * y; Dy[9] = -3.f * kY3a * (xx - yy); Dz[9] = 0.f;
            Y[10] = kY3b * x * y * z;
            Dx[10] = kY3b * y * z; Dy[10] = kY3b * x * z; Dz[10] = kY3b * x * y;
            Y[11] = -kY3c * y * (4.f * zz - xx - yy);
            Dx[11] = 2.f * kY3c * x * y; Dy[11] = -kY3c * (4.f * zz - xx - 3.f * yy); Dz[11] = -8.f * kY3c * y * z;
            Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Dx[12] = -6.f * kY3d * x * z; Dy[12] = -6.f * kY3d * y * z; Dz[12] = kY3d * (6.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kY3c * x * (4.f * zz - xx - yy);
            Dx[13] = -kY3c * (4.f * zz - 3.f * xx - yy); Dy[13] = 2.f * kY3c * x * y; Dz[13] = -8.f * kY3c * x * z;
            Y[14] = kY3e * z * (xx - yy);
            Dx[14] = 2.f * kY3e * x * z; Dy[14] = -2.f * kY3e * y * z; Dz[14] = kY3e * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.f * yy);
            Dx[15] = -3.f * kY3a * (xx - yy); Dy[15] = 6.f * kY3a * x * y; Dz[15] = 0.f;
        }
    }
    // Which channels were clamped at zero in the forward pass.
    float s[3] = {0.5f, 0.5f, 0.5f};
    for (int k = 0; k < kK; ++k)
        for (int c = 0; c < 3; ++c) s[c] = fmaf(Y[k], __ldg(src + 3 * k + c), s[c]);
    float g[3];
    for (int c = 0; c < 3; ++c) g[c] = s[c] > 0.f ? gr[c] : 0.f;
    float3 gd = make_float3(0.f, 0.f, 0.f);
    for (int k = 0; k < kK; ++k) {
        float dot = 0.f;
        for (int c = 0; c < 3; ++c) {
            dsrc[3 * k + c] = Y[k] * g[c];
            dot = fmaf(__ldg(src + 3 * k + c), g[c], dot);
        }
        gd.x = fmaf(Dx[k], dot, gd.x);
        gd.y = fmaf(Dy[k], dot, gd.y);
        gd.z = fmaf(Dz[k], dot, gd.z);
    }
    return gd;
}

// Gradients of Gaussian i's parameters from the gradients of its record
// (rec_grad, 9 floats); false, with all outputs zero, when it received none.
template <int DEG>
__device__ __forceinline__ bool project_bwd_one(const ProjectArgs &P, const GsCameraDev &K, int64_t i,
                                                const float *rec_grad, float *dsh, float *gm_out, float *gls_out,
                                                float *gq_out, float *go_out) {
    constexpr int kK = (DEG + 1) * (DEG + 1);
    float gr9[9];
    bool any = false;
    for (int f = 0; f < 9; ++f) {
        gr9[f] = rec_grad[f];
        any |= gr9[f] != 0.f;
    }
    if (!any) {
        for (int a = 0; a < 3; ++a) gm_out[a] = 0.f;
        for (int a = 0; a < 3; ++a) gls_out[a] = 0.f;
        for (int a = 0; a < 4; ++a) gq_out[a] = 0.f;
        *go_out = 0.f;
        for (int a = 0; a < kK * 3; ++a) dsh[a] = 0.f;
        return false;
    }
    // ---- forward recomputation ----
    const float mx = P.means[3 * i], my = P.means[3 * i + 1], mz = P.means[3 * i + 2];
    const float tx = fmaf(K.R[0], mx, fmaf(K.R[1], my, fmaf(K.R[2], mz, K.t[0])));
    const float ty = fmaf(K.R[3], mx, fmaf(K.R[4], my, fmaf(K.R[5], mz, K.t[1])));
    const float tz = fmaf(K.R[6], mx, fmaf(K.R[7], my, fmaf(K.R[8], mz, K.t[2])));
    const float q0 = P.quats[4 * i], q1 = P.quats[4 * i + 1], q2 = P.quats[4 * i + 2], q3 = P.quats[4 * i + 3];
    const float qn = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    const float qw = q0 / qn, qx = q1 / qn, qy = q2 / qn, qz = q3 / qn;
    const float sc[3] = {expf(P.log_scales[3 * i]), expf(P.log_scales[3 * i + 1]), expf(P.log_scales[3 * i + 2])};
    float Rm[3][3];
    Rm[0][0] = 1.f - 2.f * (qy * qy + qz * qz); Rm[0][1] = 2.f * (qx * qy - qw * qz); Rm[0][2] = 2.f * (qx * qz + qw * qy);
    Rm[1][0] = 2.f * (qx * qy + qw * qz); Rm[1][1] = 1.f - 2.f * (qx * qx + qz * qz); Rm[1][2] = 2.f * (qy * qz - qw * qx);
    Rm[2][0] = 2.f * (qx * qz - qw * qy); Rm[2][1] = 2.f * (qy * qz + qw * qx); Rm[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
    float M[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[r][c] = Rm[r][c] * sc[c];
    const float iz = 1.f / tz;
    const float rx_raw = tx * iz, ry_raw = ty * iz;
    const bool rx_free = rx_raw > -K.lim_x && rx_raw < K.lim_x;
    const bool ry_free = ry_raw > -K.lim_y && ry_raw < K.lim_y;
    const float rx = fminf(K.lim_x, fmaxf(-K.lim_x, rx_raw));
    const float ry = fminf(K.lim_y, fmaxf(-K.lim_y, ry_raw));
    float T0[3], T1[3];
    for (int c = 0; c < 3; ++c) {
        T0[c] = K.fx * iz * (K.R[c] - rx * K.R[6 + c]);
        T1[c] = K.fy * iz * (K.R[3 + c] - ry * K.R[6 + c]);
    }
    float A0[3], A1[3];
    for (int c = 0; c < 3; ++c) {
        A0[c] = T0[0] * M[0][c] + T0[1] * M[1][c] + T0[2] * M[2][c];
        A1[c] = T1[0] * M[0][c] + T1[1] * M[1][c] + T1[2] * M[2][c];
    }
    const float a = A0[0] * A0[0] + A0[1] * A0[1] + A0[2] * A0[2] + kDilation;
    const float c = A1[0] * A1[0] + A1[1] * A1[1] + A1[2] * A1[2] + kDilation;
    const float b = A0[0] * A1[0] + A0[1] * A1[1] + A0[2] * A1[2];
    const float cr0 = A0[1] * A1[2] - A0[2] * A1[1], cr1 = A0[2] * A1[0] - A0[0] * A1[2],
                cr2 = A0[0] * A1[1] - A0[1] * A1[0];
    const float det = cr0 * cr0 + cr1 * cr1 + cr2 * cr2 + kDilation * (a + c - 2.f * kDilation) +
                      kDilation * kDilation;
    const float o = 1.f / (1.f + expf(-P.logits[i]));

    // ---- backward ----
    const float gu = gr9[0], gv = gr9[1], gQ00 = gr9[2], gQ01 = gr9[3], gQ11 = gr9[4], go = gr9[5];
    // conic = (c, -b, a) / det
    const float id = 1.f / det, id2 = id * id;
    const float ga = gQ00 * (-c * c * id2) + gQ01 * (b * c * id2) + gQ11 * (id - a * c * id2);
    const float gc = gQ00 * (id - a * c * id2) + gQ01 * (a * b * id2) + gQ11 * (-a * a * id2);
    const float gb = gQ00 * (2.f * b * c * id2) + gQ01 * (-id - 2.f * b * b * id2) + gQ11 * (2.f * a * b * id2);
    float gA0[3], gA1[3];
    for (int k = 0; k < 3; ++k) {
        gA0[k] = 2.f * ga * A0[k] + gb * A1[k];
        gA1[k] = 2.f * gc * A1[k] + gb * A0[k];
    }
    // A = T M
    float gT0[3], gT1[3], gM[3][3];
    for (int r = 0; r < 3; ++r) {
        gT0[r] = gA0[0] * M[r][0] + gA0[1] * M[r][1] + gA0[2] * M[r][2];
        gT1[r] = gA1[0] * M[r][0] + gA1[1] * M[r][1] + gA1[2] * M[r][2];
        for (int k = 0; k < 3; ++k) gM[r][k] = T0[r] * gA0[k] + T1[r] * gA1[k];
    }
    // M = R diag(s)
    float gR[3][3], gls[3];
    for (int k = 0; k < 3; ++k) {
        float gs = 0.f;
        for (int r = 0; r < 3; ++r) {
            gR[r][k] = gM[r][k] * sc[k];
            gs = fmaf(gM[r][k], Rm[r][k], gs);
        }
        gls[k] = gs * sc[k];
    }
    // R(q^) then q^ = q / |q|
    const float gqw = 2.f * (-qz * gR[0][1] + qy * gR[0][2] + qz * gR[1][0] - qx * gR[1][2] - qy * gR[2][0] + qx * gR[2][1]);
    const float gqx = 2.f * (qy * gR[0][1] + qz * gR[0][2] + qy * gR[1][0] - 2.f * qx * gR[1][1] - qw * gR[1][2] +
                             qz * gR[2][0] + qw * gR[2][1] - 2.f * qx * gR[2][2]);
    const float gqy = 2.f * (-2.f * qy * gR[0][0] + qx * gR[0][1] + qw * gR[0][2] + qx * gR[1][0] + qz * gR[1][2] -
                             qw * gR[2][0] + qz * gR[2][1] - 2.f * qy * gR[2][2]);
    const float gqz = 2.f * (-2.f * qz * gR[0][0] - qw * gR[0][1] + qx * gR[0][2] + qw * gR[1][0] - 2.f * qz * gR[1][1] +
                             qy * gR[1][2] + qx * gR[2][0] + qy * gR[2][1]);
    const float qdot = qw * gqw + qx * gqx + qy * gqy + qz * gqz;
    // T0 = fx iz (W0 - rx W2), T1 = fy iz (W1 - ry W2)
    float g_rx = 0.f, g_ry = 0.f, g_iz = 0.f;
    for (int k = 0; k < 3; ++k) {
        g_rx = fmaf(gT0[k], -K.fx * iz * K.R[6 + k], g_rx);
        g_ry = fmaf(gT1[k], -K.fy * iz * K.R[6 + k], g_ry);
        g_iz = fmaf(gT0[k], K.fx * (K.R[k] - rx * K.R[6 + k]), g_iz);
        g_iz = fmaf(gT1[k], K.fy * (K.R[3 + k] - ry * K.R[6 + k]), g_iz);
    }
    float g_tx = gu * K.fx * iz, g_ty = gv * K.fy * iz;
    g_iz += gu * K.fx * tx + gv * K.fy * ty;
    if (rx_free) { g_tx += g_rx * iz; g_iz += g_rx * tx; }
    if (ry_free) { g_ty += g_ry * iz; g_iz += g_ry * ty; }
    const float g_tz = -g_iz * iz * iz;
    // t = W mu + t_c
    float gm[3];
    for (int k = 0; k < 3; ++k) gm[k] = K.R[k] * g_tx + K.R[3 + k] * g_ty + K.R[6 + k] * g_tz;
    // colour: direction d = (mu - C) / |mu - C|
    float vx = mx - K.C[0], vy = my - K.C[1], vz = mz - K.C[2];
    const float vn = sqrtf(vx * vx + vy * vy + vz * vz);
    const float dx = vx / vn, dy = vy / vn, dz = vz / vn;
    const float grgb[3] = {gr9[6], gr9[7], gr9[8]};
    const float3 gd = sh_colour_bwd<DEG>(P.sh + (size_t)i * kK * 3, dsh, dx, dy, dz, grgb);
    const float ddot = dx * gd.x + dy * gd.y + dz * gd.z;
    gm[0] += (gd.x - dx * ddot) / vn;
    gm[1] += (gd.y - dy * ddot) / vn;
    gm[2] += (gd.z - dz * ddot) / vn;

    for (int k = 0; k < 3; ++k) gm_out[k] = gm[k];
    for (int k = 0; k < 3; ++k) gls_out[k] = gls[k];
    gq_out[0] = (gqw - qw * qdot) / qn;
    gq_out[1] = (gqx - qx * qdot) / qn;
    gq_out[2] = (gqy - qy * qdot) / qn;
    gq_out[3] = (gqz - qz * qdot) / qn;
    *go_out = go * o * (1.f - o);
    return true;
}

}  // namespace


namespace {

// One thread per compact record slot of a joint batch: the gradients of
// Gaussian i under view v's camera, added to i's gradients (several views
// see the same Gaussian).
template <int DEG>
__global__ void __launch_bounds__(128)
    project_bwd_batch_kernel(const ProjectArgs P, const ViewDesc *views, const uint2 *meta, int64_t n_records,
                             const float *d_rec, const gs_grads out) {
    constexpr int kS = (DEG + 1) * (DEG + 1) * 3;
    const int64_t j = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (j >= n_records) return;
    const uint2 m = meta[j];  // (view, Gaussian)
    const int64_t i = m.y;
    float dsh[kS], gm[3], gls[3], gq[4], go;
    if (!project_bwd_one<DEG>(P, views[m.x].cam, i, d_rec + kRecGradStride * j, dsh, gm, gls, gq, &go)) return;
    for (int a = 0; a < 3; ++a) atomicAdd(out.d_means + 3 * i + a, gm[a]);
    for (int a = 0; a < 3; ++a) atomicAdd(out.d_log_scales + 3 * i + a, gls[a]);
    for (int a = 0; a < 4; ++a) atomicAdd(out.d_quats + 4 * i + a, gq[a]);
    atomicAdd(out.d_opacity_logits + i, go);
#pragma unroll
    for (int a = 0; a < kS; ++a)
        if (dsh[a] != 0.f) atomicAdd(out.d_sh + kS * i + a, dsh[a]);
}

}  // namespace

cudaError_t gs_launch_project_bwd_batch(const gs_gaussians &g, const ViewDesc *views, const uint2 *meta,
                                        int64_t n_records, const float *d_rec, const gs_grads &out, cudaStream_t s) {
    const int64_t rec_capacity = n_records;
    if (rec_capacity <= 0 || g.n == 0) return cudaSuccess;
    const ProjectArgs P{g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, g.n, GsCameraDev{}, GsGrid{},
                        nullptr, nullptr, false, false};
    const unsigned blocks = (unsigned)((rec_capacity + 127) / 128);
    switch (g.sh_degree) {
        case 0: project_bwd_batch_kernel<0><<<blocks, 128, 0, s>>>(P, views, meta, n_records, d_rec, out); break;
        case 1: project_bwd_batch_kernel<1><<<blocks, 128, 0, s>>>(P, views, meta, n_records, d_rec, out); break;
        case 2: project_bwd_batch_kernel<2><<<blocks, 128, 0, s>>>(P, views, meta, n_records, d_rec, out); break;
        default: project_bwd_batch_kernel<3><<<blocks, 128, 0, s>>>(P, views, meta, n_records, d_rec, out); break;
    }
    return cudaGetLastError();
}

namespace {
// The zeros of the gradient arrays are written by memsets (at copy speed);
// this kernel then writes, one thread per Gaussian, the gradients of the
// Gaussians whose records received any (the visible ones; a frame has few of
// them among the scene's Gaussians).
template <int DEG>
__global__ void __launch_bounds__(128) project_bwd_sparse_kernel(const ProjectBwdArgs B) {
    constexpr int kS = (DEG + 1) * (DEG + 1) * 3;
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (i >= B.P.n) return;
    float dsh[kS], gm[3], gls[3], gq[4], go;
    if (!project_bwd_one<DEG>(B.P, B.P.cam, i, B.d_rec + kRecGradStride * i, dsh, gm, gls, gq, &go)) return;
    for (int a = 0; a < 3; ++a) B.d_means[3 * i + a] = gm[a];
    for (int a = 0; a < 3; ++a) B.d_log_scales[3 * i + a] = gls[a];
    for (int a = 0; a < 4; ++a) B.d_quats[4 * i + a] = gq[a];
    B.d_logits[i] = go;
#pragma unroll
    for (int a = 0; a < kS; ++a) B.d_sh[kS * i + a] = dsh[a];
}
}  // namespace

namespace {
// Zeros of several float arrays in one launch: blockIdx.y picks the array,
// blocks stride over its 16-byte chunks (the 4-byte words before the first
// and after the last whole chunk are written one by one).
struct ZeroSpans {
    float *ptr[6];
    size_t words[6];
};

__global__ void __launch_bounds__(256) zero_spans_kernel(const ZeroSpans z) {
    float *p = z.ptr[blockIdx.y];
    const size_t n = z.words[blockIdx.y];
    if (!p || n == 0) return;
    const size_t head = ((16 - reinterpret_cast<uintptr_t>(p) % 16) % 16) / 4;  // words before a 16-byte boundary
    const size_t h = head < n ? head : n;
    const size_t chunks = (n - h) / 4;
    uint4 *body = reinterpret_cast<uint4 *>(p + h);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < chunks; i += (size_t)gridDim.x * blockDim.x)
        body[i] = make_uint4(0u, 0u, 0u, 0u);
    if (blockIdx.x == 0 && threadIdx.x < 8) {
        const size_t t = h + chunks * 4;  // first word of the tail
        if (threadIdx.x < h) p[threadIdx.x] = 0.f;
        if (t + threadIdx.x < n && threadIdx.x < 4) p[t + threadIdx.x] = 0.f;
    }
}
}  // namespace

cudaError_t gs_launch_zero_grads(const gs_gaussians &g, const gs_grads &out, float *d_rec, size_t rec_words,
                                 cudaStream_t s) {
    const size_t n = g.n > 0 ? (size_t)g.n : 0, kS = (size_t)(g.sh_degree + 1) * (g.sh_degree + 1) * 3;
    ZeroSpans z{{out.d_means, out.d_log_scales, out.d_quats, out.d_opacity_logits, out.d_sh, d_rec},
                {n * 3, n * 3, n * 4, n, n * kS, rec_words}};
    for (int i = 0; i < 6; ++i)
        if (reinterpret_cast<uintptr_t>(z.ptr[i]) % 4 != 0) return cudaErrorInvalidValue;  // float arrays
    zero_spans_kernel<<<dim3(152 * 4, 6, 1), 256, 0, s>>>(z);
    return cudaGetLastError();
}

cudaError_t gs_launch_project_bwd(const gs_gaussians &g, const GsCameraDev &cam, const GsGrid &grid,
                                  const float *d_rec, const gs_grads &out, cudaStream_t s) {
    if (g.n == 0) return cudaSuccess;
    ProjectBwdArgs B;
    B.P = ProjectArgs{g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, g.n, cam, grid, nullptr, nullptr,
                      false, false};
    B.d_rec = d_rec;
    B.d_means = out.d_means;
    B.d_log_scales = out.d_log_scales;
    B.d_quats = out.d_quats;
    B.d_logits = out.d_opacity_logits;
    B.d_sh = out.d_sh;
    // The arrays hold zeros already (gs_launch_zero_grads); only the
    // Gaussians with gradients are written: measured faster than writing
    // every Gaussian's gradients from one kernel (which wrote zeros at a
    // fraction of the copy bandwidth).
    const unsigned blocks = (unsigned)((g.n + 127) / 128);
    switch (g.sh_degree) {
        case 0: project_bwd_sparse_kernel<0><<<blocks, 128, 0, s>>>(B); break;
        case 1: project_bwd_sparse_kernel<1><<<blocks, 128, 0, s>>>(B); break;
        case 2: project_bwd_sparse_kernel<2><<<blocks, 128, 0, s>>>(B); break;
        default: project_bwd_sparse_kernel<3><<<blocks, 128, 0, s>>>(B); break;
    }
    return cudaGetLastError();
}

size_t gs_batch_scratch_bytes(int64_t rec_capacity, int64_t key_capacity, int64_t n, int n_views) {
    return front_layout(rec_capacity, key_capacity, (n + kBatchBlock - 1) / kBatchBlock * n_views * kBatchRounds,
                        false)
        .total;
}

cudaError_t gs_launch_project_bin_batch(const gs_gaussians &g, const ViewDesc *views_dev, int n_views,
                                        gs_record *records, const gs::BlendRecordOut &br, uint2 *meta, int64_t rec_capacity, uint32_t *keys,
                                        uint32_t *values, int64_t key_capacity, unsigned long long *counts,
                                        void *scratch, const GsSortScratch &sc, uint32_t *d_err, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counts, 0, 5 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int64_t nb = (g.n + kBatchBlock - 1) / kBatchBlock, n_seg = nb * n_views * kBatchRounds;
    const FrontLayout L = front_layout(rec_capacity, key_capacity, n_seg, false);
    char *base = static_cast<char *>(scratch);
    e = cudaMemsetAsync(base, 0, L.zero, s);
    if (e != cudaSuccess || g.n == 0 || n_views == 0) return e;
    ListBatchArgs A;
    A.P = ProjectArgs{g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, g.n, GsCameraDev{}, GsGrid{},
                      reinterpret_cast<float4 *>(records), nullptr,
                      reinterpret_cast<uintptr_t>(g.sh) % 16 == 0,
                      reinterpret_cast<uintptr_t>(g.quats) % 16 == 0};
    A.views = views_dev;
    A.br = br;
    A.meta = meta;
    A.rec_capacity = rec_capacity;
    A.packed = reinterpret_cast<unsigned long long *>(base);
    A.seg = reinterpret_cast<uint2 *>(base + L.seg);
    A.seg_dst = reinterpret_cast<uint32_t *>(base + L.seg_dst);
    A.lkeys = reinterpret_cast<uint64_t *>(base + L.lkeys);
    A.lvals = reinterpret_cast<uint32_t *>(base + L.lvals);
    A.dsc = gs_sort_carve_digits(base + L.dsort, rec_capacity, 0, kDepthPasses, kDepthItems);
    A.counts = counts;
    A.d_err = d_err;
    A.views_fast = nb <= 65535;
    const dim3 grid = A.views_fast ? dim3((unsigned)n_views, (unsigned)nb) : dim3((unsigned)nb, (unsigned)n_views);
    switch (g.sh_degree) {
        case 0: e = launch_project_list_batch<0>(A, grid, s); break;
        case 1: e = launch_project_list_batch<1>(A, grid, s); break;
        case 2: e = launch_project_list_batch<2>(A, grid, s); break;
        default: e = launch_project_list_batch<3>(A, grid, s); break;
    }
    if (e != cudaSuccess) return e;
    EmitArgs E{};
    E.records = reinterpret_cast<const float4 *>(records);
    E.meta = meta;
    E.views = views_dev;
    E.keys = keys;
    E.values = values;
    E.capacity = key_capacity;
    E.sc = sc;
    return launch_list_stages(L, base, rec_capacity, n_seg, A.dsc, E, 4, true, false, counts, d_err, s, nullptr);
}
