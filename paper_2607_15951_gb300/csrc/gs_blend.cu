// gs_blend.cu — per-tile front-to-back alpha compositing (Eq. 1; Sec. 4.5
// step 3). One thread block per screen tile. The tile's depth-ordered list
// is walked in batches staged in shared memory; every record is turned once
// per block into the form the inner loop wants:
//   A, B, C   the conic scaled to the base-2 exponent, so that
//             power * log2(e) = A dx^2 + B dx dy + C dy^2
//   thr       log2(1 / (255 opacity)): alpha >= 1/255  <=>  exponent >= thr
//   box       a conservative bounding box of the pixels where the record can
//             reach alpha >= 1/255 (used only by the culled variant).
//
// Variants (identical outputs):
//  * culled (default): each warp owns an 8x8 pixel block, two pixels per lane
//    sharing the x terms; per 32 records one ballot tells the warp which
//    records' boxes touch its block, and it walks only those.
//  * basic: one thread per pixel walks every record (reference schedule).
// Both evaluate a (pixel, record) pair with the same function, so a record a
// warp skips is exactly one whose evaluation would have been skipped.
#include "gs_internal.cuh"

namespace {

using namespace gs;

constexpr float kLog2e = 1.4426950408889634f;
constexpr int kBatch = 256;

struct BlendArgs {
    const float4 *records;
    const uint32_t *values;
    const uint32_t *ranges;
    GsGrid grid;
    int width, height;
    float bg[3];
    float *rgb;
    float *final_T;
    int32_t *n_contrib;
    int32_t *n_eval;
};

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Shared-memory form of one record.
struct SRec {
    float4 *a;    // (u, v, A, B)
    float4 *b;    // (C, opacity, thr, blue)
    float2 *rg;   // (red, green)
    float4 *box;  // (x0, x1, y0, y1) pixel-centre box where alpha can reach 1/255
};

// Builds the shared form of record g at slot s.
__device__ __forceinline__ void stage_record(const float4 *__restrict__ rec, uint32_t g, int s,
                                             const SRec &S, bool want_box) {
    const float4 r0 = __ldg(rec + 3 * (size_t)g);
    const float4 r1 = __ldg(rec + 3 * (size_t)g + 1);
    const float blue = __ldg(reinterpret_cast<const float *>(rec + 3 * (size_t)g + 2));
    const float q00 = r0.z, q01 = r0.w, q11 = r1.x, o = r1.y;
    const float A = -0.5f * kLog2e * q00, B = -kLog2e * q01, C = -0.5f * kLog2e * q11;
    const float thr = -log2f(255.f * o);
    S.a[s] = make_float4(r0.x, r0.y, A, B);
    S.b[s] = make_float4(C, o, thr, blue);
    S.rg[s] = make_float2(r1.z, r1.w);
    if (!want_box) return;
    // alpha >= 1/255 needs (1/2) d^T Q d <= L = ln(255 o). The axis-aligned
    // box of that ellipse has half-widths sqrt(2 L Sigma00), sqrt(2 L Sigma11)
    // with Sigma = Q^-1. L is inflated to cover the FP32 evaluation error of
    // the exponent, which is at most 8 eps kappa |exponent| for a conic of
    // condition number kappa <= (q00 + q11)^2 / det; det by Kahan's method.
    const float L = logf(255.f * o);
    float4 box = make_float4(1.f, -1.f, 1.f, -1.f);  // empty
    if (L > -1e-4f) {
        const float w = q01 * q01;
        const float e = fmaf(-q01, q01, w);
        const float det = fmaf(q00, q11, -w) + e;
        if (det > 0.f) {
            const float tr = q00 + q11;
            const float kappa = tr * tr / det;
            const float Lp = (fmaxf(L, 0.f) + 1e-4f) * (1.f + 64.f * 1.2e-7f * kappa);
            const float hx = sqrtf(2.f * Lp * (q11 / det)) * 1.0001f + 1e-3f;
            const float hy = sqrtf(2.f * Lp * (q00 / det)) * 1.0001f + 1e-3f;
            box = make_float4(r0.x - hx, r0.x + hx, r0.y - hy, r0.y + hy);
            if (!(hx < 3e38f) || !(hy < 3e38f)) box = make_float4(-3e38f, 3e38f, -3e38f, 3e38f);
        } else {
            box = make_float4(-3e38f, 3e38f, -3e38f, 3e38f);  // cannot bound: never cull
        }
    }
    S.box[s] = box;
}

// Per-pixel compositing state.
struct Pix {
    float T, r, g, b;
    int32_t last, eval;
    bool done;
};

// One (pixel, record) step of Eq. 1 with the standard rules; e = exponent in
// base 2. Returns after updating the pixel.
__device__ __forceinline__ void composite(Pix &p, float e, float o, float thr, float cr, float cg,
                                          float cb, int32_t pos) {
    if (e > 0.f || e < thr) return;  // power > 0, or alpha < 1/255
    const float alpha = fminf(kAlphaMax, o * ex2(e));
    const float Tn = p.T * (1.f - alpha);
    if (Tn < kTMin) {
        p.done = true;
        p.eval = pos;
        return;
    }
    const float w = alpha * p.T;
    p.r = fmaf(cr, w, p.r);
    p.g = fmaf(cg, w, p.g);
    p.b = fmaf(cb, w, p.b);
    p.T = Tn;
    p.last = pos;
}

__device__ __forceinline__ void write_pixel(const BlendArgs &a, int px, int py, const Pix &p) {
    if (px >= a.width || py >= a.height) return;
    const size_t i = (size_t)py * a.width + px;
    a.rgb[3 * i + 0] = fmaf(p.T, a.bg[0], p.r);
    a.rgb[3 * i + 1] = fmaf(p.T, a.bg[1], p.g);
    a.rgb[3 * i + 2] = fmaf(p.T, a.bg[2], p.b);
    if (a.final_T) a.final_T[i] = p.T;
    if (a.n_contrib) a.n_contrib[i] = p.last;
    if (a.n_eval) a.n_eval[i] = p.eval;
}

// ---------------------------------------------------------------------------
// Culled variant: warps own 8x8 blocks, two pixels per lane.
// ---------------------------------------------------------------------------
template <int TW, int TH>
__global__ void __launch_bounds__((TW / 8) * (TH / 8) * 32) blend_culled_kernel(const BlendArgs a) {
    constexpr int kWX = TW / 8, kWarps = kWX * (TH / 8), kThreads = kWarps * 32;
    __shared__ float4 s_a[kBatch], s_b[kBatch], s_box[kBatch];
    __shared__ float2 s_rg[kBatch];
    const SRec S{s_a, s_b, s_rg, s_box};

    const int tile = blockIdx.x;
    const int tx = tile % a.grid.tiles_x, ty = tile / a.grid.tiles_x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bx = tx * TW + (warp % kWX) * 8, by = ty * TH + (warp / kWX) * 8;
    const int px = bx + (lane & 7), py0 = by + (lane >> 3), py1 = py0 + 4;
    const float fx = px + 0.5f, fy0 = py0 + 0.5f, fy1 = py1 + 0.5f;
    // Pixel-centre extent of this warp's block (clipped to the image).
    const float wx0 = bx + 0.5f, wx1 = fminf(bx + 7.5f, a.width - 0.5f);
    const float wy0 = by + 0.5f, wy1 = fminf(by + 7.5f, a.height - 0.5f);

    const uint32_t first = a.ranges[2 * tile], last = a.ranges[2 * tile + 1];
    Pix p0{1.f, 0.f, 0.f, 0.f, 0, 0, !(px < a.width && py0 < a.height)};
    Pix p1{1.f, 0.f, 0.f, 0.f, 0, 0, !(px < a.width && py1 < a.height)};
    bool warp_done = __all_sync(0xffffffffu, p0.done && p1.done);

    for (uint32_t start = first; start < last; start += kBatch) {
        if (__syncthreads_count(warp_done) == kThreads) break;
        for (int s = tid; s < kBatch; s += kThreads) {
            const uint32_t k = start + s;
            if (k < last) stage_record(a.records, a.values[k], s, S, true);
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBatch, last - start);
        const int32_t pos0 = (int32_t)(start - first) + 1;  // list position of slot 0
        if (!warp_done) {
            for (int c = 0; c < cnt; c += 32) {
                const int j = c + lane;
                bool hit = false;
                if (j < cnt) {
                    const float4 bx4 = s_box[j];
                    hit = bx4.x <= wx1 && bx4.y >= wx0 && bx4.z <= wy1 && bx4.w >= wy0;
                }
                uint32_t bits = __ballot_sync(0xffffffffu, hit);
                while (bits) {
                    const int jj = c + __ffs(bits) - 1;
                    bits &= bits - 1;
                    const float4 ra = s_a[jj];
                    const float4 rb = s_b[jj];
                    const float2 rg = s_rg[jj];
                    const float dx = fx - ra.x;
                    const float adx2 = ra.z * dx * dx, bdx = ra.w * dx;
                    if (!p0.done) {
                        const float dy = fy0 - ra.y;
                        composite(p0, fmaf(dy, fmaf(rb.x, dy, bdx), adx2), rb.y, rb.z, rg.x, rg.y, rb.w,
                                  pos0 + jj);
                    }
                    if (!p1.done) {
                        const float dy = fy1 - ra.y;
                        composite(p1, fmaf(dy, fmaf(rb.x, dy, bdx), adx2), rb.y, rb.z, rg.x, rg.y, rb.w,
                                  pos0 + jj);
                    }
                }
                warp_done = __all_sync(0xffffffffu, p0.done && p1.done);
                if (warp_done) break;
            }
        }
    }
    const int32_t n_list = (int32_t)(last - first);
    if (!p0.done) p0.eval = n_list;
    if (!p1.done) p1.eval = n_list;
    write_pixel(a, px, py0, p0);
    write_pixel(a, px, py1, p1);
}

// ---------------------------------------------------------------------------
// Basic variant: one thread per pixel, every record evaluated.
// ---------------------------------------------------------------------------
template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) blend_basic_kernel(const BlendArgs a) {
    constexpr int kN = TW * TH;
    __shared__ float4 s_a[kBatch], s_b[kBatch];
    __shared__ float2 s_rg[kBatch];
    const SRec S{s_a, s_b, s_rg, nullptr};

    const int tile = blockIdx.x;
    const int tx = tile % a.grid.tiles_x, ty = tile / a.grid.tiles_x;
    const int tid = threadIdx.x;
    const int px = tx * TW + tid % TW, py = ty * TH + tid / TW;
    const float fx = px + 0.5f, fy = py + 0.5f;
    const uint32_t first = a.ranges[2 * tile], last = a.ranges[2 * tile + 1];
    Pix p{1.f, 0.f, 0.f, 0.f, 0, 0, !(px < a.width && py < a.height)};

    for (uint32_t start = first; start < last; start += kBatch) {
        if (__syncthreads_count(p.done) == kN) break;
        for (int s = tid; s < kBatch; s += kN) {
            const uint32_t k = start + s;
            if (k < last) stage_record(a.records, a.values[k], s, S, false);
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBatch, last - start);
        const int32_t pos0 = (int32_t)(start - first) + 1;
        for (int j = 0; j < cnt && !p.done; ++j) {
            const float4 ra = s_a[j];
            const float4 rb = s_b[j];
            const float2 rg = s_rg[j];
            const float dx = fx - ra.x, dy = fy - ra.y;
            const float e = fmaf(dy, fmaf(rb.x, dy, ra.w * dx), ra.z * dx * dx);
            composite(p, e, rb.y, rb.z, rg.x, rg.y, rb.w, pos0 + j);
        }
    }
    if (!p.done) p.eval = (int32_t)(last - first);
    write_pixel(a, px, py, p);
}

}  // namespace

cudaError_t gs_launch_blend(const gs_record *records, const uint32_t *values, const uint32_t *ranges,
                            const GsGrid &grid, int width, int height, const float bg[3],
                            const gs_framebuffer &fb, int variant, cudaStream_t s) {
    BlendArgs a{reinterpret_cast<const float4 *>(records), values, ranges, grid, width, height,
                {bg[0], bg[1], bg[2]}, fb.rgb, fb.final_T, fb.n_contrib, fb.n_eval};
    const unsigned blocks = (unsigned)(grid.tiles_x * grid.tiles_y);
    const int tw = grid.tile_w, th = grid.tile_h;
    if (variant == GS_BLEND_BASIC) {
        if (tw == 16 && th == 16) blend_basic_kernel<16, 16><<<blocks, 256, 0, s>>>(a);
        else if (tw == 16 && th == 8) blend_basic_kernel<16, 8><<<blocks, 128, 0, s>>>(a);
        else blend_basic_kernel<8, 8><<<blocks, 64, 0, s>>>(a);
    } else {
        if (tw == 16 && th == 16) blend_culled_kernel<16, 16><<<blocks, 128, 0, s>>>(a);
        else if (tw == 16 && th == 8) blend_culled_kernel<16, 8><<<blocks, 64, 0, s>>>(a);
        else blend_culled_kernel<8, 8><<<blocks, 32, 0, s>>>(a);
    }
    return cudaGetLastError();
}
