// gs_blend.cu — per-tile front-to-back alpha compositing (Eq. 1; Sec. 4.5
// step 3). One thread block per screen tile. The tile's depth-ordered list
// is walked in batches staged in shared memory, in the form the inner loop
// wants (the blend record written by the render path's projection, or the
// same constants computed from a caller's gs_record):
//   A, B, C   the conic scaled to the base-2 exponent, so that
//             power * log2(e) = A dx^2 + B dx dy + C dy^2
//   thr       log2(1 / (255 opacity)): alpha >= 1/255  <=>  exponent >= thr
//   box       a conservative bounding box of the pixels where the record can
//             reach alpha >= 1/255 (used only by the culled variants).
//
// Variants (identical outputs):
//  * culled (default): each warp owns an 8x4 pixel block, one pixel per lane;
//    per 32 records one ballot tells the warp which records' boxes touch its
//    block, and it walks only those.
//  * culled 8x8 / wide / tile: the same with 8x8 blocks (2 pixels per lane
//    sharing the x terms), 16x8 blocks (4) or one warp per 16x16 tile (8).
//    Finer blocks cull more records than the wider ones save in per-record
//    overhead (one 1080p frame alone: 8x4 0.197 ms, 8x8 0.229; with the box
//    test only, 16x8 0.369 and 16x16 0.694). 8x8 blocks issue the fewest
//    instructions and win when several frames' kernels share the GPU.
//  * basic: one thread per pixel walks every record (reference schedule).
// Both evaluate a (pixel, record) pair with the same function, so a record a
// warp skips is exactly one whose evaluation would have been skipped.
#include "gs_internal.cuh"

namespace {

using namespace gs;

constexpr int kBatch = 256;

struct BlendArgs {
    RecordReader rd;
    const uint32_t *values;
    const uint32_t *ranges;
    GsGrid grid;
    int width, height;
    float bg[3];
    float *rgb;
    float *final_T;
    int32_t *n_contrib;
    int32_t *n_eval;
    // Block b blends (list) tile order[b] (longest list first) when set, else tile b.
    const uint32_t *order;
};

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Shared-memory form of one record.
// The alpha test reads only a and b; col is read for the pairs that pass it.
struct SRec {
    float4 *a;    // (u, v, A, B)
    float2 *b;    // (C, thr)
    float4 *col;  // (opacity, red, green, blue)
    float4 *box;  // (x0, x1, y0, y1) pixel-centre box where alpha can reach 1/255
};

// Builds the shared form of a record at slot s from its blend-record words
// (geo = u, v, A, B; aux = C, thr, hxy; col = opacity, red, green, blue).
__device__ __forceinline__ void stage_values(const float4 &geo, const float4 &aux, const float4 &col, int s,
                                             const SRec &S, bool want_box) {
    S.a[s] = geo;
    S.b[s] = make_float2(aux.x, aux.y);
    S.col[s] = col;
    if (!want_box) return;
    const float2 h = blend_box_half(aux.z);
    S.box[s] = make_float4(geo.x - h.x, geo.x + h.x, geo.y - h.y, geo.y + h.y);
}

// Builds the shared form of record g at slot s (RAW: from a gs_record).
template <bool RAW = false>
__device__ __forceinline__ void stage_record(const RecordReader &rd, uint32_t g, int s,
                                             const SRec &S, bool want_box) {
    float4 geo, aux, col;
    rd.load<RAW>(g, geo, aux, col);
    stage_values(geo, aux, col, s, S, want_box);
}

// Can a record reach alpha >= 1/255 at some pixel centre of the rectangle
// [x0, x1] x [y0, y1]? First its conservative box, then the exact maximum of
// the exponent e(d) = A dx^2 + B dx dy + C dy^2 (A, C < 0: a concave
// quadratic) over the rectangle: 0 if the mean is inside, else the largest of
// the four edge maxima, each at the clamped stationary point of e along that
// edge. The margin covers the FP32 rounding of both this maximum and the
// per-pixel exponent (far above a few ulps of the summed term magnitudes),
// so a record this rejects is one every pixel of the rectangle would skip.
__device__ __forceinline__ bool record_touches(const float4 &ra, const float2 &rb, const float4 &box, float x0,
                                               float x1, float y0, float y1) {
    if (!(box.x <= x1 && box.y >= x0 && box.z <= y1 && box.w >= y0)) return false;
    const float dx0 = x0 - ra.x, dx1 = x1 - ra.x, dy0 = y0 - ra.y, dy1 = y1 - ra.y;
    if (dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f) return true;
    const float A = ra.z, B = ra.w, C = rb.x, thr = rb.y;
    const float i2a = -0.5f / A, i2c = -0.5f / C;  // stationary points: dx = -B dy / 2A, dy = -B dx / 2C
    auto e = [&](float dx, float dy) { return fmaf(dy, fmaf(C, dy, B * dx), A * dx * dx); };
    const float ya = fminf(fmaxf(B * dx0 * i2c, dy0), dy1), yb = fminf(fmaxf(B * dx1 * i2c, dy0), dy1);
    const float xa = fminf(fmaxf(B * dy0 * i2a, dx0), dx1), xb = fminf(fmaxf(B * dy1 * i2a, dx0), dx1);
    const float m = fmaxf(fmaxf(e(dx0, ya), e(dx1, yb)), fmaxf(e(xa, dy0), e(xb, dy1)));
    const float dxm = fmaxf(fabsf(dx0), fabsf(dx1)), dym = fmaxf(fabsf(dy0), fabsf(dy1));
    const float scale = fmaf(-A, dxm * dxm, fmaf(fabsf(B), dxm * dym, -C * dym * dym));
    return m >= thr - (1e-5f * scale + 1e-6f);
}

// Per-pixel compositing state.
struct Pix {
    float T, r, g, b;
    int32_t last, eval;
    bool done;
};

// One (pixel, record) step of Eq. 1 with the standard rules; e = exponent in
// base 2. Returns after updating the pixel.
__device__ __forceinline__ void composite(Pix &p, float e, float thr, const float4 *col, int32_t pos) {
    if (e > 0.f || e < thr) return;  // power > 0, or alpha < 1/255
    const float4 c = *col;           // opacity, red, green, blue
    const float cr = c.y, cg = c.z, cb = c.w;
    const float alpha = fminf(kAlphaMax, c.x * ex2(e));
    const float w = alpha * p.T;  // this Gaussian's weight; T (1 - alpha) = T - w
    const float Tn = p.T - w;
    if (Tn < kTMin) {
        p.done = true;
        p.eval = pos;
        return;
    }
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
// Culled variant: warps own BW x BH pixel blocks (BW * BH / 32 pixels per
// lane, a column of pixels kRows apart sharing the x terms of a record).
// 8x8 blocks (default) cull finely; wider blocks amortise each record's
// ballot, shared-memory reads and x terms over more pixels.
// ---------------------------------------------------------------------------
template <int TW, int TH, int BW, int BH, int DEPTH = kBatch, bool RAW = false>
__device__ __forceinline__ void blend_tile_culled(const BlendArgs &a, int tile) {
    constexpr int kWX = TW / BW, kWarps = kWX * (TH / BH), kThreads = kWarps * 32;
    constexpr int kRows = 32 / BW;     // rows covered by the warp's lanes at once
    constexpr int kNP = BW * BH / 32;  // pixels per lane
    static_assert(kNP >= 1 && kRows * kNP == BH, "block shape");
    __shared__ float4 s_a[DEPTH], s_col[DEPTH], s_box[DEPTH];
    __shared__ float2 s_b[DEPTH];
    const SRec S{s_a, s_b, s_col, s_box};

    const int tx = tile % a.grid.tiles_x, ty = tile / a.grid.tiles_x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bx = tx * TW + (warp % kWX) * BW, by = ty * TH + (warp / kWX) * BH;
    const int px = bx + (lane % BW), py_base = by + lane / BW;
    const float fx = px + 0.5f;
    // Pixel-centre extent of this warp's block (clipped to the image).
    const float wx0 = bx + 0.5f, wx1 = fminf(bx + BW - 0.5f, a.width - 0.5f);
    const float wy0 = by + 0.5f, wy1 = fminf(by + BH - 0.5f, a.height - 0.5f);

    const uint32_t first = a.ranges[2 * tile], last = a.ranges[2 * tile + 1];
    Pix p[kNP];
    bool mine_done = true;
#pragma unroll
    for (int q = 0; q < kNP; ++q) {
        p[q] = Pix{1.f, 0.f, 0.f, 0.f, 0, 0, !(px < a.width && py_base + q * kRows < a.height)};
        mine_done = mine_done && p[q].done;
    }
    bool warp_done = __all_sync(0xffffffffu, mine_done);

    for (uint32_t start = first; start < last; start += DEPTH) {
        if (__syncthreads_count(warp_done) == kThreads) break;
        for (int s = tid; s < DEPTH; s += kThreads) {
            const uint32_t k = start + s;
            if (k < last) stage_record<RAW>(a.rd, a.values[k], s, S, true);
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)DEPTH, last - start);
        const int32_t pos0 = (int32_t)(start - first) + 1;  // list position of slot 0
        if (!warp_done) {
            for (int c = 0; c < cnt; c += 32) {
                const int j = c + lane;
                const bool hit = j < cnt && record_touches(s_a[j], s_b[j], s_box[j], wx0, wx1, wy0, wy1);
                uint32_t bits = __ballot_sync(0xffffffffu, hit);
                while (bits) {
                    const int jj = c + __ffs(bits) - 1;
                    bits &= bits - 1;
                    const float4 ra = s_a[jj];
                    const float2 rb = s_b[jj];
                    const float dx = fx - ra.x;
                    const float adx2 = ra.z * dx * dx, bdx = ra.w * dx;
#pragma unroll
                    for (int q = 0; q < kNP; ++q) {
                        if (!p[q].done) {
                            const float dy = (float)(py_base + q * kRows) + 0.5f - ra.y;
                            composite(p[q], fmaf(dy, fmaf(rb.x, dy, bdx), adx2), rb.y, &s_col[jj], pos0 + jj);
                        }
                    }
                }
                mine_done = true;
#pragma unroll
                for (int q = 0; q < kNP; ++q) mine_done = mine_done && p[q].done;
                warp_done = __all_sync(0xffffffffu, mine_done);
                if (warp_done) break;
            }
        }
    }
    const int32_t n_list = (int32_t)(last - first);
#pragma unroll
    for (int q = 0; q < kNP; ++q) {
        if (!p[q].done) p[q].eval = n_list;
        write_pixel(a, px, py_base + q * kRows, p[q]);
    }
}

// ---------------------------------------------------------------------------
// Two pixels per lane in packed FP32 pairs (8x8 blocks: the pixels of a lane
// share their column, rows r and r + 4). Blackwell's fma / mul / sub .f32x2
// instructions do one step for both pixels, each element rounded to nearest
// like the scalar operation, and the steps are the scalar schedule's, so the
// outputs equal it bit for bit. Every value the two pixels share is staged
// duplicated, as a pair ((u, u), (v, v), ...), so no instruction has to
// build a pair from a scalar.
// ---------------------------------------------------------------------------
typedef unsigned long long f32x2;

// Records staged per batch by the single-frame packed blend: 128 (10 KB of
// shared memory) rather than 256, so that other frames' kernels fit beside
// its blocks (eight 1080p frames in flight: 0.162 against 0.165 ms per frame;
// alone the same 0.352 ms).
constexpr int kBatchX2 = 128;

__device__ __forceinline__ f32x2 x2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void x2_split(f32x2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ float x2_lo(f32x2 v) {
    float lo, hi;
    x2_split(v, lo, hi);
    return lo;
}
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Shared-memory form of a record for the packed schedule (80 bytes):
// d0 = ((u, u), (v, v)), d1 = ((A, A), (B, B)), d2 = ((C, C), (o, o)),
// c01 = ((red, red), (green, green)), c2 = ((blue, blue), (thr, hxy)).
struct SRecX2 {
    ulonglong2 *d0, *d1, *d2, *c01, *c2;
};

// Stages a record from its blend-record words (geo, aux, col as RecordReader
// loads them).
__device__ __forceinline__ void stage_values_x2(const float4 &geo, const float4 &aux, const float4 &col, int s,
                                                const SRecX2 &S) {
    S.d0[s] = make_ulonglong2(x2(geo.x, geo.x), x2(geo.y, geo.y));
    S.d1[s] = make_ulonglong2(x2(geo.z, geo.z), x2(geo.w, geo.w));
    S.d2[s] = make_ulonglong2(x2(aux.x, aux.x), x2(col.x, col.x));
    S.c01[s] = make_ulonglong2(x2(col.y, col.y), x2(col.z, col.z));
    S.c2[s] = make_ulonglong2(x2(col.w, col.w), x2(aux.y, aux.z));
}

template <bool RAW = false>
__device__ __forceinline__ void stage_record_x2(const RecordReader &rd, uint32_t g, int s, const SRecX2 &S) {
    float4 geo, aux, col;
    rd.load<RAW>(g, geo, aux, col);
    stage_values_x2(geo, aux, col, s, S);
}

// record_touches on a packed record (the box from u, v and the half-widths).
__device__ __forceinline__ bool record_touches_x2(const SRecX2 &S, int j, float x0, float x1, float y0, float y1) {
    const float u = x2_lo(S.d0[j].x), v = x2_lo(S.d0[j].y);
    const ulonglong2 d1 = S.d1[j];
    float thr, hxy;
    x2_split(S.c2[j].y, thr, hxy);
    const float2 h = blend_box_half(hxy);
    return record_touches(make_float4(u, v, x2_lo(d1.x), x2_lo(d1.y)), make_float2(x2_lo(S.d2[j].x), thr),
                          make_float4(u - h.x, u + h.x, v - h.y, v + h.y), x0, x1, y0, y1);
}

// Compositing state of a lane's two pixels.
struct PixX2 {
    f32x2 T2, R2, G2, B2;
    int32_t last0, last1, eval0, eval1;
    bool done0, done1;
};

// One staged batch of cnt records (list positions pos0 + slot, or s_pos[slot]
// when given) blended into the lane's NP pixel pairs (all in one column, so
// the x terms of a record are computed once), in batch order, with the warp
// culling of the scalar schedule. Returns whether all the warp's pixels have
// stopped.
template <int NP>
__device__ __forceinline__ bool all_done_x2(const PixX2 (&P)[NP]) {
    bool mine = true;
#pragma unroll
    for (int q = 0; q < NP; ++q) mine = mine && P[q].done0 && P[q].done1;
    return __all_sync(0xffffffffu, mine);
}

template <int NP>
__device__ __forceinline__ bool blend_batch_x2(PixX2 (&P)[NP], const SRecX2 &S, const int32_t *s_pos, int32_t pos0,
                                               int cnt, f32x2 fx2, const f32x2 (&fy2)[NP], float wx0, float wx1,
                                               float wy0, float wy1, int lane) {
    for (int c = 0; c < cnt; c += 32) {
        const int j = c + lane;
        const bool hit = j < cnt && record_touches_x2(S, j, wx0, wx1, wy0, wy1);
        uint32_t bits = __ballot_sync(0xffffffffu, hit);
        while (bits) {
            const int jj = c + __ffs(bits) - 1;
            bits &= bits - 1;
            const ulonglong2 d0 = S.d0[jj], d1 = S.d1[jj];
            const f32x2 dx2 = x2_sub(fx2, d0.x);
            const f32x2 adx2 = x2_mul(x2_mul(d1.x, dx2), dx2), bdx2 = x2_mul(d1.y, dx2);
            const ulonglong2 d2 = S.d2[jj];
            const ulonglong2 c2 = S.c2[jj];
            float thr, hxy;
            x2_split(c2.y, thr, hxy);
            const int32_t pos = s_pos ? s_pos[jj] : pos0 + jj;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                PixX2 &Q = P[q];
                const f32x2 dy2 = x2_sub(fy2[q], d0.y);
                float e0, e1;
                x2_split(x2_fma(dy2, x2_fma(d2.x, dy2, bdx2), adx2), e0, e1);
                // power > 0, or alpha < 1/255: the pixel skips the record
                const bool t0 = !Q.done0 && !(e0 > 0.f || e0 < thr);
                const bool t1 = !Q.done1 && !(e1 > 0.f || e1 < thr);
                if (!(t0 || t1)) continue;
                float a0, a1;
                x2_split(x2_mul(d2.y, x2(ex2(e0), ex2(e1))), a0, a1);
                const f32x2 w2 = x2_mul(x2(fminf(kAlphaMax, a0), fminf(kAlphaMax, a1)), Q.T2);
                float w0, w1, tn0, tn1;
                x2_split(w2, w0, w1);
                x2_split(x2_sub(Q.T2, w2), tn0, tn1);
                // T would fall below the limit: the pixel stops before this record.
                const bool s0 = t0 && tn0 < kTMin, s1 = t1 && tn1 < kTMin;
                const bool u0 = t0 && !s0, u1 = t1 && !s1;
                const f32x2 we2 = x2(u0 ? w0 : 0.f, u1 ? w1 : 0.f);  // weights of the pixels that take it
                Q.T2 = x2_sub(Q.T2, we2);
                const ulonglong2 c01 = S.c01[jj];
                Q.R2 = x2_fma(c01.x, we2, Q.R2);
                Q.G2 = x2_fma(c01.y, we2, Q.G2);
                Q.B2 = x2_fma(c2.x, we2, Q.B2);
                Q.last0 = u0 ? pos : Q.last0;
                Q.last1 = u1 ? pos : Q.last1;
                if (s0 || s1) {
                    if (s0) Q.done0 = true, Q.eval0 = pos;
                    if (s1) Q.done1 = true, Q.eval1 = pos;
                }
            }
        }
        if (all_done_x2(P)) return true;
    }
    return all_done_x2(P);
}

// A lane's pixels in a BW x 8 warp block (BW = 8: two, BW = 16: four), all in
// column px: pair q holds rows py(q) and py(q) + 4, py(q) = by + lane / BW +
// q * 32 / BW.
template <int BW>
struct LaneX2 {
    static constexpr int NP = BW / 8, kRows = 32 / BW;
    int px, pyb;
    f32x2 fx2, fy2[NP];
    PixX2 P[NP];
    __device__ __forceinline__ LaneX2(const BlendArgs &a, int bx, int by, int lane) {
        px = bx + (lane % BW);
        pyb = by + lane / BW;
        fx2 = x2(px + 0.5f, px + 0.5f);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            const int y0 = pyb + q * kRows, y1 = y0 + 4;
            fy2[q] = x2((float)y0 + 0.5f, (float)y1 + 0.5f);
            P[q] = PixX2{x2(1.f, 1.f), x2(0.f, 0.f), x2(0.f, 0.f), x2(0.f, 0.f), 0, 0, 0, 0,
                         !(px < a.width && y0 < a.height), !(px < a.width && y1 < a.height)};
        }
    }
};

// Writes the lane's two pixels (n_list: list length, the n_eval of pixels
// that never stopped).
__device__ __forceinline__ void write_pixels_x2(const BlendArgs &a, const PixX2 &P, int px, int py0, int py1,
                                                int32_t n_list) {
    Pix p0, p1;
    x2_split(P.T2, p0.T, p1.T);
    x2_split(P.R2, p0.r, p1.r);
    x2_split(P.G2, p0.g, p1.g);
    x2_split(P.B2, p0.b, p1.b);
    p0.last = P.last0, p1.last = P.last1;
    p0.eval = P.done0 ? P.eval0 : n_list, p1.eval = P.done1 ? P.eval1 : n_list;
    write_pixel(a, px, py0, p0);
    write_pixel(a, px, py1, p1);
}

template <int TW, int TH, int BW, int DEPTH, bool RAW>
__device__ __forceinline__ void blend_tile_culled_x2(const BlendArgs &a, int tile) {
    constexpr int BH = 8;
    constexpr int kWX = TW / BW, kWarps = kWX * (TH / BH), kThreads = kWarps * 32;
    __shared__ ulonglong2 s_d0[DEPTH], s_d1[DEPTH], s_d2[DEPTH], s_c01[DEPTH], s_c2[DEPTH];
    const SRecX2 S{s_d0, s_d1, s_d2, s_c01, s_c2};

    const int tx = tile % a.grid.tiles_x, ty = tile / a.grid.tiles_x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bx = tx * TW + (warp % kWX) * BW, by = ty * TH + (warp / kWX) * BH;
    LaneX2<BW> L(a, bx, by, lane);
    const float wx0 = bx + 0.5f, wx1 = fminf(bx + BW - 0.5f, a.width - 0.5f);
    const float wy0 = by + 0.5f, wy1 = fminf(by + BH - 0.5f, a.height - 0.5f);

    const uint32_t first = a.ranges[2 * tile], last = a.ranges[2 * tile + 1];
    bool warp_done = all_done_x2(L.P);
    for (uint32_t start = first; start < last; start += DEPTH) {
        if (__syncthreads_count(warp_done) == kThreads) break;
        for (int s = tid; s < DEPTH; s += kThreads) {
            const uint32_t k = start + s;
            if (k < last) stage_record_x2<RAW>(a.rd, a.values[k], s, S);
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)DEPTH, last - start);
        const int32_t pos0 = (int32_t)(start - first) + 1;  // list position of slot 0
        if (!warp_done)
            warp_done = blend_batch_x2(L.P, S, nullptr, pos0, cnt, L.fx2, L.fy2, wx0, wx1, wy0, wy1, lane);
    }
    const int32_t n_list = (int32_t)(last - first);
#pragma unroll
    for (int q = 0; q < LaneX2<BW>::NP; ++q) {
        const int y0 = L.pyb + q * LaneX2<BW>::kRows;
        write_pixels_x2(a, L.P[q], L.px, y0, y0 + 4, n_list);
    }
}

// Resident blocks per SM the register allocation must allow. Two pixels per
// lane (8x8 blocks): 36 warps per SM (56 registers), measured 8 % more
// frames/s with frames in flight than the unconstrained 64 registers and the
// same time alone. Four pixels per lane (16x8 blocks, two packed pairs): 28
// warps per SM (72 registers). One pixel per lane: no constraint; stating it
// lets the allocator use 54 registers instead of 46, 4 % faster alone (0.205
// -> 0.197 ms on a 1080p frame) although one block fewer fits per SM.
constexpr int blend_min_blocks(int warps, int pixels_per_lane) {
    return pixels_per_lane == 2 ? (36 / warps < 32 ? 36 / warps : 32)  // at most 32 blocks per SM
         : pixels_per_lane == 4 ? (28 / warps < 32 ? 28 / warps : 32)
                                : 1;
}

template <int TW, int TH, int BW, int BH, bool RAW>
__global__ void __launch_bounds__((TW / BW) * (TH / BH) * 32,
                                  blend_min_blocks((TW / BW) * (TH / BH), BW * BH / 32))
    blend_culled_kernel(const BlendArgs a) {
    const int tile = a.order ? (int)a.order[blockIdx.x] : (int)blockIdx.x;
    if constexpr (BH == 8 && (BW == 8 || BW == 16) && !RAW)
        blend_tile_culled_x2<TW, TH, BW, kBatchX2, false>(a, tile);
    else blend_tile_culled<TW, TH, BW, BH, kBatch, RAW>(a, tile);
}

// ---------------------------------------------------------------------------
// Cluster variant: the per-tile lists are built for list tiles of CX x CY
// screen tiles of 16 x 16 pixels (32 x 16 or 32 x 32 pixels), and the CX x CY
// thread blocks of one list tile form a thread-block cluster that shares the
// list's batches through distributed shared memory: per batch of CX CY S
// records each block stages S of them (one global / L2 read per record and
// cluster instead of one per screen tile; entries are dealt out round-robin)
// and marks the cluster tiles each may reach: those in the record's 16 x 16
// tile rect (the rule of the default lists) that its conservative box meets.
// After a cluster barrier every block copies, in list order, the records
// marked for its own tile from its peers' shared memory into its local batch
// and blends it with the culled schedule, so every tile walks its default
// list, in the same (depth, index) order, less records that cannot reach it.
// The cluster keeps staging until every one of its blocks is done (a flag per
// block, read after a cluster barrier, so all blocks take the same number of
// barriers). List positions (n_contrib, n_eval) refer to the list tile's
// list; colours and transmittance equal those of the per-16x16-tile lists
// bit for bit, because each pixel sees the same records in the same order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Cluster-wide barrier; release / acquire order shared-memory writes before
// it with peers' reads after it.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of the same shared-memory location in the block of cluster rank r.
__device__ __forceinline__ uint32_t peer_addr(const void *p, uint32_t r) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(p)), "r"(r));
    return a;
}

__device__ __forceinline__ float4 ld_peer_f4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a)
                 : "memory");
    return v;
}

__device__ __forceinline__ float2 ld_peer_f2(uint32_t a) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_peer_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

template <int CX, int CY, int BW, int BH, int S>
__global__ void __launch_bounds__((16 / BW) * (16 / BH) * 32) blend_cluster_kernel(const BlendArgs a) {
    constexpr int TW = 16, TH = 16, NC = CX * CY, L = NC * S;
    constexpr int kWX = TW / BW, kThreads = kWX * (TH / BH) * 32, kWarps = kThreads / 32;
    constexpr int kRows = 32 / BW, kNP = BW * BH / 32;
    static_assert(kRows * kNP == BH && kThreads <= 256, "block shape");
    static_assert(L % kThreads == 0 && S <= kThreads, "batch shape");
    // This block's share of a batch, read by the whole cluster.
    __shared__ float4 s_sa[S], s_scol[S], s_sbox[S];
    __shared__ float2 s_sb[S];
    __shared__ uint32_t s_smask[S];
    // The records of the batch that can reach this block's tile, in list order.
    __shared__ float4 s_a[L], s_col[L], s_box[L];
    __shared__ float2 s_b[L];
    __shared__ int32_t s_pos[L];
    __shared__ float4 s_rect[NC];  // pixel-centre rectangles of the cluster's tiles, by rank
    __shared__ int2 s_ptile[NC];   // the cluster's screen tiles, by rank
    __shared__ int2 s_tile;        // this block's screen tile (read by peers)
    __shared__ int s_done;         // all of this block's pixels have stopped (read by peers)
    __shared__ uint32_t s_wcnt[2][kWarps];

    const uint32_t rank = cluster_ctarank();
    const int tx = blockIdx.x, ty = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bx = tx * TW + (warp % kWX) * BW, by = ty * TH + (warp / kWX) * BH;
    const int px = bx + (lane % BW), py_base = by + lane / BW;
    const float fx = px + 0.5f;
    const float wx0 = bx + 0.5f, wx1 = fminf(bx + BW - 0.5f, a.width - 0.5f);
    const float wy0 = by + 0.5f, wy1 = fminf(by + BH - 0.5f, a.height - 0.5f);
    const int lt = (ty / CY) * a.grid.tiles_x + tx / CX;  // the list tile (same for the whole cluster)
    const uint32_t first = a.ranges[2 * lt], last = a.ranges[2 * lt + 1];

    Pix p[kNP];
    bool mine_done = true;
#pragma unroll
    for (int q = 0; q < kNP; ++q) {
        p[q] = Pix{1.f, 0.f, 0.f, 0.f, 0, 0, !(px < a.width && py_base + q * kRows < a.height)};
        mine_done = mine_done && p[q].done;
    }
    bool warp_done = __all_sync(0xffffffffu, mine_done);
    if (tid == 0) s_tile = make_int2(tx, ty);
    __syncthreads();
    cluster_sync_all();
    if (tid < NC) {
        const uint32_t ta = peer_addr(&s_tile, (uint32_t)tid);
        const int ptx = (int)ld_peer_u32(ta), pty = (int)ld_peer_u32(ta + 4);
        s_ptile[tid] = make_int2(ptx, pty);
        // Pixel-centre extent of that tile, clipped to the image (empty when
        // the tile lies outside it: x0 > x1).
        s_rect[tid] = make_float4(ptx * TW + 0.5f, fminf(ptx * TW + TW - 0.5f, a.width - 0.5f), pty * TH + 0.5f,
                                  fminf(pty * TH + TH - 0.5f, a.height - 0.5f));
    }
    __syncthreads();

    const SRec SL{s_sa, s_sb, s_scol, s_sbox};
    for (uint32_t start = first; start < last; start += L) {
        // Done flags of the previous batch, published by the barrier below;
        // every block reads the same flags, so all leave together (before
        // staging a batch nobody needs). The barrier also ends every peer's
        // reads of this block's previous share.
        const int cta_done = __syncthreads_and(warp_done);
        if (tid == 0) s_done = cta_done;
        cluster_sync_all();
        const int peer_done = tid < NC ? (int)ld_peer_u32(peer_addr(&s_done, (uint32_t)tid)) : 1;
        if (__syncthreads_and(peer_done)) break;
        // Stage this block's share of the batch (list entries start + rank,
        // start + rank + NC, ...) and mark the cluster tiles each can reach.
        const int n_batch = (int)min((uint32_t)L, last - start);
        for (int i = tid; i < S; i += kThreads) {
            const uint32_t k = start + rank + (uint32_t)(NC * i);
            uint32_t m = 0;
            if (k < last) {
                const uint32_t gi = a.values[k];
                stage_record(a.rd, gi, i, SL, true);
                // A tile takes the record only if its 16 x 16 tile rect (the
                // rule of the default lists, from the record's integer
                // radius) holds the tile and the record's conservative box
                // meets the tile (the warps test the exact ellipse later).
                const float4 ra = s_sa[i], bx = s_sbox[i];
                const int rad = __ldg(reinterpret_cast<const int *>(a.rd.rec32 + 3 * (size_t)gi + 2) + 2);
                const Rect R16 = tile_rect(ra.x, ra.y, rad, TW, TH, 1 << 30, 1 << 30);
#pragma unroll
                for (int r = 0; r < NC; ++r) {
                    const float4 R = s_rect[r];
                    const int2 t = s_ptile[r];
                    if (t.x >= R16.x0 && t.x < R16.x1 && t.y >= R16.y0 && t.y < R16.y1 && R.x <= R.y &&
                        R.z <= R.w && bx.x <= R.y && bx.y >= R.x && bx.z <= R.w && bx.w >= R.z)
                        m |= 1u << r;
                }
            }
            s_smask[i] = m;
        }
        cluster_sync_all();  // every share staged
        if (cta_done) continue;  // this tile is finished: it only stages for its peers
        // Gather the records marked for this tile, in list order (entry
        // start + j sits in slot j / NC of rank j % NC); per round of
        // kThreads entries, warp counts give each warp its place.
        int cnt = 0;
        for (int j0 = 0, rd_ = 0; j0 < n_batch; j0 += kThreads, rd_ ^= 1) {
            const int j = j0 + tid, sl = j % NC, i = j / NC;
            const uint32_t m = j < n_batch ? ld_peer_u32(peer_addr(&s_smask[i], (uint32_t)sl)) : 0u;
            const bool keep = (m >> rank) & 1u;
            const uint32_t ballot = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) s_wcnt[rd_][warp] = __popc(ballot);
            __syncthreads();
            int before = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const int c = (int)s_wcnt[rd_][w];
                before += w < warp ? c : 0;
                total += c;
            }
            if (keep) {
                const int d = cnt + before + __popc(ballot & lanemask_lt());
                s_a[d] = ld_peer_f4(peer_addr(&s_sa[i], (uint32_t)sl));
                s_b[d] = ld_peer_f2(peer_addr(&s_sb[i], (uint32_t)sl));
                s_col[d] = ld_peer_f4(peer_addr(&s_scol[i], (uint32_t)sl));
                s_box[d] = ld_peer_f4(peer_addr(&s_sbox[i], (uint32_t)sl));
                s_pos[d] = (int32_t)(start - first) + j + 1;
            }
            cnt += total;
        }
        __syncthreads();
        if (!warp_done) {
            for (int c = 0; c < cnt; c += 32) {
                const int j = c + lane;
                const bool hit = j < cnt && record_touches(s_a[j], s_b[j], s_box[j], wx0, wx1, wy0, wy1);
                uint32_t bits = __ballot_sync(0xffffffffu, hit);
                while (bits) {
                    const int jj = c + __ffs(bits) - 1;
                    bits &= bits - 1;
                    const float4 ra = s_a[jj];
                    const float2 rb = s_b[jj];
                    const float dx = fx - ra.x;
                    const float adx2 = ra.z * dx * dx, bdx = ra.w * dx;
                    const int32_t pos = s_pos[jj];
#pragma unroll
                    for (int q = 0; q < kNP; ++q) {
                        if (!p[q].done) {
                            const float dy = (float)(py_base + q * kRows) + 0.5f - ra.y;
                            composite(p[q], fmaf(dy, fmaf(rb.x, dy, bdx), adx2), rb.y, &s_col[jj], pos);
                        }
                    }
                }
                mine_done = true;
#pragma unroll
                for (int q = 0; q < kNP; ++q) mine_done = mine_done && p[q].done;
                warp_done = __all_sync(0xffffffffu, mine_done);
                if (warp_done) break;
            }
        }
    }
    // No block leaves while a peer may still read its shared memory.
    cluster_sync_all();
    const int32_t n_list = (int32_t)(last - first);
#pragma unroll
    for (int q = 0; q < kNP; ++q) {
        if (!p[q].done) p[q].eval = n_list;
        write_pixel(a, px, py_base + q * kRows, p[q]);
    }
}

// ---------------------------------------------------------------------------
// List-tile variant: the lists of list tiles of CX x CY screen tiles, each
// 16 x 16 screen tile blended by its own thread block, without a cluster: the
// block reads its list tile's list itself and keeps the records whose 16 x 16
// tile rect (the rule of the default lists; packed per record by the
// projection) holds its tile, compacted in list order into its batch; the
// batch is blended in packed pairs as by blend_tile_culled_x2 (whose warp
// culling drops the records that cannot reach a warp's pixels). Colours and
// transmittance equal those of the default lists bit for bit; list positions
// are the list tile's, as in the cluster blend.
// ---------------------------------------------------------------------------
// BW = 8 (8x8 warp blocks, four warps per tile): nine resident blocks per SM
// (56 registers, as the per-tile blend), measured 1-5 % faster than eight
// with 64 registers (1080p frame, 4K imbalance view). BW = 16 (16x8 warp
// blocks, two warps per tile, two pixel pairs per lane): fourteen (72
// registers), as the per-tile form.
constexpr int listtile_min_blocks(int bw) { return bw == 8 ? 9 : 14; }

template <int CX, int CY, int BW, int DEPTH>
__device__ __forceinline__ void blend_listtile_tile(const BlendArgs &a, int tx, int ty) {
    constexpr int TW = 16, TH = 16, BH = 8;
    constexpr int kWX = TW / BW, kWarps = kWX * (TH / BH), kThreads = kWarps * 32;
    static_assert(DEPTH % kThreads == 0 && DEPTH >= 2 * kThreads, "batch shape");
    __shared__ ulonglong2 s_d0[DEPTH], s_d1[DEPTH], s_d2[DEPTH], s_c01[DEPTH], s_c2[DEPTH];
    __shared__ int32_t s_pos[DEPTH];
    __shared__ uint32_t s_wcnt[2][kWarps];
    const SRecX2 S{s_d0, s_d1, s_d2, s_c01, s_c2};

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bx = tx * TW + (warp % kWX) * BW, by = ty * TH + (warp / kWX) * BH;
    LaneX2<BW> L(a, bx, by, lane);
    const float wx0 = bx + 0.5f, wx1 = fminf(bx + BW - 0.5f, a.width - 0.5f);
    const float wy0 = by + 0.5f, wy1 = fminf(by + BH - 0.5f, a.height - 0.5f);
    const int lt = (ty / CY) * a.grid.tiles_x + tx / CX;
    const uint32_t first = a.ranges[2 * lt], last = a.ranges[2 * lt + 1];

    bool warp_done = all_done_x2(L.P);
    uint32_t next = first;
    int rd_ = 0;
    // The list reads run ahead of the rounds that use them: a thread holds
    // its entry of the round being filled (gi0) with that entry's tile range
    // (r0), and its entry of the next round (gi1); each round issues the next
    // round's range load and the value load two rounds ahead, so neither
    // waits in the round (nor in the blend) that follows. An entry past the
    // list has range (0, 0), which no tile holds.
    uint32_t gi0 = 0, gi1 = 0;
    uint2 r0 = make_uint2(0u, 0u);
    {
        const uint32_t k0 = first + (uint32_t)tid, k1 = k0 + kThreads;
        if (k0 < last) gi0 = a.values[k0];
        if (k1 < last) gi1 = a.values[k1];
        if (k0 < last) r0 = __ldg(a.rd.rect16 + gi0);
    }
    while (next < last) {
        if (__syncthreads_count(warp_done) == kThreads) break;
        // Fill the batch: rounds of kThreads list entries, the kept ones
        // compacted in list order (per-warp counts give each warp its place).
        int cnt = 0;
        while (next < last && cnt <= DEPTH - kThreads) {
            const uint32_t k = next + (uint32_t)tid;
            const uint32_t gi = gi0;
            const uint2 r = r0;
            const uint32_t k1 = k + kThreads, k2 = k1 + kThreads;
            r0 = k1 < last ? __ldg(a.rd.rect16 + gi1) : make_uint2(0u, 0u);
            gi0 = gi1;
            gi1 = k2 < last ? a.values[k2] : 0u;
            const bool keep = (uint32_t)tx >= (r.x & 0xffffu) && (uint32_t)tx < (r.x >> 16) &&
                              (uint32_t)ty >= (r.y & 0xffffu) && (uint32_t)ty < (r.y >> 16);
            const uint32_t ballot = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) s_wcnt[rd_][warp] = __popc(ballot);
            __syncthreads();
            int before = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const int c = (int)s_wcnt[rd_][w];
                before += w < warp ? c : 0;
                total += c;
            }
            if (keep) {
                const int d = cnt + before + __popc(ballot & lanemask_lt());
                stage_record_x2<false>(a.rd, gi, d, S);
                s_pos[d] = (int32_t)(k - first) + 1;
            }
            cnt += total;
            next += kThreads;
            rd_ ^= 1;
        }
        __syncthreads();
        if (!warp_done) warp_done = blend_batch_x2(L.P, S, s_pos, 0, cnt, L.fx2, L.fy2, wx0, wx1, wy0, wy1, lane);
    }
    const int32_t n_list = (int32_t)(last - first);
#pragma unroll
    for (int q = 0; q < LaneX2<BW>::NP; ++q) {
        const int y0 = L.pyb + q * LaneX2<BW>::kRows;
        write_pixels_x2(a, L.P[q], L.px, y0, y0 + 4, n_list);
    }
}

template <int CX, int CY, int BW, int DEPTH>
__global__ void __launch_bounds__(BW == 8 ? 128 : 64, listtile_min_blocks(BW))
    blend_listtile_kernel(const BlendArgs a) {
    // Ordered: a 1-D grid of CX CY blocks per list tile, the list tiles
    // longest list first; else the 2-D grid of screen tiles.
    int tx = blockIdx.x, ty = blockIdx.y;
    if (a.order) {
        const int lt = (int)a.order[blockIdx.x / (CX * CY)], sub = (int)(blockIdx.x % (CX * CY));
        tx = (lt % a.grid.tiles_x) * CX + sub % CX;
        ty = (lt / a.grid.tiles_x) * CY + sub / CX;
    }
    if (tx * 16 >= a.width || ty * 16 >= a.height) return;  // padding of the list grid (whole block)
    blend_listtile_tile<CX, CY, BW, DEPTH>(a, tx, ty);
}

// Persistent blend over many views: blocks take global tiles from a queue
// (largest lists first); each tile is rendered with its view's parameters.
struct BlendBatchArgs {
    RecordReader rd;
    const uint32_t *values;
    const uint32_t *ranges;   // indexed by global tile
    const ViewDesc *views;
    int n_views;
    const uint32_t *order;    // queue order: global tiles (with list tiles: global tile x sub-tiles + sub-tile)
    int32_t n_tiles;          // items in the queue
    uint32_t *queue_head;
};

// With list tiles (LX x LY screen tiles of 16 x 16 per list tile) the queue
// holds one item per (list tile, screen tile of it), in list-length order,
// and each item is blended as by blend_listtile_kernel.
template <int TW, int TH, int DEPTH, int LX = 1, int LY = 1>
__global__ void __launch_bounds__((TW / 8) * (TH / 8) * 32) blend_batch_kernel(const BlendBatchArgs b) {
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(b.queue_head, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= b.n_tiles) return;
        const uint32_t code = b.order[item];
        const uint32_t gt = code / (LX * LY);  // global (list) tile
        int lo = 0, hi = b.n_views - 1;        // last view whose first tile <= gt
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.views[mid].tile_base <= gt) lo = mid; else hi = mid - 1;
        }
        const ViewDesc &V = b.views[lo];
        BlendArgs a{b.rd, b.values, b.ranges + 2 * (size_t)V.tile_base, V.grid, V.cam.width, V.cam.height,
                    {V.bg[0], V.bg[1], V.bg[2]}, V.rgb, V.final_T, V.n_contrib, V.n_eval};
        const int lt = (int)(gt - V.tile_base);
        if constexpr (LX * LY == 1) {
            blend_tile_culled_x2<TW, TH, 8, DEPTH, false>(a, lt);
        } else {
            const int sub = (int)(code % (LX * LY));
            const int tx = (lt % V.grid.tiles_x) * LX + sub % LX, ty = (lt / V.grid.tiles_x) * LY + sub / LX;
            if (tx * 16 < V.cam.width && ty * 16 < V.cam.height)  // block-uniform
                blend_listtile_tile<LX, LY, 8, 256>(a, tx, ty);
        }
    }
}

// ---------------------------------------------------------------------------
// Bulk-copy variant. A gather kernel writes each key's blend record (decoded
// to FP32: geo, aux, col; 48 bytes) in list order, so a tile's records are
// contiguous; the blend stages them 128 at a time with one cp.async.bulk
// copy into shared memory, double-buffered (the copy of batch b + 1 overlaps batch b), each
// completing on an mbarrier. The compute is the culled schedule's, so the
// outputs are identical. Every wait is bounded in time and sets the error
// word instead of hanging; a block waits for its copies in flight before it
// exits.
// ---------------------------------------------------------------------------
constexpr int kTmaBatch = 128;  // records per bulk copy (6 KB)

__global__ void __launch_bounds__(256) gather_records_kernel(RecordReader rd, const uint32_t *__restrict__ values,
                                                             const unsigned long long *d_n, int64_t n_cap,
                                                             float4 *__restrict__ out) {
    const int64_t n = d_n ? (int64_t)*d_n : n_cap;
    for (int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x; k < n && k < n_cap;
         k += (int64_t)gridDim.x * 256) {
        float4 geo, aux, col;
        rd.load(values[k], geo, aux, col);
        out[3 * k] = geo;
        out[3 * k + 1] = aux;
        out[3 * k + 2] = col;
    }
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    // Generic-proxy accesses of this buffer (made visible by the preceding
    // block barrier) are ordered before the async-proxy write.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Waits for the phase with the given parity to complete; gives up after
// kSpinTimeoutNs (sets kErrTimeout) so that a copy that never lands cannot
// hang the GPU.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t *d_err) {
    unsigned long long t0 = 0;
    for (uint32_t i = 0;; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 63u) == 0u) {
            const unsigned long long now = global_ns();
            if (i == 0) t0 = now;
            else if (now - t0 > kSpinTimeoutNs || (ld_relaxed_u32(d_err) & kErrTimeout)) {
                atomicOr(d_err, kErrTimeout);
                return false;
            }
        }
    }
}

template <int TW, int TH, int BW, int BH>
__global__ void __launch_bounds__((TW / BW) * (TH / BH) * 32)
    blend_tma_kernel(const BlendArgs a, const float4 *__restrict__ srec, uint32_t *d_err) {
    constexpr int kWX = TW / BW, kWarps = kWX * (TH / BH), kThreads = kWarps * 32;
    constexpr int kRows = 32 / BW, kNP = BW * BH / 32;
    __shared__ __align__(128) float4 s_raw[2][kTmaBatch * 3];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ float4 s_a[kTmaBatch], s_col[kTmaBatch], s_box[kTmaBatch];
    __shared__ float2 s_b[kTmaBatch];
    const SRec S{s_a, s_b, s_col, s_box};

    const int tile = blockIdx.x;
    const int tx = tile % a.grid.tiles_x, ty = tile / a.grid.tiles_x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bx = tx * TW + (warp % kWX) * BW, by = ty * TH + (warp / kWX) * BH;
    const int px = bx + (lane % BW), py_base = by + lane / BW;
    const float fx = px + 0.5f;
    const float wx0 = bx + 0.5f, wx1 = fminf(bx + BW - 0.5f, a.width - 0.5f);
    const float wy0 = by + 0.5f, wy1 = fminf(by + BH - 0.5f, a.height - 0.5f);

    const uint32_t first = a.ranges[2 * tile], last = a.ranges[2 * tile + 1];
    const int n_list = (int)(last - first);
    const int nb = (n_list + kTmaBatch - 1) / kTmaBatch;
    Pix p[kNP];
    bool mine_done = true;
#pragma unroll
    for (int q = 0; q < kNP; ++q) {
        p[q] = Pix{1.f, 0.f, 0.f, 0.f, 0, 0, !(px < a.width && py_base + q * kRows < a.height)};
        mine_done = mine_done && p[q].done;
    }
    bool warp_done = __all_sync(0xffffffffu, mine_done);
    auto issue = [&](int b) {
        const uint32_t k0 = first + (uint32_t)b * kTmaBatch;
        const uint32_t cnt = min((uint32_t)kTmaBatch, last - k0);
        bulk_load(s_raw[b & 1], srec + 3 * (size_t)k0, cnt * 48u, &s_bar[b & 1]);
    };
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (nb > 0) issue(0);
    }
    __syncthreads();
    int issued = nb > 0 ? 1 : 0, consumed = 0;
    for (int b = 0; b < nb; ++b) {
        if (__syncthreads_count(warp_done) == kThreads) break;
        if (b + 1 < nb) {
            if (tid == 0) issue(b + 1);  // its buffer was last read before the barrier above
            issued = b + 2;
        }
        const bool ok = mbar_wait(&s_bar[b & 1], (uint32_t)(b >> 1) & 1u, d_err);
        consumed = b + 1;
        if (__syncthreads_or(!ok)) break;
        const int cnt = min(kTmaBatch, n_list - b * kTmaBatch);
        for (int s = tid; s < cnt; s += kThreads) {
            const float4 *r = &s_raw[b & 1][3 * s];
            stage_values(r[0], r[1], r[2], s, S, true);
        }
        __syncthreads();
        const int32_t pos0 = b * kTmaBatch + 1;
        if (!warp_done) {
            for (int c = 0; c < cnt; c += 32) {
                const int j = c + lane;
                const bool hit = j < cnt && record_touches(s_a[j], s_b[j], s_box[j], wx0, wx1, wy0, wy1);
                uint32_t bits = __ballot_sync(0xffffffffu, hit);
                while (bits) {
                    const int jj = c + __ffs(bits) - 1;
                    bits &= bits - 1;
                    const float4 ra = s_a[jj];
                    const float2 rb = s_b[jj];
                    const float dx = fx - ra.x;
                    const float adx2 = ra.z * dx * dx, bdx = ra.w * dx;
#pragma unroll
                    for (int q = 0; q < kNP; ++q) {
                        if (!p[q].done) {
                            const float dy = (float)(py_base + q * kRows) + 0.5f - ra.y;
                            composite(p[q], fmaf(dy, fmaf(rb.x, dy, bdx), adx2), rb.y, &s_col[jj], pos0 + jj);
                        }
                    }
                }
                mine_done = true;
#pragma unroll
                for (int q = 0; q < kNP; ++q) mine_done = mine_done && p[q].done;
                warp_done = __all_sync(0xffffffffu, mine_done);
                if (warp_done) break;
            }
        }
    }
    // A copy still in flight (the block stopped early) must land before the
    // block's shared memory is released.
    if (tid == 0)
        for (int b = consumed; b < issued; ++b) mbar_wait(&s_bar[b & 1], (uint32_t)(b >> 1) & 1u, d_err);
#pragma unroll
    for (int q = 0; q < kNP; ++q) {
        if (!p[q].done) p[q].eval = n_list;
        write_pixel(a, px, py_base + q * kRows, p[q]);
    }
}

// ---------------------------------------------------------------------------
// Basic variant: one thread per pixel, every record evaluated.
// ---------------------------------------------------------------------------
template <int TW, int TH, bool RAW>
__global__ void __launch_bounds__(TW *TH) blend_basic_kernel(const BlendArgs a) {
    constexpr int kN = TW * TH;
    __shared__ float4 s_a[kBatch], s_col[kBatch];
    __shared__ float2 s_b[kBatch];
    const SRec S{s_a, s_b, s_col, nullptr};

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
            if (k < last) stage_record<RAW>(a.rd, a.values[k], s, S, false);
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBatch, last - start);
        const int32_t pos0 = (int32_t)(start - first) + 1;
        for (int j = 0; j < cnt && !p.done; ++j) {
            const float4 ra = s_a[j];
            const float2 rb = s_b[j];
            const float dx = fx - ra.x, dy = fy - ra.y;
            const float e = fmaf(dy, fmaf(rb.x, dy, ra.w * dx), ra.z * dx * dx);
            composite(p, e, rb.y, &s_col[j], pos0 + j);
        }
    }
    if (!p.done) p.eval = (int32_t)(last - first);
    write_pixel(a, px, py, p);
}

}  // namespace

namespace {
template <int TW, int TH, int DEPTH, int LX = 1, int LY = 1>
void launch_blend_batch(const BlendBatchArgs &b, int sms, cudaStream_t s) {
    constexpr int kThreads = (TW / 8) * (TH / 8) * 32;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, blend_batch_kernel<TW, TH, DEPTH, LX, LY>, kThreads, 0);
    blend_batch_kernel<TW, TH, DEPTH, LX, LY><<<(unsigned)(sms * (per_sm > 0 ? per_sm : 1)), kThreads, 0, s>>>(b);
}

template <int DEPTH>
void launch_blend_batch_shape(const BlendBatchArgs &b, int tile_w, int tile_h, int sms, cudaStream_t s) {
    if (tile_w == 16 && tile_h == 16) launch_blend_batch<16, 16, DEPTH>(b, sms, s);
    else if (tile_w == 16 && tile_h == 8) launch_blend_batch<16, 8, DEPTH>(b, sms, s);
    else launch_blend_batch<8, 8, DEPTH>(b, sms, s);
}
}  // namespace

cudaError_t gs_launch_blend_batch(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                                  const ViewDesc *views_dev, int n_views, int tile_w, int tile_h, int depth,
                                  const uint32_t *order, int32_t n_items, uint32_t *queue_head, int lists,
                                  cudaStream_t s) {
    BlendBatchArgs b{rd, values, ranges, views_dev, n_views, order, n_items, queue_head};
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (lists > 1) {  // list tiles: 16x16 screen tiles, 256 records staged per batch
        if (lists == GS_LISTS_2X1) launch_blend_batch<16, 16, 256, 2, 1>(b, sms, s);
        else if (lists == GS_LISTS_2X2) launch_blend_batch<16, 16, 256, 2, 2>(b, sms, s);
        else if (lists == GS_LISTS_4X4) launch_blend_batch<16, 16, 256, 4, 4>(b, sms, s);
        else if (lists == GS_LISTS_8X8) launch_blend_batch<16, 16, 256, 8, 8>(b, sms, s);
        else return cudaErrorInvalidValue;
        return cudaGetLastError();
    }
    // Persistent grid sized by occupancy; 8x8 warp blocks (in the queue loop
    // the 8x4 blocks' larger thread blocks measured slower: 7770 vs 8985
    // views/s on 64 views). depth = records staged per shared-memory batch.
    if (depth == 64) launch_blend_batch_shape<64>(b, tile_w, tile_h, sms, s);
    else if (depth == 128) launch_blend_batch_shape<128>(b, tile_w, tile_h, sms, s);
    else launch_blend_batch_shape<256>(b, tile_w, tile_h, sms, s);
    return cudaGetLastError();
}

cudaError_t gs_launch_blend_tma(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                                const GsGrid &grid, int width, int height, const float bg[3],
                                const gs_framebuffer &fb, float4 *gather, const unsigned long long *d_n,
                                int64_t n_cap, uint32_t *d_err, cudaStream_t s) {
    if (n_cap > 0) {
        int64_t blocks = (n_cap + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        gather_records_kernel<<<(unsigned)blocks, 256, 0, s>>>(rd, values, d_n, n_cap, gather);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    BlendArgs a{rd, values, ranges, grid, width, height,
                {bg[0], bg[1], bg[2]}, fb.rgb, fb.final_T, fb.n_contrib, fb.n_eval};
    const unsigned blocks = (unsigned)(grid.tiles_x * grid.tiles_y);
    const int tw = grid.tile_w, th = grid.tile_h;
    if (tw == 16 && th == 16) blend_tma_kernel<16, 16, 8, 4><<<blocks, 256, 0, s>>>(a, gather, d_err);
    else if (tw == 16 && th == 8) blend_tma_kernel<16, 8, 8, 4><<<blocks, 128, 0, s>>>(a, gather, d_err);
    else blend_tma_kernel<8, 8, 8, 4><<<blocks, 64, 0, s>>>(a, gather, d_err);
    return cudaGetLastError();
}

namespace {
template <bool RAW>
void launch_blend_variant(const BlendArgs &a, const GsGrid &grid, int variant, cudaStream_t s) {
    const unsigned blocks = (unsigned)(grid.tiles_x * grid.tiles_y);
    const int tw = grid.tile_w, th = grid.tile_h;
    if (variant == GS_BLEND_BASIC) {
        if (tw == 16 && th == 16) blend_basic_kernel<16, 16, RAW><<<blocks, 256, 0, s>>>(a);
        else if (tw == 16 && th == 8) blend_basic_kernel<16, 8, RAW><<<blocks, 128, 0, s>>>(a);
        else blend_basic_kernel<8, 8, RAW><<<blocks, 64, 0, s>>>(a);
    } else if (variant == GS_BLEND_CULLED_WIDE && tw == 16) {
        if (th == 16) blend_culled_kernel<16, 16, 16, 8, RAW><<<blocks, 64, 0, s>>>(a);
        else blend_culled_kernel<16, 8, 16, 8, RAW><<<blocks, 32, 0, s>>>(a);
    } else if (variant == GS_BLEND_CULLED_TILE && tw == 16 && th == 16) {
        blend_culled_kernel<16, 16, 16, 16, RAW><<<blocks, 32, 0, s>>>(a);
    } else if (variant == GS_BLEND_CULLED_8X8) {
        if (tw == 16 && th == 16) blend_culled_kernel<16, 16, 8, 8, RAW><<<blocks, 128, 0, s>>>(a);
        else if (tw == 16 && th == 8) blend_culled_kernel<16, 8, 8, 8, RAW><<<blocks, 64, 0, s>>>(a);
        else blend_culled_kernel<8, 8, 8, 8, RAW><<<blocks, 32, 0, s>>>(a);
    } else {
        // GS_BLEND_CULLED (8x4 blocks), and the wide variants on tiles they do not divide
        if (tw == 16 && th == 16) blend_culled_kernel<16, 16, 8, 4, RAW><<<blocks, 256, 0, s>>>(a);
        else if (tw == 16 && th == 8) blend_culled_kernel<16, 8, 8, 4, RAW><<<blocks, 128, 0, s>>>(a);
        else blend_culled_kernel<8, 8, 8, 4, RAW><<<blocks, 64, 0, s>>>(a);
    }
}
}  // namespace

namespace {
template <int CX, int CY, int BW, int BH>
cudaError_t launch_cluster(const BlendArgs &a, int width, int height, cudaStream_t s) {
    constexpr int S = 128;  // records staged per block and batch
    const int t16x = (width + 15) / 16, t16y = (height + 15) / 16;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((t16x + CX - 1) / CX * CX), (unsigned)((t16y + CY - 1) / CY * CY), 1);
    cfg.blockDim = dim3((16 / BW) * (16 / BH) * 32, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CX;
    attr[0].val.clusterDim.y = CY;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, blend_cluster_kernel<CX, CY, BW, BH, S>, a);
}
}  // namespace

cudaError_t gs_launch_blend_listtile(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                                     const GsGrid &list_grid, int lists, int width, int height, const float bg[3],
                                     const gs_framebuffer &fb, bool wide_blocks, const uint32_t *order,
                                     cudaStream_t s) {
    BlendArgs a{rd, values, ranges, list_grid, width, height,
                {bg[0], bg[1], bg[2]}, fb.rgb, fb.final_T, fb.n_contrib, fb.n_eval, order};
    const dim3 grid = order ? dim3((unsigned)(list_grid.tiles_x * list_grid.tiles_y * lists), 1, 1)
                            : dim3((unsigned)((width + 15) / 16), (unsigned)((height + 15) / 16), 1);
    if (wide_blocks) {
        if (lists == GS_LISTS_2X1) blend_listtile_kernel<2, 1, 16, 128><<<grid, 64, 0, s>>>(a);
        else if (lists == GS_LISTS_2X2) blend_listtile_kernel<2, 2, 16, 128><<<grid, 64, 0, s>>>(a);
        else if (lists == GS_LISTS_4X4) blend_listtile_kernel<4, 4, 16, 128><<<grid, 64, 0, s>>>(a);
        else if (lists == GS_LISTS_8X8) blend_listtile_kernel<8, 8, 16, 128><<<grid, 64, 0, s>>>(a);
        else return cudaErrorInvalidValue;
    } else {
        if (lists == GS_LISTS_2X1) blend_listtile_kernel<2, 1, 8, 256><<<grid, 128, 0, s>>>(a);
        else if (lists == GS_LISTS_2X2) blend_listtile_kernel<2, 2, 8, 256><<<grid, 128, 0, s>>>(a);
        else if (lists == GS_LISTS_4X4) blend_listtile_kernel<4, 4, 8, 256><<<grid, 128, 0, s>>>(a);
        else if (lists == GS_LISTS_8X8) blend_listtile_kernel<8, 8, 8, 256><<<grid, 128, 0, s>>>(a);
        else return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t gs_launch_blend_cluster(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                                    const GsGrid &list_grid, int cluster, int width, int height, const float bg[3],
                                    const gs_framebuffer &fb, bool wide_blocks, cudaStream_t s) {
    BlendArgs a{rd, values, ranges, list_grid, width, height,
                {bg[0], bg[1], bg[2]}, fb.rgb, fb.final_T, fb.n_contrib, fb.n_eval};
    if (cluster == 2) return wide_blocks ? launch_cluster<2, 1, 8, 8>(a, width, height, s)
                                         : launch_cluster<2, 1, 8, 4>(a, width, height, s);
    if (cluster == 4) return wide_blocks ? launch_cluster<2, 2, 8, 8>(a, width, height, s)
                                         : launch_cluster<2, 2, 8, 4>(a, width, height, s);
    return cudaErrorInvalidValue;
}

cudaError_t gs_launch_blend(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                            const GsGrid &grid, int width, int height, const float bg[3],
                            const gs_framebuffer &fb, int variant, cudaStream_t s, const uint32_t *order) {
    // order: only the culled variants take it (block b blends tile order[b]).
    BlendArgs a{rd, values, ranges, grid, width, height,
                {bg[0], bg[1], bg[2]}, fb.rgb, fb.final_T, fb.n_contrib, fb.n_eval, order};
    // Caller-provided gs_records (the stage API) get the per-key constants
    // computed while staging; the render path's blend records carry them.
    if (rd.mode == kRecRaw) launch_blend_variant<true>(a, grid, variant, s);
    else launch_blend_variant<false>(a, grid, variant, s);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Backward of the blend (Eq. 1 differentiated). For a pixel with contributors
// k = 1..m (alpha_k, T_k the transmittance in front of k, T_N the final one):
//   dC/dc_k     = alpha_k T_k
//   dC/dalpha_k = c_k T_k - (S_k + bg T_N) / (1 - alpha_k),
//   S_k = sum_{l>k} c_l alpha_l T_l,
// and alpha = min(0.99, o G) (no derivative where clamped), G = 2^e. Each tile
// is walked back to front from its pixels' last contributors; T_k is
// recovered as T_{k+1} / (1 - alpha_k) from the stored final T, and S grows as
// the walk goes. Same warp layout and the same conservative record culling
// as the forward kernel. Per record the 9 gradients
// (u, v, Q00, Q01, Q11, opacity, r, g, b) are summed over the warp (transpose
// reduction), over the block in shared memory, then added to global memory.
// ---------------------------------------------------------------------------
namespace {

struct BlendBwdArgs {
    RecordReader rd;
    const uint32_t *values;
    const uint32_t *ranges;
    GsGrid grid;
    int width, height;
    float bg[3];
    const float *d_rgb;
    const float *final_T;
    const int32_t *n_contrib;
    float *d_rec;  // n rows of kRecGradStride floats
    // Blocks cover TW x TH screen tiles, cta_tiles_x of them per row; the
    // lists belong to list tiles of lcx x lcy screen tiles (1 x 1 unless the
    // frame was blended in thread-block clusters).
    int cta_tiles_x, lcx, lcy;
};

constexpr float kLn2 = 0.6931471805599453f;

// Sum of 9 values over the warp; lane l ends with slot (l >> 1) & 15.
__device__ __forceinline__ float warp_sum9(float v[16], int lane) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool up = lane & 16;
        const float send = up ? v[i] : v[i + 8];
        const float keep = up ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = lane & 8;
        const float send = up ? v[i] : v[i + 4];
        const float keep = up ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = lane & 4;
        const float send = up ? v[i] : v[i + 2];
        const float keep = up ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool up = lane & 2;
        const float send = up ? v[0] : v[1];
        const float keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Backward state of a lane's two pixels (8x8 warp blocks: one column, rows r
// and r + 4), in packed pairs: T going back up the list, the final T, the
// suffix sums S of later contributions and dL/dC, per channel.
struct PixBX2 {
    f32x2 T2, TN2, S2[3], g2[3];
    int32_t last0, last1;
};

template <int TW, int TH>
__device__ __forceinline__ void blend_bwd_tile(const BlendBwdArgs &a, int tile) {
    constexpr int BW = 8, BH = 8, kRows = 4;
    constexpr int kWX = TW / BW, kWarps = kWX * (TH / BH), kThreads = kWarps * 32;
    __shared__ ulonglong2 s_d0[kBatch], s_d1[kBatch], s_d2[kBatch], s_c01[kBatch], s_c2[kBatch];
    __shared__ float s_grad[kBatch * 9];
    __shared__ uint32_t s_g[kBatch];
    __shared__ int s_maxlast;
    const SRecX2 S{s_d0, s_d1, s_d2, s_c01, s_c2};

    const int tx = tile % a.cta_tiles_x, ty = tile / a.cta_tiles_x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bx = tx * TW + (warp % kWX) * BW, by = ty * TH + (warp / kWX) * BH;
    const int px = bx + (lane % BW), py0 = by + lane / BW, py1 = py0 + kRows;
    const f32x2 fx2 = x2(px + 0.5f, px + 0.5f);
    const f32x2 fy2 = x2((float)py0 + 0.5f, (float)py1 + 0.5f);
    const float wx0 = bx + 0.5f, wx1 = fminf(bx + BW - 0.5f, a.width - 0.5f);
    const float wy0 = by + 0.5f, wy1 = fminf(by + BH - 0.5f, a.height - 0.5f);
    const uint32_t first = a.ranges[2 * ((ty / a.lcy) * a.grid.tiles_x + tx / a.lcx)];

    PixBX2 P;
    {
        const bool in0 = px < a.width && py0 < a.height, in1 = px < a.width && py1 < a.height;
        const size_t i0 = in0 ? (size_t)py0 * a.width + px : 0, i1 = in1 ? (size_t)py1 * a.width + px : 0;
        const float t0 = in0 ? a.final_T[i0] : 1.f, t1 = in1 ? a.final_T[i1] : 1.f;
        P.T2 = P.TN2 = x2(t0, t1);
        P.last0 = in0 ? a.n_contrib[i0] : 0;
        P.last1 = in1 ? a.n_contrib[i1] : 0;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            P.S2[ch] = x2(0.f, 0.f);
            P.g2[ch] = x2(in0 ? a.d_rgb[3 * i0 + ch] : 0.f, in1 ? a.d_rgb[3 * i1 + ch] : 0.f);
        }
    }
    const f32x2 bg2[3] = {x2(a.bg[0], a.bg[0]), x2(a.bg[1], a.bg[1]), x2(a.bg[2], a.bg[2])};
    const f32x2 one2 = x2(1.f, 1.f);
    if (tid == 0) s_maxlast = 0;
    for (int s = tid; s < kBatch * 9; s += kThreads) s_grad[s] = 0.f;
    __syncthreads();
    const int wmax = __reduce_max_sync(0xffffffffu, max(P.last0, P.last1));
    if (lane == 0) atomicMax(&s_maxlast, wmax);
    __syncthreads();
    const int max_last = s_maxlast;

    // Batches of positions (end - kBatch, end], end going down from max_last.
    for (int end = max_last; end > 0; end -= kBatch) {
        const int beg = max(0, end - kBatch);  // positions beg+1 .. end
        const int cnt = end - beg;
        for (int s = tid; s < cnt; s += kThreads) {
            const uint32_t g = a.values[first + beg + s];
            s_g[s] = g;
            float4 geo, aux, col;
            a.rd.load(g, geo, aux, col);
            if (a.lcx > 1 || a.lcy > 1) {
                // The lists belong to list tiles; this tile blended only the
                // records whose 16 x 16 tile rect holds it (others: an empty box).
                const int rad = __ldg(reinterpret_cast<const int *>(a.rd.rec32 + 3 * (size_t)g + 2) + 2);
                const Rect R = tile_rect(geo.x, geo.y, rad, TW, TH, 1 << 30, 1 << 30);
                if (!(tx >= R.x0 && tx < R.x1 && ty >= R.y0 && ty < R.y1)) {
                    const __half2 never = __floats2half2_rn(-INFINITY, -INFINITY);
                    aux.z = *reinterpret_cast<const float *>(&never);
                }
            }
            stage_values_x2(geo, aux, col, s, S);
        }
        __syncthreads();
        if (wmax > beg) {
            for (int c = ((cnt - 1) / 32) * 32; c >= 0; c -= 32) {
                const int j = c + lane;
                const bool hit = j < cnt && record_touches_x2(S, j, wx0, wx1, wy0, wy1);
                uint32_t bits = __ballot_sync(0xffffffffu, hit);
                while (bits) {
                    const int hb = 31 - __clz(bits);
                    bits &= ~(1u << hb);
                    const int jj = c + hb;
                    const int pos = beg + jj + 1;
                    const ulonglong2 d0 = S.d0[jj], d1 = S.d1[jj], d2 = S.d2[jj], c2r = S.c2[jj];
                    const f32x2 dx2 = x2_sub(fx2, d0.x), dy2 = x2_sub(fy2, d0.y);
                    const f32x2 adx2 = x2_mul(x2_mul(d1.x, dx2), dx2), bdx2 = x2_mul(d1.y, dx2);
                    float e0, e1, thr, hxy;
                    x2_split(x2_fma(dy2, x2_fma(d2.x, dy2, bdx2), adx2), e0, e1);
                    x2_split(c2r.y, thr, hxy);
                    // The pixels that took the record in the forward pass.
                    const bool k0 = pos <= P.last0 && !(e0 > 0.f || e0 < thr);
                    const bool k1 = pos <= P.last1 && !(e1 > 0.f || e1 < thr);
                    if (!__any_sync(0xffffffffu, k0 || k1)) continue;
                    float acc[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k) acc[k] = 0.f;
                    if (k0 || k1) {
                        // A pixel that skipped the record gets G = 0, so alpha = 0:
                        // its S stays as it was (alpha T = 0), every gradient term
                        // it adds is 0, and its T is kept by a select.
                        const float G0 = k0 ? ex2(e0) : 0.f, G1 = k1 ? ex2(e1) : 0.f;
                        const f32x2 G2 = x2(G0, G1);
                        float r0, r1;
                        const f32x2 raw2 = x2_mul(d2.y, G2);
                        x2_split(raw2, r0, r1);
                        const f32x2 alpha2 = x2(fminf(kAlphaMax, r0), fminf(kAlphaMax, r1));
                        float m0, m1;
                        x2_split(x2_sub(one2, alpha2), m0, m1);
                        // 1 - alpha lies in [0.01, 1]: the fast reciprocal (within
                        // 2 ulp) is far inside the gradients' tolerance.
                        const float i0 = __fdividef(1.f, m0), i1 = __fdividef(1.f, m1);
                        const f32x2 inv2 = x2(i0, i1), ninv2 = x2(-i0, -i1);
                        const f32x2 Tk2 = x2_mul(P.T2, inv2);
                        const f32x2 at2 = x2_mul(alpha2, Tk2);  // alpha_k T_k
                        const ulonglong2 c01 = S.c01[jj];
                        const f32x2 col2[3] = {c01.x, c01.y, c2r.x};
                        f32x2 dL2 = x2(0.f, 0.f);  // dL / dalpha_k
                        f32x2 a6[3];
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) {
                            // c_k T_k - (S_k + bg T_N) / (1 - alpha_k)
                            const f32x2 later = x2_mul(x2_fma(bg2[ch], P.TN2, P.S2[ch]), ninv2);
                            dL2 = x2_fma(P.g2[ch], x2_fma(col2[ch], Tk2, later), dL2);
                            a6[ch] = x2_mul(P.g2[ch], at2);
                            P.S2[ch] = x2_fma(col2[ch], at2, P.S2[ch]);
                        }
                        float tk0, tk1, tc0, tc1;
                        x2_split(Tk2, tk0, tk1);
                        x2_split(P.T2, tc0, tc1);
                        P.T2 = x2(k0 ? tk0 : tc0, k1 ? tk1 : tc1);
                        // No gradient through a clamped alpha.
                        const bool n0 = k0 && r0 < kAlphaMax, n1 = k1 && r1 < kAlphaMax;
                        const f32x2 Gm2 = x2(n0 ? G0 : 0.f, n1 ? G1 : 0.f);
                        const f32x2 rm2 = x2(n0 ? r0 : 0.f, n1 ? r1 : 0.f);
                        const f32x2 a5 = x2_mul(dL2, Gm2);
                        const f32x2 dp2 = x2_mul(dL2, rm2);  // dL / dpower
                        // Conic (Q00, Q01, Q11) from the base-2 form: Q00 = -2 ln2 A,
                        // Q01 = -ln2 B, Q11 = -2 ln2 C.
                        const f32x2 q00 = x2_mul(d1.x, x2(-2.f * kLn2, -2.f * kLn2));
                        const f32x2 q01 = x2_mul(d1.y, x2(-kLn2, -kLn2));
                        const f32x2 q11 = x2_mul(d2.x, x2(-2.f * kLn2, -2.f * kLn2));
                        const f32x2 a0 = x2_mul(dp2, x2_fma(q00, dx2, x2_mul(q01, dy2)));
                        const f32x2 a1 = x2_mul(dp2, x2_fma(q01, dx2, x2_mul(q11, dy2)));
                        const f32x2 a2 = x2_mul(dp2, x2_mul(x2(-0.5f, -0.5f), x2_mul(dx2, dx2)));
                        const f32x2 a3 = x2_mul(dp2, x2_mul(x2(-1.f, -1.f), x2_mul(dx2, dy2)));
                        const f32x2 a4 = x2_mul(dp2, x2_mul(x2(-0.5f, -0.5f), x2_mul(dy2, dy2)));
                        const f32x2 parts[9] = {a0, a1, a2, a3, a4, a5, a6[0], a6[1], a6[2]};
#pragma unroll
                        for (int k = 0; k < 9; ++k) {
                            float lo, hi;
                            x2_split(parts[k], lo, hi);
                            acc[k] = lo + hi;
                        }
                    }
                    const float v = warp_sum9(acc, lane);
                    const int slot = (lane >> 1) & 15;
                    if ((lane & 1) == 0 && slot < 9 && v != 0.f) atomicAdd(&s_grad[jj * 9 + slot], v);
                }
            }
        }
        __syncthreads();
        // The batch's record gradients into global memory: one thread per
        // record, a vector reduction per nonzero group of four.
        for (int r = tid; r < cnt; r += kThreads) {
            float *src = s_grad + 9 * r;
            const float4 g0 = make_float4(src[0], src[1], src[2], src[3]);
            const float4 g1 = make_float4(src[4], src[5], src[6], src[7]);
            const float g8 = src[8];
#pragma unroll
            for (int k = 0; k < 9; ++k) src[k] = 0.f;
            float *dst = a.d_rec + (size_t)s_g[r] * kRecGradStride;
            if (g0.x != 0.f || g0.y != 0.f || g0.z != 0.f || g0.w != 0.f)
                asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(g0.x), "f"(g0.y),
                             "f"(g0.z), "f"(g0.w)
                             : "memory");
            if (g1.x != 0.f || g1.y != 0.f || g1.z != 0.f || g1.w != 0.f)
                asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst + 4), "f"(g1.x), "f"(g1.y),
                             "f"(g1.z), "f"(g1.w)
                             : "memory");
            if (g8 != 0.f) atomicAdd(dst + 8, g8);
        }
        __syncthreads();
    }
}

template <int TW, int TH>
__global__ void __launch_bounds__((TW / 8) * (TH / 8) * 32) blend_bwd_kernel(const BlendBwdArgs a) {
    blend_bwd_tile<TW, TH>(a, blockIdx.x);
}

// Backward of a joint batch: block b takes global tile b of the batch and
// differentiates it with its view's parameters; record gradients are indexed
// by compact record slot (one per visible (view, Gaussian) pair).
struct BlendBwdBatchArgs {
    RecordReader rd;
    const uint32_t *values;     // compact record slots, per-tile lists
    const uint32_t *ranges;     // by global tile
    const ViewDesc *views;
    const GsBwdView *bviews;    // d_rgb, final_T, n_contrib per view
    int n_views;
    float *d_rec;               // record slots x kRecGradStride
};

template <int TW, int TH>
__global__ void __launch_bounds__((TW / 8) * (TH / 8) * 32) blend_bwd_batch_kernel(const BlendBwdBatchArgs b) {
    const uint32_t gt = blockIdx.x;
    int lo = 0, hi = b.n_views - 1;  // last view whose first tile <= gt
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.views[mid].tile_base <= gt) lo = mid; else hi = mid - 1;
    }
    const ViewDesc &V = b.views[lo];
    const GsBwdView &W = b.bviews[lo];
    BlendBwdArgs a{b.rd, b.values, b.ranges + 2 * (size_t)V.tile_base, V.grid, V.cam.width, V.cam.height,
                   {V.bg[0], V.bg[1], V.bg[2]}, W.d_rgb, W.final_T, W.n_contrib, b.d_rec, V.grid.tiles_x, 1, 1};
    blend_bwd_tile<TW, TH>(a, (int)(gt - V.tile_base));
}

}  // namespace

cudaError_t gs_launch_blend_bwd_batch(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                                      const ViewDesc *views, const GsBwdView *bviews, int n_views, int tile_w,
                                      int tile_h, int32_t total_tiles, float *d_rec, cudaStream_t s) {
    if (total_tiles <= 0) return cudaSuccess;
    BlendBwdBatchArgs b{rd, values, ranges, views, bviews, n_views, d_rec};
    if (tile_w == 16 && tile_h == 16) blend_bwd_batch_kernel<16, 16><<<(unsigned)total_tiles, 128, 0, s>>>(b);
    else if (tile_w == 16 && tile_h == 8) blend_bwd_batch_kernel<16, 8><<<(unsigned)total_tiles, 64, 0, s>>>(b);
    else blend_bwd_batch_kernel<8, 8><<<(unsigned)total_tiles, 32, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t gs_launch_blend_bwd(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                                const GsGrid &grid, int width, int height, const float bg[3],
                                const float *d_rgb, const float *final_T, const int32_t *n_contrib,
                                float *d_rec, cudaStream_t s, int cluster) {
    // A cluster frame's lists belong to list tiles of 2 x 1 or 2 x 2 screen
    // tiles of 16 x 16; each block still differentiates one 16 x 16 tile.
    int lcx = 1, lcy = 1;
    list_tile_dims(cluster, &lcx, &lcy);
    const int tw = grid.tile_w / lcx, th = grid.tile_h / lcy;
    const int ctx_ = (width + tw - 1) / tw, cty = (height + th - 1) / th;
    BlendBwdArgs a{rd, values, ranges, grid, width, height,
                   {bg[0], bg[1], bg[2]}, d_rgb, final_T, n_contrib, d_rec, ctx_, lcx, lcy};
    const unsigned blocks = (unsigned)(ctx_ * cty);
    // Warp blocks 8x8, the two pixels of a lane in packed pairs (finer 8x4
    // blocks measured 3 % slower in the scalar form: more warp reductions of
    // the record gradients per record).
    if (tw == 16 && th == 16) blend_bwd_kernel<16, 16><<<blocks, 128, 0, s>>>(a);
    else if (tw == 16 && th == 8) blend_bwd_kernel<16, 8><<<blocks, 64, 0, s>>>(a);
    else blend_bwd_kernel<8, 8><<<blocks, 32, 0, s>>>(a);
    return cudaGetLastError();
}
