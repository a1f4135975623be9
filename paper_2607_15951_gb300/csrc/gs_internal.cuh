// gs_internal.cuh — device-side definitions shared by the library's kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs.h"

// Shared-memory carveout preference for the kernels of the render path
// (-1: leave the CUDA runtime's default).
#ifndef GS_CARVEOUT
#define GS_CARVEOUT -1
#endif
template <class F>
inline void gs_carveout(F *kernel) {
    if (GS_CARVEOUT >= 0)
        cudaFuncSetAttribute(reinterpret_cast<const void *>(kernel), cudaFuncAttributePreferredSharedMemoryCarveout,
                             GS_CARVEOUT);
}

namespace gs {

// Key slots per block of the key emission kernel (2^11 = 2048).
constexpr int kKeyBlockLog2 = 11;

// Constants of the standard 3DGS formulation (the paper cites it for Eq. 1
// and for the 3-sigma bound of Sec. 4.4 but prints none of them).
constexpr float kDilation = 0.3f;         // px^2 added to the 2D covariance diagonal
constexpr float kAlphaMax = 0.99f;        // opacity clamp
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;            // stop before T would fall below this
constexpr float kGuard = 1.3f;            // Jacobian view-ratio clamp, x tan(half fov)
constexpr int kMaxRadius = 1 << 30;       // radius clamp so tile arithmetic fits int64

// Device error word bits (gs_context::d_err).
// kErrTemporal: an incremental re-binning could not produce this frame's
// lists (the caller rebuilds them with the full binning); not a user error.
enum : uint32_t { kErrTimeout = 1u, kErrCapacity = 2u, kErrRange = 4u, kErrTemporal = 8u };

// Every spin-wait on another block gives up after this much wall time and
// sets kErrTimeout; other waiting blocks see the error word and leave early.
constexpr unsigned long long kSpinTimeoutNs = 2000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Look-back status words: top two bits flag, low 62 bits value.
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagIncl = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;

// Warp-wide decoupled look-back over per-partition status words: returns
// the sum of the values of all partitions before p. Lanes inspect 32
// predecessors at a time; a window is consumed once every lane sees a
// published flag, up to and including the nearest inclusive prefix.
// Sets kErrTimeout (and returns a meaningless sum) if a predecessor stays
// unpublished for kSpinTimeoutNs or another block already timed out.
__device__ __forceinline__ unsigned long long warp_lookback(const unsigned long long *status, long long p,
                                            uint32_t *d_err, bool *timed_out,
                                            unsigned long long timeout_ns = kSpinTimeoutNs) {
    const int lane = threadIdx.x & 31;
    unsigned long long excl = 0;
    long long q = p - 1;
    // The clock starts at the first unpublished read and is checked every
    // 16th poll, so a look-back that finds its prefix at once reads no timer.
    unsigned long long t0 = 0;
    uint32_t polls = 0;
    *timed_out = false;
    while (true) {
        const long long idx = q - lane;
        const unsigned long long s = idx >= 0 ? ld_relaxed_u64(status + idx) : kFlagIncl;
        if (!__all_sync(0xffffffffu, (s >> 62) != 0)) {
            bool give_up = false;
            if ((polls++ & 15u) == 0u) {
                const unsigned long long now = global_ns();
                if (polls == 1) t0 = now;
                give_up = (now - t0 > timeout_ns) || (ld_relaxed_u32(d_err) & kErrTimeout);
            }
            if (__any_sync(0xffffffffu, give_up)) {
                if (lane == 0) atomicOr(d_err, kErrTimeout);
                *timed_out = true;
                return excl;
            }
            __nanosleep(32);
            continue;
        }
        const uint32_t incl = __ballot_sync(0xffffffffu, (s >> 62) == 2);
        const int first = incl ? __ffs(incl) - 1 : 31;
        unsigned long long v = lane <= first ? (s & kValueMask) : 0ull;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (incl) return excl;
        q -= 32;
    }
}

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t v, uint32_t *s_tmp /* 8 */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_tmp[warp] = incl;
    __syncthreads();
    uint32_t pre = 0;
    for (int w = 0; w < warp; ++w) pre += s_tmp[w];
    __syncthreads();
    return pre + incl - v;
}

// Tile rectangle of a record: columns [floor((u-r)/tw), floor((u+r+tw-1)/tw))
// and rows likewise, clamped to the grid. floor((u +- n)/t) for an integer n
// equals floor((floor(u) +- n)/t), so the bounds are exact integer arithmetic
// on floor(u) (a shift, the tile sides being powers of two); |u| is clamped
// to 2^31, which cannot change an answer once the radius is clamped to 2^30.
struct Rect {
    int x0, y0, x1, y1;
};

// floor(a / 2^s): an arithmetic right shift (tile sides are powers of two).
__device__ __forceinline__ long long floordiv_pow2(long long a, int s) { return a >> s; }

__device__ __forceinline__ int clamp_tile(long long v, int limit) {
    return v < 0 ? 0 : (v > limit ? limit : (int)v);
}

__device__ __forceinline__ Rect tile_rect(float u, float v, int r, int tw, int th, int tiles_x,
                                          int tiles_y) {
    const float lim = 2147483648.0f;
    long long fu = (long long)floorf(fminf(fmaxf(u, -lim), lim));
    long long fv = (long long)floorf(fminf(fmaxf(v, -lim), lim));
    Rect R;
    const int sx = __ffs(tw) - 1, sy = __ffs(th) - 1;
    R.x0 = clamp_tile(floordiv_pow2(fu - r, sx), tiles_x);
    R.x1 = clamp_tile(floordiv_pow2(fu + r + tw - 1, sx), tiles_x);
    R.y0 = clamp_tile(floordiv_pow2(fv - r, sy), tiles_y);
    R.y1 = clamp_tile(floordiv_pow2(fv + r + th - 1, sy), tiles_y);
    return R;
}

// What the blend needs of a record, computed once per visible Gaussian by
// the render path's projections (and per staged key when the blend reads
// caller-provided gs_records):
//   A, B, C  the conic scaled to the base-2 exponent,
//            power * log2(e) = A dx^2 + B dx dy + C dy^2;
//   thr      log2(1 / (255 opacity)) of the FP32 opacity: alpha >= 1/255
//            <=> exponent >= thr, so every record precision takes the alpha
//            decisions of the FP32 path;
//   hxy      half-widths (hx, hy) of a conservative box around the mean
//            outside which alpha < 1/255, two FP16 rounded up (+inf: never
//            cull; -inf: alpha never reaches 1/255).
// alpha >= 1/255 needs (1/2) d^T Q d <= L = ln(255 o); that ellipse's
// axis-aligned box has half-widths sqrt(2 L Sigma00), sqrt(2 L Sigma11) with
// Sigma = Q^-1. L is inflated to cover the FP32 evaluation error of the
// exponent, at most 8 eps kappa |exponent| for a conic of condition number
// kappa <= (q00 + q11)^2 / det (det by Kahan's method).
struct BlendPre {
    float A, B, C, thr;
    uint32_t hxy;
};

constexpr float kLog2eF = 1.4426950408889634f;

__device__ __forceinline__ BlendPre blend_pre(float q00, float q01, float q11, float o) {
    BlendPre p;
    p.A = -0.5f * kLog2eF * q00;
    p.B = -kLog2eF * q01;
    p.C = -0.5f * kLog2eF * q11;
    p.thr = -log2f(255.f * o);
    const float L = logf(255.f * o);
    float hx = -INFINITY, hy = -INFINITY;  // alpha never reaches 1/255
    if (L > -1e-4f) {
        hx = hy = INFINITY;  // cannot bound: never cull
        const float w = q01 * q01;
        const float e = fmaf(-q01, q01, w);
        const float det = fmaf(q00, q11, -w) + e;
        if (det > 0.f) {
            const float tr = q00 + q11;
            const float kappa = tr * tr / det;
            const float Lp = (fmaxf(L, 0.f) + 1e-4f) * (1.f + 64.f * 1.2e-7f * kappa);
            const float bx = sqrtf(2.f * Lp * (q11 / det)) * 1.0001f + 1e-3f;
            const float by = sqrtf(2.f * Lp * (q00 / det)) * 1.0001f + 1e-3f;
            if (bx < 3e38f && by < 3e38f) {
                hx = bx;
                hy = by;
            }
        }
    }
    const __half2 h = __halves2half2(__float2half_ru(hx), __float2half_ru(hy));
    p.hxy = *reinterpret_cast<const uint32_t *>(&h);
    return p;
}

// Record forms the blend can read (RecordReader::mode). The render path
// writes a blend record of three arrays per visible Gaussian (or per record
// slot of a batch):
//   geo  float4  (u, v, A, B)
//   aux  float4  (C, thr, hxy bits, w)
//   col  kRecF32:  float4 (red, green, blue, 0), w = opacity (48 bytes);
//        kRecF16:  uint32 FP16 pair (green, blue), w = FP16 pair (opacity,
//                  red) (36 bytes);
//        kRecBF16: uint32 BF16 pair (green - 1, blue - 1), w = (FP16
//                  opacity, BF16 red - 1) (36 bytes).
// The 2D mean, the conic and the alpha threshold stay FP32: the exponent's
// error is the conic's relative error times |power| (up to ln 255 at the
// 1/255 edge), which with 16-bit conics exceeds the image bound on dense
// scenes. With BF16 colours the opacity is FP16 (a product o G needs more
// than BF16's 8 significant bits to stay within the image bound) and the
// colours are stored less 1: colours lie in [0, 2) in practice, where
// c - 1 in [-1, 1) keeps BF16's rounding error at or below 2^-9, half of
// what c itself would get in [1, 2). kRecRaw reads gs_records (the stage
// API's blend input) and computes the constants per staged key.
enum : int { kRecRaw = 0, kRecF32 = 1, kRecF16 = 2, kRecBF16 = 3 };

__device__ __forceinline__ uint32_t pack_f16x2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ uint32_t pack_bf16x2_less1(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a - 1.f, b - 1.f);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// w word of aux and the col word of the 16-bit forms.
__device__ __forceinline__ uint32_t pack_op_red(float o, float r, int mode) {
    if (mode == kRecBF16) {
        const __half ho = __float2half_rn(o);
        const __nv_bfloat16 br = __float2bfloat16_rn(r - 1.f);
        return (uint32_t)*reinterpret_cast<const uint16_t *>(&ho) |
               ((uint32_t)*reinterpret_cast<const uint16_t *>(&br) << 16);
    }
    return pack_f16x2(o, r);
}

__device__ __forceinline__ uint32_t pack_green_blue(float g, float b, int mode) {
    return mode == kRecBF16 ? pack_bf16x2_less1(g, b) : pack_f16x2(g, b);
}

// Writes blend record slot j (geo, aux, col) from the gs_record words
// (r0 = u, v, Q00, Q01; Q11; opacity; red, green, blue).
struct BlendRecordOut {
    float4 *geo;
    float4 *aux;
    void *col;  // float4 (kRecF32) or uint32 (16-bit forms)
    int mode;   // kRecF32, kRecF16 or kRecBF16
    // Optional (list tiles): the 16 x 16 screen tiles that take the record,
    // packed as (x0 | x1 << 16, y0 | y1 << 16): those of its tile rect (the
    // rule of the 16 x 16 lists, from the integer radius rad, clamped to
    // t16x x t16y) whose pixel centres its conservative box can reach (a
    // superset of the exact test; an empty range when it reaches none).
    uint2 *rect16;
    int t16x, t16y;
    __device__ __forceinline__ void write(size_t j, const float4 &r0, float q11, float o, float r, float g,
                                          float b, int rad = 0) const {
        const BlendPre p = blend_pre(r0.z, r0.w, q11, o);
        geo[j] = make_float4(r0.x, r0.y, p.A, p.B);
        if (rect16) {
            Rect R = tile_rect(r0.x, r0.y, rad, 16, 16, t16x, t16y);
            const uint32_t hw = p.hxy;
            const float2 h = __half22float2(*reinterpret_cast<const __half2 *>(&hw));
            if (!(h.x >= 0.f && h.y >= 0.f)) {
                R.x1 = R.x0;  // alpha never reaches 1/255
            } else if (h.x < 1e6f && h.y < 1e6f) {
                // Tile t's pixel centres span [16 t + 0.5, 16 t + 15.5]; the
                // box [u - hx, u + hx] can only meet tiles t with
                // floor((u - hx - 0.5) / 16) <= t <= floor((u + hx) / 16).
                R.x0 = max(R.x0, (int)floorf((r0.x - h.x - 0.5f) * 0.0625f));
                R.x1 = min(R.x1, (int)floorf((r0.x + h.x) * 0.0625f) + 1);
                R.y0 = max(R.y0, (int)floorf((r0.y - h.y - 0.5f) * 0.0625f));
                R.y1 = min(R.y1, (int)floorf((r0.y + h.y) * 0.0625f) + 1);
            }
            rect16[j] = R.x0 < R.x1 && R.y0 < R.y1
                            ? make_uint2((uint32_t)R.x0 | ((uint32_t)R.x1 << 16), (uint32_t)R.y0 | ((uint32_t)R.y1 << 16))
                            : make_uint2(0u, 0u);
        }
        if (mode == kRecF32) {
            aux[j] = make_float4(p.C, p.thr, __uint_as_float(p.hxy), o);
            static_cast<float4 *>(col)[j] = make_float4(r, g, b, 0.f);
        } else {
            aux[j] = make_float4(p.C, p.thr, __uint_as_float(p.hxy), __uint_as_float(pack_op_red(o, r, mode)));
            static_cast<uint32_t *>(col)[j] = pack_green_blue(g, b, mode);
        }
    }
};

// What the blend kernels read of a record, in any form: geo = (u, v, A, B),
// aux = (C, thr, hxy bits, -), col = (opacity, red, green, blue).
struct RecordReader {
    const float4 *rec32;  // kRecRaw: gs_record array
    const float4 *geo;
    const float4 *aux;
    const void *col;
    int mode;
    const uint2 *rect16;  // the 16 x 16 tile rects (list-tile frames), as BlendRecordOut writes them
    // Any form (RAW: the caller guarantees mode == kRecRaw; kernels that only
    // ever read blend records instantiate RAW = false and carry no code for
    // the per-key constants).
    template <bool RAW = false>
    __device__ __forceinline__ void load(uint32_t g, float4 &og, float4 &oa, float4 &oc) const {
        if (RAW) {
            const float4 r0 = __ldg(rec32 + 3 * (size_t)g);
            const float4 r1 = __ldg(rec32 + 3 * (size_t)g + 1);
            const float blue = __ldg(reinterpret_cast<const float *>(rec32 + 3 * (size_t)g + 2));
            const BlendPre p = blend_pre(r0.z, r0.w, r1.x, r1.y);
            og = make_float4(r0.x, r0.y, p.A, p.B);
            oa = make_float4(p.C, p.thr, __uint_as_float(p.hxy), 0.f);
            oc = make_float4(r1.y, r1.z, r1.w, blue);
            return;
        }
        og = __ldg(geo + g);
        oa = __ldg(aux + g);
        oc = load_col(g, oa);
    }
    // (opacity, red, green, blue) of a blend record whose aux word is oa.
    __device__ __forceinline__ float4 load_col(uint32_t g, const float4 &oa) const {
        if (mode == kRecF32) {
            const float4 c = __ldg(static_cast<const float4 *>(col) + g);
            return make_float4(oa.w, c.x, c.y, c.z);
        }
        const uint32_t w = __float_as_uint(oa.w), gb = __ldg(static_cast<const uint32_t *>(col) + g);
        if (mode == kRecBF16) {
            const __half ho = *reinterpret_cast<const __half *>(&w);
            const uint32_t rb = w >> 16;
            const float red = __uint_as_float(rb << 16) + 1.f;  // BF16 -> FP32 is a shift
            const float green = __uint_as_float(gb << 16) + 1.f, blue = __uint_as_float(gb & 0xffff0000u) + 1.f;
            return make_float4(__half2float(ho), red, green, blue);
        }
        const float2 orr = __half22float2(*reinterpret_cast<const __half2 *>(&w));
        const float2 gbb = __half22float2(*reinterpret_cast<const __half2 *>(&gb));
        return make_float4(orr.x, orr.y, gbb.x, gbb.y);
    }
};

// Half-widths of a blend record's box (hxy bits of aux.z).
__device__ __forceinline__ float2 blend_box_half(float hxy_bits) {
    const uint32_t w = __float_as_uint(hxy_bits);
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}

// Records as three float4s (the gs_record layout):
//   r0 = (u, v, Q00, Q01), r1 = (Q11, opacity, red, green),
//   r2 = (blue, depth, radius bits, tiles bits).
struct Rec {
    float4 r0, r1, r2;
};
static_assert(sizeof(gs_record) == 48, "gs_record must be 48 bytes");

}  // namespace gs

using gs::RecordReader;

// ---------------------------------------------------------------------------
// Host-side launch helpers (implemented in the kernel files).
// ---------------------------------------------------------------------------
struct GsCameraDev {
    float R[9];
    float t[3];
    float C[3];  // camera centre -R^T t
    float fx, fy, cx, cy, near_z;
    float lim_x, lim_y;  // 1.3 tan(half fov) per axis
    float rn[3];         // row norms of R, rounded up (the conservative screen bound)
    int width, height;
};

struct GsGrid {
    int tile_w, tile_h, tiles_x, tiles_y;
};

// One view of a batched render (device table, filled by the host per call).
struct ViewDesc {
    GsCameraDev cam;
    GsGrid grid;
    uint32_t tile_base;  // global id of this view's first tile
    float bg[3];
    float *rgb;
    float *final_T;
    int32_t *n_contrib;
    int32_t *n_eval;
};

// Per-view inputs of a batched backward.
struct GsBwdView {
    const float *d_rgb;
    const float *final_T;
    const int32_t *n_contrib;
};

cudaError_t gs_launch_project(const gs_gaussians &g, const GsCameraDev &cam, const GsGrid &grid,
                              gs_record *records, uint32_t *tiles, cudaStream_t s);

// Exclusive scan of tiles[0..n) into offsets (u64); counts[0] = total,
// counts[1] = number of non-zero entries. `scratch` holds the look-back
// state: gs_scan_scratch_bytes(n) bytes, zeroed inside the call.
size_t gs_scan_scratch_bytes(int64_t n);
cudaError_t gs_launch_scan(const uint32_t *tiles, int64_t n, unsigned long long *offsets,
                           unsigned long long *counts, void *scratch, uint32_t *d_err,
                           cudaStream_t s);
// Self-test of the bounded waits: runs the scan (kind 0) or one onesweep pass
// (kind 1) on n zero items with the partition counter preset to 1, so that
// partition 0 never publishes; every block waiting on it must give up after
// timeout_ns and set kErrTimeout. Scratch: gs_selftest_scratch_bytes(n).
size_t gs_selftest_scratch_bytes(int64_t n);
cudaError_t gs_launch_selftest_wait(int kind, int64_t n, void *scratch, uint32_t *d_err,
                                    unsigned long long timeout_ns, cudaStream_t s);

cudaError_t gs_launch_emit(const gs_record *records, const uint32_t *tiles,
                           const unsigned long long *offsets, int64_t n, const GsGrid &grid,
                           uint64_t *keys, uint32_t *values, int64_t capacity, uint32_t *d_err,
                           cudaStream_t s);

cudaError_t gs_launch_ranges(const uint64_t *keys, int64_t n, int32_t n_tiles, uint32_t *ranges,
                             uint32_t *d_err, cudaStream_t s);




// Onesweep radix sort. Pairs per partition (one block's share of a pass):
#ifndef GS_SORT_ITEMS
#define GS_SORT_ITEMS 16
#endif
#ifndef GS_SORT_LOOKAHEAD
#define GS_SORT_LOOKAHEAD 8
#endif
constexpr int kSortThreads = 256;
constexpr int kSortTile = kSortThreads * GS_SORT_ITEMS;
// Scratch: gs_sort_scratch_bytes(n, key_bits) bytes, laid out as
// GsSortScratch (digit histograms, their exclusive bucket offsets, one
// partition counter per pass, a ticket, and the look-back status words).
struct GsSortScratch {
    uint32_t *hist;    // passes x 256 digit counts
    uint32_t *bucket;  // passes x 256 exclusive bucket offsets
    uint32_t *counter; // passes partition counters
    uint32_t *ticket;  // last-block ticket of the histogram producer
    unsigned long long *status;  // passes x parts x 256
    int passes;
    int64_t parts;     // partitions of the capacity the passes are launched for
    int digit0;        // pass p sorts the 8-bit digit digit0 + p of the key
    int items;         // pairs per thread of a partition (256 threads): 8 or GS_SORT_ITEMS
    bool diverse_last; // the last digit is diverse too (rank it with ballots, as the others)
};
size_t gs_sort_scratch_bytes(int64_t n, int key_bits);
GsSortScratch gs_sort_carve(void *base, int64_t n_capacity, int key_bits);
// Scratch for `passes` digit passes starting at digit `digit0`, with
// partitions of 256 x items pairs: 8 (short lists: shorter per-partition
// latency), GS_SORT_ITEMS, 12 (long lists, three blocks per SM), or 0 to
// choose by capacity (gs_sort_items_for).
int gs_sort_items_for(int64_t n_capacity);
size_t gs_sort_scratch_bytes_digits(int64_t n, int passes, int items = 0);
GsSortScratch gs_sort_carve_digits(void *base, int64_t n_capacity, int digit0, int passes, int items = 0);
int gs_sort_passes(int key_bits);
// Sorts (keys, values) using (alt_keys, alt_values) as the ping-pong pair;
// *result_in_alt tells which pair holds the result. Zeroes the scratch and
// builds the histograms itself.
cudaError_t gs_launch_sort(uint64_t *keys, uint32_t *values, uint64_t *alt_keys,
                           uint32_t *alt_values, int64_t n, int key_bits, void *scratch,
                           uint32_t *d_err, bool *result_in_alt, cudaStream_t s);
// Digit passes only, for a producer that already filled sc.hist / sc.bucket.
// The grid covers n_capacity pairs; the pair count is read from *d_n.
cudaError_t gs_launch_sort_passes(uint64_t *keys, uint32_t *values, uint64_t *alt_keys,
                                  uint32_t *alt_values, int64_t n_capacity,
                                  const unsigned long long *d_n, const GsSortScratch &sc,
                                  uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                  unsigned long long timeout_ns = gs::kSpinTimeoutNs, int max_passes = 64,
                                  int first_pass = 0);
// The same over 32- and 16-bit keys (tile ids of a frame's tile sort).
cudaError_t gs_launch_sort_passes(uint32_t *keys, uint32_t *values, uint32_t *alt_keys,
                                  uint32_t *alt_values, int64_t n_capacity,
                                  const unsigned long long *d_n, const GsSortScratch &sc,
                                  uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                  unsigned long long timeout_ns = gs::kSpinTimeoutNs, int max_passes = 64,
                                  int first_pass = 0);
cudaError_t gs_launch_sort_passes(uint16_t *keys, uint32_t *values, uint16_t *alt_keys,
                                  uint32_t *alt_values, int64_t n_capacity,
                                  const unsigned long long *d_n, const GsSortScratch &sc,
                                  uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                  unsigned long long timeout_ns = gs::kSpinTimeoutNs, int max_passes = 64,
                                  int first_pass = 0);

// Reduce-then-scan digit passes (long lists; see gs_sort.cu): the same
// result as gs_launch_sort_passes with partitions of 3072 pairs that never
// wait on one another. rts_scratch: gs_sort_rts_scratch_bytes(n_capacity).
// sc supplies the passes, digit0 and the bucket offsets of every pass.
constexpr int64_t kRtsMinPairs = int64_t(1) << 23;  // capacities from here on use it
size_t gs_sort_rts_scratch_bytes(int64_t n_capacity);
cudaError_t gs_launch_sort_passes_rts(uint16_t *keys, uint32_t *values, uint16_t *alt_keys, uint32_t *alt_values,
                                      int64_t n_capacity, const unsigned long long *d_n, const GsSortScratch &sc,
                                      void *rts_scratch, uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                      int first_pass = 0);
cudaError_t gs_launch_sort_passes_rts(uint32_t *keys, uint32_t *values, uint32_t *alt_keys, uint32_t *alt_values,
                                      int64_t n_capacity, const unsigned long long *d_n, const GsSortScratch &sc,
                                      void *rts_scratch, uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                      int first_pass = 0);
cudaError_t gs_launch_sort_passes_rts(uint64_t *keys, uint32_t *values, uint64_t *alt_keys, uint32_t *alt_values,
                                      int64_t n_capacity, const unsigned long long *d_n, const GsSortScratch &sc,
                                      void *rts_scratch, uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                      int first_pass = 0);

// order (optional, the culled variants only): block b blends tile order[b]
// (a longest-list-first order from gs_launch_tile_order).
cudaError_t gs_launch_blend(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                            const GsGrid &grid, int width, int height, const float bg[3],
                            const gs_framebuffer &fb, int variant, cudaStream_t s, const uint32_t *order = nullptr);
// Thread-block-cluster blend: the lists belong to list tiles of cluster
// screen tiles of 16 x 16 (cluster 2: 2 x 1, 4: 2 x 2; list_grid is their
// grid); the blocks of a list tile form one cluster and share its batches
// through distributed shared memory. wide_blocks: 8x8 warp blocks.
// Rows of the record-gradient buffers: the 9 gradients of a record
// (u, v, Q00, Q01, Q11, opacity, red, green, blue) padded to 12 floats, so a
// row is 16-byte aligned and the blend backward adds it with vector
// reductions.
constexpr int kRecGradStride = 12;

// Screen tiles per list tile (1, 2: 2 x 1, 4: 2 x 2, 16: 4 x 4, 64: 8 x 8)
// as columns x rows.
inline void list_tile_dims(int code, int *lx, int *ly) {
    *lx = code >= 64 ? 8 : code >= 16 ? 4 : code >= 2 ? 2 : 1;
    *ly = code >= 64 ? 8 : code >= 16 ? 4 : code >= 4 ? 2 : 1;
}

// Blend of list tiles (lists: a list_tile_dims code above 1, 16 x 16 screen tiles)
// without clusters: each screen tile's block reads its list tile's list
// (wide_blocks: 16x8 warp blocks with two pixel pairs per lane, else 8x8);
// order (optional): the list tiles in the order their blocks start.
cudaError_t gs_launch_blend_listtile(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                                     const GsGrid &list_grid, int lists, int width, int height, const float bg[3],
                                     const gs_framebuffer &fb, bool wide_blocks, const uint32_t *order,
                                     cudaStream_t s);
cudaError_t gs_launch_blend_cluster(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                                    const GsGrid &list_grid, int cluster, int width, int height, const float bg[3],
                                    const gs_framebuffer &fb, bool wide_blocks, cudaStream_t s);
// GS_BLEND_TMA: gathers the records of the sorted list (*d_n pairs, or n_cap
// without a device count) into `gather` (n_cap x 48 bytes, 16-byte aligned),
// then blends with bulk copies of contiguous record batches.
cudaError_t gs_launch_blend_tma(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                                const GsGrid &grid, int width, int height, const float bg[3],
                                const gs_framebuffer &fb, float4 *gather, const unsigned long long *d_n,
                                int64_t n_cap, uint32_t *d_err, cudaStream_t s);

// Per-frame binning front end, depth first: (1) projection of every Gaussian,
// appending each visible one to a compact list as (tiles << 32 | depth bits,
// index), in index order (the list slots come from a decoupled look-back
// scan), with the depth digit histograms; (2) a stable radix sort of that
// list by depth (4 digit passes over the visible Gaussians only), which so
// orders it by (depth bits, index); (3) a scan of the tile counts in depth
// order giving each entry its first key slot; (4) emission of the keys in
// that order: with xy_keys (grids at most 256 tiles wide) the key is (row <<
// 8 | column), the tile sort's digit histograms are counted from the rects
// in (1) and the emission is fused with the sort's first pass, whose output
// lands in keys / values (the caller runs passes 1..); otherwise the key is
// the tile id, counted by the emission, and all passes are the caller's.
// key_bytes = 2 or 4; `sc` is the tile sort's scratch (digit0 = 0, at least
// one pass). The stable tile sort leaves every tile's list in (depth bits,
// index) order.
// counts[0] = K, counts[1] = visible Gaussians, counts[2] = K if it fits in
// `capacity` else 0 (the tile sort and ranges then see an empty list and the
// overflow bit is set in d_err), counts[3] = visible Gaussians (the depth
// sort's count). `scan_scratch`: gs_fused_scratch_bytes(n, capacity).
size_t gs_fused_scratch_bytes(int64_t n, int64_t capacity);
size_t gs_key_block_bytes(int64_t capacity);
// Per-tile [first, last + 1) of tile keys sorted by gs_launch_project_bin
// + the tile sort (key_bytes 2 or 4; *d_n keys, the grid covering
// n_capacity); empty tiles get [0, 0). Keys are tile ids, or (row << 8 |
// column) when xy_tiles_x (the grid's width in tiles) is non-zero.
cudaError_t gs_launch_ranges_tiles(const void *keys, int key_bytes, int64_t n_capacity,
                                   const unsigned long long *d_n, int32_t n_tiles, uint32_t *ranges,
                                   uint32_t *d_err, cudaStream_t s, int xy_tiles_x = 0);
cudaError_t gs_launch_project_bin(const gs_gaussians &g, const GsCameraDev &cam, const GsGrid &grid,
                                  gs_record *records, const gs::BlendRecordOut &br,
                                  void *keys, int key_bytes, bool xy_keys, uint32_t *values,
                                  int64_t capacity, unsigned long long *counts, void *scan_scratch,
                                  const GsSortScratch &sc, uint32_t *d_err, cudaStream_t s,
                                  const cudaEvent_t *marks = nullptr /* 3 events or null */,
                                  uint2 *prect = nullptr /* n packed tile rects, for re-binning */,
                                  const uint2 *prev_rect = nullptr /* previous frame's: */,
                                  unsigned long long *moved = nullptr /* count of rects that differ */);

// CUDA graphs of gs_render frames: is `node` (of a captured graph) the
// projection's launch (gs_launch_project_bin or gs_launch_project_temporal),
// and set the camera that launch takes in an instantiated graph (the rest of
// its arguments stays as captured).
bool gs_is_camera_node(cudaGraphNode_t node);
cudaError_t gs_set_node_camera(cudaGraphExec_t exec, cudaGraphNode_t node, const GsCameraDev &cam);
// Temporal re-binning (gs_temporal.cu). Projection step: records as
// gs_launch_project_bin, plus per Gaussian its packed tile rect (`rect`),
// compared with the previous frame's (`prev_rect`): `moved` flags, work
// items (index << 32 | chunk, one per 256 tiles of the larger of a moved
// Gaussian's two rects) and counters (zeroed): [0] visible << 33 | keys,
// [1] moved Gaussians, [2] work items.
cudaError_t gs_launch_project_temporal(const gs_gaussians &g, const GsCameraDev &cam, const GsGrid &grid,
                                       gs_record *records, const gs::BlendRecordOut &br, const uint2 *prev_rect, uint2 *rect, uint8_t *moved,
                                       unsigned long long *items, int64_t item_capacity,
                                       unsigned long long *counters, uint32_t *d_err, cudaStream_t s);
struct GsTemporalRebin {
    const float4 *records;          // FP32 records of this frame
    const uint32_t *prev_vals, *prev_ranges;
    const uint8_t *moved;
    uint32_t *removed, *added;      // per tile, zeroed
    const unsigned long long *items;   // moved-Gaussian work items
    const unsigned long long *n_items;
    int64_t item_capacity;
    const uint2 *prev_rect, *rect;  // previous and this frame's packed rects
    int32_t n_tiles, tiles_x;
    int64_t n_gaussians;
    uint32_t *ranges;               // out
    uint32_t *vals;                 // out
    int64_t capacity;               // entries vals holds
    uint32_t *ins_first, *ins_cursor, *ins_vals;  // ins_cursor zeroed
    int64_t ins_capacity;
    unsigned long long *totals;     // out: [0] entries, [1] arrivals
    uint32_t *scan_counter;         // zeroed
    unsigned long long *scan_status;  // zeroed, gs_temporal_scan_status_bytes
    int cap_entries;                // per-tile entry limit (power of two)
    uint32_t *d_err;
};
size_t gs_temporal_merge_smem(int cap_entries);
size_t gs_temporal_scan_status_bytes(int32_t n_tiles);
cudaError_t gs_launch_temporal_rebin(const GsTemporalRebin &r, cudaStream_t s);

// Backward kernels. gs_launch_zero_grads zeroes the five gradient arrays of
// g's Gaussians and the rec_words floats of d_rec in one launch (before the
// blend backward adds into d_rec and the projection backward writes the
// gradients of the Gaussians that received any).
cudaError_t gs_launch_zero_grads(const gs_gaussians &g, const gs_grads &out, float *d_rec, size_t rec_words,
                                 cudaStream_t s);
cudaError_t gs_launch_blend_bwd(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                                const GsGrid &grid, int width, int height, const float bg[3],
                                const float *d_rgb, const float *final_T, const int32_t *n_contrib,
                                float *d_rec, cudaStream_t s, int cluster = 1);
// Backward of a joint batch (gs_render_batch): blend gradients per compact
// record slot over all views' tiles, then, per record slot (view, Gaussian),
// the projection gradients under that view's camera, added to the Gaussian's
// gradients (which the caller zeroed).
cudaError_t gs_launch_blend_bwd_batch(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                                      const ViewDesc *views, const GsBwdView *bviews, int n_views, int tile_w,
                                      int tile_h, int32_t total_tiles, float *d_rec, cudaStream_t s);
cudaError_t gs_launch_project_bwd_batch(const gs_gaussians &g, const ViewDesc *views, const uint2 *meta,
                                        int64_t n_records, const float *d_rec, const gs_grads &out, cudaStream_t s);
cudaError_t gs_launch_project_bwd(const gs_gaussians &g, const GsCameraDev &cam, const GsGrid &grid,
                                  const float *d_rec, const gs_grads &out, cudaStream_t s);

// Batched front end, depth first as gs_launch_project_bin: projection of
// every (view, Gaussian) pair into compact records (slot j: record, meta =
// (view, Gaussian index)), the list of slots gathered into (view, index)
// order and sorted by depth, then emission of 32-bit global tile ids (the
// view's first tile + tile) whose values are compact slots, with the tile
// sort's histograms + bucket offsets in sc (digit0 = 0). counts as in
// gs_launch_project_bin, with [1] = records used.
size_t gs_batch_scratch_bytes(int64_t rec_capacity, int64_t key_capacity, int64_t n, int n_views);
cudaError_t gs_launch_project_bin_batch(const gs_gaussians &g, const ViewDesc *views_dev, int n_views,
                                        gs_record *records, const gs::BlendRecordOut &br, uint2 *meta, int64_t rec_capacity, uint32_t *keys,
                                        uint32_t *values, int64_t key_capacity, unsigned long long *counts,
                                        void *scratch, const GsSortScratch &sc, uint32_t *d_err, cudaStream_t s);
// Persistent blend over a queue of global tiles (largest lists first); with
// list tiles (lists > 1, a list_tile_dims code) the queue holds one item per
// (global list tile, screen tile of it).
cudaError_t gs_launch_blend_batch(const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                                  const ViewDesc *views_dev, int n_views, int tile_w, int tile_h, int depth,
                                  const uint32_t *order, int32_t n_items, uint32_t *queue_head, int lists,
                                  cudaStream_t s);
// Longest-list-first order of one frame's n_tiles (list) tiles into order
// (n_tiles entries), from their ranges; one small kernel.
cudaError_t gs_launch_tile_order(const uint32_t *ranges, int32_t n_tiles, uint32_t *order, cudaStream_t s);
// Largest-first work queue of global tiles, subs items per tile (item t
// names tile t / subs); qs: gs_queue_scratch_bytes(), the queue head the
// blend takes items from is qs[193].
size_t gs_queue_scratch_bytes();
cudaError_t gs_launch_queue(const uint32_t *ranges, int32_t n_tiles, uint32_t *qs, uint32_t *order,
                            cudaStream_t s, int subs = 1);
