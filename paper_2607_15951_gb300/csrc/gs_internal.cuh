// gs_internal.cuh — device-side definitions shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gs {

// Constants of the standard 3DGS formulation (the paper cites it for Eq. 1
// and for the 3-sigma bound of Sec. 4.4 but prints none of them).
constexpr float kDilation = 0.3f;         // px^2 added to the 2D covariance diagonal
constexpr float kAlphaMax = 0.99f;        // opacity clamp
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;            // stop before T would fall below this
constexpr float kGuard = 1.3f;            // Jacobian view-ratio clamp, x tan(half fov)
constexpr int kMaxRadius = 1 << 30;       // radius clamp so tile arithmetic fits int64

// Device error word bits (gs_context::d_err).
enum : uint32_t { kErrTimeout = 1u, kErrCapacity = 2u, kErrRange = 4u };

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

// Tile rectangle of a record: columns [floor((u-r)/tw), floor((u+r+tw-1)/tw))
// and rows likewise, clamped to the grid. floor((u +- n)/t) for an integer n
// equals floordiv(floor(u) +- n, t), so the bounds are exact integer
// arithmetic on floor(u); |u| is clamped to 2^31, which cannot change an
// answer once the radius is clamped to 2^30.
struct Rect {
    int x0, y0, x1, y1;
};

__device__ __forceinline__ long long floordiv(long long a, int b) {
    long long q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

__device__ __forceinline__ int clamp_tile(long long v, int limit) {
    return v < 0 ? 0 : (v > limit ? limit : (int)v);
}

__device__ __forceinline__ Rect tile_rect(float u, float v, int r, int tw, int th, int tiles_x,
                                          int tiles_y) {
    const float lim = 2147483648.0f;
    long long fu = (long long)floorf(fminf(fmaxf(u, -lim), lim));
    long long fv = (long long)floorf(fminf(fmaxf(v, -lim), lim));
    Rect R;
    R.x0 = clamp_tile(floordiv(fu - r, tw), tiles_x);
    R.x1 = clamp_tile(floordiv(fu + r + tw - 1, tw), tiles_x);
    R.y0 = clamp_tile(floordiv(fv - r, th), tiles_y);
    R.y1 = clamp_tile(floordiv(fv + r + th - 1, th), tiles_y);
    return R;
}

// Records as three float4s (the gs_record layout):
//   r0 = (u, v, Q00, Q01), r1 = (Q11, opacity, red, green),
//   r2 = (blue, depth, radius bits, tiles bits).
struct Rec {
    float4 r0, r1, r2;
};
static_assert(sizeof(gs_record) == 48, "gs_record must be 48 bytes");

}  // namespace gs

// ---------------------------------------------------------------------------
// Host-side launch helpers (implemented in the kernel files).
// ---------------------------------------------------------------------------
struct GsCameraDev {
    float R[9];
    float t[3];
    float C[3];  // camera centre -R^T t
    float fx, fy, cx, cy, near_z;
    float lim_x, lim_y;  // 1.3 tan(half fov) per axis
    int width, height;
};

struct GsGrid {
    int tile_w, tile_h, tiles_x, tiles_y;
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

cudaError_t gs_launch_emit(const gs_record *records, const uint32_t *tiles,
                           const unsigned long long *offsets, int64_t n, const GsGrid &grid,
                           uint64_t *keys, uint32_t *values, int64_t capacity, uint32_t *d_err,
                           cudaStream_t s);

cudaError_t gs_launch_ranges(const uint64_t *keys, int64_t n, int32_t n_tiles, uint32_t *ranges,
                             uint32_t *d_err, cudaStream_t s);

// Onesweep radix sort. Scratch: gs_sort_scratch_bytes(n, key_bits) bytes.
// Sorts (keys, values) using (alt_keys, alt_values) as the ping-pong pair;
// *result_in_alt tells which pair holds the result.
size_t gs_sort_scratch_bytes(int64_t n, int key_bits);
cudaError_t gs_launch_sort(uint64_t *keys, uint32_t *values, uint64_t *alt_keys,
                           uint32_t *alt_values, int64_t n, int key_bits, void *scratch,
                           uint32_t *d_err, bool *result_in_alt, cudaStream_t s);
int gs_sort_passes(int key_bits);

cudaError_t gs_launch_blend(const gs_record *records, const uint32_t *values, const uint32_t *ranges,
                            const GsGrid &grid, int width, int height, const float bg[3],
                            const gs_framebuffer &fb, int variant, cudaStream_t s);
