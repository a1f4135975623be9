// gs_bin.cu — screen-tile binning (Sec. 3.1 stage 3; Sec. 4.5 step 2):
// for the gs_bin stage entry point, the exclusive scan of per-Gaussian tile
// counts and the emission of (tile << 32 | depth bits, index) pairs; for
// every path, the per-tile ranges of the sorted keys (64-bit keys, or the
// 16/32-bit tile keys of gs_render and gs_render_batch) and the batch blend's
// longest-list-first work queue. gs_render emits its keys in depth order in
// gs_project.cu; the sort itself is gs_sort.cu.
#include "gs_internal.cuh"

namespace {

using namespace gs;

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Single-pass exclusive scan of u32 counts into u64 offsets (decoupled
// look-back; partitions taken in launch order from an atomic counter so a
// block only ever waits on blocks that are already running).
__global__ void __launch_bounds__(kScanThreads)
scan_kernel(const uint32_t *__restrict__ in, int64_t n, unsigned long long *__restrict__ out,
            unsigned long long *counts, uint32_t *counter, unsigned long long *status,
            int64_t num_parts, uint32_t *d_err, unsigned long long timeout_ns) {
    __shared__ uint32_t s_part;
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    __shared__ uint32_t s_vis[kScanThreads / 32];
    __shared__ unsigned long long s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_part = atomicAdd(counter, 1u);
    __syncthreads();
    const long long p = s_part;
    const long long base = p * kScanTile + (long long)tid * kScanItems;

    uint32_t v[kScanItems];
    unsigned long long sum = 0;
    uint32_t vis = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const long long idx = base + j;
        v[j] = idx < n ? in[idx] : 0u;
        sum += v[j];
        vis += v[j] != 0u;
    }
    // Block-wide exclusive scan of the per-thread sums.
    unsigned long long incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    for (int o = 16; o > 0; o >>= 1) vis += __shfl_xor_sync(0xffffffffu, vis, o);
    if (lane == 31) s_warp[warp] = incl;
    if (lane == 0) s_vis[warp] = vis;
    __syncthreads();
    unsigned long long warp_prefix = 0, block_total = 0;
    uint32_t block_vis = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        if (w < warp) warp_prefix += s_warp[w];
        block_total += s_warp[w];
        block_vis += s_vis[w];
    }
    const unsigned long long thread_excl = warp_prefix + incl - sum;

    if (warp == 0) {
        unsigned long long prefix = 0;
        if (p == 0) {
            if (lane == 0) st_relaxed_u64(status, kFlagIncl | block_total);
        } else {
            if (lane == 0) st_relaxed_u64(status + p, kFlagAgg | block_total);
            bool to;
            prefix = warp_lookback(status, p, d_err, &to, timeout_ns);
            if (lane == 0) st_relaxed_u64(status + p, kFlagIncl | ((prefix + block_total) & kValueMask));
        }
        if (lane == 0) {
            s_prefix = prefix;
            if (block_vis) atomicAdd(counts + 1, (unsigned long long)block_vis);
            if (p == num_parts - 1) counts[0] = prefix + block_total;
        }
    }
    __syncthreads();
    unsigned long long run = s_prefix + thread_excl;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const long long idx = base + j;
        if (idx < n) out[idx] = run;
        run += v[j];
    }
}

// Key emission. Gaussian i owns keys [offsets[i], offsets[i] + tiles[i]);
// it writes one key per tile of its rect, row by row:
//   key = tile_id << 32 | bits(depth), value = i.
// Gaussians covering at most 32 tiles are written by their own thread; larger
// ones are written by the whole warp, one at a time, with coalesced stores.
__global__ void __launch_bounds__(256)
emit_kernel(const float4 *__restrict__ rec, const uint32_t *__restrict__ tiles,
            const unsigned long long *__restrict__ offsets, int64_t n, GsGrid grid,
            uint64_t *__restrict__ keys, uint32_t *__restrict__ values, int64_t capacity,
            uint32_t *d_err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    uint32_t t = i < n ? tiles[i] : 0u;
    Rect R = {0, 0, 0, 0};
    uint32_t dbits = 0;
    unsigned long long off = 0;
    if (t) {
        const float4 r0 = rec[3 * i], r2 = rec[3 * i + 2];
        R = tile_rect(r0.x, r0.y, __float_as_int(r2.z), grid.tile_w, grid.tile_h, grid.tiles_x,
                      grid.tiles_y);
        dbits = __float_as_uint(r2.y);
        off = offsets[i];
        const long long area = (long long)(R.x1 - R.x0) * (R.y1 - R.y0);
        if (area != (long long)t) {
            atomicOr(d_err, kErrRange);
            t = 0;
        } else if (off + t > (unsigned long long)capacity) {
            atomicOr(d_err, kErrCapacity);
            t = 0;
        }
    }
    const bool big = t > 32u;
    if (t && !big) {
        unsigned long long k = off;
        for (int ty = R.y0; ty < R.y1; ++ty)
            for (int tx = R.x0; tx < R.x1; ++tx, ++k) {
                keys[k] = ((uint64_t)(ty * grid.tiles_x + tx) << 32) | dbits;
                values[k] = (uint32_t)i;
            }
    }
    uint32_t bigmask = __ballot_sync(0xffffffffu, big);
    while (bigmask) {
        const int src = __ffs(bigmask) - 1;
        bigmask &= bigmask - 1;
        const int x0 = __shfl_sync(0xffffffffu, R.x0, src);
        const int y0 = __shfl_sync(0xffffffffu, R.y0, src);
        const int w = __shfl_sync(0xffffffffu, R.x1 - R.x0, src);
        const uint32_t cnt = __shfl_sync(0xffffffffu, t, src);
        const uint32_t db = __shfl_sync(0xffffffffu, dbits, src);
        const unsigned long long o = __shfl_sync(0xffffffffu, off, src);
        const uint32_t gi = (uint32_t)(i - lane + src);
        for (uint32_t k = lane; k < cnt; k += 32) {
            const int ty = y0 + (int)(k / (uint32_t)w), tx = x0 + (int)(k % (uint32_t)w);
            keys[o + k] = ((uint64_t)(ty * grid.tiles_x + tx) << 32) | db;
            values[o + k] = gi;
        }
    }
}

// Per-tile [first, last+1) of n sorted (tile << 32 | depth bits) keys;
// ranges must be zeroed first.
__global__ void ranges_kernel(const uint64_t *__restrict__ keys, int64_t n, int32_t n_tiles,
                              uint32_t *__restrict__ ranges, uint32_t *d_err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t tile = keys[i] >> 32;
    if (tile >= (uint64_t)n_tiles) {
        atomicOr(d_err, kErrRange);
        return;
    }
    if (i == 0) {
        ranges[2 * tile] = 0;
    } else {
        const uint64_t prev = keys[i - 1] >> 32;
        if (prev != tile) {
            ranges[2 * tile] = (uint32_t)i;
            if (prev < (uint64_t)n_tiles) ranges[2 * prev + 1] = (uint32_t)i;
        }
    }
    if (i == n - 1) ranges[2 * tile + 1] = (uint32_t)n;
}

// Per-tile [first, last+1) of sorted tile-id keys; ranges must be zeroed
// first. Thread t looks at keys [8t, 8t + 8) (one or two 16-byte loads while
// the capacity allows, so the grid covers the capacity) and the key before
// them; a boundary between keys i-1 and i opens tile key[i] and closes tile
// key[i-1].
template <typename KT>
__global__ void __launch_bounds__(256) ranges_tiles_kernel(const KT *__restrict__ keys, int64_t n_capacity,
                                                          const unsigned long long *d_n, int32_t n_tiles,
                                                          uint32_t *__restrict__ ranges, uint32_t *d_err,
                                                          int xy_tiles_x) {
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8;
    const int64_t n = (int64_t)*d_n;
    if (i0 >= n) return;
    uint32_t k[8];
    if (i0 + 8 <= n_capacity) {
        const uint4 a = reinterpret_cast<const uint4 *>(keys + i0)[0];
        if (sizeof(KT) == 2) {
            k[0] = a.x & 0xffffu; k[1] = a.x >> 16; k[2] = a.y & 0xffffu; k[3] = a.y >> 16;
            k[4] = a.z & 0xffffu; k[5] = a.z >> 16; k[6] = a.w & 0xffffu; k[7] = a.w >> 16;
        } else {
            const uint4 b = reinterpret_cast<const uint4 *>(keys + i0)[1];
            k[0] = a.x; k[1] = a.y; k[2] = a.z; k[3] = a.w;
            k[4] = b.x; k[5] = b.y; k[6] = b.z; k[7] = b.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) k[j] = i0 + j < n ? (uint32_t)keys[i0 + j] : 0u;
    }
    // (row << 8 | column) keys to tile ids (the order is the same).
    auto tile_of = [&](uint32_t key) {
        return xy_tiles_x ? (key >> 8) * (uint32_t)xy_tiles_x + (key & 255u) : key;
    };
    uint32_t prev = i0 > 0 ? tile_of((uint32_t)keys[i0 - 1]) : 0xffffffffu;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int64_t i = i0 + j;
        if (i >= n) break;
        const uint32_t t = tile_of(k[j]);
        if (t >= (uint32_t)n_tiles) {
            atomicOr(d_err, kErrRange);
            return;
        }
        if (t != prev) {
            ranges[2 * t] = (uint32_t)i;
            if (prev < (uint32_t)n_tiles) ranges[2 * prev + 1] = (uint32_t)i;
        }
        if (i == n - 1) ranges[2 * t + 1] = (uint32_t)n;
        prev = t;
    }
}

}  // namespace

cudaError_t gs_launch_ranges_tiles(const void *keys, int key_bytes, int64_t n_capacity,
                                   const unsigned long long *d_n, int32_t n_tiles, uint32_t *ranges,
                                   uint32_t *d_err, cudaStream_t s, int xy_tiles_x) {
    if (key_bytes != 2 && key_bytes != 4) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(ranges, 0, (size_t)n_tiles * 2 * sizeof(uint32_t), s);
    if (e != cudaSuccess || n_capacity == 0) return e;
    const unsigned blocks = (unsigned)((n_capacity + 8 * 256 - 1) / (8 * 256));
    if (key_bytes == 2)
        ranges_tiles_kernel<uint16_t><<<blocks, 256, 0, s>>>(static_cast<const uint16_t *>(keys), n_capacity, d_n,
                                                            n_tiles, ranges, d_err, xy_tiles_x);
    else
        ranges_tiles_kernel<uint32_t><<<blocks, 256, 0, s>>>(static_cast<const uint32_t *>(keys), n_capacity, d_n,
                                                            n_tiles, ranges, d_err, xy_tiles_x);
    return cudaGetLastError();
}

size_t gs_scan_scratch_bytes(int64_t n) {
    const int64_t parts = (n + kScanTile - 1) / kScanTile;
    return 16 + (size_t)(parts > 0 ? parts : 1) * sizeof(unsigned long long);
}

cudaError_t gs_launch_scan(const uint32_t *tiles, int64_t n, unsigned long long *offsets,
                           unsigned long long *counts, void *scratch, uint32_t *d_err,
                           cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess || n == 0) return e;
    e = cudaMemsetAsync(scratch, 0, gs_scan_scratch_bytes(n), s);
    if (e != cudaSuccess) return e;
    const int64_t parts = (n + kScanTile - 1) / kScanTile;
    uint32_t *counter = static_cast<uint32_t *>(scratch);
    unsigned long long *status =
        reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) + 16);
    scan_kernel<<<(unsigned)parts, kScanThreads, 0, s>>>(tiles, n, offsets, counts, counter, status,
                                                         parts, d_err, kSpinTimeoutNs);
    return cudaGetLastError();
}

cudaError_t gs_launch_emit(const gs_record *records, const uint32_t *tiles,
                           const unsigned long long *offsets, int64_t n, const GsGrid &grid,
                           uint64_t *keys, uint32_t *values, int64_t capacity, uint32_t *d_err,
                           cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    emit_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const float4 *>(records), tiles, offsets, n,
                                       grid, keys, values, capacity, d_err);
    return cudaGetLastError();
}

cudaError_t gs_launch_ranges(const uint64_t *keys, int64_t n, int32_t n_tiles, uint32_t *ranges,
                             uint32_t *d_err, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ranges, 0, (size_t)n_tiles * 2 * sizeof(uint32_t), s);
    if (e != cudaSuccess || n == 0) return e;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    ranges_kernel<<<blocks, 256, 0, s>>>(keys, n, n_tiles, ranges, d_err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Work queue of a batched blend: global tiles ordered by the bit length of
// their list (longest first), so that the largest tiles start first and the
// short ones fill the tail. Order inside a bucket is arbitrary (it does not
// change any output).
// ---------------------------------------------------------------------------
namespace {

constexpr int kBuckets = 33;

__global__ void queue_count_kernel(const uint32_t *__restrict__ ranges, int64_t n_items, int subs, uint32_t *qs) {
    // qs: [0,64) counts, [64,128) starts, [128,192) cursors, 192 ticket, 193 head
    __shared__ uint32_t s_c[kBuckets];
    __shared__ bool s_last;
    for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) s_c[b] = 0;
    __syncthreads();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_items;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tile = t / subs;
        const uint32_t len = ranges[2 * tile + 1] - ranges[2 * tile];
        atomicAdd(&s_c[len ? 32 - __clz(len) : 0], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBuckets; b += blockDim.x)
        if (s_c[b]) atomicAdd(&qs[b], s_c[b]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&qs[192], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    uint32_t run = 0;
    for (int b = kBuckets - 1; b >= 0; --b) {
        qs[64 + b] = run;
        run += __ldcg(&qs[b]);
    }
}

__global__ void queue_scatter_kernel(const uint32_t *__restrict__ ranges, int64_t n_items, int subs, uint32_t *qs,
                                     uint32_t *__restrict__ order) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_items) return;
    const int64_t tile = t / subs;
    const uint32_t len = ranges[2 * tile + 1] - ranges[2 * tile];
    const int b = len ? 32 - __clz(len) : 0;
    order[qs[64 + b] + atomicAdd(&qs[128 + b], 1u)] = (uint32_t)t;
}

}  // namespace

namespace {

// Longest-list-first order of one frame's (list) tiles, one block: a
// counting sort of the tiles by the bit length of their list, longest first
// (tiles in one bucket keep an arbitrary order). Each thread loads the ranges
// of up to kOrderUnroll tiles at once; lanes of a warp that fall in the same
// bucket take one shared-memory atomic between them; the buckets of the
// first kOrderCache tiles are kept in shared memory for the second pass.
constexpr int kOrderThreads = 1024, kOrderUnroll = 8, kOrderCache = 32768;

__device__ __forceinline__ int order_bucket(uint2 r) {
    const uint32_t len = r.y - r.x;
    return len ? 32 - __clz(len) : 0;
}

__global__ void __launch_bounds__(kOrderThreads) tile_order_kernel(const uint2 *__restrict__ ranges,
                                                                   int32_t n_tiles, uint32_t *__restrict__ order) {
    __shared__ uint32_t s_count[kBuckets], s_next[kBuckets];
    __shared__ uint8_t s_bucket[kOrderCache];
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < kBuckets) s_count[tid] = 0;
    __syncthreads();
    // Tile base + j kOrderThreads + lane for j < kOrderUnroll (base: the
    // warp's first tile, warp-uniform, so every lane takes each match).
    for (int base = tid - lane; base < n_tiles; base += kOrderThreads * kOrderUnroll) {
        uint2 r[kOrderUnroll];
#pragma unroll
        for (int j = 0; j < kOrderUnroll; ++j) {
            const int t = base + j * kOrderThreads + lane;
            r[j] = t < n_tiles ? ranges[t] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int j = 0; j < kOrderUnroll; ++j) {
            const int t = base + j * kOrderThreads + lane;
            const int b = t < n_tiles ? order_bucket(r[j]) : kBuckets;  // kBuckets: no tile
            const uint32_t peers = __match_any_sync(0xffffffffu, b);
            if (b < kBuckets && lane == __ffs(peers) - 1) atomicAdd(&s_count[b], (uint32_t)__popc(peers));
            if (t < n_tiles && t < kOrderCache) s_bucket[t] = (uint8_t)b;
        }
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t run = 0;
        for (int b = kBuckets - 1; b >= 0; --b) {
            s_next[b] = run;
            run += s_count[b];
        }
    }
    __syncthreads();
    for (int base = tid - lane; base < n_tiles; base += kOrderThreads) {
        const int t = base + lane;
        const int b = t >= n_tiles ? kBuckets : t < kOrderCache ? (int)s_bucket[t] : order_bucket(ranges[t]);
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        uint32_t first = 0;
        if (b < kBuckets && lane == leader) first = atomicAdd(&s_next[b], (uint32_t)__popc(peers));
        first = __shfl_sync(0xffffffffu, first, leader);
        if (b < kBuckets) order[first + __popc(peers & lanemask_lt())] = (uint32_t)t;
    }
}

}  // namespace

cudaError_t gs_launch_tile_order(const uint32_t *ranges, int32_t n_tiles, uint32_t *order, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    // ranges: 2 n_tiles words from cudaMalloc, so 8-byte aligned pairs
    tile_order_kernel<<<1, kOrderThreads, 0, s>>>(reinterpret_cast<const uint2 *>(ranges), n_tiles, order);
    return cudaGetLastError();
}

size_t gs_queue_scratch_bytes() { return 256 * sizeof(uint32_t); }

cudaError_t gs_launch_queue(const uint32_t *ranges, int32_t n_tiles, uint32_t *qs, uint32_t *order,
                            cudaStream_t s, int subs) {
    cudaError_t e = cudaMemsetAsync(qs, 0, gs_queue_scratch_bytes(), s);
    const int64_t n_items = (int64_t)n_tiles * subs;
    if (e != cudaSuccess || n_items == 0) return e;
    const unsigned blocks = (unsigned)((n_items + 255) / 256);
    queue_count_kernel<<<blocks < 608 ? blocks : 608, 256, 0, s>>>(ranges, n_items, subs, qs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    queue_scatter_kernel<<<blocks, 256, 0, s>>>(ranges, n_items, subs, qs, order);
    return cudaGetLastError();
}

size_t gs_selftest_scratch_bytes(int64_t n) {
    // scan: counter + status (parts + 1) + offsets + counts; sort: keys,
    // values, their copies and the sort scratch
    const int64_t parts = (n + kScanTile - 1) / kScanTile + 1;
    const size_t scan = 256 + (size_t)parts * 8 + (size_t)n * 8 + 64;
    const size_t sort = (size_t)n * 24 + gs_sort_scratch_bytes(n, 8) + 4096;
    return scan > sort ? scan : sort;
}

cudaError_t gs_launch_selftest_wait(int kind, int64_t n, void *scratch, uint32_t *d_err,
                                    unsigned long long timeout_ns, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(scratch, 0, gs_selftest_scratch_bytes(n), s);
    if (e != cudaSuccess) return e;
    char *base = static_cast<char *>(scratch);
    const uint32_t one = 1;
    if (kind == 0) {
        const int64_t parts = (n + kScanTile - 1) / kScanTile;
        uint32_t *counter = reinterpret_cast<uint32_t *>(base);
        unsigned long long *status = reinterpret_cast<unsigned long long *>(base + 256);
        unsigned long long *offsets = status + parts + 1;
        unsigned long long *counts = offsets + n;
        const uint32_t *tiles = reinterpret_cast<const uint32_t *>(counts + 4);  // zeros
        e = cudaMemcpyAsync(counter, &one, 4, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        // Blocks take partitions 1 .. parts; partition 0 is never taken.
        scan_kernel<<<(unsigned)parts, kScanThreads, 0, s>>>(tiles, n, offsets, counts, counter, status,
                                                             parts + 1, d_err, timeout_ns);
        return cudaGetLastError();
    }
    uint64_t *keys = reinterpret_cast<uint64_t *>(base);
    uint32_t *vals = reinterpret_cast<uint32_t *>(keys + n);
    uint64_t *akeys = reinterpret_cast<uint64_t *>(vals + n);
    uint32_t *avals = reinterpret_cast<uint32_t *>(akeys + n);
    char *sbase = reinterpret_cast<char *>(avals + n);
    sbase += (256 - reinterpret_cast<uintptr_t>(sbase) % 256) % 256;
    const GsSortScratch sc = gs_sort_carve(sbase, n, 8);
    e = cudaMemcpyAsync(sc.counter, &one, 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    bool in_alt = false;
    return gs_launch_sort_passes(keys, vals, akeys, avals, n, nullptr, sc, d_err, &in_alt, s, timeout_ns, 1);
}
