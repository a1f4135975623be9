// gs_temporal.cu — temporal re-binning: the per-tile lists of a frame are
// rebuilt from those of the previous frame (the paper's temporal-locality
// idea, Sec. 5.4 and Sec. 6: when the view changes gradually most Gaussians
// stay in the screen tiles they were in).
//
// After the temporal projection (gs_project.cu) has listed the Gaussians
// whose tile rect changed ("moved"):
//  1. moved_count_kernel: one warp per work item (a moved Gaussian, or a
//     256-tile chunk of a large one) counts, per tile, the entries that leave
//     (its old rect) and arrive (its new rect);
//  2. tile_scan_kernel: new per-tile counts (old - removed + added) and the
//     first slot of every tile in the new value array and in the array of
//     arriving entries (decoupled look-back over partitions of tiles);
//  3. moved_emit_kernel: one warp per work item writes the Gaussian's index
//     into the arriving entries of each of its tiles (eight slot atomics in
//     flight per lane: one round trip per chunk, however large the splat);
//  4. tile_merge_kernel: one block per tile keeps the old entries whose
//     Gaussian did not move (in their old order), restores their order under
//     this frame's (depth bits, Gaussian index) with a few odd-even
//     transposition rounds (a bitonic sort if that is not enough), sorts the
//     arriving ones and merges the two runs.
// The result is exactly the list the full binning would produce. The merge
// runs twice: for tiles of up to 1024 entries with little shared memory per
// block, then for the larger ones. A tile above the per-tile limit, a key
// count above the capacity or state that does not match the frame sets
// kErrTemporal: the caller rebuilds the frame.
#include "gs_internal.cuh"

namespace {

using namespace gs;

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // tiles per scan partition
constexpr int kMergeThreads = 256;

struct TileScanArgs {
    const uint32_t *prev_ranges;  // n_tiles x 2
    const uint32_t *removed, *added;
    int32_t n_tiles;
    uint32_t *ranges;             // out: n_tiles x 2
    uint32_t *ins_first;          // out: first arriving-entry slot of each tile
    unsigned long long *totals;   // out: [0] entries, [1] arriving entries
    uint32_t *counter;            // zeroed
    unsigned long long *status;   // zeroed, one per partition
    uint32_t *d_err;
};

// Packed per-tile value: entries << 32 | arrivals (both sums stay below 2^30
// while the key count fits the capacity checked below).
__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(const TileScanArgs A) {
    __shared__ uint32_t s_part;
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    __shared__ unsigned long long s_prefix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_part = atomicAdd(A.counter, 1u);
    __syncthreads();
    const int64_t p = s_part;
    const int64_t base = p * kScanTile + (int64_t)tid * kScanItems;
    unsigned long long v[kScanItems];
    unsigned long long sum = 0;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t t = base + j;
        v[j] = 0;
        if (t < A.n_tiles) {
            const uint32_t n_old = A.prev_ranges[2 * t + 1] - A.prev_ranges[2 * t];
            const uint32_t rem = A.removed[t], add = A.added[t];
            bad |= rem > n_old;
            const uint32_t n_new = rem > n_old ? add : n_old - rem + add;
            v[j] = ((unsigned long long)n_new << 32) | add;
        }
        sum += v[j];
    }
    if (bad) atomicOr(A.d_err, kErrTemporal);
    unsigned long long incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    unsigned long long warp_prefix = 0, block_total = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        if (w < warp) warp_prefix += s_warp[w];
        block_total += s_warp[w];
    }
    const int64_t parts = (A.n_tiles + kScanTile - 1) / kScanTile;
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
        if (lane == 0) {
            s_prefix = prefix;
            if (p == parts - 1) {
                const unsigned long long tot = prefix + block_total;
                A.totals[0] = tot >> 32;
                A.totals[1] = tot & 0xffffffffull;
            }
        }
    }
    __syncthreads();
    unsigned long long run = s_prefix + warp_prefix + incl - sum;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        const int64_t t = base + j;
        if (t < A.n_tiles) {
            const uint32_t first = (uint32_t)(run >> 32);
            A.ranges[2 * t] = first;
            A.ranges[2 * t + 1] = first + (uint32_t)(v[j] >> 32);
            A.ins_first[t] = (uint32_t)(run & 0xffffffffull);
        }
        run += v[j];
    }
}

constexpr int kChunkTiles = 256;  // tiles of a rect per work item (as in the projection)

struct MovedArgs {
    const unsigned long long *items;   // index << 32 | chunk
    const unsigned long long *n_list;  // device count of the items (may exceed item_capacity:
    int64_t item_capacity;             // the projection then flagged the frame)
    const uint2 *prev_rect, *rect;     // packed rects, previous and this frame
    int32_t tiles_x;
    uint32_t *removed, *added;         // per tile (moved_count_kernel)
    const uint32_t *ins_first;         // per tile (moved_emit_kernel)
    uint32_t *ins_cursor;              // zeroed, per tile
    uint32_t *ins_vals;
    int64_t ins_capacity;
    uint32_t *d_err;
};

struct RectSpan {
    int x0, y0, w, n;  // n = w * h tiles, 0 when empty
};

__device__ __forceinline__ RectSpan unpack_span(uint2 r) {
    RectSpan s;
    s.x0 = (int)(r.x & 0xffffu);
    s.y0 = (int)(r.y & 0xffffu);
    s.w = (int)(r.x >> 16) - s.x0;
    const int h = (int)(r.y >> 16) - s.y0;
    s.n = (s.w > 0 && h > 0) ? s.w * h : 0;
    return s;
}

// One warp per moved Gaussian: every tile of its old rect loses an entry,
// every tile of its new rect gains one (reductions, no returned values).
__global__ void __launch_bounds__(256) moved_count_kernel(const MovedArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t warp_id = ((int64_t)blockIdx.x * 256 + threadIdx.x) >> 5;
    const int64_t n_warps = (int64_t)gridDim.x * 8;
    const int64_t n = (int64_t)*A.n_list < A.item_capacity ? (int64_t)*A.n_list : A.item_capacity;
    for (int64_t q = warp_id; q < n; q += n_warps) {
        const unsigned long long item = A.items[q];
        const uint32_t g = (uint32_t)(item >> 32);
        const int k0 = (int)(item & 0xffffffffu) * kChunkTiles;
        const RectSpan o = unpack_span(A.prev_rect[g]), r = unpack_span(A.rect[g]);
        const int oe = o.n < k0 + kChunkTiles ? o.n : k0 + kChunkTiles;
        const int re = r.n < k0 + kChunkTiles ? r.n : k0 + kChunkTiles;
        for (int k = k0 + lane; k < oe; k += 32)
            atomicAdd(&A.removed[(o.y0 + k / o.w) * A.tiles_x + o.x0 + k % o.w], 1u);
        for (int k = k0 + lane; k < re; k += 32)
            atomicAdd(&A.added[(r.y0 + k / r.w) * A.tiles_x + r.x0 + k % r.w], 1u);
    }
}

// One warp per moved Gaussian: its index goes into the arriving entries of
// every tile of its new rect, at a slot taken from the tile's cursor.
__global__ void __launch_bounds__(256) moved_emit_kernel(const MovedArgs A) {
    constexpr int kUnroll = 8;
    const int lane = threadIdx.x & 31;
    const int64_t warp_id = ((int64_t)blockIdx.x * 256 + threadIdx.x) >> 5;
    const int64_t n_warps = (int64_t)gridDim.x * 8;
    const int64_t n = (int64_t)*A.n_list < A.item_capacity ? (int64_t)*A.n_list : A.item_capacity;
    for (int64_t q = warp_id; q < n; q += n_warps) {
        const unsigned long long item = A.items[q];
        const uint32_t g = (uint32_t)(item >> 32);
        const int kb = (int)(item & 0xffffffffu) * kChunkTiles;
        const RectSpan r = unpack_span(A.rect[g]);
        const int ke = r.n < kb + kChunkTiles ? r.n : kb + kChunkTiles;
        for (int k0 = kb; k0 < ke; k0 += 32 * kUnroll) {
            int tile[kUnroll];
            uint32_t c[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int k = k0 + u * 32 + lane;
                tile[u] = k < ke ? (r.y0 + k / r.w) * A.tiles_x + r.x0 + k % r.w : -1;
                c[u] = tile[u] >= 0 ? atomicAdd(&A.ins_cursor[tile[u]], 1u) : 0u;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                if (tile[u] < 0) continue;
                const uint64_t slot = (uint64_t)A.ins_first[tile[u]] + c[u];
                if (slot < (uint64_t)A.ins_capacity)
                    A.ins_vals[slot] = g;
                else
                    atomicOr(A.d_err, kErrTemporal);
            }
        }
    }
}

struct MergeArgs {
    const float4 *records;         // FP32 records (depth in word 9)
    const uint32_t *prev_vals, *prev_ranges;
    const uint8_t *moved;
    const uint32_t *removed, *added, *ins_first, *ins_vals;
    const uint32_t *ranges;        // this frame's
    uint32_t *vals;                // out
    int64_t capacity;              // of vals
    uint32_t min_entries;          // this launch merges tiles with min_entries < entries <= cap_entries
    int cap_entries;               // (shared memory); above the largest class is an error
    bool last_class;
    uint32_t *d_err;
};

__device__ __forceinline__ unsigned long long depth_key(const float4 *rec, uint32_t g) {
    return ((unsigned long long)__float_as_uint(__ldg(&rec[3 * (size_t)g + 2].y)) << 32) | g;
}

// Bitonic sort of s[0, n) in shared memory, padded to a power of two with
// keys above every real one (the depth word of a real key is a finite float).
__device__ void block_bitonic(unsigned long long *s, uint32_t n) {
    const int tid = threadIdx.x;
    uint32_t p2 = 1;
    while (p2 < n) p2 <<= 1;
    for (uint32_t i = n + tid; i < p2; i += kMergeThreads) s[i] = ~0ull;
    __syncthreads();
    for (uint32_t k = 2; k <= p2; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = tid; i < p2; i += kMergeThreads) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = s[i], b = s[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

constexpr int kRepairRounds = 16;  // odd-even transposition rounds before a full sort

__global__ void __launch_bounds__(kMergeThreads) tile_merge_kernel(const MergeArgs A) {
    extern __shared__ unsigned long long s_key[];  // kept entries [cap], then arrivals [cap]
    __shared__ uint32_t s_wcnt[kMergeThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int t = blockIdx.x;
    const uint32_t old_first = A.prev_ranges[2 * t], n_old = A.prev_ranges[2 * t + 1] - old_first;
    const uint32_t rem = A.removed[t], add = A.added[t];
    const uint32_t out_first = A.ranges[2 * t], n_new = A.ranges[2 * t + 1] - out_first;
    if (n_new <= A.min_entries) return;
    if (n_new > (uint32_t)A.cap_entries && !A.last_class) return;
    if (rem > n_old || n_new != n_old - rem + add || n_new > (uint32_t)A.cap_entries ||
        (uint64_t)out_first + n_new > (uint64_t)A.capacity) {
        if (tid == 0) atomicOr(A.d_err, kErrTemporal);
        return;
    }
    unsigned long long *s_arr = s_key + A.cap_entries;
    // 1. Entries that stay, in their old order (stable compaction by warp
    // ballots). The loads of kUnroll entries per thread (index, moved flag,
    // depth) are issued together, so a long list costs few memory round trips.
    constexpr int kUnroll = 4;
    uint32_t n_kept = 0;
    for (uint32_t b = 0; b < n_old; b += kMergeThreads * kUnroll) {
        uint32_t g[kUnroll];
        bool keep[kUnroll];
        unsigned long long key[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint32_t k = b + u * kMergeThreads + tid;
            g[u] = k < n_old ? A.prev_vals[old_first + k] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint32_t k = b + u * kMergeThreads + tid;
            keep[u] = k < n_old && A.moved[g[u]] == 0;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) key[u] = keep[u] ? depth_key(A.records, g[u]) : 0ull;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const uint32_t ball = __ballot_sync(0xffffffffu, keep[u]);
            if (lane == 0) s_wcnt[warp] = __popc(ball);
            __syncthreads();
            uint32_t off = 0, total = 0;
            for (int w = 0; w < kMergeThreads / 32; ++w) {
                off += w < warp ? s_wcnt[w] : 0u;
                total += s_wcnt[w];
            }
            const uint32_t pos = n_kept + off + __popc(ball & lanemask_lt());
            if (keep[u] && pos < (uint32_t)A.cap_entries) s_key[pos] = key[u];
            n_kept += total;
            __syncthreads();
        }
    }
    if (n_kept + add != n_new) {
        if (tid == 0) atomicOr(A.d_err, kErrTemporal);
        return;
    }
    // 2. Arriving entries.
    const uint32_t ins0 = A.ins_first[t];
    for (uint32_t j = tid; j < add; j += kMergeThreads) s_arr[j] = depth_key(A.records, A.ins_vals[ins0 + j]);
    // 3. The kept entries were in the previous frame's depth order; depths
    // changed a little, so a few odd-even transposition rounds usually restore
    // the order (keys are distinct: the index is in them). Otherwise sort.
    __syncthreads();
    bool in_order = false;
    for (int r = 0; r < kRepairRounds && !in_order; ++r) {
        bool swapped = false;
        for (uint32_t phase = 0; phase < 2; ++phase) {
            for (uint32_t i = 2 * tid + phase; i + 1 < n_kept; i += 2 * kMergeThreads) {
                const unsigned long long a = s_key[i], b = s_key[i + 1];
                if (a > b) {
                    s_key[i] = b;
                    s_key[i + 1] = a;
                    swapped = true;
                }
            }
            __syncthreads();
        }
        in_order = !__syncthreads_or(swapped);
    }
    if (!in_order) block_bitonic(s_key, n_kept);
    if (add > 1) block_bitonic(s_arr, add);
    // 4. Merge: every entry goes to (its rank in its own run) + (entries of the
    // other run below it), found by binary search.
    uint32_t *out = A.vals + out_first;
    for (uint32_t i = tid; i < n_kept; i += kMergeThreads) {
        const unsigned long long ki = s_key[i];
        uint32_t lo = 0, hi = add;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_arr[mid] < ki) lo = mid + 1; else hi = mid;
        }
        out[i + lo] = (uint32_t)ki;
    }
    for (uint32_t j = tid; j < add; j += kMergeThreads) {
        const unsigned long long kj = s_arr[j];
        uint32_t lo = 0, hi = n_kept;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_key[mid] < kj) lo = mid + 1; else hi = mid;
        }
        out[j + lo] = (uint32_t)kj;
    }
}

}  // namespace

size_t gs_temporal_merge_smem(int cap_entries) { return (size_t)cap_entries * 2 * sizeof(unsigned long long); }

size_t gs_temporal_scan_status_bytes(int32_t n_tiles) {
    return ((size_t)(n_tiles + kScanTile - 1) / kScanTile + 1) * sizeof(unsigned long long);
}

cudaError_t gs_launch_temporal_rebin(const GsTemporalRebin &R, cudaStream_t s) {
    if (R.n_tiles <= 0) return cudaSuccess;
    int64_t blocks = (R.n_gaussians + 255) / 256;
    if (blocks > 1216) blocks = 1216;
    if (blocks < 1) blocks = 1;
    MovedArgs M{R.items, R.n_items, R.item_capacity, R.prev_rect, R.rect, R.tiles_x, R.removed, R.added, R.ins_first,
                R.ins_cursor, R.ins_vals, R.ins_capacity, R.d_err};
    moved_count_kernel<<<(unsigned)blocks, 256, 0, s>>>(M);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    TileScanArgs S{R.prev_ranges, R.removed, R.added, R.n_tiles, R.ranges, R.ins_first, R.totals,
                   R.scan_counter, R.scan_status, R.d_err};
    tile_scan_kernel<<<(unsigned)((R.n_tiles + kScanTile - 1) / kScanTile), kScanThreads, 0, s>>>(S);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    moved_emit_kernel<<<(unsigned)blocks, 256, 0, s>>>(M);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // Two size classes: small tiles with little shared memory per block (many
    // blocks per SM), then the large ones.
    const int small_cap = R.cap_entries < 1024 ? R.cap_entries : 1024;
    const size_t big_smem = gs_temporal_merge_smem(R.cap_entries);
    e = cudaFuncSetAttribute(tile_merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem);
    if (e != cudaSuccess) return e;
    MergeArgs G{R.records, R.prev_vals, R.prev_ranges, R.moved, R.removed, R.added, R.ins_first, R.ins_vals,
                R.ranges, R.vals, R.capacity, 0u, small_cap, small_cap == R.cap_entries, R.d_err};
    tile_merge_kernel<<<(unsigned)R.n_tiles, kMergeThreads, gs_temporal_merge_smem(small_cap), s>>>(G);
    e = cudaGetLastError();
    if (e != cudaSuccess || small_cap == R.cap_entries) return e;
    G.min_entries = (uint32_t)small_cap;
    G.cap_entries = R.cap_entries;
    G.last_class = true;
    tile_merge_kernel<<<(unsigned)R.n_tiles, kMergeThreads, big_smem, s>>>(G);
    return cudaGetLastError();
}
