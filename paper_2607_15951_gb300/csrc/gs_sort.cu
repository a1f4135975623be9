// gs_sort.cu — stable LSD radix sort of (key, u32 value) pairs, written
// from the Onesweep design (Adinets and Merrill, 2022): one up-front pass
// builds the digit histograms of every pass at once, then each 8-bit digit
// pass is a single launch in which every block
//   1. takes the next partition of kSortTile pairs (atomic counter, so blocks
//      only wait on blocks that are already running),
//   2. ranks its pairs by digit, stably, with warp match + per-warp counters,
//   3. publishes its per-digit counts and resolves its global per-digit
//      offsets by decoupled look-back over earlier partitions' status words
//      (one thread per digit; every wait is bounded in time),
//   4. reorders the pairs in shared memory by digit and writes them out in
//      digit-contiguous runs, so global stores are coalesced.
// Keys are 64-bit (tile << 32 | depth bits, the staged binning entry points),
// or 16/32-bit tile ids (a frame's tile sort, whose keys arrive in depth
// order: the sort moves 6 or 8 bytes per pair and pass instead of 12).
#include "gs_internal.cuh"

#ifndef GS_SORT_MIN_BLOCKS
#define GS_SORT_MIN_BLOCKS 2
#endif
#ifndef GS_SORT_HIST_AGG
#define GS_SORT_HIST_AGG 0
#endif


namespace {

using namespace gs;

constexpr int kThreads = kSortThreads;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = GS_SORT_ITEMS;     // items per thread of the default variant
constexpr int kLargeItems = 12;           // ... of the variant for long lists
constexpr int64_t kLargeSortPairs = int64_t(1) << 23;  // capacities from here on use it
constexpr int kLookAhead = GS_SORT_LOOKAHEAD;  // status words read per look-back step
constexpr int kRadix = 256;
constexpr int kMaxPasses = 8;

inline int64_t num_parts(int64_t n, int items = kItems) {
    const int64_t tile = (int64_t)kThreads * items;
    return (n + tile - 1) / tile;
}

inline size_t header_bytes(int passes) {
    size_t b = (size_t)passes * kRadix * 4 * 2 + (size_t)passes * 4 + 4;
    return (b + 255) & ~(size_t)255;
}

using SortScratch = GsSortScratch;

// Histograms of every digit pass; the last block to finish turns them into
// exclusive bucket offsets.
__global__ void __launch_bounds__(kThreads)
histogram_kernel(const uint64_t *__restrict__ keys, int64_t n, int passes, SortScratch sc) {
    __shared__ uint32_t s_hist[kMaxPasses * kRadix];
    __shared__ uint32_t s_tmp[kWarps];
    __shared__ bool s_last;
    for (int i = threadIdx.x; i < passes * kRadix; i += kThreads) s_hist[i] = 0;
    __syncthreads();
    // Neighbouring keys often share digits (the tiles of one Gaussian share
    // its depth bits), so lanes with equal digits add once through a leader.
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    const int64_t n_up = (n + 31) & ~(int64_t)31;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n_up; i += stride) {
        const bool ok = i < n;
        const uint64_t k = ok ? keys[i] : 0ull;
        for (int p = 0; p < passes; ++p) {
            const uint32_t d = ok ? (uint32_t)((k >> (8 * p)) & 255) : 256u;
#if GS_SORT_HIST_AGG
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (d < 256u && (peers & lanemask_lt()) == 0u)
                atomicAdd(&s_hist[p * kRadix + d], (uint32_t)__popc(peers));
#else
            if (d < 256u) atomicAdd(&s_hist[p * kRadix + d], 1u);
#endif
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kThreads)
        if (s_hist[i]) atomicAdd(&sc.hist[i], s_hist[i]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(sc.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int p = 0; p < passes; ++p) {
        const uint32_t c = __ldcg(&sc.hist[p * kRadix + threadIdx.x]);
        const uint32_t e = block_exclusive_scan_256(c, s_tmp);
        sc.bucket[p * kRadix + threadIdx.x] = e;
    }
}

template <typename KT, int ITEMS, int MIN_BLOCKS>
__global__ void __launch_bounds__(kThreads, MIN_BLOCKS)
onesweep_kernel(const KT *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
                KT *__restrict__ keys_out, uint32_t *__restrict__ vals_out, int64_t n_host,
                const unsigned long long *d_n, int pass, int64_t parts, SortScratch sc,
                uint32_t *d_err, unsigned long long timeout_ns, bool ballot_rank) {
    constexpr int kItems = ITEMS, kTile = kThreads * ITEMS;
    extern __shared__ __align__(16) unsigned char smem[];
    KT *s_keys = reinterpret_cast<KT *>(smem);                                  // kTile
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_keys + kTile);            // kTile
    uint32_t *s_whist = s_vals + kTile;                                         // kWarps x 256
    uint32_t *s_doff = s_whist + kWarps * kRadix;                               // 256
    uint32_t *s_gbase = s_doff + kRadix;                                        // 256
    uint32_t *s_tmp = s_gbase + kRadix;                                         // kWarps
    uint32_t *s_part = s_tmp + kWarps;                                          // 1

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int shift = 8 * (pass + sc.digit0);
    if (tid == 0) *s_part = atomicAdd(sc.counter + pass, 1u);
    __syncthreads();
    const int64_t p = *s_part;
    const int64_t base = p * kTile;
    // With a device-side count the grid covers the capacity; partitions past
    // the count have nothing to do (no later partition waits on them).
    const int64_t n = d_n ? (int64_t)*d_n : n_host;
    if (base >= n) return;
    for (int i = tid; i < kWarps * kRadix; i += kThreads) s_whist[i] = 0;
    __syncthreads();

    // Warp-striped load: warp w holds pairs [w*32*kItems, (w+1)*32*kItems) of
    // the partition, item j of lane l at offset j*32 + l (coalesced).
    KT key[kItems];
    uint32_t val[kItems];
    uint32_t rank[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t idx = base + (int64_t)warp * 32 * kItems + j * 32 + lane;
        key[j] = idx < n ? keys_in[idx] : (KT)~(KT)0;
        val[j] = idx < n ? vals_in[idx] : 0u;
    }
    // Stable rank within the warp, in (item, lane) order. Out-of-range items
    // get digit 256, which matches nothing real and is never counted.
    uint32_t *my_hist = s_whist + warp * kRadix;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t idx = base + (int64_t)warp * 32 * kItems + j * 32 + lane;
        const uint32_t d = idx < n ? (uint32_t)((key[j] >> shift) & 255) : 256u;
        // Lanes with equal digits: warp match (fast when a warp holds few
        // distinct digits), or 9 ballots, one per bit of 0..256 (constant
        // cost, faster when digits are diverse).
        uint32_t peers;
        if (ballot_rank) {
            peers = 0xffffffffu;
#pragma unroll
            for (int b = 0; b < 9; ++b) {
                const bool bit = (d >> b) & 1u;
                const uint32_t m = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? m : ~m;
            }
        } else {
            peers = __match_any_sync(0xffffffffu, d);
        }
        const uint32_t lt = peers & lanemask_lt();
        const uint32_t before = d < 256u ? my_hist[d] : 0u;
        __syncwarp();
        rank[j] = before + __popc(lt);
        if (d < 256u && lt == 0u) my_hist[d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();

    // Thread tid owns digit tid: prefix over warps, block total for the digit.
    const uint32_t digit = tid;
    uint32_t total = 0;
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = s_whist[w * kRadix + digit];
        s_whist[w * kRadix + digit] = total;
        total += c;
    }
    unsigned long long *st = sc.status + ((int64_t)pass * parts + p) * kRadix + digit;
    if (p == 0) {
        st_relaxed_u64(st, kFlagIncl | total);
    } else {
        st_relaxed_u64(st, kFlagAgg | total);
    }
    const uint32_t doff = block_exclusive_scan_256(total, s_tmp);
    s_doff[digit] = doff;

    // Decoupled look-back for this digit over partitions p-1, p-2, ...,
    // reading kLookAhead status words per step so a chain of aggregates costs
    // one memory latency per kLookAhead partitions.
    unsigned long long excl = 0;
    if (p > 0) {
        unsigned long long t0 = 0;  // read at the first unpublished status word
        int64_t q = p - 1;
        uint32_t polls = 0;
        bool found = false;
        while (q >= 0 && !found) {
            unsigned long long sw[kLookAhead];
#pragma unroll
            for (int k = 0; k < kLookAhead; ++k)
                sw[k] = (q - k >= 0) ? ld_relaxed_u64(st - (p - (q - k)) * kRadix) : 0ull;
            int consumed = 0;
#pragma unroll
            for (int k = 0; k < kLookAhead; ++k) {
                if (q - k < 0 || consumed != k) break;
                const unsigned long long f = sw[k] >> 62;
                if (f == 0) break;
                excl += sw[k] & kValueMask;
                ++consumed;
                if (f == 2) {
                    found = true;
                    break;
                }
            }
            q -= consumed;
            if (!found && consumed == 0) {
                if (polls == 0) t0 = global_ns();
                if ((++polls & 63u) == 0u &&
                    ((global_ns() - t0 > timeout_ns) || (ld_relaxed_u32(d_err) & kErrTimeout))) {
                    atomicOr(d_err, kErrTimeout);
                    __threadfence();
                    break;
                }
            }
        }
        st_relaxed_u64(st, kFlagIncl | ((excl + total) & kValueMask));
    }
    s_gbase[digit] = sc.bucket[pass * kRadix + digit] + (uint32_t)excl;
    __syncthreads();

    // Reorder by digit in shared memory.
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t idx = base + (int64_t)warp * 32 * kItems + j * 32 + lane;
        if (idx < n) {
            const uint32_t d = (uint32_t)((key[j] >> shift) & 255);
            const uint32_t pos = s_doff[d] + my_hist[d] + rank[j];
            s_keys[pos] = key[j];
            s_vals[pos] = val[j];
        }
    }
    __syncthreads();
    const int valid = (int)((n - base) < kTile ? (n - base) : kTile);
    for (int i = tid; i < valid; i += kThreads) {
        const KT k = s_keys[i];
        const uint32_t d = (uint32_t)((k >> shift) & 255);
        const uint64_t gp = (uint64_t)s_gbase[d] + (uint32_t)(i - s_doff[d]);
        // Only reachable after a timed-out look-back left offsets meaningless.
        if (gp >= (uint64_t)n) {
            atomicOr(d_err, kErrRange);
            continue;
        }
        keys_out[gp] = k;
        vals_out[gp] = s_vals[i];
    }
}

template <typename KT, int ITEMS>
constexpr size_t onesweep_smem() {
    return (size_t)kThreads * ITEMS * (sizeof(KT) + 4) + (size_t)kWarps * kRadix * 4 + 2 * kRadix * 4 +
           kWarps * 4 + 16;
}

template <typename KT, int ITEMS, int MIN_BLOCKS>
cudaError_t prepare_shape() {
    return cudaFuncSetAttribute(onesweep_kernel<KT, ITEMS, MIN_BLOCKS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)onesweep_smem<KT, ITEMS>());
}

// The digit passes of sc over n_capacity pairs (count *d_n when given),
// ping-ponging between the two buffers.
template <typename KT>
cudaError_t launch_passes(KT *keys, uint32_t *values, KT *alt_keys, uint32_t *alt_values, int64_t n_capacity,
                          const unsigned long long *d_n, const GsSortScratch &sc, uint32_t *d_err,
                          bool *result_in_alt, cudaStream_t s, unsigned long long timeout_ns, int max_passes) {
    *result_in_alt = false;
    // Three partition shapes: 8 items per thread for short lists (shorter
    // per-partition latency), GS_SORT_ITEMS (16) by default, 12 items with
    // three blocks per SM for long lists (more partitions in flight).
    if (sc.items != 8 && sc.items != kItems && sc.items != kLargeItems) return cudaErrorInvalidValue;
    const int shape = sc.items == kLargeItems && kLargeItems != kItems ? 2 : (sc.items == 8 && kItems != 8 ? 0 : 1);
    const size_t smem = shape == 0 ? onesweep_smem<KT, 8>() : shape == 2 ? onesweep_smem<KT, kLargeItems>()
                                                                         : onesweep_smem<KT, kItems>();
    cudaError_t e = shape == 0   ? prepare_shape<KT, 8, GS_SORT_MIN_BLOCKS>()
                    : shape == 2 ? prepare_shape<KT, kLargeItems, 3>()
                                 : prepare_shape<KT, kItems, GS_SORT_MIN_BLOCKS>();
    if (e != cudaSuccess) return e;
    const KT *kin = keys;
    const uint32_t *vin = values;
    KT *kout = alt_keys;
    uint32_t *vout = alt_values;
    const int passes = sc.passes < max_passes ? sc.passes : max_passes;
    for (int pass = 0; pass < passes; ++pass) {
        // Lower digits of depth bits and tile ids are diverse within a warp;
        // the top digit (exponent byte, high tile bits) takes few values.
        const bool ballot = pass + 1 < sc.passes;
        if (shape == 0)
            onesweep_kernel<KT, 8, GS_SORT_MIN_BLOCKS><<<(unsigned)sc.parts, kThreads, smem, s>>>(
                kin, vin, kout, vout, n_capacity, d_n, pass, sc.parts, sc, d_err, timeout_ns, ballot);
        else if (shape == 2)
            onesweep_kernel<KT, kLargeItems, 3><<<(unsigned)sc.parts, kThreads, smem, s>>>(
                kin, vin, kout, vout, n_capacity, d_n, pass, sc.parts, sc, d_err, timeout_ns, ballot);
        else
            onesweep_kernel<KT, kItems, GS_SORT_MIN_BLOCKS><<<(unsigned)sc.parts, kThreads, smem, s>>>(
                kin, vin, kout, vout, n_capacity, d_n, pass, sc.parts, sc, d_err, timeout_ns, ballot);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        kin = kout;
        vin = vout;
        kout = (kout == alt_keys) ? keys : alt_keys;
        vout = (vout == alt_values) ? values : alt_values;
    }
    *result_in_alt = (passes & 1) != 0;
    return cudaSuccess;
}

}  // namespace

int gs_sort_passes(int key_bits) { return (key_bits + 7) / 8; }

size_t gs_sort_scratch_bytes(int64_t n, int key_bits) {
    return gs_sort_scratch_bytes_digits(n, gs_sort_passes(key_bits));
}

GsSortScratch gs_sort_carve(void *base, int64_t n_capacity, int key_bits) {
    return gs_sort_carve_digits(base, n_capacity, 0, gs_sort_passes(key_bits));
}

int gs_sort_items_for(int64_t n) { return n >= kLargeSortPairs ? kLargeItems : kItems; }

size_t gs_sort_scratch_bytes_digits(int64_t n, int passes, int items) {
    if (items == 0) items = gs_sort_items_for(n);
    const int64_t parts = num_parts(n, items) > 0 ? num_parts(n, items) : 1;
    return header_bytes(passes) + (size_t)passes * parts * kRadix * sizeof(unsigned long long);
}

GsSortScratch gs_sort_carve_digits(void *base, int64_t n_capacity, int digit0, int passes, int items) {
    if (items == 0) items = gs_sort_items_for(n_capacity);
    char *p = static_cast<char *>(base);
    GsSortScratch s;
    s.hist = reinterpret_cast<uint32_t *>(p);
    s.bucket = s.hist + passes * kRadix;
    s.counter = s.bucket + passes * kRadix;
    s.ticket = s.counter + passes;
    s.status = reinterpret_cast<unsigned long long *>(p + header_bytes(passes));
    s.passes = passes;
    s.parts = num_parts(n_capacity, items) > 0 ? num_parts(n_capacity, items) : 1;
    s.digit0 = digit0;
    s.items = items;
    return s;
}

cudaError_t gs_launch_sort_passes(uint64_t *keys, uint32_t *values, uint64_t *alt_keys,
                                  uint32_t *alt_values, int64_t n_capacity,
                                  const unsigned long long *d_n, const GsSortScratch &sc,
                                  uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                  unsigned long long timeout_ns, int max_passes) {
    return launch_passes<uint64_t>(keys, values, alt_keys, alt_values, n_capacity, d_n, sc, d_err, result_in_alt, s,
                                   timeout_ns, max_passes);
}

cudaError_t gs_launch_sort_passes(uint32_t *keys, uint32_t *values, uint32_t *alt_keys,
                                  uint32_t *alt_values, int64_t n_capacity,
                                  const unsigned long long *d_n, const GsSortScratch &sc,
                                  uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                  unsigned long long timeout_ns, int max_passes) {
    return launch_passes<uint32_t>(keys, values, alt_keys, alt_values, n_capacity, d_n, sc, d_err, result_in_alt, s,
                                   timeout_ns, max_passes);
}

cudaError_t gs_launch_sort_passes(uint16_t *keys, uint32_t *values, uint16_t *alt_keys,
                                  uint32_t *alt_values, int64_t n_capacity,
                                  const unsigned long long *d_n, const GsSortScratch &sc,
                                  uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                  unsigned long long timeout_ns, int max_passes) {
    return launch_passes<uint16_t>(keys, values, alt_keys, alt_values, n_capacity, d_n, sc, d_err, result_in_alt, s,
                                   timeout_ns, max_passes);
}

cudaError_t gs_launch_sort(uint64_t *keys, uint32_t *values, uint64_t *alt_keys,
                           uint32_t *alt_values, int64_t n, int key_bits, void *scratch,
                           uint32_t *d_err, bool *result_in_alt, cudaStream_t s) {
    *result_in_alt = false;
    if (n <= 1 || key_bits <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(scratch, 0, gs_sort_scratch_bytes(n, key_bits), s);
    if (e != cudaSuccess) return e;
    const GsSortScratch sc = gs_sort_carve(scratch, n, key_bits);
    const unsigned hist_blocks = (unsigned)(sc.parts < 608 ? sc.parts : 608);
    histogram_kernel<<<hist_blocks, kThreads, 0, s>>>(keys, n, sc.passes, sc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return gs_launch_sort_passes(keys, values, alt_keys, alt_values, n, nullptr, sc, d_err,
                                 result_in_alt, s);
}
