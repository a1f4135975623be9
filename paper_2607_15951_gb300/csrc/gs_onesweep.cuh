// gs_onesweep.cuh — one partition of an Onesweep digit pass (Adinets and
// Merrill, 2022): stable ranking of the partition's pairs by the digit,
// publication of its digit counts, decoupled look-back for the counts of all
// earlier partitions (bounded waits), reorder in shared memory and
// digit-contiguous (coalesced) stores. Shared by the radix sort passes and by
// kernels that produce their partition's keys themselves.
#pragma once

#include "gs_internal.cuh"

namespace gs {

constexpr int kOsThreads = kSortThreads;  // 256: one thread per digit
constexpr int kOsWarps = kOsThreads / 32;
constexpr int kOsRadix = 256;
constexpr int kOsLookAhead = GS_SORT_LOOKAHEAD;  // status words read per look-back step

// Shared memory the partition needs: the reordered pairs, per-warp digit
// counters, digit offsets and bases, scan scratch.
template <typename KT, int ITEMS>
__host__ __device__ constexpr size_t onesweep_partition_smem() {
    return (size_t)kOsThreads * ITEMS * (sizeof(KT) + 4) + (size_t)kOsWarps * kOsRadix * 4 + 2 * kOsRadix * 4 +
           kOsWarps * 4 + 16;
}

// key/val: the partition's pairs, warp-striped (item j of lane l of warp w
// is pair base + w*32*ITEMS + j*32 + l; pairs at or past n are ignored).
// p: the partition's index in the order partitions were taken (a partition
// only waits on earlier ones). status: this pass's look-back words
// (parts x 256, zeroed); bucket: the pass's 256 exclusive digit offsets.
// All 256 threads of the block call it.
template <typename KT, int ITEMS>
__device__ __forceinline__ void onesweep_partition(const KT (&key)[ITEMS], const uint32_t (&val)[ITEMS], int64_t base,
                                                   int64_t n, int64_t p, int shift, unsigned long long *status,
                                                   const uint32_t *bucket, KT *__restrict__ keys_out,
                                                   uint32_t *__restrict__ vals_out, uint32_t *d_err,
                                                   unsigned long long timeout_ns, bool ballot_rank,
                                                   unsigned char *smem) {
    constexpr int kItems = ITEMS, kTile = kOsThreads * ITEMS, kThreads = kOsThreads, kWarps = kOsWarps,
                  kRadix = kOsRadix;
    KT *s_keys = reinterpret_cast<KT *>(smem);                                  // kTile
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_keys + kTile);            // kTile
    uint32_t *s_whist = s_vals + kTile;                                         // kWarps x 256
    uint32_t *s_doff = s_whist + kWarps * kRadix;                               // 256
    uint32_t *s_gbase = s_doff + kRadix;                                        // 256
    uint32_t *s_tmp = s_gbase + kRadix;                                         // kWarps
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kWarps * kRadix; i += kThreads) s_whist[i] = 0;
    __syncthreads();
    uint32_t rank[kItems];
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
    unsigned long long *st = status + p * kRadix + digit;
    if (p == 0) {
        st_relaxed_u64(st, kFlagIncl | total);
    } else {
        st_relaxed_u64(st, kFlagAgg | total);
    }
    const uint32_t doff = block_exclusive_scan_256(total, s_tmp);
    s_doff[digit] = doff;

    // Decoupled look-back for this digit over partitions p-1, p-2, ...,
    // reading kOsLookAhead status words per step so a chain of aggregates costs
    // one memory latency per kOsLookAhead partitions.
    unsigned long long excl = 0;
    if (p > 0) {
        unsigned long long t0 = 0;  // read at the first unpublished status word
        int64_t q = p - 1;
        uint32_t polls = 0;
        bool found = false;
        while (q >= 0 && !found) {
            unsigned long long sw[kOsLookAhead];
#pragma unroll
            for (int k = 0; k < kOsLookAhead; ++k)
                sw[k] = (q - k >= 0) ? ld_relaxed_u64(st - (p - (q - k)) * kRadix) : 0ull;
            int consumed = 0;
#pragma unroll
            for (int k = 0; k < kOsLookAhead; ++k) {
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
    s_gbase[digit] = bucket[digit] + (uint32_t)excl;
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

}  // namespace gs
