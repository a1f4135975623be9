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
// counters (later the digits' start offsets within the partition), the
// digits' global destinations, scan scratch.
template <typename KT, int ITEMS>
__host__ __device__ constexpr size_t onesweep_partition_smem() {
    return (size_t)kOsThreads * ITEMS * (sizeof(KT) + 4) + (size_t)kOsWarps * kOsRadix * 4 + kOsRadix * 4 +
           kOsWarps * 4 + 16;
}

// The partition proper. FULL: all kTile pairs are in range (every partition
// but the last), so no item needs a range test.
template <typename KT, int ITEMS, bool FULL>
__device__ __forceinline__ void onesweep_partition_body(const KT (&key)[ITEMS], const uint32_t (&val)[ITEMS],
                                                        int valid, int64_t n, int64_t p, int shift,
                                                        unsigned long long *status, const uint32_t *bucket,
                                                        KT *__restrict__ keys_out, uint32_t *__restrict__ vals_out,
                                                        uint32_t *d_err, unsigned long long timeout_ns,
                                                        bool ballot_rank, unsigned char *smem,
                                                        const uint32_t *rts, int64_t rts_stride) {
    constexpr int kItems = ITEMS, kTile = kOsThreads * ITEMS, kThreads = kOsThreads, kWarps = kOsWarps,
                  kRadix = kOsRadix;
    KT *s_keys = reinterpret_cast<KT *>(smem);                                  // kTile
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_keys + kTile);            // kTile
    uint32_t *s_whist = s_vals + kTile;                                         // kWarps x 256
    uint32_t *s_gdst = s_whist + kWarps * kRadix;                               // 256
    uint32_t *s_tmp = s_gdst + kRadix;                                          // kWarps
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kWarps * kRadix; i += kThreads) s_whist[i] = 0;
    __syncthreads();
    uint32_t rank[kItems];
    // Stable rank within the warp, in (item, lane) order; out-of-range items
    // (only in the last partition) are never counted.
    uint32_t *my_hist = s_whist + warp * kRadix;
    const uint32_t lt_mask = lanemask_lt();
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const bool in = FULL || warp * 32 * kItems + j * 32 + lane < valid;
        const uint32_t d = (uint32_t)(key[j] >> shift) & 255u;
        // Lanes with equal digits: warp match (fast when a warp holds few
        // distinct digits), or one ballot per digit bit (constant cost,
        // faster when digits are diverse).
        uint32_t peers;
        if (ballot_rank) {
            peers = FULL ? 0xffffffffu : __ballot_sync(0xffffffffu, in);
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const bool bit = (d >> b) & 1u;
                const uint32_t m = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? m : ~m;
            }
        } else {
            peers = __match_any_sync(0xffffffffu, in ? d : 256u);
        }
        const uint32_t lt = peers & lt_mask;
        const uint32_t before = in ? my_hist[d] : 0u;
        __syncwarp();
        rank[j] = before + __popc(lt);
        if (in && lt == 0u) my_hist[d] = before + __popc(peers);
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
    if (!rts) {
        if (p == 0) {
            st_relaxed_u64(st, kFlagIncl | total);
        } else {
            st_relaxed_u64(st, kFlagAgg | total);
        }
    }
    const uint32_t doff = block_exclusive_scan_256(total, s_tmp);
    // Warp w's items of this digit start at doff + (earlier warps' count).
    for (int w = 0; w < kWarps; ++w) s_whist[w * kRadix + digit] += doff;
    if (rts) {
        // Reduce-then-scan: the partition's global offset per digit is known.
        s_gdst[digit] = rts[(int64_t)digit * rts_stride] - doff;
    }

    // Decoupled look-back for this digit over partitions p-1, p-2, ...,
    // reading kOsLookAhead status words per step so a chain of aggregates costs
    // one memory latency per kOsLookAhead partitions.
    unsigned long long excl = 0;
    if (!rts && p > 0) {
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
    // Global slot of the partition's i-th pair of this digit: gdst + i (pair
    // counts stay below 2^32, so the arithmetic is modulo 2^32).
    if (!rts) s_gdst[digit] = bucket[digit] + (uint32_t)excl - doff;
    __syncthreads();

    // Reorder by digit in shared memory.
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        if (FULL || warp * 32 * kItems + j * 32 + lane < valid) {
            const uint32_t d = (uint32_t)(key[j] >> shift) & 255u;
            const uint32_t pos = my_hist[d] + rank[j];
            s_keys[pos] = key[j];
            s_vals[pos] = val[j];
        }
    }
    __syncthreads();
    for (int i = tid; i < valid; i += kThreads) {
        const KT k = s_keys[i];
        const uint32_t gp = s_gdst[(uint32_t)(k >> shift) & 255u] + (uint32_t)i;
        // Only reachable after a timed-out look-back left offsets meaningless.
        if ((int64_t)gp >= n) {
            atomicOr(d_err, kErrRange);
            continue;
        }
        keys_out[gp] = k;
        vals_out[gp] = s_vals[i];
    }
}

// key/val: the partition's pairs, warp-striped (item j of lane l of warp w
// is pair base + w*32*ITEMS + j*32 + l; pairs at or past n are ignored).
// p: the partition's index in the order partitions were taken (a partition
// only waits on earlier ones). status: this pass's look-back words
// (parts x 256, zeroed); bucket: the pass's 256 exclusive digit offsets.
// rts (reduce-then-scan passes): instead of the look-back, the partition's
// global offset of digit d is rts[d * rts_stride] (status and bucket unused).
// All 256 threads of the block call it.
template <typename KT, int ITEMS>
__device__ __forceinline__ void onesweep_partition(const KT (&key)[ITEMS], const uint32_t (&val)[ITEMS], int64_t base,
                                                   int64_t n, int64_t p, int shift, unsigned long long *status,
                                                   const uint32_t *bucket, KT *__restrict__ keys_out,
                                                   uint32_t *__restrict__ vals_out, uint32_t *d_err,
                                                   unsigned long long timeout_ns, bool ballot_rank,
                                                   unsigned char *smem, const uint32_t *rts = nullptr,
                                                   int64_t rts_stride = 0) {
    constexpr int kTile = kOsThreads * ITEMS;
    const int valid = (int)(n - base < kTile ? n - base : kTile);
    if (valid == kTile)
        onesweep_partition_body<KT, ITEMS, true>(key, val, valid, n, p, shift, status, bucket, keys_out, vals_out,
                                                 d_err, timeout_ns, ballot_rank, smem, rts, rts_stride);
    else
        onesweep_partition_body<KT, ITEMS, false>(key, val, valid, n, p, shift, status, bucket, keys_out, vals_out,
                                                  d_err, timeout_ns, ballot_rank, smem, rts, rts_stride);
}

}  // namespace gs
