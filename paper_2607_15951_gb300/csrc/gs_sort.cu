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
#include "gs_onesweep.cuh"

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
    __shared__ uint32_t s_part;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int shift = 8 * (pass + sc.digit0);
    if (tid == 0) s_part = atomicAdd(sc.counter + pass, 1u);
    __syncthreads();
    const int64_t p = s_part;
    const int64_t base = p * kTile;
    // With a device-side count the grid covers the capacity; partitions past
    // the count have nothing to do (no later partition waits on them).
    const int64_t n = d_n ? (int64_t)*d_n : n_host;
    if (base >= n) return;

    // Warp-striped load: warp w holds pairs [w*32*kItems, (w+1)*32*kItems) of
    // the partition, item j of lane l at offset j*32 + l (coalesced).
    KT key[kItems];
    uint32_t val[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t idx = base + (int64_t)warp * 32 * kItems + j * 32 + lane;
        key[j] = idx < n ? keys_in[idx] : (KT)~(KT)0;
        val[j] = idx < n ? vals_in[idx] : 0u;
    }
    onesweep_partition<KT, kItems>(key, val, base, n, p, shift, sc.status + (int64_t)pass * parts * kRadix,
                                   sc.bucket + pass * kRadix, keys_out, vals_out, d_err, timeout_ns, ballot_rank,
                                   smem);
}

template <typename KT, int ITEMS>
constexpr size_t onesweep_smem() {
    return onesweep_partition_smem<KT, ITEMS>();
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
                          bool *result_in_alt, cudaStream_t s, unsigned long long timeout_ns, int max_passes,
                          int first_pass) {
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
    for (int pass = first_pass; pass < passes; ++pass) {
        // Lower digits of depth bits and tile ids are diverse within a warp;
        // the top digit (exponent byte, high tile bits) takes few values.
        const bool ballot = pass + 1 < sc.passes || sc.diverse_last;
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
    *result_in_alt = passes > first_pass && ((passes - first_pass) & 1) != 0;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Reduce-then-scan digit passes, for long lists. A onesweep pass over many
// partitions is held back by its look-back chains: every block walks back to
// the nearest inclusive prefix while hundreds of partitions are in flight
// (on a 174M-pair pass each 3072-pair partition lived ~80 us against ~10 us
// of work). Here a pass is three launches and no block waits on another:
//   1. each partition's 256 digit counts (reads the keys only);
//   2. per digit, an exclusive scan over the partitions plus the digit's
//      bucket offset: every partition's global offset per digit;
//   3. the partition ranking and scatter of the onesweep pass, with those
//      offsets in place of the look-back.
// ---------------------------------------------------------------------------
constexpr int kRtsItems = kLargeItems;
constexpr int kRtsTile = kThreads * kRtsItems;
constexpr int kRtsScanThreads = 1024;

inline int64_t rts_parts(int64_t n) { return (n + kRtsTile - 1) / kRtsTile > 0 ? (n + kRtsTile - 1) / kRtsTile : 1; }

template <typename KT>
__global__ void __launch_bounds__(kThreads) rts_hist_kernel(const KT *__restrict__ keys, int64_t n_cap,
                                                            const unsigned long long *d_n, int shift,
                                                            int64_t stride, uint32_t *__restrict__ counts) {
    __shared__ uint32_t h[kRadix];
    const int tid = threadIdx.x;
    const int64_t n = d_n ? (int64_t)*d_n : n_cap;
    const int64_t base = (int64_t)blockIdx.x * kRtsTile;
    if (base >= n) return;  // the scan reads only the partitions of the n pairs
    h[tid] = 0;
    __syncthreads();
    const int cnt = (int)(n - base < kRtsTile ? n - base : kRtsTile);
    for (int i = tid; i < cnt; i += kThreads) atomicAdd(&h[(uint32_t)(keys[base + i] >> shift) & 255u], 1u);
    __syncthreads();
    counts[(int64_t)tid * stride + blockIdx.x] = h[tid];
}

// Block d: exclusive scan of digit d's counts over the partitions, plus the
// digit's bucket offset.
__global__ void __launch_bounds__(kRtsScanThreads) rts_scan_kernel(const uint32_t *__restrict__ counts,
                                                                   const uint32_t *__restrict__ bucket,
                                                                   int64_t n_cap, const unsigned long long *d_n,
                                                                   int64_t stride, uint32_t *__restrict__ offsets) {
    __shared__ uint32_t s_w[kRtsScanThreads / 32];
    __shared__ uint32_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = d_n ? (int64_t)*d_n : n_cap;
    const int64_t parts = (n + kRtsTile - 1) / kRtsTile;
    const uint32_t *c = counts + (int64_t)blockIdx.x * stride;
    uint32_t *o = offsets + (int64_t)blockIdx.x * stride;
    if (tid == 0) s_carry = bucket[blockIdx.x];
    __syncthreads();
    constexpr int kPer = 4;
    for (int64_t c0 = 0; c0 < parts; c0 += (int64_t)kRtsScanThreads * kPer) {
        uint32_t v[kPer], sum = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t q = c0 + (int64_t)tid * kPer + k;
            v[k] = q < parts ? c[q] : 0u;
            sum += v[k];
        }
        uint32_t incl = sum;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = s_w[lane];
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += t;
            }
            s_w[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const uint32_t carry = s_carry;
        uint32_t run = carry + (warp ? s_w[warp - 1] : 0u) + incl - sum;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t q = c0 + (int64_t)tid * kPer + k;
            if (q < parts) o[q] = run;
            run += v[k];
        }
        __syncthreads();
        if (tid == kRtsScanThreads - 1) s_carry = carry + s_w[31];
        __syncthreads();
    }
}

template <typename KT>
__global__ void __launch_bounds__(kThreads, 3)
rts_scatter_kernel(const KT *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, KT *__restrict__ keys_out,
                   uint32_t *__restrict__ vals_out, int64_t n_cap, const unsigned long long *d_n, int shift,
                   int64_t stride, const uint32_t *__restrict__ offsets, uint32_t *d_err, bool ballot_rank) {
    constexpr int kItems = kRtsItems;
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = d_n ? (int64_t)*d_n : n_cap;
    const int64_t p = blockIdx.x;
    const int64_t base = p * kRtsTile;
    if (base >= n) return;
    KT key[kItems];
    uint32_t val[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const int64_t idx = base + (int64_t)warp * 32 * kItems + j * 32 + lane;
        key[j] = idx < n ? keys_in[idx] : (KT)~(KT)0;
        val[j] = idx < n ? vals_in[idx] : 0u;
    }
    onesweep_partition<KT, kItems>(key, val, base, n, p, shift, nullptr, nullptr, keys_out, vals_out, d_err, 0ull,
                                   ballot_rank, smem, offsets + p, stride);
}

template <typename KT>
cudaError_t launch_passes_rts(KT *keys, uint32_t *values, KT *alt_keys, uint32_t *alt_values, int64_t n_capacity,
                              const unsigned long long *d_n, const GsSortScratch &sc, void *rts_scratch,
                              uint32_t *d_err, bool *result_in_alt, cudaStream_t s, int first_pass) {
    *result_in_alt = false;
    const int64_t parts = rts_parts(n_capacity);
    uint32_t *counts = static_cast<uint32_t *>(rts_scratch);
    uint32_t *offsets = counts + (int64_t)kRadix * parts;
    const size_t smem = onesweep_smem<KT, kRtsItems>();
    cudaError_t e = cudaFuncSetAttribute(rts_scatter_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const KT *kin = keys;
    const uint32_t *vin = values;
    KT *kout = alt_keys;
    uint32_t *vout = alt_values;
    for (int pass = first_pass; pass < sc.passes; ++pass) {
        const int shift = 8 * (pass + sc.digit0);
        const bool ballot = pass + 1 < sc.passes || sc.diverse_last;
        rts_hist_kernel<KT><<<(unsigned)parts, kThreads, 0, s>>>(kin, n_capacity, d_n, shift, parts, counts);
        rts_scan_kernel<<<kRadix, kRtsScanThreads, 0, s>>>(counts, sc.bucket + pass * kRadix, n_capacity, d_n, parts,
                                                           offsets);
        rts_scatter_kernel<KT><<<(unsigned)parts, kThreads, smem, s>>>(kin, vin, kout, vout, n_capacity, d_n, shift,
                                                                       parts, offsets, d_err, ballot);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        kin = kout;
        vin = vout;
        kout = (kout == alt_keys) ? keys : alt_keys;
        vout = (vout == alt_values) ? values : alt_values;
    }
    *result_in_alt = sc.passes > first_pass && ((sc.passes - first_pass) & 1) != 0;
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
    s.diverse_last = false;
    return s;
}

cudaError_t gs_launch_sort_passes(uint64_t *keys, uint32_t *values, uint64_t *alt_keys,
                                  uint32_t *alt_values, int64_t n_capacity,
                                  const unsigned long long *d_n, const GsSortScratch &sc,
                                  uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                  unsigned long long timeout_ns, int max_passes, int first_pass) {
    return launch_passes<uint64_t>(keys, values, alt_keys, alt_values, n_capacity, d_n, sc, d_err, result_in_alt, s,
                                   timeout_ns, max_passes, first_pass);
}

cudaError_t gs_launch_sort_passes(uint32_t *keys, uint32_t *values, uint32_t *alt_keys,
                                  uint32_t *alt_values, int64_t n_capacity,
                                  const unsigned long long *d_n, const GsSortScratch &sc,
                                  uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                  unsigned long long timeout_ns, int max_passes, int first_pass) {
    return launch_passes<uint32_t>(keys, values, alt_keys, alt_values, n_capacity, d_n, sc, d_err, result_in_alt, s,
                                   timeout_ns, max_passes, first_pass);
}

cudaError_t gs_launch_sort_passes(uint16_t *keys, uint32_t *values, uint16_t *alt_keys,
                                  uint32_t *alt_values, int64_t n_capacity,
                                  const unsigned long long *d_n, const GsSortScratch &sc,
                                  uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                  unsigned long long timeout_ns, int max_passes, int first_pass) {
    return launch_passes<uint16_t>(keys, values, alt_keys, alt_values, n_capacity, d_n, sc, d_err, result_in_alt, s,
                                   timeout_ns, max_passes, first_pass);
}

cudaError_t gs_launch_sort(uint64_t *keys, uint32_t *values, uint64_t *alt_keys,
                           uint32_t *alt_values, int64_t n, int key_bits, void *scratch,
                           uint32_t *d_err, bool *result_in_alt, cudaStream_t s) {
    *result_in_alt = false;
    if (n <= 1 || key_bits <= 0) return cudaSuccess;
    if (n >= kRtsMinPairs) {
        // Long lists: reduce-then-scan passes. Their per-partition counts and
        // offsets (2 KB per 3072 pairs) fit where the onesweep look-back
        // words (2 KB per 3072 pairs and pass) would go.
        const int passes = gs_sort_passes(key_bits);
        const size_t head = header_bytes(passes);  // histograms, buckets, ticket
        cudaError_t e = cudaMemsetAsync(scratch, 0, head, s);
        if (e != cudaSuccess) return e;
        const GsSortScratch sc = gs_sort_carve_digits(scratch, 1, 0, passes);
        const unsigned hist_blocks = (unsigned)(rts_parts(n) < 608 ? rts_parts(n) : 608);
        histogram_kernel<<<hist_blocks, kThreads, 0, s>>>(keys, n, sc.passes, sc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_passes_rts<uint64_t>(keys, values, alt_keys, alt_values, n, nullptr, sc,
                                           static_cast<char *>(scratch) + head, d_err, result_in_alt, s, 0);
    }
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

size_t gs_sort_rts_scratch_bytes(int64_t n_capacity) { return (size_t)2 * kRadix * rts_parts(n_capacity) * 4; }

cudaError_t gs_launch_sort_passes_rts(uint16_t *keys, uint32_t *values, uint16_t *alt_keys, uint32_t *alt_values,
                                      int64_t n_capacity, const unsigned long long *d_n, const GsSortScratch &sc,
                                      void *rts_scratch, uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                      int first_pass) {
    return launch_passes_rts<uint16_t>(keys, values, alt_keys, alt_values, n_capacity, d_n, sc, rts_scratch, d_err,
                                       result_in_alt, s, first_pass);
}

cudaError_t gs_launch_sort_passes_rts(uint32_t *keys, uint32_t *values, uint32_t *alt_keys, uint32_t *alt_values,
                                      int64_t n_capacity, const unsigned long long *d_n, const GsSortScratch &sc,
                                      void *rts_scratch, uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                      int first_pass) {
    return launch_passes_rts<uint32_t>(keys, values, alt_keys, alt_values, n_capacity, d_n, sc, rts_scratch, d_err,
                                       result_in_alt, s, first_pass);
}

cudaError_t gs_launch_sort_passes_rts(uint64_t *keys, uint32_t *values, uint64_t *alt_keys, uint32_t *alt_values,
                                      int64_t n_capacity, const unsigned long long *d_n, const GsSortScratch &sc,
                                      void *rts_scratch, uint32_t *d_err, bool *result_in_alt, cudaStream_t s,
                                      int first_pass) {
    return launch_passes_rts<uint64_t>(keys, values, alt_keys, alt_values, n_capacity, d_n, sc, rts_scratch, d_err,
                                       result_in_alt, s, first_pass);
}
