// gs_noalloc.cu — gs_sort_pairs_noalloc: the radix sort of gs_sort_pairs for
// callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not safe —
// inside a custom allocator or memory-pool callback, in a real-time loop whose
// memory footprint is fixed up front, or in a host that owns all device
// memory itself and forbids libraries from taking more. Such callers cannot
// create a gs_context (its workspace grows with cudaMalloc). This entry point
// takes its scratch from one array that is part of the library image
// instead: a file-scope __device__ array of kScratchBytes (about 4 MiB:
// 4,227,328 bytes with the default partition size), which every GPU that
// loads libgs.so holds until the process exits.
//
// Rules of use:
//  * n is limited to GS_NOALLOC_SORT_MAX_PAIRS pairs; larger requests fail
//    with GS_ERR_CAPACITY before anything is launched.
//  * All calls, from every thread and stream, share the one array. Calls that
//    overlap on the GPU (different streams, or host threads racing) corrupt
//    each other's results; serialise them.
//  * The first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current. The address is kept
//    for the life of the process, so the device must not be reset
//    (cudaDeviceReset) after that first call. Devices with an index of 64 or more are not served
//    (GS_ERR_CUDA).
//  * The call returns after the sort has finished on `stream` (it waits for
//    that stream once to read the device error word).
#include <mutex>

#include "gs_internal.cuh"

namespace {

constexpr int64_t kMaxPairs = GS_NOALLOC_SORT_MAX_PAIRS;
constexpr size_t kAltKeysBytes = (size_t)kMaxPairs * 8;
constexpr size_t kAltValsBytes = (size_t)kMaxPairs * 4;
// Sort scratch for 64-bit keys (8 passes): a header of histograms and
// counters below 32 KiB, and 8 x ceil(n / kSortTile) x 256 status words.
constexpr size_t kSortScratchBytes =
    32768 + (size_t)8 * ((kMaxPairs + kSortTile - 1) / kSortTile) * 256 * 8;
constexpr size_t kErrOffset = kAltKeysBytes + kAltValsBytes + kSortScratchBytes;
constexpr size_t kScratchBytes = kErrOffset + 256;

// The scratch itself. In host code this name is only a stand-in for the
// symbol, never a device address: the address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_dev_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(int device, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_dev_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_dev_ptr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_dev_ptr[device]);
    return cudaSuccess;
}

}  // namespace

extern "C" gs_status gs_sort_pairs_noalloc(uint64_t *keys, uint32_t *values, int64_t n,
                                           int32_t key_bits, void *stream) {
    if (n < 0 || key_bits < 1 || key_bits > 64) return GS_ERR_INVALID_ARG;
    if (n > kMaxPairs) return GS_ERR_CAPACITY;
    if (n > 0 && (!keys || !values)) return GS_ERR_INVALID_ARG;
    if (n <= 1) return GS_OK;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices)
        return GS_ERR_CUDA;
    unsigned char *base = nullptr;
    if (scratch_address(device, &base) != cudaSuccess) return GS_ERR_CUDA;
    if (gs_sort_scratch_bytes(n, key_bits) > kSortScratchBytes) return GS_ERR_CAPACITY;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t *alt_keys = reinterpret_cast<uint64_t *>(base);
    uint32_t *alt_vals = reinterpret_cast<uint32_t *>(base + kAltKeysBytes);
    void *sort_scratch = base + kAltKeysBytes + kAltValsBytes;
    uint32_t *d_err = reinterpret_cast<uint32_t *>(base + kErrOffset);

    // The array keeps the previous call's contents: clear the error word here;
    // gs_launch_sort clears the histogram and look-back state it uses.
    if (cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s) != cudaSuccess) return GS_ERR_CUDA;
    bool in_alt = false;
    if (gs_launch_sort(keys, values, alt_keys, alt_vals, n, key_bits, sort_scratch, d_err, &in_alt, s) !=
        cudaSuccess)
        return GS_ERR_CUDA;
    if (in_alt) {
        if (cudaMemcpyAsync(keys, alt_keys, (size_t)n * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(values, alt_vals, (size_t)n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return GS_ERR_CUDA;
    }
    // The error word is read on the caller's stream, so the wait covers that
    // stream only.
    uint32_t err = 0;
    if (cudaMemcpyAsync(&err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GS_ERR_CUDA;
    if (err & gs::kErrTimeout) return GS_ERR_TIMEOUT;
    return err ? GS_ERR_INVALID_ARG : GS_OK;
}
