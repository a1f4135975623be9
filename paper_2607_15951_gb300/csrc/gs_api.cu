// gs_api.cu — the C ABI (include/gs.h): argument validation, the context
// and its grow-only workspace, and the launch sequences of each entry point.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gs_internal.cuh"

namespace {

// Grow-only device buffer.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct gs_context {
    int device = 0;
    std::string last_error;
    uint32_t *d_err = nullptr;               // device error word
    unsigned long long *d_counts = nullptr;  // [K, n_visible, K if it fitted, visible, rects changed, pad...]
    unsigned long long *h_counts = nullptr;  // pinned mirror of d_counts
    uint32_t *h_err = nullptr;               // pinned mirror of d_err
    DevBuf records, tiles, offsets, scan_scratch, keys, values, alt_keys, alt_values, sort_scratch,
        ranges;
    gs_render_stats stats{};
    // State of the last gs_render, for gs_render_backward: the frame's
    // number, its scene arrays, camera and options, and where its lists are.
    bool have_last = false;
    uint64_t frame_id = 0;  // number of the last gs_render (1, 2, ...; 0: none)
    gs_gaussians last_g{};
    gs_camera last_cam{};
    float last_bg[3] = {0.f, 0.f, 0.f};
    int64_t last_n = 0;
    int last_w = 0, last_h = 0, last_tw = 0, last_th = 0, last_cluster = 1;
    GsGrid last_grid{};  // the grid of the frame's lists
    const uint32_t *last_values = nullptr;
    DevBuf d_rec;
    DevBuf br_geo, br_aux, br_col;  // blend records of the render path (16 B per slot each)
    DevBuf br_rect;                 // their 16 x 16 tile rects, for list-tile frames (8 B per slot)
    DevBuf tile_order;              // the blend's longest-list-first tile order (4 B per list tile)
    // gs_render's captured frames: the launches of one frame as a CUDA
    // graph, replayed (with the frame's camera set in the projection's
    // launch) while the scene arrays, image size, options, framebuffer, key
    // capacity, blend schedule and the context's buffers stay the same; a few
    // are kept (least recently used replaced), so frames that alternate
    // framebuffers or scenes still replay. buf_gen counts the reallocations
    // of the context's buffers. After kGraphMissRun captures in a row the
    // next graph_skip_len frames launch directly (32 at first, doubling up to
    // 1024 while the pattern repeats, back to 32 after a replay).
    uint64_t buf_gen = 0;
    static constexpr int kGraphs = 8, kGraphMissRun = 4, kGraphSkip = 32, kGraphSkipMax = 1024;
    int graph_skip_len = kGraphSkip;
    struct FrameGraph {
        bool valid = false;
        uint64_t last_use = 0;
        int kind = 0;                 // 0: a full binning, 1: a re-binned frame
        const void *extra[8] = {};    // further addresses the launches take (temporal state)
        gs_gaussians g{};
        gs_options o{};
        gs_framebuffer fb{};
        int w = 0, h = 0, variant = 0;
        int64_t cap = 0;
        uint64_t buf_gen = 0;
        uint32_t *sv = nullptr;  // where the frame's sorted lists end up
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t project = nullptr;
    } fg[kGraphs];
    uint64_t graph_clock = 0;
    int graph_miss_run = 0, graph_skip = 0;
    cudaStream_t capture_stream = nullptr;
    // Batched path (own buffers: a captured graph holds their addresses).
    struct Batch {
        DevBuf views, rec, meta, geo, aux, col, scratch, ranges, order, queue, keys, vals, akeys, avals, sort, rts;
        DevBuf rect;  // 16 x 16 tile ranges of the records (list tiles)
        ViewDesc *h_views = nullptr;
        int h_views_cap = 0;
        int64_t rec_cap = 0, key_cap = 0;
        cudaGraphExec_t exec = nullptr;
        cudaStream_t capture = nullptr;  // the graph is captured here, launched on the caller's stream
        std::vector<int64_t> sig;  // what the captured graph was built for
        int64_t keys_per_view = 0;  // of the last batch (chooses GS_BATCH_AUTO's schedule)
        // The last joint batch, for gs_render_batch_backward.
        bool have_joint = false;
        int64_t joint_n = 0, joint_records = 0;
        int joint_views = 0, joint_tw = 0, joint_th = 0, joint_dtype = 0, joint_lists = 1;
        int32_t joint_tiles = 0;
        const uint32_t *joint_values = nullptr;
        DevBuf d_rec, bviews;
    } batch;
    int last_dtype = GS_RECORD_F32;
    int64_t key_capacity = 0;  // pairs the render path's key buffers hold
    bool pinned_capacity = false;  // set by gs_reserve_keys: do not shrink
    DevBuf fused_scratch;
    DevBuf gathered;  // records in list order (GS_BLEND_TMA)
    DevBuf rts_scratch;  // per-partition digit counts and offsets of reduce-then-scan passes
    bool timing = false;
    bool timed_once = false;
    cudaEvent_t ev[8] = {};
    // Frames rendered with GS_SYNC_DEFERRED whose counts are not checked yet
    // (a ring, oldest at ring_head). h_ring holds per slot the four counts and
    // the error word, copied back after the frame.
    static constexpr int kRing = 4;
    struct Pending {
        cudaEvent_t done = nullptr;
        uint64_t seq = 0;
        int64_t cap = 0;
        int n_tiles = 0, bits = 0;
    } ring[kRing];
    unsigned long long *h_ring = nullptr;
    int ring_head = 0, ring_count = 0;
    uint64_t next_seq = 1;   // sequence number of the next deferred frame
    uint64_t clear_seq = 0;  // frames before this one saw an error word already reported
    uint64_t last_seq = 0;   // the last gs_render, if it was deferred
    const uint32_t *last_ranges = nullptr;  // per-tile ranges of the last gs_render
    // Temporal re-binning state: the lists and tile rects of the last frame
    // rendered with opts->temporal (prev_* may point into the full path's
    // buffers; an incremental frame writes vals[cur] / ranges[cur]).
    struct Temporal {
        bool valid = false;
        int64_t n = 0;
        int tiles_x = 0, tiles_y = 0, tw = 0, th = 0;
        DevBuf rects[2], moved, moved_list, tile_scratch, vals[2], ranges[2], ins_vals;
        const uint32_t *prev_vals = nullptr, *prev_ranges = nullptr;
        int cur = 0;
        int rcur = 0;         // rects[rcur] holds the last frame's packed tile rects
        int64_t rects_n = -1;  // ... for this many Gaussians (-1: none)
        double last_churn = 0.0;  // moved / visible of the last frame
        // Adaptive gate (opts->temporal == 1): device time of the binning
        // (projection to ranges) of re-binned and of full frames, averaged
        // over recent frames, and a counter of frames binned in full since
        // re-binning last measured slower.
        cudaEvent_t ev[2] = {nullptr, nullptr};
        double full_ms = 0.0, rebin_ms = 0.0;
        int full_seen = 0, rebin_seen = 0;  // frames of each kind timed so far
        uint32_t gate = 0;
        // Adaptive mode only: frames still to render without tracking rects
        // (after a frame whose churn, or whose measured re-binning time,
        // ruled re-binning out).
        uint32_t cooldown = 0;
    } temporal;
};

namespace {

gs_status fail(gs_context *ctx, gs_status st, const std::string &msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

gs_status cuda_fail(gs_context *ctx, cudaError_t e, const char *where) {
    return fail(ctx, GS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define GS_CUDA(ctx, call)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

gs_status ensure(gs_context *ctx, DevBuf &b, size_t bytes, const char *what) {
    if (bytes <= b.bytes) return GS_OK;
    ++ctx->buf_gen;
    size_t want = bytes + bytes / 4 + 256;
    if (b.ptr) {
        cudaError_t e = cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree");
    }
    cudaError_t e = cudaMalloc(&b.ptr, want);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ctx, GS_ERR_OOM, std::string("cannot allocate ") + std::to_string(want) +
                                         " bytes for " + what);
    }
    b.bytes = want;
    return GS_OK;
}

bool finite(float v) { return std::isfinite(v); }

gs_status check_camera(gs_context *ctx, const gs_camera *cam) {
    if (!cam) return fail(ctx, GS_ERR_INVALID_ARG, "camera is NULL");
    if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
        return fail(ctx, GS_ERR_INVALID_ARG, "camera width/height must be in 1..16384");
    if (!(cam->fx > 0) || !(cam->fy > 0) || !finite(cam->fx) || !finite(cam->fy) ||
        !finite(cam->cx) || !finite(cam->cy))
        return fail(ctx, GS_ERR_INVALID_ARG, "camera intrinsics must be finite with fx, fy > 0");
    if (!(cam->near_z > 0) || !finite(cam->near_z))
        return fail(ctx, GS_ERR_INVALID_ARG, "camera near_z must be finite and > 0");
    for (int i = 0; i < 12; ++i)
        if (!finite(cam->world_to_cam[i]))
            return fail(ctx, GS_ERR_INVALID_ARG, "camera world_to_cam must be finite");
    return GS_OK;
}

gs_status check_options(gs_context *ctx, const gs_options *o) {
    if (!o) return fail(ctx, GS_ERR_INVALID_ARG, "options are NULL");
    const bool ok_tile = (o->tile_w == 16 && o->tile_h == 16) || (o->tile_w == 16 && o->tile_h == 8) ||
                         (o->tile_w == 8 && o->tile_h == 8);
    if (!ok_tile) return fail(ctx, GS_ERR_INVALID_ARG, "tile must be 16x16, 16x8 or 8x8");
    if (o->record_dtype != GS_RECORD_F32 && o->record_dtype != GS_RECORD_F16 && o->record_dtype != GS_RECORD_BF16)
        return fail(ctx, GS_ERR_INVALID_ARG, "record_dtype must be GS_RECORD_F32, _F16 or _BF16");
    if (o->blend_variant < GS_BLEND_CULLED || o->blend_variant > GS_BLEND_TMA)
        return fail(ctx, GS_ERR_INVALID_ARG, "blend_variant must be one of the GS_BLEND_* schedules");
    if (o->direct_launch != 0 && o->direct_launch != 1)
        return fail(ctx, GS_ERR_INVALID_ARG, "direct_launch must be 0 or 1");
    if (o->sync_mode != GS_SYNC_FRAME && o->sync_mode != GS_SYNC_DEFERRED)
        return fail(ctx, GS_ERR_INVALID_ARG, "sync_mode must be GS_SYNC_FRAME or GS_SYNC_DEFERRED");
    if (o->temporal < 0 || o->temporal > 2) return fail(ctx, GS_ERR_INVALID_ARG, "temporal must be 0, 1 or 2");
    if (o->temporal && o->sync_mode != GS_SYNC_FRAME)
        return fail(ctx, GS_ERR_INVALID_ARG, "temporal re-binning needs sync_mode GS_SYNC_FRAME");
    if (o->batch_mode < GS_BATCH_AUTO || o->batch_mode > GS_BATCH_PER_VIEW)
        return fail(ctx, GS_ERR_INVALID_ARG, "batch_mode must be GS_BATCH_AUTO, _JOINT or _PER_VIEW");
    if (o->batch_depth != 0 && o->batch_depth != 64 && o->batch_depth != 128 && o->batch_depth != 256)
        return fail(ctx, GS_ERR_INVALID_ARG, "batch_depth must be 0, 64, 128 or 256");
    if (o->cluster != GS_CLUSTER_NONE && o->cluster != 1 && o->cluster != GS_CLUSTER_2X1 &&
        o->cluster != GS_CLUSTER_2X2)
        return fail(ctx, GS_ERR_INVALID_ARG, "cluster must be GS_CLUSTER_NONE (0 or 1), _2X1 or _2X2");
    if (o->cluster > 1 && !(o->tile_w == 16 && o->tile_h == 16))
        return fail(ctx, GS_ERR_INVALID_ARG, "thread-block clusters need 16x16 tiles");
    if (o->cluster > 1 && o->temporal)
        return fail(ctx, GS_ERR_UNSUPPORTED, "temporal re-binning does not take thread-block clusters");
    if (o->list_tiles != GS_LISTS_1X1 && o->list_tiles != 1 && o->list_tiles != GS_LISTS_2X1 &&
        o->list_tiles != GS_LISTS_2X2 && o->list_tiles != GS_LISTS_4X4 && o->list_tiles != GS_LISTS_8X8)
        return fail(ctx, GS_ERR_INVALID_ARG, "list_tiles must be GS_LISTS_1X1 (0 or 1), _2X1, _2X2, _4X4 or _8X8");
    if (o->list_tiles > 1 && o->cluster > 1)
        return fail(ctx, GS_ERR_INVALID_ARG, "list_tiles and cluster are exclusive");
    if (o->list_tiles > 1 && !(o->tile_w == 16 && o->tile_h == 16))
        return fail(ctx, GS_ERR_INVALID_ARG, "list tiles need 16x16 tiles");
    if (o->list_tiles > 1 && o->temporal)
        return fail(ctx, GS_ERR_UNSUPPORTED, "temporal re-binning does not take list tiles");
    if (o->tile_order != GS_ORDER_LONGEST_FIRST && o->tile_order != GS_ORDER_GRID)
        return fail(ctx, GS_ERR_INVALID_ARG, "tile_order must be GS_ORDER_LONGEST_FIRST or GS_ORDER_GRID");
    for (int i = 0; i < 3; ++i)
        if (!finite(o->bg[i])) return fail(ctx, GS_ERR_INVALID_ARG, "bg must be finite");
    return GS_OK;
}

gs_status check_gaussians(gs_context *ctx, const gs_gaussians *g) {
    if (!g) return fail(ctx, GS_ERR_INVALID_ARG, "gaussians are NULL");
    if (g->n < 0 || g->n >= (int64_t(1) << 31))
        return fail(ctx, GS_ERR_INVALID_ARG, "n must be in 0 .. 2^31-1");
    if (g->sh_degree < 0 || g->sh_degree > 3)
        return fail(ctx, GS_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
        return fail(ctx, GS_ERR_INVALID_ARG, "a Gaussian array is NULL");
    return GS_OK;
}

// Screen tiles per list tile (a list_tile_dims code), from the cluster or
// list-tile option.
int list_shape(const gs_options *o) {
    return o->cluster > 1 ? o->cluster : (o->list_tiles > 1 ? o->list_tiles : 1);
}

// The grid of the per-tile lists: the screen tiles, or with thread-block
// clusters or list tiles the list tiles of 2 x 1 / 2 x 2 screen tiles.
GsGrid make_grid(const gs_camera *cam, const gs_options *o) {
    GsGrid gr;
    int lx = 1, ly = 1;
    list_tile_dims(list_shape(o), &lx, &ly);
    gr.tile_w = lx * o->tile_w;
    gr.tile_h = ly * o->tile_h;
    gr.tiles_x = (cam->width + gr.tile_w - 1) / gr.tile_w;
    gr.tiles_y = (cam->height + gr.tile_h - 1) / gr.tile_h;
    return gr;
}

GsCameraDev make_cam(const gs_camera *c) {
    GsCameraDev k;
    for (int r = 0; r < 3; ++r) {
        for (int j = 0; j < 3; ++j) k.R[3 * r + j] = c->world_to_cam[4 * r + j];
        k.t[r] = c->world_to_cam[4 * r + 3];
    }
    for (int j = 0; j < 3; ++j)  // C = -R^T t (in double, then rounded)
        k.C[j] = (float)-((double)k.R[j] * k.t[0] + (double)k.R[3 + j] * k.t[1] +
                          (double)k.R[6 + j] * k.t[2]);
    k.fx = c->fx;
    k.fy = c->fy;
    k.cx = c->cx;
    k.cy = c->cy;
    k.near_z = c->near_z;
    k.lim_x = gs::kGuard * (0.5f * c->width / c->fx);
    k.lim_y = gs::kGuard * (0.5f * c->height / c->fy);
    for (int r = 0; r < 3; ++r) {
        const double nr = std::sqrt((double)k.R[3 * r] * k.R[3 * r] + (double)k.R[3 * r + 1] * k.R[3 * r + 1] +
                                    (double)k.R[3 * r + 2] * k.R[3 * r + 2]);
        k.rn[r] = (float)(nr * (1.0 + 1e-6));
    }
    k.width = c->width;
    k.height = c->height;
    return k;
}

int key_bits_for(int n_tiles) {
    int b = 0;
    while ((1ll << b) < n_tiles) ++b;
    return 32 + b;
}

// Reads the device error word after a synchronisation point.
gs_status collect_device_error(gs_context *ctx, cudaStream_t s) {
    GS_CUDA(ctx, cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GS_CUDA(ctx, cudaStreamSynchronize(s));
    const uint32_t w = *ctx->h_err;
    if (w == 0) return GS_OK;
    GS_CUDA(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), s));
    if (w & gs::kErrTimeout)
        return fail(ctx, GS_ERR_TIMEOUT, "a device-side wait gave up (look-back timeout)");
    if (w & gs::kErrCapacity) return fail(ctx, GS_ERR_CAPACITY, "a device buffer was too small");
    return fail(ctx, GS_ERR_INVALID_ARG, "records inconsistent with their tile counts");
}

// Checks the oldest deferred frame: with wait, blocks until it is done;
// otherwise returns at once if it is still running (*retired = false).
gs_status retire_oldest(gs_context *ctx, bool wait, cudaStream_t s, bool *retired) {
    *retired = false;
    if (ctx->ring_count == 0) return GS_OK;
    const int i = ctx->ring_head;
    const gs_context::Pending p = ctx->ring[i];
    const cudaError_t e = wait ? cudaEventSynchronize(p.done) : cudaEventQuery(p.done);
    if (e == cudaErrorNotReady) return GS_OK;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "deferred frame");
    *retired = true;
    ctx->ring_head = (i + 1) % gs_context::kRing;
    --ctx->ring_count;
    const unsigned long long *h = ctx->h_ring + 5 * i;
    const unsigned long long K = h[0];
    const uint32_t w = static_cast<uint32_t>(h[4]);
    ctx->stats.n_visible = (int64_t)h[1];
    ctx->stats.n_keys = (int64_t)K;
    ctx->stats.n_tiles = p.n_tiles;
    ctx->stats.key_bits = p.bits;
    const bool overflow = (int64_t)K > p.cap;
    if (overflow && p.seq == ctx->last_seq) ctx->have_last = false;
    // The error word is sticky: frames enqueued before it was cleared see the
    // bits of an earlier frame, which are reported once.
    const bool fresh = p.seq >= ctx->clear_seq;
    if ((overflow || w) && fresh) {
        GS_CUDA(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), s));
        ctx->clear_seq = ctx->next_seq;
    }
    if (K >= (1ull << 32) - 1)
        return fail(ctx, GS_ERR_CAPACITY, "more than 2^32-2 (tile, Gaussian) pairs in one frame");
    if (overflow) {
        ctx->key_capacity = std::max<int64_t>(ctx->key_capacity, (int64_t)(K + K / 4 + 1024));
        return fail(ctx, GS_ERR_CAPACITY,
                    "a deferred frame needed " + std::to_string(K) + " key pairs but the buffers held " +
                        std::to_string(p.cap) + "; its image is incomplete. The buffers have grown: render it again");
    }
    if (w && fresh) {
        if (w & gs::kErrTimeout)
            return fail(ctx, GS_ERR_TIMEOUT, "a device-side wait gave up (look-back timeout)");
        if (w & gs::kErrCapacity) return fail(ctx, GS_ERR_CAPACITY, "a device buffer was too small");
        return fail(ctx, GS_ERR_INVALID_ARG, "records inconsistent with their tile counts");
    }
    return GS_OK;
}

// Checks deferred frames, oldest first: all of them (waiting) or those that
// are done. Stops at the first error.
gs_status drain_deferred(gs_context *ctx, bool wait, cudaStream_t s) {
    while (ctx->ring_count > 0) {
        bool retired = false;
        const gs_status st = retire_oldest(ctx, wait, s, &retired);
        if (st != GS_OK) return st;
        if (!retired) break;
    }
    return GS_OK;
}

enum { EV_START, EV_PROJECT, EV_DEPTH, EV_SCAN, EV_EMIT, EV_SORT, EV_RANGES, EV_BLEND, EV_COUNT };

void mark(gs_context *ctx, int which, cudaStream_t s) {
    if (ctx->timing) cudaEventRecord(ctx->ev[which], s);
}

// Record form of the blend records written for record precision dtype.
int rec_mode(int dtype) {
    return dtype == GS_RECORD_F16 ? gs::kRecF16 : dtype == GS_RECORD_BF16 ? gs::kRecBF16 : gs::kRecF32;
}

// The blend records of the render path (or, with raw, caller's gs_records).
RecordReader reader(gs_context *ctx, const gs_record *rec, int dtype, bool raw = false) {
    RecordReader r;
    r.rec32 = reinterpret_cast<const float4 *>(rec);
    r.geo = static_cast<const float4 *>(ctx->br_geo.ptr);
    r.aux = static_cast<const float4 *>(ctx->br_aux.ptr);
    r.col = ctx->br_col.ptr;
    r.mode = raw ? gs::kRecRaw : rec_mode(dtype);
    r.rect16 = static_cast<const uint2 *>(ctx->br_rect.ptr);
    return r;
}

// Where the render path's projection writes its blend records (with cam:
// also their 16 x 16 tile rects, which the list-tile blend reads).
gs::BlendRecordOut blend_out(gs_context *ctx, int dtype, const gs_camera *cam = nullptr) {
    return gs::BlendRecordOut{static_cast<float4 *>(ctx->br_geo.ptr),
                              static_cast<float4 *>(ctx->br_aux.ptr),
                              ctx->br_col.ptr,
                              rec_mode(dtype),
                              cam ? static_cast<uint2 *>(ctx->br_rect.ptr) : nullptr,
                              cam ? (cam->width + 15) / 16 : 0,
                              cam ? (cam->height + 15) / 16 : 0};
}

// The blend records of the last joint batch (one per compact record slot).
RecordReader batch_reader(gs_context *ctx, int dtype) {
    RecordReader r;
    r.rec32 = static_cast<const float4 *>(ctx->batch.rec.ptr);
    r.geo = static_cast<const float4 *>(ctx->batch.geo.ptr);
    r.aux = static_cast<const float4 *>(ctx->batch.aux.ptr);
    r.col = ctx->batch.col.ptr;
    r.mode = rec_mode(dtype);
    r.rect16 = static_cast<const uint2 *>(ctx->batch.rect.ptr);
    return r;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Scan + emit + sort + ranges into the given key/value buffers (which must
// hold `capacity` pairs); the other pair of buffers comes from the context.
// The stage entry points reuse the context's key buffers, which the temporal
// state and the last frame's lists (read by gs_render_backward) point into:
// they drop both.
void drop_temporal(gs_context *ctx) {
    ctx->temporal.valid = false;
    ctx->have_last = false;
}

// Temporal mode's binning time: events around projection .. ranges.
// (Not inside a capture: a graph's frames are timed around its launch.)
void temporal_mark(gs_context *ctx, int k, cudaStream_t s) {
    if (ctx->temporal.ev[k] && s != ctx->capture_stream) cudaEventRecord(ctx->temporal.ev[k], s);
}

// After a synchronised temporal frame: folds its binning time into the
// average of its kind. The first frame of each kind on a context is not
// counted: it may include the kernels' first-launch loading.
void temporal_sample(gs_context *ctx, bool rebinned) {
    auto &T = ctx->temporal;
    float ms = 0.f;
    if (!T.ev[0] || cudaEventElapsedTime(&ms, T.ev[0], T.ev[1]) != cudaSuccess) return;
    if ((rebinned ? T.rebin_seen : T.full_seen)++ == 0) return;
    double &avg = rebinned ? T.rebin_ms : T.full_ms;
    avg = avg > 0.0 ? 0.5 * avg + 0.5 * ms : ms;
}

// Whether a frame that may be re-binned should be. temporal == 2 always
// re-bins; temporal == 1 re-bins while re-binned frames measured no slower
// than full ones (2 % margin), and otherwise bins in full, re-binning one
// frame in 8 to measure again (the scene, the camera motion or the GPU's
// load may change).
bool temporal_rebin_now(gs_context *ctx, int temporal) {
    auto &T = ctx->temporal;
    if (temporal == 2 || T.rebin_ms <= 0.0 || T.full_ms <= 0.0 || T.rebin_ms <= 1.02 * T.full_ms) {
        T.gate = 0;
        return true;
    }
    return (++T.gate % 8u) == 0u;
}

// Adaptive mode: frames rendered without tracking rects once re-binning is
// ruled out. Tracking (writing this frame's rects and comparing them with
// the last frame's) costs every full frame some time, so after a frame that
// found the churn above the limit, or that the gate sent to the full binning,
// the next kTemporalCooldown frames skip it; the two frames after them track
// again (the first writes rects, the second bins in full and measures the
// churn), one frame in eight, as the gate re-measures.
constexpr uint32_t kTemporalCooldown = 6;

// Records what gs_render_backward needs of the frame just enqueued (seq: its
// deferred sequence number, 0 for a synchronised frame).
void remember_frame(gs_context *ctx, const gs_gaussians *g, const gs_camera *cam, const gs_options *opts,
                    const GsGrid &grid, const uint32_t *values, const uint32_t *ranges, uint64_t seq) {
    ctx->have_last = true;
    ctx->frame_id += 1;
    ctx->last_seq = seq;
    ctx->last_g = *g;
    ctx->last_cam = *cam;
    for (int c = 0; c < 3; ++c) ctx->last_bg[c] = opts->bg[c];
    ctx->last_n = g->n;
    ctx->last_w = cam->width;
    ctx->last_h = cam->height;
    ctx->last_tw = opts->tile_w;
    ctx->last_th = opts->tile_h;
    ctx->last_cluster = list_shape(opts);
    ctx->last_grid = grid;
    ctx->last_values = values;
    ctx->last_ranges = ranges;
    ctx->last_dtype = opts->record_dtype;
}

// Is (g, cam, opts) the frame remembered by remember_frame? Compares the
// scene's array pointers, count and SH degree, every camera field, the tile
// shape, the background and the record precision.
bool same_frame(const gs_context *ctx, const gs_gaussians *g, const gs_camera *cam, const gs_options *opts) {
    const gs_gaussians &a = ctx->last_g;
    if (a.means != g->means || a.log_scales != g->log_scales || a.quats != g->quats ||
        a.opacity_logits != g->opacity_logits || a.sh != g->sh || a.n != g->n || a.sh_degree != g->sh_degree)
        return false;
    const gs_camera &c = ctx->last_cam;
    for (int i = 0; i < 12; ++i)
        if (c.world_to_cam[i] != cam->world_to_cam[i]) return false;
    if (c.fx != cam->fx || c.fy != cam->fy || c.cx != cam->cx || c.cy != cam->cy || c.width != cam->width ||
        c.height != cam->height || c.near_z != cam->near_z)
        return false;
    for (int i = 0; i < 3; ++i)
        if (ctx->last_bg[i] != opts->bg[i]) return false;
    return ctx->last_tw == opts->tile_w && ctx->last_th == opts->tile_h && ctx->last_dtype == opts->record_dtype &&
           ctx->last_cluster == list_shape(opts);
}

gs_status bin_impl(gs_context *ctx, const gs_record *records, const uint32_t *tiles, int64_t n,
                   const GsGrid &grid, uint64_t *keys, uint32_t *values, int64_t capacity,
                   bool capacity_is_ctx, uint32_t *ranges, int64_t *n_keys, cudaStream_t s) {
    drop_temporal(ctx);
    gs_status st;
    const int n_tiles = grid.tiles_x * grid.tiles_y;
    if ((st = ensure(ctx, ctx->offsets, (size_t)(n > 0 ? n : 1) * 8, "offsets")) != GS_OK) return st;
    if ((st = ensure(ctx, ctx->scan_scratch, gs_scan_scratch_bytes(n), "scan scratch")) != GS_OK)
        return st;
    GS_CUDA(ctx, gs_launch_scan(tiles, n, static_cast<unsigned long long *>(ctx->offsets.ptr),
                                ctx->d_counts, ctx->scan_scratch.ptr, ctx->d_err, s));
    GS_CUDA(ctx, cudaMemcpyAsync(ctx->h_counts, ctx->d_counts, 2 * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, s));
    if ((st = collect_device_error(ctx, s)) != GS_OK) return st;
    const unsigned long long K = ctx->h_counts[0];
    *n_keys = (int64_t)K;
    ctx->stats.n_visible = (int64_t)ctx->h_counts[1];
    ctx->stats.n_keys = (int64_t)K;
    ctx->stats.n_tiles = n_tiles;
    ctx->stats.key_bits = key_bits_for(n_tiles);
    if (K >= (1ull << 32) - 1)
        return fail(ctx, GS_ERR_CAPACITY, "more than 2^32-2 (tile, Gaussian) pairs in one pass");
    if (capacity_is_ctx) {
        if ((st = ensure(ctx, ctx->keys, (K + 1) * 8, "keys")) != GS_OK) return st;
        if ((st = ensure(ctx, ctx->values, (K + 1) * 4, "values")) != GS_OK) return st;
        keys = static_cast<uint64_t *>(ctx->keys.ptr);
        values = static_cast<uint32_t *>(ctx->values.ptr);
        capacity = (int64_t)(K + 1);
    } else if ((int64_t)K > capacity) {
        return fail(ctx, GS_ERR_CAPACITY, "key buffer capacity " + std::to_string(capacity) +
                                              " < " + std::to_string(K) + " pairs");
    }
    if ((st = ensure(ctx, ctx->alt_keys, (K + 1) * 8, "alt keys")) != GS_OK) return st;
    if ((st = ensure(ctx, ctx->alt_values, (K + 1) * 4, "alt values")) != GS_OK) return st;
    const int bits = key_bits_for(n_tiles);
    if ((st = ensure(ctx, ctx->sort_scratch, gs_sort_scratch_bytes((int64_t)K, bits), "sort scratch")) !=
        GS_OK)
        return st;
    // Emit into whichever buffer makes the sorted result land in `keys`.
    const bool odd = (gs_sort_passes(bits) & 1) != 0 && K > 1;
    uint64_t *ek = odd ? static_cast<uint64_t *>(ctx->alt_keys.ptr) : keys;
    uint32_t *ev = odd ? static_cast<uint32_t *>(ctx->alt_values.ptr) : values;
    uint64_t *ok = odd ? keys : static_cast<uint64_t *>(ctx->alt_keys.ptr);
    uint32_t *ov = odd ? values : static_cast<uint32_t *>(ctx->alt_values.ptr);
    GS_CUDA(ctx, gs_launch_emit(records, tiles, static_cast<unsigned long long *>(ctx->offsets.ptr), n,
                                grid, ek, ev, (int64_t)K, ctx->d_err, s));
    bool in_alt = false;
    GS_CUDA(ctx, gs_launch_sort(ek, ev, ok, ov, (int64_t)K, bits, ctx->sort_scratch.ptr, ctx->d_err,
                                &in_alt, s));
    (void)capacity;
    GS_CUDA(ctx, gs_launch_ranges(keys, (int64_t)K, n_tiles, ranges, ctx->d_err, s));
    return GS_OK;
}

// The default culled blend of gs_render uses 8x8 warp blocks, whose two
// pixels per lane go through packed FP32 pair instructions (measured 0.188
// against 0.197 ms for 8x4 blocks at 141 entries per tile on a 1080p frame,
// and faster at thousands per tile). The cluster blend computes one pixel at
// a time: 8x4 blocks for shallow lists, 8x8 for deep ones (more than 1024
// entries per list tile in the previous frame). All give identical images.
int blend_schedule(const gs_context *ctx, const gs_options *opts, int n_tiles) {
    if (opts->blend_variant != GS_BLEND_CULLED) return opts->blend_variant;
    if (opts->cluster > 1)
        return ctx->stats.n_keys > (int64_t)1024 * n_tiles ? GS_BLEND_CULLED_8X8 : GS_BLEND_CULLED;
    return GS_BLEND_CULLED_8X8;
}

// Longest lists first (GS_ORDER_LONGEST_FIRST): the culled and list-tile
// blends take their tiles in the order of a small sort kernel, launched here
// after the frame's ranges; *order stays null for grid order and for the
// blends that do not take an order.
gs_status launch_tile_order(gs_context *ctx, const uint32_t *ranges, const GsGrid &grid, const gs_options *opts,
                            cudaStream_t s, const uint32_t **order) {
    *order = nullptr;
    const int n_tiles = grid.tiles_x * grid.tiles_y;
    const int variant = blend_schedule(ctx, opts, n_tiles);
    if (opts->tile_order != GS_ORDER_LONGEST_FIRST || opts->cluster > 1 ||
        (opts->list_tiles <= 1 && (variant == GS_BLEND_BASIC || variant == GS_BLEND_TMA)))
        return GS_OK;
    gs_status st = ensure(ctx, ctx->tile_order, (size_t)(n_tiles > 0 ? n_tiles : 1) * 4, "tile order");
    if (st != GS_OK) return st;
    GS_CUDA(ctx, gs_launch_tile_order(ranges, n_tiles, static_cast<uint32_t *>(ctx->tile_order.ptr), s));
    *order = static_cast<const uint32_t *>(ctx->tile_order.ptr);
    return GS_OK;
}

// The blend of a gs_render frame with `d_n` (device count, at most n_cap)
// pairs in its lists; order: from launch_tile_order.
gs_status launch_blend(gs_context *ctx, const RecordReader &rd, const uint32_t *values, const uint32_t *ranges,
                       const GsGrid &grid, const gs_camera *cam, const gs_options *opts, const gs_framebuffer *fb,
                       const unsigned long long *d_n, int64_t n_cap, const uint32_t *order, cudaStream_t s) {
    const int variant = blend_schedule(ctx, opts, grid.tiles_x * grid.tiles_y);
    if (opts->list_tiles > 1) {
        GS_CUDA(ctx, gs_launch_blend_listtile(rd, values, ranges, grid, opts->list_tiles, cam->width, cam->height,
                                              opts->bg, *fb, variant == GS_BLEND_CULLED_WIDE, order, s));
        return GS_OK;
    }
    if (opts->cluster > 1) {
        GS_CUDA(ctx, gs_launch_blend_cluster(rd, values, ranges, grid, opts->cluster, cam->width, cam->height,
                                             opts->bg, *fb, variant == GS_BLEND_CULLED_8X8, s));
        return GS_OK;
    }
    if (variant == GS_BLEND_TMA) {
        gs_status st = ensure(ctx, ctx->gathered, (size_t)(n_cap > 0 ? n_cap : 1) * 48, "gathered records");
        if (st != GS_OK) return st;
        GS_CUDA(ctx, gs_launch_blend_tma(rd, values, ranges, grid, cam->width, cam->height, opts->bg, *fb,
                                         static_cast<float4 *>(ctx->gathered.ptr), d_n, n_cap, ctx->d_err, s));
        return GS_OK;
    }
    GS_CUDA(ctx, gs_launch_blend(rd, values, ranges, grid, cam->width, cam->height, opts->bg, *fb, variant, s,
                                 order));
    return GS_OK;
}

void drop_frame_graph(gs_context::FrameGraph &F) {
    if (F.exec) cudaGraphExecDestroy(F.exec);
    if (F.graph) cudaGraphDestroy(F.graph);
    F = gs_context::FrameGraph{};
}

// Does the captured frame F serve (g, cam, opts, fb) with this key capacity,
// blend schedule and the context's current buffers? (The camera pose and
// intrinsics are set per replay; the sync mode acts after the graph.)
bool frame_graph_fits(const gs_context *ctx, const gs_context::FrameGraph &F, int kind, const void *const extra[8],
                      const gs_gaussians *g, const gs_camera *cam, const gs_options *opts, const gs_framebuffer *fb,
                      int64_t cap, int variant) {
    if (!F.valid || F.kind != kind) return false;
    for (int i = 0; i < 8; ++i)
        if (F.extra[i] != extra[i]) return false;
    gs_options a = F.o, b = *opts;  // 4-byte fields only: no padding
    a.sync_mode = b.sync_mode = 0;
    return F.g.means == g->means && F.g.log_scales == g->log_scales && F.g.quats == g->quats &&
           F.g.opacity_logits == g->opacity_logits && F.g.sh == g->sh && F.g.n == g->n &&
           F.g.sh_degree == g->sh_degree && F.w == cam->width && F.h == cam->height &&
           std::memcmp(&a, &b, sizeof a) == 0 && F.fb.rgb == fb->rgb && F.fb.final_T == fb->final_T &&
           F.fb.n_contrib == fb->n_contrib && F.fb.n_eval == fb->n_eval && F.cap == cap && F.variant == variant &&
           F.buf_gen == ctx->buf_gen;
}

// Enqueues a gs_render frame on s through one of the context's CUDA graphs:
// a graph that fits the frame is launched with the frame's camera set in the
// projection's launch; otherwise the least recently used slot captures the
// frame's launches (on the context's own stream, so nothing runs) first. A
// context whose frames keep missing (kGraphMissRun captures in a row)
// launches its next graph_skip_len frames directly. enqueue(q) issues the
// frame's launches on q and sets *sv.
template <class Enqueue>
gs_status replay_frame(gs_context *ctx, int kind, const void *const extra[8], const gs_gaussians *g,
                       const gs_camera *cam, const gs_options *opts, const gs_framebuffer *fb, int64_t cap,
                       int variant, const GsCameraDev &dcam, cudaStream_t s, Enqueue &enqueue, uint32_t **sv) {
    if (ctx->graph_skip > 0) {
        --ctx->graph_skip;
        return enqueue(s);
    }
    // A caller capturing its own graph on s gets the launches themselves.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        (void)cudaGetLastError();
        return enqueue(s);
    }
    gs_context::FrameGraph *F = nullptr, *lru = &ctx->fg[0];
    for (auto &c : ctx->fg) {
        if (frame_graph_fits(ctx, c, kind, extra, g, cam, opts, fb, cap, variant)) F = &c;
        if (!c.valid || (lru->valid && c.last_use < lru->last_use)) lru = &c;
    }
    if (F) {
        ctx->graph_miss_run = 0;
        ctx->graph_skip_len = gs_context::kGraphSkip;
    } else {
        if (++ctx->graph_miss_run >= gs_context::kGraphMissRun) {
            ctx->graph_miss_run = 0;
            ctx->graph_skip = ctx->graph_skip_len;
            ctx->graph_skip_len = std::min(2 * ctx->graph_skip_len, gs_context::kGraphSkipMax);
            return enqueue(s);
        }
        F = lru;
        drop_frame_graph(*F);
        if (!ctx->capture_stream)
            GS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        GS_CUDA(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        const gs_status st = enqueue(ctx->capture_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &graph);
        if (st != GS_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            (void)cudaGetLastError();
            return st != GS_OK ? st : cuda_fail(ctx, e, "cudaStreamEndCapture");
        }
        size_t count = 0;
        cudaError_t e2 = cudaGraphGetNodes(graph, nullptr, &count);
        std::vector<cudaGraphNode_t> nodes(count);
        if (e2 == cudaSuccess && count > 0) e2 = cudaGraphGetNodes(graph, nodes.data(), &count);
        cudaGraphNode_t project = nullptr;
        int found = 0;
        for (size_t i = 0; e2 == cudaSuccess && i < count; ++i)
            if (gs_is_camera_node(nodes[i])) project = nodes[i], ++found;
        cudaGraphExec_t exec = nullptr;
        if (e2 == cudaSuccess) e2 = cudaGraphInstantiate(&exec, graph, 0);
        if (e2 != cudaSuccess || found != (g->n > 0 ? 1 : 0)) {
            if (exec) cudaGraphExecDestroy(exec);
            cudaGraphDestroy(graph);
            return e2 != cudaSuccess ? cuda_fail(ctx, e2, "CUDA graph of the frame")
                                     : fail(ctx, GS_ERR_CUDA, "CUDA graph of the frame: projection launch not found");
        }
        F->valid = true;
        F->kind = kind;
        for (int i = 0; i < 8; ++i) F->extra[i] = extra[i];
        F->g = *g;
        F->o = *opts;
        F->fb = *fb;
        F->w = cam->width;
        F->h = cam->height;
        F->variant = variant;
        F->cap = cap;
        F->buf_gen = ctx->buf_gen;
        F->sv = *sv;
        F->graph = graph;
        F->exec = exec;
        F->project = project;
    }
    F->last_use = ++ctx->graph_clock;
    if (F->project) GS_CUDA(ctx, gs_set_node_camera(F->exec, F->project, dcam));
    GS_CUDA(ctx, cudaGraphLaunch(F->exec, s));
    *sv = F->sv;
    return GS_OK;
}

// Above this fraction of moved Gaussians (of the visible ones) in the last
// frame, the next frame is binned from scratch: re-binning pays off only
// while few tiles change (measured break-even near 10 % on a 1M-Gaussian
// 1080p scene).
constexpr double kTemporalMaxChurn = 0.08;
// GS_BATCH_AUTO renders views one by one after a batch with more keys per view.
constexpr int64_t kBatchPerViewKeys = int64_t(8) << 20;
// Largest tile list the per-tile merge holds in shared memory (a power of two).
constexpr int kTemporalTileCap = 4096;

// One frame with temporal re-binning. *done = false (and GS_OK) when the
// frame has to be binned from scratch instead: a tile above the per-tile
// limit, more pairs than the buffers hold, or state inconsistent with it.
gs_status render_rebinned(gs_context *ctx, const gs_gaussians *g, const gs_camera *cam, const gs_options *opts,
                          const gs_framebuffer *fb, cudaStream_t s, bool *done) {
    *done = false;
    auto &T = ctx->temporal;
    gs_status st;
    const GsGrid grid = make_grid(cam, opts);
    const int64_t n = g->n;
    const int n_tiles = grid.tiles_x * grid.tiles_y;
    const int64_t cap = ctx->key_capacity;
    const int dtype = opts->record_dtype;
    const size_t tiles4 = ((size_t)n_tiles * 4 + 255) / 256 * 256;
    const size_t status_bytes = (gs_temporal_scan_status_bytes(n_tiles) + 255) / 256 * 256;
    // tile scratch: removed, added, ins_cursor (zeroed), ins_first, then 256 B
    // of counters (zeroed) and the scan status (zeroed)
    const size_t zero_bytes = 3 * tiles4 + 256 + status_bytes;
    const int out = T.cur;
    // Work items: one per moved Gaussian plus one per 256 tiles of its rects.
    const int64_t item_cap = n + 2 * (cap / 256) + 4096;
    if ((st = ensure(ctx, T.rects[T.rcur ^ 1], (size_t)n * 8, "temporal rects")) != GS_OK ||
        (st = ensure(ctx, T.moved, (size_t)n, "temporal flags")) != GS_OK ||
        (st = ensure(ctx, T.moved_list, (size_t)item_cap * 8, "temporal work items")) != GS_OK ||
        (st = ensure(ctx, T.tile_scratch, zero_bytes + tiles4, "temporal tile scratch")) != GS_OK ||
        (st = ensure(ctx, T.vals[out], (size_t)cap * 4, "temporal values")) != GS_OK ||
        (st = ensure(ctx, T.ranges[out], (size_t)n_tiles * 8, "temporal ranges")) != GS_OK ||
        (st = ensure(ctx, T.ins_vals, (size_t)cap * 4, "temporal arrivals")) != GS_OK)
        return st;
    char *ts = static_cast<char *>(T.tile_scratch.ptr);
    uint32_t *removed = reinterpret_cast<uint32_t *>(ts);
    uint32_t *added = reinterpret_cast<uint32_t *>(ts + tiles4);
    uint32_t *ins_cursor = reinterpret_cast<uint32_t *>(ts + 2 * tiles4);
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(ts + 3 * tiles4);
    unsigned long long *status = reinterpret_cast<unsigned long long *>(ts + 3 * tiles4 + 256);
    uint32_t *ins_first = reinterpret_cast<uint32_t *>(ts + zero_bytes);
    // counters: [0] visible << 33 | keys, [1] moved Gaussians, [2] their work items,
    // [3] entries, [4] arrivals, [5] the scan's partition counter
    gs_record *rec = static_cast<gs_record *>(ctx->records.ptr);
    uint32_t *vals = static_cast<uint32_t *>(T.vals[out].ptr);
    uint32_t *ranges = static_cast<uint32_t *>(T.ranges[out].ptr);
    const uint2 *prev_rect = static_cast<const uint2 *>(T.rects[T.rcur].ptr);
    uint2 *rect = static_cast<uint2 *>(T.rects[T.rcur ^ 1].ptr);
    const GsCameraDev dcam = make_cam(cam);
    // The frame's launches on stream q (enqueued directly or captured into
    // the context's CUDA graph of re-binned frames, as in gs_render).
    auto enqueue = [&](cudaStream_t q) -> gs_status {
        GS_CUDA(ctx, cudaMemsetAsync(ts, 0, zero_bytes, q));
        mark(ctx, EV_START, q);
        temporal_mark(ctx, 0, q);
        GS_CUDA(ctx, gs_launch_project_temporal(*g, dcam, grid, rec, blend_out(ctx, dtype), prev_rect, rect,
                                                static_cast<uint8_t *>(T.moved.ptr),
                                                static_cast<unsigned long long *>(T.moved_list.ptr), item_cap,
                                                counters, ctx->d_err, q));
        mark(ctx, EV_PROJECT, q);
        mark(ctx, EV_DEPTH, q);
        mark(ctx, EV_SCAN, q);
        mark(ctx, EV_EMIT, q);
        GsTemporalRebin R;
        R.records = reinterpret_cast<const float4 *>(rec);
        R.prev_vals = T.prev_vals;
        R.prev_ranges = T.prev_ranges;
        R.moved = static_cast<const uint8_t *>(T.moved.ptr);
        R.removed = removed;
        R.added = added;
        R.items = static_cast<const unsigned long long *>(T.moved_list.ptr);
        R.n_items = counters + 2;
        R.item_capacity = item_cap;
        R.prev_rect = prev_rect;
        R.rect = rect;
        R.n_tiles = n_tiles;
        R.tiles_x = grid.tiles_x;
        R.n_gaussians = n;
        R.ranges = ranges;
        R.vals = vals;
        R.capacity = cap;
        R.ins_first = ins_first;
        R.ins_cursor = ins_cursor;
        R.ins_vals = static_cast<uint32_t *>(T.ins_vals.ptr);
        R.ins_capacity = cap;
        R.totals = counters + 3;
        R.scan_counter = reinterpret_cast<uint32_t *>(counters + 5);
        R.scan_status = status;
        R.cap_entries = kTemporalTileCap;
        R.d_err = ctx->d_err;
        GS_CUDA(ctx, gs_launch_temporal_rebin(R, q));
        temporal_mark(ctx, 1, q);
        mark(ctx, EV_SORT, q);
        const uint32_t *order = nullptr;
        gs_status st2;
        if ((st2 = launch_tile_order(ctx, ranges, grid, opts, q, &order)) != GS_OK) return st2;
        mark(ctx, EV_RANGES, q);
        return launch_blend(ctx, reader(ctx, rec, dtype), vals, ranges, grid, cam, opts, fb, counters + 3, cap, order,
                            q);
    };
    const int variant = blend_schedule(ctx, opts, n_tiles);
    if (!ctx->timing && opts->direct_launch == 0 && variant != GS_BLEND_TMA) {
        const void *extra[8] = {T.prev_vals, T.prev_ranges, prev_rect, rect, vals, ranges,
                                reinterpret_cast<const void *>(static_cast<uintptr_t>(item_cap))};
        uint32_t *sv = vals;
        temporal_mark(ctx, 0, s);
        if ((st = replay_frame(ctx, 1, extra, g, cam, opts, fb, cap, variant, dcam, s, enqueue, &sv)) != GS_OK)
            return st;
        temporal_mark(ctx, 1, s);
    } else if ((st = enqueue(s)) != GS_OK) {
        return st;
    }
    mark(ctx, EV_BLEND, s);
    unsigned long long *h = ctx->h_ring;  // no deferred frame is in flight (drained before)
    h[5] = 0;
    GS_CUDA(ctx, cudaMemcpyAsync(h, counters, 5 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    GS_CUDA(ctx, cudaMemcpyAsync(h + 5, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GS_CUDA(ctx, cudaStreamSynchronize(s));
    const uint32_t w = static_cast<uint32_t>(h[5]);
    const unsigned long long K = h[3];
    if ((w & gs::kErrTemporal) || (int64_t)K > cap) {
        // Rebuild this frame from scratch (it also recaptures the state).
        GS_CUDA(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), s));
        T.valid = false;
        if ((int64_t)K > cap) ctx->key_capacity = (int64_t)(K + K / 4 + 1024);
        return GS_OK;
    }
    const int64_t visible = (int64_t)(h[0] >> 33);
    ctx->stats.n_visible = visible;
    ctx->stats.n_keys = (int64_t)K;
    ctx->stats.n_tiles = n_tiles;
    ctx->stats.key_bits = key_bits_for(n_tiles);
    ctx->stats.n_moved = (int64_t)h[1];
    ctx->stats.rebinned = 1;
    T.prev_vals = vals;
    T.prev_ranges = ranges;
    T.cur = out ^ 1;
    T.rcur ^= 1;
    T.rects_n = n;
    T.last_churn = visible > 0 ? (double)h[1] / (double)visible : 0.0;
    if (opts->temporal == 1 && T.last_churn > kTemporalMaxChurn) T.cooldown = kTemporalCooldown;
    temporal_sample(ctx, true);
    if (ctx->timing) ctx->timed_once = true;
    remember_frame(ctx, g, cam, opts, grid, vals, ranges, 0);
    *done = true;
    if (w) return collect_device_error(ctx, s);
    return GS_OK;
}

}  // namespace

extern "C" {

void gs_default_options(gs_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tile_w = 16;
    o->tile_h = 16;
}

gs_status gs_create(gs_context **out, int device) {
    if (!out) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        (void)cudaGetLastError();
        return GS_ERR_INVALID_ARG;
    }
    gs_context *ctx = new gs_context();
    ctx->device = device;
    DeviceGuard g(device);
    if (cudaMalloc(&ctx->d_err, 256) != cudaSuccess ||
        cudaMalloc(&ctx->d_counts, 8 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_counts, 8 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_err, sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_ring, 5 * gs_context::kRing * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(ctx->d_err, 0, 256) != cudaSuccess) {
        (void)cudaGetLastError();
        gs_destroy(ctx);
        return GS_ERR_CUDA;
    }
    for (auto &p : ctx->ring) {
        if (cudaEventCreateWithFlags(&p.done, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            gs_destroy(ctx);
            return GS_ERR_CUDA;
        }
    }
    *out = ctx;
    return GS_OK;
}

void gs_destroy(gs_context *ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    for (auto &F : ctx->fg) drop_frame_graph(F);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    DevBuf *bufs[] = {&ctx->records, &ctx->tiles, &ctx->offsets, &ctx->scan_scratch, &ctx->keys,
                      &ctx->values, &ctx->alt_keys, &ctx->alt_values, &ctx->sort_scratch, &ctx->ranges,
                      &ctx->fused_scratch, &ctx->d_rec, &ctx->br_geo, &ctx->br_aux, &ctx->br_col, &ctx->gathered,
                      &ctx->rts_scratch, &ctx->br_rect, &ctx->tile_order};
    for (DevBuf *b : bufs)
        if (b->ptr) cudaFree(b->ptr);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_counts) cudaFree(ctx->d_counts);
    if (ctx->h_counts) cudaFreeHost(ctx->h_counts);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    if (ctx->ring_count > 0) cudaDeviceSynchronize();  // frames in flight still write h_ring
    if (ctx->h_ring) cudaFreeHost(ctx->h_ring);
    for (auto &p : ctx->ring)
        if (p.done) cudaEventDestroy(p.done);
    for (int i = 0; i < EV_COUNT; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    for (auto &e : ctx->temporal.ev)
        if (e) cudaEventDestroy(e);
    auto &B = ctx->batch;
    DevBuf *bb[] = {&B.rect, &B.views, &B.rec, &B.meta, &B.geo, &B.aux, &B.col, &B.scratch, &B.ranges, &B.order,
                    &B.queue, &B.keys, &B.vals, &B.akeys, &B.avals, &B.sort, &B.d_rec, &B.bviews, &B.rts};
    for (DevBuf *b : bb)
        if (b->ptr) cudaFree(b->ptr);
    if (B.exec) cudaGraphExecDestroy(B.exec);
    if (B.capture) cudaStreamDestroy(B.capture);
    if (B.h_views) cudaFreeHost(B.h_views);
    delete ctx;
}

const char *gs_last_error(const gs_context *ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

gs_status gs_sync_status(gs_context *ctx, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess && e != cudaErrorNotReady) return cuda_fail(ctx, e, "pending CUDA error");
    gs_status st = drain_deferred(ctx, true, s);
    if (st != GS_OK) return st;
    return collect_device_error(ctx, s);
}

size_t gs_workspace_bytes(const gs_context *ctx) {
    if (!ctx) return 0;
    const DevBuf *bufs[] = {&ctx->records, &ctx->tiles, &ctx->offsets, &ctx->scan_scratch, &ctx->keys,
                            &ctx->values, &ctx->alt_keys, &ctx->alt_values, &ctx->sort_scratch,
                            &ctx->ranges, &ctx->fused_scratch, &ctx->d_rec, &ctx->br_geo, &ctx->br_aux, &ctx->br_col,
                            &ctx->gathered, &ctx->rts_scratch, &ctx->br_rect, &ctx->tile_order};
    size_t t = 0;
    for (const DevBuf *b : bufs) t += b->bytes;
    return t;
}

gs_status gs_project(gs_context *ctx, const gs_gaussians *g, const gs_camera *cam,
                     const gs_options *opts, gs_record *records, uint32_t *tiles, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    gs_status st;
    if ((st = check_gaussians(ctx, g)) != GS_OK || (st = check_camera(ctx, cam)) != GS_OK ||
        (st = check_options(ctx, opts)) != GS_OK)
        return st;
    if (g->n > 0 && (!records || !tiles))
        return fail(ctx, GS_ERR_INVALID_ARG, "records/tiles are NULL");
    if (reinterpret_cast<uintptr_t>(records) % 16 != 0)
        return fail(ctx, GS_ERR_INVALID_ARG, "records must be 16-byte aligned");
    if (list_shape(opts) > 1)
        return fail(ctx, GS_ERR_UNSUPPORTED, "thread-block clusters and list tiles are gs_render options");
    DeviceGuard dg(ctx->device);
    GS_CUDA(ctx, gs_launch_project(*g, make_cam(cam), make_grid(cam, opts), records, tiles,
                                   static_cast<cudaStream_t>(stream)));
    return GS_OK;
}

gs_status gs_bin(gs_context *ctx, const gs_record *records, const uint32_t *tiles, int64_t n,
                 const gs_camera *cam, const gs_options *opts, uint64_t *keys, uint32_t *values,
                 int64_t capacity, uint32_t *ranges, int64_t *n_keys, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    gs_status st;
    if ((st = check_camera(ctx, cam)) != GS_OK || (st = check_options(ctx, opts)) != GS_OK) return st;
    if (!n_keys || !ranges || n < 0 || n >= (int64_t(1) << 31) || capacity < 0)
        return fail(ctx, GS_ERR_INVALID_ARG, "bad n, capacity, ranges or n_keys");
    if (n > 0 && (!records || !tiles)) return fail(ctx, GS_ERR_INVALID_ARG, "records/tiles are NULL");
    if (capacity > 0 && (!keys || !values)) return fail(ctx, GS_ERR_INVALID_ARG, "keys/values are NULL");
    if (reinterpret_cast<uintptr_t>(records) % 16 != 0)
        return fail(ctx, GS_ERR_INVALID_ARG, "records must be 16-byte aligned");
    if (list_shape(opts) > 1)
        return fail(ctx, GS_ERR_UNSUPPORTED, "thread-block clusters and list tiles are gs_render options");
    DeviceGuard dg(ctx->device);
    *n_keys = 0;
    st = bin_impl(ctx, records, tiles, n, make_grid(cam, opts), keys, values, capacity, false, ranges,
                  n_keys, static_cast<cudaStream_t>(stream));
    return st;
}

gs_status gs_sort_pairs(gs_context *ctx, uint64_t *keys, uint32_t *values, int64_t n, int32_t key_bits,
                        void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (n < 0 || n >= (int64_t(1) << 32) - 1 || key_bits < 1 || key_bits > 64)
        return fail(ctx, GS_ERR_INVALID_ARG, "n must be in 0..2^32-2 and key_bits in 1..64");
    if (n > 0 && (!keys || !values)) return fail(ctx, GS_ERR_INVALID_ARG, "keys/values are NULL");
    if (n <= 1) return GS_OK;
    drop_temporal(ctx);
    DeviceGuard dg(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gs_status st;
    if ((st = ensure(ctx, ctx->alt_keys, (size_t)n * 8, "alt keys")) != GS_OK) return st;
    if ((st = ensure(ctx, ctx->alt_values, (size_t)n * 4, "alt values")) != GS_OK) return st;
    if ((st = ensure(ctx, ctx->sort_scratch, gs_sort_scratch_bytes(n, key_bits), "sort scratch")) != GS_OK)
        return st;
    bool in_alt = false;
    GS_CUDA(ctx, gs_launch_sort(keys, values, static_cast<uint64_t *>(ctx->alt_keys.ptr),
                                static_cast<uint32_t *>(ctx->alt_values.ptr), n, key_bits,
                                ctx->sort_scratch.ptr, ctx->d_err, &in_alt, s));
    if (in_alt) {
        GS_CUDA(ctx, cudaMemcpyAsync(keys, ctx->alt_keys.ptr, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
        GS_CUDA(ctx, cudaMemcpyAsync(values, ctx->alt_values.ptr, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    }
    return GS_OK;
}

gs_status gs_tile_ranges(gs_context *ctx, const uint64_t *keys, int64_t n, int32_t n_tiles,
                         uint32_t *ranges, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (n < 0 || n >= (int64_t(1) << 32) - 1 || n_tiles < 1 || !ranges || (n > 0 && !keys))
        return fail(ctx, GS_ERR_INVALID_ARG, "bad keys, n, n_tiles or ranges");
    DeviceGuard dg(ctx->device);
    GS_CUDA(ctx, gs_launch_ranges(keys, n, n_tiles, ranges, ctx->d_err, static_cast<cudaStream_t>(stream)));
    return GS_OK;
}

gs_status gs_blend(gs_context *ctx, const gs_record *records, const uint32_t *values,
                   const uint32_t *ranges, const gs_camera *cam, const gs_options *opts,
                   const gs_framebuffer *fb, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    gs_status st;
    if ((st = check_camera(ctx, cam)) != GS_OK || (st = check_options(ctx, opts)) != GS_OK) return st;
    if (!fb || !fb->rgb || !ranges) return fail(ctx, GS_ERR_INVALID_ARG, "framebuffer rgb/ranges NULL");
    if (reinterpret_cast<uintptr_t>(records) % 16 != 0)
        return fail(ctx, GS_ERR_INVALID_ARG, "records must be 16-byte aligned");
    DeviceGuard dg(ctx->device);
    if (opts->record_dtype != GS_RECORD_F32)
        return fail(ctx, GS_ERR_UNSUPPORTED, "gs_blend reads FP32 gs_records; use gs_render for F16/BF16");
    if (list_shape(opts) > 1)
        return fail(ctx, GS_ERR_UNSUPPORTED, "thread-block clusters and list tiles are gs_render options");
    GS_CUDA(ctx, gs_launch_blend(reader(ctx, records, GS_RECORD_F32, true), values, ranges, make_grid(cam, opts),
                                 cam->width, cam->height, opts->bg, *fb, opts->blend_variant,
                                 static_cast<cudaStream_t>(stream)));
    return GS_OK;
}

gs_status gs_render(gs_context *ctx, const gs_gaussians *g, const gs_camera *cam,
                    const gs_options *opts, const gs_framebuffer *fb, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    gs_status st;
    if ((st = check_gaussians(ctx, g)) != GS_OK || (st = check_camera(ctx, cam)) != GS_OK ||
        (st = check_options(ctx, opts)) != GS_OK)
        return st;
    if (!fb || !fb->rgb) return fail(ctx, GS_ERR_INVALID_ARG, "framebuffer rgb is NULL");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const GsGrid grid = make_grid(cam, opts);
    const GsCameraDev dcam = make_cam(cam);
    const int64_t n = g->n;
    const int n_tiles = grid.tiles_x * grid.tiles_y;
    const int bits = key_bits_for(n_tiles);
    // Tile keys: (row << 8 | column) for grids at most 256 tiles wide (the
    // tile sort's histograms then come from the rects and its first pass is
    // fused with the emission), else tile ids. Both orders are the tile
    // order, and both fit the same key width on grids of at most 256 x 256.
    int row_bits = 0;
    while ((1 << row_bits) < grid.tiles_y) ++row_bits;
    const bool xy_possible = grid.tiles_x <= 256;
    const int dtype = opts->record_dtype;
    if ((st = ensure(ctx, ctx->br_geo, (size_t)(n > 0 ? n : 1) * 16, "blend records")) != GS_OK ||
        (st = ensure(ctx, ctx->br_aux, (size_t)(n > 0 ? n : 1) * 16, "blend records")) != GS_OK ||
        (st = ensure(ctx, ctx->br_col, (size_t)(n > 0 ? n : 1) * 16, "blend records")) != GS_OK ||
        (opts->list_tiles > 1 &&
         (st = ensure(ctx, ctx->br_rect, (size_t)(n > 0 ? n : 1) * 8, "blend record rects")) != GS_OK))
        return st;
    if ((st = ensure(ctx, ctx->records, (size_t)(n > 0 ? n : 1) * sizeof(gs_record), "records")) != GS_OK ||
        (st = ensure(ctx, ctx->ranges, (size_t)n_tiles * 8, "ranges")) != GS_OK ||
        (st = ensure(ctx, ctx->tile_order, (size_t)n_tiles * 4 + 4, "tile order")) != GS_OK)
        return st;
    const bool deferred = opts->sync_mode == GS_SYNC_DEFERRED;
    // Earlier deferred frames: all of them before a synchronised frame, the
    // finished ones otherwise (and the oldest if the ring is full).
    if ((st = drain_deferred(ctx, !deferred, s)) != GS_OK) return st;
    if (deferred && ctx->ring_count == gs_context::kRing) {
        bool retired = false;
        if ((st = retire_oldest(ctx, true, s, &retired)) != GS_OK) return st;
    }
    if (ctx->key_capacity == 0) ctx->key_capacity = std::max<int64_t>(int64_t(1) << 20, 2 * n);
    gs_record *rec = static_cast<gs_record *>(ctx->records.ptr);
    uint32_t *ranges = static_cast<uint32_t *>(ctx->ranges.ptr);
    auto &T = ctx->temporal;
    // temporal: the frame is rendered in temporal mode; track: it also
    // writes and compares tile rects (not during an adaptive cool-down).
    const bool temporal = opts->temporal != 0;
    bool track = temporal;
    if (temporal && opts->temporal == 1 && T.cooldown > 0) {
        --T.cooldown;
        track = false;
    }
    if (!track) {
        T.valid = false;
        T.rects_n = -1;
    } else {
        if (T.valid && (T.n != n || T.tiles_x != grid.tiles_x || T.tiles_y != grid.tiles_y ||
                        T.tw != grid.tile_w || T.th != grid.tile_h))
            T.valid = false;
        for (int k = 0; k < 2; ++k)
            if (!T.ev[k]) GS_CUDA(ctx, cudaEventCreate(&T.ev[k]));
        if (T.valid && T.last_churn <= kTemporalMaxChurn && n > 0) {
            if (temporal_rebin_now(ctx, opts->temporal)) {
                bool done = false;
                if ((st = render_rebinned(ctx, g, cam, opts, fb, s, &done)) != GS_OK) return st;
                if (done) return GS_OK;
            } else {
                // The gate chose the full binning: cool down, and let the
                // gate re-bin the first frame it is asked about afterwards.
                T.cooldown = kTemporalCooldown;
                T.gate = 7;
            }
        }
        if ((st = ensure(ctx, T.rects[0], (size_t)(n > 0 ? n : 1) * 8, "temporal rects")) != GS_OK ||
            (st = ensure(ctx, T.rects[1], (size_t)(n > 0 ? n : 1) * 8, "temporal rects")) != GS_OK)
            return st;
    }
    // A full frame with temporal re-binning on writes this frame's rects next
    // to the previous frame's (if that frame had the same Gaussians and tile
    // grid) and counts the rects that changed: the churn that decides how the
    // next frame is binned.
    const bool have_prev_rects = track && T.rects_n == n && T.tiles_x == grid.tiles_x &&
                                 T.tiles_y == grid.tiles_y && T.tw == grid.tile_w && T.th == grid.tile_h;
    uint2 *prect = track ? static_cast<uint2 *>(T.rects[T.rcur ^ (have_prev_rects ? 1 : 0)].ptr) : nullptr;
    const uint2 *prev_rect = have_prev_rects ? static_cast<const uint2 *>(T.rects[T.rcur].ptr) : nullptr;

    // The key buffers are sized from earlier frames; if this frame needs more,
    // the overflow is detected at the end and the frame is rendered again.
    for (int attempt = 0; attempt < 3; ++attempt) {
        const int64_t cap = ctx->key_capacity;
        // Long lists sort their tile keys with reduce-then-scan passes (no
        // look-back chains) after a plain emission of tile ids; short ones
        // with onesweep passes, the first fused with the emission.
        const bool rts = cap >= kRtsMinPairs;
        const bool xy_keys = xy_possible && !rts;
        const int tkey_bits = xy_keys ? 8 + row_bits : bits - 32;
        const int tile_passes = (tkey_bits + 7) / 8;
        const int sort_passes = tile_passes > 0 ? tile_passes : 1;
        const int key_bytes = tkey_bits <= 16 ? 2 : 4;
        const int64_t status_cap = rts ? 1 : cap;  // onesweep look-back words (none with rts)
        if ((st = ensure(ctx, ctx->keys, (size_t)cap * key_bytes, "keys")) != GS_OK ||
            (st = ensure(ctx, ctx->values, (size_t)cap * 4, "values")) != GS_OK ||
            (st = ensure(ctx, ctx->alt_keys, (size_t)cap * key_bytes, "alt keys")) != GS_OK ||
            (st = ensure(ctx, ctx->alt_values, (size_t)cap * 4, "alt values")) != GS_OK ||
            (st = ensure(ctx, ctx->sort_scratch, gs_sort_scratch_bytes_digits(status_cap, sort_passes),
                         "sort scratch")) != GS_OK ||
            (rts && (st = ensure(ctx, ctx->rts_scratch, gs_sort_rts_scratch_bytes(cap), "sort scratch")) != GS_OK) ||
            (st = ensure(ctx, ctx->fused_scratch, gs_fused_scratch_bytes(n, cap), "front-end scratch")) != GS_OK)
            return st;
        void *keys = ctx->keys.ptr, *akeys = ctx->alt_keys.ptr;
        uint32_t *vals = static_cast<uint32_t *>(ctx->values.ptr);
        uint32_t *avals = static_cast<uint32_t *>(ctx->alt_values.ptr);
        // The frame's launches, from the tile sort's scratch reset to the
        // blend, on stream q: enqueued directly, or captured once into a CUDA
        // graph that later frames replay with their own camera.
        uint32_t *sv = nullptr;
        auto enqueue = [&](cudaStream_t q) -> gs_status {
            // The tile sort: keys are tile ids emitted in (depth, index)
            // order, so the stable sort on them alone gives each tile's list
            // in order. Its digit histograms are counted from the tile rects
            // during the projection, and its first pass is fused with the
            // emission (whose output lands in the alternate buffers); at
            // least one pass runs.
            GS_CUDA(ctx, cudaMemsetAsync(ctx->sort_scratch.ptr, 0, gs_sort_scratch_bytes_digits(status_cap, sort_passes),
                                         q));
            GsSortScratch sc = gs_sort_carve_digits(ctx->sort_scratch.ptr, status_cap, 0, sort_passes);
            // The row digit takes many values within a warp; so does the high
            // byte of tile ids once the low byte is sorted.
            sc.diverse_last = xy_keys || rts;
            mark(ctx, EV_START, q);
            if (track) temporal_mark(ctx, 0, q);
            cudaEvent_t ev3[3] = {nullptr, nullptr, nullptr};
            if (ctx->timing) {
                ev3[0] = ctx->ev[EV_PROJECT];
                ev3[1] = ctx->ev[EV_DEPTH];
                ev3[2] = ctx->ev[EV_SCAN];
            }
            GS_CUDA(ctx, gs_launch_project_bin(*g, dcam, grid, rec, blend_out(ctx, dtype, opts->list_tiles > 1 ? cam : nullptr),
                                               xy_keys ? akeys : keys, key_bytes, xy_keys, xy_keys ? avals : vals,
                                               cap, ctx->d_counts,
                                               ctx->fused_scratch.ptr, sc, ctx->d_err, q, ev3, prect, prev_rect,
                                               ctx->d_counts + 4));
            mark(ctx, EV_EMIT, q);
            // The remaining passes, from the emission's output (the alternate
            // buffers after the fused first pass, else keys / vals).
            void *in_k = xy_keys ? akeys : keys, *out_k = xy_keys ? keys : akeys;
            uint32_t *in_v = xy_keys ? avals : vals, *out_v = xy_keys ? vals : avals;
            const int first_pass = xy_keys ? 1 : 0;
            bool moved = false;
            if (rts && key_bytes == 2)
                GS_CUDA(ctx, gs_launch_sort_passes_rts(static_cast<uint16_t *>(in_k), in_v, static_cast<uint16_t *>(out_k),
                                                       out_v, cap, ctx->d_counts + 2, sc, ctx->rts_scratch.ptr,
                                                       ctx->d_err, &moved, q, first_pass));
            else if (rts)
                GS_CUDA(ctx, gs_launch_sort_passes_rts(static_cast<uint32_t *>(in_k), in_v, static_cast<uint32_t *>(out_k),
                                                       out_v, cap, ctx->d_counts + 2, sc, ctx->rts_scratch.ptr,
                                                       ctx->d_err, &moved, q, first_pass));
            else if (key_bytes == 2)
                GS_CUDA(ctx, gs_launch_sort_passes(static_cast<uint16_t *>(in_k), in_v, static_cast<uint16_t *>(out_k),
                                                   out_v, cap, ctx->d_counts + 2, sc, ctx->d_err, &moved, q,
                                                   gs::kSpinTimeoutNs, 64, first_pass));
            else
                GS_CUDA(ctx, gs_launch_sort_passes(static_cast<uint32_t *>(in_k), in_v, static_cast<uint32_t *>(out_k),
                                                   out_v, cap, ctx->d_counts + 2, sc, ctx->d_err, &moved, q,
                                                   gs::kSpinTimeoutNs, 64, first_pass));
            mark(ctx, EV_SORT, q);
            const void *sk = moved ? out_k : in_k;
            sv = moved ? out_v : in_v;
            GS_CUDA(ctx, gs_launch_ranges_tiles(sk, key_bytes, cap, ctx->d_counts + 2, n_tiles, ranges, ctx->d_err, q,
                                                xy_keys ? grid.tiles_x : 0));
            // (The temporal binning time ends with the ranges, as that of a
            // re-binned frame does.)
            if (track) temporal_mark(ctx, 1, q);
            const uint32_t *order = nullptr;
            gs_status st;
            if ((st = launch_tile_order(ctx, ranges, grid, opts, q, &order)) != GS_OK) return st;
            mark(ctx, EV_RANGES, q);
            if ((st = launch_blend(ctx, reader(ctx, rec, dtype), sv, ranges, grid, cam, opts, fb, ctx->d_counts + 2,
                                   cap, order, q)) != GS_OK)
                return st;
            return GS_OK;
        };
        const int variant = blend_schedule(ctx, opts, n_tiles);
        if (!ctx->timing && opts->direct_launch == 0 && variant != GS_BLEND_TMA) {
            // With tile rects tracked, the temporal gate times the whole
            // graph (binning and blend) of both kinds of frames.
            const void *extra[8] = {prect, prev_rect};
            if (track) temporal_mark(ctx, 0, s);
            if ((st = replay_frame(ctx, 0, extra, g, cam, opts, fb, cap, variant, dcam, s, enqueue, &sv)) != GS_OK)
                return st;
            if (track) temporal_mark(ctx, 1, s);
        } else if ((st = enqueue(s)) != GS_OK) {
            return st;
        }
        mark(ctx, EV_BLEND, s);
        if (deferred) {
            const int slot = (ctx->ring_head + ctx->ring_count) % gs_context::kRing;
            unsigned long long *h = ctx->h_ring + 5 * slot;
            h[4] = 0;
            GS_CUDA(ctx, cudaMemcpyAsync(h, ctx->d_counts, 4 * sizeof(unsigned long long),
                                         cudaMemcpyDeviceToHost, s));
            GS_CUDA(ctx, cudaMemcpyAsync(h + 4, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            gs_context::Pending &p = ctx->ring[slot];
            GS_CUDA(ctx, cudaEventRecord(p.done, s));
            p.seq = ctx->next_seq++;
            p.cap = cap;
            p.n_tiles = n_tiles;
            p.bits = bits;
            ++ctx->ring_count;
            if (ctx->timing) ctx->timed_once = true;
            remember_frame(ctx, g, cam, opts, grid, sv, ranges, p.seq);
            return GS_OK;
        }
        GS_CUDA(ctx, cudaMemcpyAsync(ctx->h_counts, ctx->d_counts, 5 * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, s));
        GS_CUDA(ctx, cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        GS_CUDA(ctx, cudaStreamSynchronize(s));
        const unsigned long long K = ctx->h_counts[0];
        ctx->stats.n_visible = (int64_t)ctx->h_counts[1];
        ctx->stats.n_keys = (int64_t)K;
        ctx->stats.n_tiles = n_tiles;
        ctx->stats.key_bits = bits;
        if (K >= (1ull << 32) - 1)
            return fail(ctx, GS_ERR_CAPACITY, "more than 2^32-2 (tile, Gaussian) pairs in one frame");
        if ((int64_t)K > cap) {
            // Overflow: nothing past the buffers was written and the frame
            // composited empty lists; grow and render again.
            GS_CUDA(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), s));
            ctx->key_capacity = (int64_t)(K + K / 4 + 1024);
            continue;
        }
        if (ctx->timing) ctx->timed_once = true;
        remember_frame(ctx, g, cam, opts, grid, sv, ranges, 0);
        ctx->stats.n_moved = have_prev_rects ? (int64_t)ctx->h_counts[4] : 0;
        ctx->stats.rebinned = 0;
        if (track) {
            T.valid = true;
            T.n = n;
            T.tiles_x = grid.tiles_x;
            T.tiles_y = grid.tiles_y;
            T.tw = grid.tile_w;
            T.th = grid.tile_h;
            T.prev_vals = sv;
            T.prev_ranges = ranges;
            T.cur = 0;
            if (have_prev_rects) T.rcur ^= 1;
            T.rects_n = n;
            // Churn unknown (no earlier rects): temporal = 2 tries
            // re-binning on the next frame; temporal = 1 first measures the
            // churn on a full binning (a fast camera would make a re-binned
            // frame cost more than the full binning saves).
            T.last_churn = have_prev_rects && ctx->stats.n_visible > 0
                               ? (double)ctx->h_counts[4] / (double)ctx->stats.n_visible
                           : (!have_prev_rects && opts->temporal == 1) ? 1.0
                                                                       : 0.0;
            // Only frames that compared rects with a previous frame's are
            // the full-binning side of the gate's comparison.
            if (have_prev_rects) temporal_sample(ctx, false);
            if (opts->temporal == 1 && have_prev_rects && T.last_churn > kTemporalMaxChurn)
                T.cooldown = kTemporalCooldown;
        }
        // The sort grids cover the capacity: when it is far above this frame's
        // count, bring it down to twice the count (the buffers themselves only
        // grow). A smaller margin would make the next frame of a larger view
        // overflow, which deferred frames report as an error.
        if (!temporal && !ctx->pinned_capacity && (int64_t)K * 3 < cap)
            ctx->key_capacity = std::max<int64_t>(65536, (int64_t)(2 * K + 1024));
        if (*ctx->h_err) return collect_device_error(ctx, s);
        return GS_OK;
    }
    return fail(ctx, GS_ERR_CAPACITY, "key buffers could not be sized for this frame");
}

gs_status gs_render_backward(gs_context *ctx, const gs_gaussians *g, const gs_camera *cam,
                             const gs_options *opts, const gs_framebuffer *fb, const float *d_rgb,
                             const gs_grads *out, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    gs_status st;
    if ((st = check_gaussians(ctx, g)) != GS_OK || (st = check_camera(ctx, cam)) != GS_OK ||
        (st = check_options(ctx, opts)) != GS_OK)
        return st;
    if (!fb || !fb->final_T || !fb->n_contrib || !d_rgb || !out)
        return fail(ctx, GS_ERR_INVALID_ARG, "final_T, n_contrib, d_rgb and the gradient struct are required");
    if (g->n > 0 && (!out->d_means || !out->d_log_scales || !out->d_quats || !out->d_opacity_logits || !out->d_sh))
        return fail(ctx, GS_ERR_INVALID_ARG, "a gradient array is NULL");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // A deferred forward frame must have fitted its key buffers.
    while (ctx->last_seq != 0 && ctx->ring_count > 0 && ctx->ring[ctx->ring_head].seq <= ctx->last_seq) {
        bool retired = false;
        if ((st = retire_oldest(ctx, true, s, &retired)) != GS_OK) return st;
    }
    if (!ctx->have_last)
        return fail(ctx, GS_ERR_INVALID_ARG, "gs_render_backward needs a completed gs_render on this context");
    if (!same_frame(ctx, g, cam, opts))
        return fail(ctx, GS_ERR_INVALID_ARG,
                    "gs_render_backward must follow gs_render of the same scene arrays, camera and options: the "
                    "context's last frame (number " + std::to_string(ctx->frame_id) + ") differs");
    const GsGrid grid = make_grid(cam, opts);
    const int64_t n = g->n;
    if ((st = ensure(ctx, ctx->d_rec, (size_t)(n > 0 ? n : 1) * kRecGradStride * sizeof(float),
                     "record gradients")) != GS_OK)
        return st;
    float *d_rec = static_cast<float *>(ctx->d_rec.ptr);
    GS_CUDA(ctx, gs_launch_zero_grads(*g, *out, d_rec, (size_t)n * kRecGradStride, s));
    GS_CUDA(ctx, gs_launch_blend_bwd(reader(ctx, static_cast<gs_record *>(ctx->records.ptr), ctx->last_dtype),
                                     ctx->last_values, ctx->last_ranges, grid, cam->width, cam->height,
                                     opts->bg, d_rgb, fb->final_T, fb->n_contrib, d_rec, s, ctx->last_cluster));
    GS_CUDA(ctx, gs_launch_project_bwd(*g, make_cam(cam), grid, d_rec, *out, s));
    if (out->d_records && n > 0)
        GS_CUDA(ctx, cudaMemcpy2DAsync(out->d_records, 9 * sizeof(float), d_rec, kRecGradStride * sizeof(float),
                                       9 * sizeof(float), (size_t)n, cudaMemcpyDeviceToDevice, s));
    return GS_OK;
}

namespace {

// Enqueues one whole batched frame on s (also used under stream capture).
gs_status enqueue_batch(gs_context *ctx, const gs_gaussians *g, int n_views, const gs_options *opts,
                        int32_t total_tiles, int bits, cudaStream_t s) {
    auto &B = ctx->batch;
    const int dtype = opts->record_dtype;
    const ViewDesc *views = static_cast<const ViewDesc *>(B.views.ptr);
    GS_CUDA(ctx, cudaMemcpyAsync(B.views.ptr, B.h_views, (size_t)n_views * sizeof(ViewDesc),
                                 cudaMemcpyHostToDevice, s));
    // The tile sort: 32-bit global tile ids emitted in (depth, view, index)
    // order, so the stable sort on them alone orders every tile's list.
    // Long key lists sort with reduce-then-scan passes (no look-back words).
    const int tile_passes = (bits - 32 + 7) / 8;
    const bool rts = B.key_cap >= kRtsMinPairs;
    const int64_t status_cap = rts ? 1 : B.key_cap;
    GS_CUDA(ctx, cudaMemsetAsync(B.sort.ptr, 0, gs_sort_scratch_bytes_digits(status_cap, tile_passes), s));
    const GsSortScratch sc = gs_sort_carve_digits(B.sort.ptr, status_cap, 0, tile_passes);
    uint32_t *keys = static_cast<uint32_t *>(B.keys.ptr), *akeys = static_cast<uint32_t *>(B.akeys.ptr);
    uint32_t *vals = static_cast<uint32_t *>(B.vals.ptr), *avals = static_cast<uint32_t *>(B.avals.ptr);
    uint2 *meta = static_cast<uint2 *>(B.meta.ptr);
    const int lists = opts->list_tiles > 1 ? opts->list_tiles : 1;
    int lx = 1, ly = 1;
    list_tile_dims(lists, &lx, &ly);
    gs::BlendRecordOut bro{static_cast<float4 *>(B.geo.ptr), static_cast<float4 *>(B.aux.ptr), B.col.ptr,
                           rec_mode(dtype), lists > 1 ? static_cast<uint2 *>(B.rect.ptr) : nullptr};
    GS_CUDA(ctx, gs_launch_project_bin_batch(*g, views, n_views, static_cast<gs_record *>(B.rec.ptr), bro, meta,
                                             B.rec_cap, keys,
                                             vals, B.key_cap, ctx->d_counts, B.scratch.ptr, sc, ctx->d_err, s));
    bool in_alt = false;
    if (rts)
        GS_CUDA(ctx, gs_launch_sort_passes_rts(keys, vals, akeys, avals, B.key_cap, ctx->d_counts + 2, sc, B.rts.ptr,
                                               ctx->d_err, &in_alt, s));
    else
        GS_CUDA(ctx, gs_launch_sort_passes(keys, vals, akeys, avals, B.key_cap, ctx->d_counts + 2, sc, ctx->d_err,
                                           &in_alt, s));
    const uint32_t *sk = in_alt ? akeys : keys;
    uint32_t *sv = in_alt ? avals : vals;
    B.joint_values = sv;
    uint32_t *ranges = static_cast<uint32_t *>(B.ranges.ptr);
    GS_CUDA(ctx, gs_launch_ranges_tiles(sk, 4, B.key_cap, ctx->d_counts + 2, total_tiles, ranges, ctx->d_err, s));
    uint32_t *qs = static_cast<uint32_t *>(B.queue.ptr);
    uint32_t *order = static_cast<uint32_t *>(B.order.ptr);
    // With list tiles, one queue item per (list tile, screen tile of it).
    GS_CUDA(ctx, gs_launch_queue(ranges, total_tiles, qs, order, s, lx * ly));
    const RecordReader rd = batch_reader(ctx, dtype);
    GS_CUDA(ctx, gs_launch_blend_batch(rd, sv, ranges, views, n_views, opts->tile_w, opts->tile_h,
                                       opts->batch_depth ? opts->batch_depth : 256, order,
                                       (int32_t)(total_tiles * lx * ly), qs + 193, lists, s));
    GS_CUDA(ctx, cudaMemcpyAsync(ctx->h_counts, ctx->d_counts, 4 * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, s));
    GS_CUDA(ctx, cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    return GS_OK;
}

}  // namespace

gs_status gs_render_batch(gs_context *ctx, const gs_gaussians *g, const gs_camera *cams, int32_t n_views,
                          const gs_options *opts, const gs_framebuffer *fbs, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    gs_status st;
    if ((st = check_gaussians(ctx, g)) != GS_OK || (st = check_options(ctx, opts)) != GS_OK) return st;
    if (n_views < 1 || n_views > 4096 || !cams || !fbs)
        return fail(ctx, GS_ERR_INVALID_ARG, "n_views must be in 1..4096 with cameras and framebuffers");
    for (int v = 0; v < n_views; ++v) {
        if ((st = check_camera(ctx, &cams[v])) != GS_OK) return st;
        if (!fbs[v].rgb) return fail(ctx, GS_ERR_INVALID_ARG, "a framebuffer rgb is NULL");
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto &B = ctx->batch;
    const int64_t n = g->n;
    // Thread-block clusters are a property of the single-view blend: such a
    // batch renders view by view (list tiles render jointly as well).
    const bool per_view = opts->batch_mode == GS_BATCH_PER_VIEW || opts->cluster > 1 ||
                          (opts->batch_mode == GS_BATCH_AUTO && B.keys_per_view > kBatchPerViewKeys);
    B.have_joint = false;
    if (per_view) {
        gs_options o = *opts;
        o.sync_mode = GS_SYNC_FRAME;
        o.temporal = 0;
        o.batch_mode = GS_BATCH_AUTO;
        // Each view has its own framebuffer: more views than the context
        // keeps frame graphs would capture every frame, so they launch
        // directly.
        if (n_views > gs_context::kGraphs) o.direct_launch = 1;
        int64_t keys = 0, visible = 0, tiles = 0;
        for (int v = 0; v < n_views; ++v) {
            if ((st = gs_render(ctx, g, &cams[v], &o, &fbs[v], stream)) != GS_OK) return st;
            keys += ctx->stats.n_keys;
            visible += ctx->stats.n_visible;
            tiles += ctx->stats.n_tiles;
        }
        ctx->stats.n_keys = keys;
        ctx->stats.n_visible = visible;
        ctx->stats.n_tiles = (int32_t)tiles;
        B.keys_per_view = keys / n_views;
        return GS_OK;
    }
    // Host view table (pinned, read by the frame's first copy).
    if (B.h_views_cap < n_views) {
        if (B.h_views) cudaFreeHost(B.h_views);
        B.h_views = nullptr;
        B.h_views_cap = 0;
        if (cudaMallocHost(&B.h_views, (size_t)n_views * sizeof(ViewDesc)) != cudaSuccess)
            return fail(ctx, GS_ERR_OOM, "cannot allocate the pinned view table");
        B.h_views_cap = n_views;
        if (B.exec) { cudaGraphExecDestroy(B.exec); B.exec = nullptr; }
    }
    int64_t total_tiles = 0;
    std::vector<int64_t> sig = {n, g->sh_degree, (int64_t)(uintptr_t)g->means, (int64_t)(uintptr_t)g->log_scales,
                                (int64_t)(uintptr_t)g->quats, (int64_t)(uintptr_t)g->opacity_logits,
                                (int64_t)(uintptr_t)g->sh, n_views, opts->tile_w, opts->tile_h,
                                opts->record_dtype, opts->batch_depth, opts->list_tiles};
    for (int v = 0; v < n_views; ++v) {
        ViewDesc &V = B.h_views[v];
        V.cam = make_cam(&cams[v]);
        V.grid = make_grid(&cams[v], opts);
        V.tile_base = (uint32_t)total_tiles;
        for (int c = 0; c < 3; ++c) V.bg[c] = opts->bg[c];
        V.rgb = fbs[v].rgb;
        V.final_T = fbs[v].final_T;
        V.n_contrib = fbs[v].n_contrib;
        V.n_eval = fbs[v].n_eval;
        total_tiles += (int64_t)V.grid.tiles_x * V.grid.tiles_y;
        sig.push_back(cams[v].width);
        sig.push_back(cams[v].height);
    }
    {
        int lx = 1, ly = 1;
        list_tile_dims(opts->list_tiles > 1 ? opts->list_tiles : 1, &lx, &ly);
        if (total_tiles * lx * ly >= (int64_t(1) << 31))
            return fail(ctx, GS_ERR_INVALID_ARG, "too many tiles in one batch");
    }
    const int bits = key_bits_for((int)total_tiles);
    if (B.rec_cap == 0) B.rec_cap = std::max<int64_t>(int64_t(1) << 20, n * n_views / 8);
    if (B.key_cap == 0) B.key_cap = std::max<int64_t>(int64_t(1) << 22, 4 * B.rec_cap);
    for (int attempt = 0; attempt < 3; ++attempt) {
        const int64_t rc = B.rec_cap, kc = B.key_cap;
        void *before[] = {B.views.ptr, B.rec.ptr, B.meta.ptr, B.geo.ptr, B.aux.ptr, B.col.ptr, B.scratch.ptr,
                          B.ranges.ptr, B.order.ptr, B.queue.ptr, B.keys.ptr, B.vals.ptr, B.akeys.ptr,
                          B.avals.ptr, B.sort.ptr, B.rts.ptr, B.rect.ptr};
        int qlx = 1, qly = 1;  // queue items per global tile
        list_tile_dims(opts->list_tiles > 1 ? opts->list_tiles : 1, &qlx, &qly);
        if ((st = ensure(ctx, B.views, (size_t)n_views * sizeof(ViewDesc), "view table")) != GS_OK ||
            (st = ensure(ctx, B.rec, (size_t)rc * sizeof(gs_record), "batch records")) != GS_OK ||
            (st = ensure(ctx, B.meta, (size_t)rc * 8, "batch record meta")) != GS_OK ||
            (st = ensure(ctx, B.geo, (size_t)rc * 16, "batch blend records")) != GS_OK ||
            (st = ensure(ctx, B.aux, (size_t)rc * 16, "batch blend records")) != GS_OK ||
            (st = ensure(ctx, B.col, (size_t)rc * 16, "batch blend records")) != GS_OK ||
            (st = ensure(ctx, B.scratch, gs_batch_scratch_bytes(rc, kc, n, n_views), "batch scratch")) != GS_OK ||
            (st = ensure(ctx, B.ranges, (size_t)total_tiles * 8, "batch ranges")) != GS_OK ||
            (st = ensure(ctx, B.order, (size_t)total_tiles * qlx * qly * 4, "batch queue")) != GS_OK ||
            (opts->list_tiles > 1 && (st = ensure(ctx, B.rect, (size_t)rc * 8, "batch record rects")) != GS_OK) ||
            (st = ensure(ctx, B.queue, gs_queue_scratch_bytes(), "batch queue")) != GS_OK ||
            (st = ensure(ctx, B.keys, (size_t)kc * 4, "batch keys")) != GS_OK ||
            (st = ensure(ctx, B.vals, (size_t)kc * 4, "batch values")) != GS_OK ||
            (st = ensure(ctx, B.akeys, (size_t)kc * 4, "batch keys")) != GS_OK ||
            (st = ensure(ctx, B.avals, (size_t)kc * 4, "batch values")) != GS_OK ||
            (st = ensure(ctx, B.sort,
                         gs_sort_scratch_bytes_digits(kc >= kRtsMinPairs ? 1 : kc, (bits - 32 + 7) / 8),
                         "batch sort scratch")) != GS_OK ||
            (kc >= kRtsMinPairs &&
             (st = ensure(ctx, B.rts, gs_sort_rts_scratch_bytes(kc), "batch sort scratch")) != GS_OK))
            return st;
        void *after[] = {B.views.ptr, B.rec.ptr, B.meta.ptr, B.geo.ptr, B.aux.ptr, B.col.ptr, B.scratch.ptr,
                         B.ranges.ptr, B.order.ptr, B.queue.ptr, B.keys.ptr, B.vals.ptr, B.akeys.ptr,
                         B.avals.ptr, B.sort.ptr, B.rts.ptr, B.rect.ptr};
        std::vector<int64_t> full = sig;
        full.push_back(rc);
        full.push_back(kc);
        bool moved = false;
        for (size_t k = 0; k < sizeof(before) / sizeof(before[0]); ++k) moved |= before[k] != after[k];
        if (moved || full != B.sig) {
            if (B.exec) { cudaGraphExecDestroy(B.exec); B.exec = nullptr; }
        }
        if (opts->direct_launch == 0) {  // graph path (default)
            if (!B.exec) {
                if (!B.capture) GS_CUDA(ctx, cudaStreamCreateWithFlags(&B.capture, cudaStreamNonBlocking));
                // Work already queued on the caller's stream comes first.
                GS_CUDA(ctx, cudaStreamSynchronize(s));
                cudaGraph_t graph = nullptr;
                GS_CUDA(ctx, cudaStreamBeginCapture(B.capture, cudaStreamCaptureModeThreadLocal));
                st = enqueue_batch(ctx, g, n_views, opts, (int32_t)total_tiles, bits, B.capture);
                const cudaError_t ec = cudaStreamEndCapture(B.capture, &graph);
                if (st != GS_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return st;
                }
                if (ec != cudaSuccess) return cuda_fail(ctx, ec, "cudaStreamEndCapture");
                const cudaError_t ei = cudaGraphInstantiate(&B.exec, graph, 0);
                cudaGraphDestroy(graph);
                if (ei != cudaSuccess) return cuda_fail(ctx, ei, "cudaGraphInstantiate");
                B.sig = full;
            }
            GS_CUDA(ctx, cudaGraphLaunch(B.exec, s));
        } else {
            if ((st = enqueue_batch(ctx, g, n_views, opts, (int32_t)total_tiles, bits, s)) != GS_OK) return st;
        }
        GS_CUDA(ctx, cudaStreamSynchronize(s));
        const unsigned long long K = ctx->h_counts[0], nv = ctx->h_counts[1];
        ctx->stats.n_keys = (int64_t)K;
        ctx->stats.n_visible = (int64_t)nv;
        ctx->stats.n_tiles = (int32_t)total_tiles;
        ctx->stats.key_bits = bits;
        if (K >= (1ull << 32) - 1)
            return fail(ctx, GS_ERR_CAPACITY, "more than 2^32-2 (tile, Gaussian) pairs in one batch");
        if ((int64_t)K > kc || (int64_t)nv > rc) {
            GS_CUDA(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), s));
            if ((int64_t)K > kc) B.key_cap = (int64_t)(K + K / 4 + 4096);
            if ((int64_t)nv > rc) B.rec_cap = (int64_t)(nv + nv / 4 + 4096);
            continue;
        }
        B.keys_per_view = (int64_t)K / n_views;
        B.have_joint = true;
        B.joint_n = n;
        B.joint_records = (int64_t)nv;
        B.joint_views = n_views;
        B.joint_tw = opts->tile_w;
        B.joint_th = opts->tile_h;
        B.joint_dtype = opts->record_dtype;
        B.joint_lists = opts->list_tiles > 1 ? opts->list_tiles : 1;
        B.joint_tiles = (int32_t)total_tiles;
        if (*ctx->h_err) return collect_device_error(ctx, s);
        return GS_OK;
    }
    return fail(ctx, GS_ERR_CAPACITY, "batch buffers could not be sized");
}

gs_status gs_render_batch_backward(gs_context *ctx, const gs_gaussians *g, const gs_camera *cams, int32_t n_views,
                                   const gs_options *opts, const gs_framebuffer *fbs, const float *const *d_rgb,
                                   const gs_grads *out, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    gs_status st;
    if ((st = check_gaussians(ctx, g)) != GS_OK || (st = check_options(ctx, opts)) != GS_OK) return st;
    if (n_views < 1 || !cams || !fbs || !d_rgb || !out)
        return fail(ctx, GS_ERR_INVALID_ARG, "cameras, framebuffers, d_rgb and the gradient struct are required");
    auto &B = ctx->batch;
    if (!B.have_joint || B.joint_n != g->n || B.joint_views != n_views || B.joint_tw != opts->tile_w ||
        B.joint_th != opts->tile_h || B.joint_dtype != opts->record_dtype ||
        B.joint_lists != (opts->list_tiles > 1 ? opts->list_tiles : 1))
        return fail(ctx, GS_ERR_INVALID_ARG,
                    "gs_render_batch_backward must follow a joint gs_render_batch of the same scene, views and options");
    if (B.joint_lists > 1)
        return fail(ctx, GS_ERR_UNSUPPORTED, "gs_render_batch_backward does not take list tiles");
    if (g->n > 0 && (!out->d_means || !out->d_log_scales || !out->d_quats || !out->d_opacity_logits || !out->d_sh))
        return fail(ctx, GS_ERR_INVALID_ARG, "a gradient array is NULL");
    std::vector<GsBwdView> bv((size_t)n_views);
    for (int v = 0; v < n_views; ++v) {
        if ((st = check_camera(ctx, &cams[v])) != GS_OK) return st;
        if (!fbs[v].final_T || !fbs[v].n_contrib || !d_rgb[v])
            return fail(ctx, GS_ERR_INVALID_ARG, "every view needs final_T, n_contrib and d_rgb");
        bv[v] = GsBwdView{d_rgb[v], fbs[v].final_T, fbs[v].n_contrib};
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = g->n, nr = B.joint_records;
    if ((st = ensure(ctx, B.d_rec, (size_t)(nr > 0 ? nr : 1) * kRecGradStride * sizeof(float),
                     "batch record gradients")) !=
            GS_OK ||
        (st = ensure(ctx, B.bviews, (size_t)n_views * sizeof(GsBwdView), "batch backward views")) != GS_OK)
        return st;
    // A copy from pageable memory: the host table may be reused at once.
    GS_CUDA(ctx, cudaMemcpyAsync(B.bviews.ptr, bv.data(), bv.size() * sizeof(GsBwdView), cudaMemcpyHostToDevice, s));
    float *d_rec = static_cast<float *>(B.d_rec.ptr);
    GS_CUDA(ctx, cudaMemsetAsync(d_rec, 0, (size_t)(nr > 0 ? nr : 1) * kRecGradStride * sizeof(float), s));
    const size_t kS = (size_t)(g->sh_degree + 1) * (g->sh_degree + 1) * 3;
    if (n > 0) {
        GS_CUDA(ctx, cudaMemsetAsync(out->d_means, 0, (size_t)n * 3 * sizeof(float), s));
        GS_CUDA(ctx, cudaMemsetAsync(out->d_log_scales, 0, (size_t)n * 3 * sizeof(float), s));
        GS_CUDA(ctx, cudaMemsetAsync(out->d_quats, 0, (size_t)n * 4 * sizeof(float), s));
        GS_CUDA(ctx, cudaMemsetAsync(out->d_opacity_logits, 0, (size_t)n * sizeof(float), s));
        GS_CUDA(ctx, cudaMemsetAsync(out->d_sh, 0, (size_t)n * kS * sizeof(float), s));
    }
    const RecordReader rd = batch_reader(ctx, opts->record_dtype);
    const ViewDesc *views = static_cast<const ViewDesc *>(B.views.ptr);
    GS_CUDA(ctx, gs_launch_blend_bwd_batch(rd, B.joint_values, static_cast<const uint32_t *>(B.ranges.ptr), views,
                                           static_cast<const GsBwdView *>(B.bviews.ptr), n_views, opts->tile_w,
                                           opts->tile_h, B.joint_tiles, d_rec, s));
    GS_CUDA(ctx, gs_launch_project_bwd_batch(*g, views, static_cast<const uint2 *>(B.meta.ptr), nr, d_rec, *out, s));
    if (out->d_records && nr > 0)
        GS_CUDA(ctx, cudaMemcpy2DAsync(out->d_records, 9 * sizeof(float), d_rec, kRecGradStride * sizeof(float),
                                       9 * sizeof(float), (size_t)nr, cudaMemcpyDeviceToDevice,
                                     s));
    return GS_OK;
}

gs_status gs_autotune_batch(gs_context *ctx, const gs_gaussians *g, const gs_camera *cams, int32_t n_views,
                            gs_options *opts, const gs_framebuffer *fbs, void *stream, float *ms_out) {
    if (!ctx || !opts) return GS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Screen tile (w, h), thread-block cluster and list tiles of each candidate.
    constexpr int kShapes = 9;
    const int shapes[kShapes][4] = {{16, 16, 0, 0},
                                    {16, 8, 0, 0},
                                    {8, 8, 0, 0},
                                    {16, 16, GS_CLUSTER_2X1, 0},
                                    {16, 16, GS_CLUSTER_2X2, 0},
                                    {16, 16, 0, GS_LISTS_2X1},
                                    {16, 16, 0, GS_LISTS_2X2},
                                    {16, 16, 0, GS_LISTS_4X4},
                                    {16, 16, 0, GS_LISTS_8X8}};
    const int depths[3] = {256, 128, 64};
    cudaEvent_t e0, e1;
    GS_CUDA(ctx, cudaEventCreate(&e0));
    GS_CUDA(ctx, cudaEventCreate(&e1));
    float best = 1e30f;
    int best_k = 0, best_d = 0;
    gs_status st = GS_OK;
    for (int k = 0; k < kShapes && st == GS_OK; ++k) {
        float best_shape = 1e30f;
        for (int d = 0; d < 3 && st == GS_OK; ++d) {
            gs_options o = *opts;
            o.tile_w = shapes[k][0];
            o.tile_h = shapes[k][1];
            o.cluster = shapes[k][2];
            o.list_tiles = shapes[k][3];
            o.batch_depth = depths[d];
            for (int w = 0; w < 2 && st == GS_OK; ++w) st = gs_render_batch(ctx, g, cams, n_views, &o, fbs, stream);
            // The depth only matters to the joint schedule without list tiles.
            const bool joint = ctx->batch.have_joint && o.list_tiles <= 1;
            float total = 0.f;
            for (int r = 0; r < 3 && st == GS_OK; ++r) {
                cudaEventRecord(e0, s);
                st = gs_render_batch(ctx, g, cams, n_views, &o, fbs, stream);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                total += ms;
            }
            if (st == GS_OK && total < best_shape) best_shape = total;
            if (st == GS_OK && total < best) {
                best = total;
                best_k = k;
                best_d = d;
            }
            if (!joint) break;
        }
        if (ms_out) ms_out[k] = best_shape / 3.f;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GS_OK) return st;
    opts->tile_w = shapes[best_k][0];
    opts->tile_h = shapes[best_k][1];
    opts->cluster = shapes[best_k][2];
    opts->list_tiles = shapes[best_k][3];
    opts->batch_depth = depths[best_d];
    return GS_OK;
}

gs_status gs_selftest_bounded_wait(gs_context *ctx, int32_t kind, int64_t timeout_ns, void *stream) {
    if (!ctx || (kind != 0 && kind != 1) || timeout_ns < 1000 || timeout_ns > 5000000000ll)
        return GS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = 1 << 20;  // a few hundred blocks, all waiting on partition 0
    gs_status st;
    DevBuf buf;
    if ((st = ensure(ctx, buf, gs_selftest_scratch_bytes(n), "self-test scratch")) != GS_OK) return st;
    GS_CUDA(ctx, cudaStreamSynchronize(s));
    GS_CUDA(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), s));
    cudaError_t e = gs_launch_selftest_wait(kind, n, buf.ptr, ctx->d_err, (unsigned long long)timeout_ns, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf.ptr);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bounded-wait self-test");
    return collect_device_error(ctx, s);
}

gs_status gs_reserve_keys(gs_context *ctx, int64_t key_capacity) {
    if (!ctx || key_capacity < 1 || key_capacity >= (int64_t(1) << 32) - 1) return GS_ERR_INVALID_ARG;
    ctx->key_capacity = key_capacity;
    ctx->pinned_capacity = true;
    return GS_OK;
}

gs_status gs_set_stage_timing(gs_context *ctx, int enable) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    if (enable && !ctx->ev[0])
        for (int i = 0; i < EV_COUNT; ++i) GS_CUDA(ctx, cudaEventCreate(&ctx->ev[i]));
    ctx->timing = enable != 0;
    return GS_OK;
}

gs_status gs_last_stage_times(gs_context *ctx, gs_stage_times *out) {
    if (!ctx || !out) return GS_ERR_INVALID_ARG;
    if (!ctx->timed_once) return fail(ctx, GS_ERR_INVALID_ARG, "no timed gs_render yet");
    DeviceGuard dg(ctx->device);
    GS_CUDA(ctx, cudaEventSynchronize(ctx->ev[EV_BLEND]));
    auto el = [&](int a, int b) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev[a], ctx->ev[b]);
        return ms;
    };
    out->project_ms = el(EV_START, EV_PROJECT);
    out->depth_sort_ms = el(EV_PROJECT, EV_DEPTH);
    out->entry_scan_ms = el(EV_DEPTH, EV_SCAN);
    out->emit_ms = el(EV_SCAN, EV_EMIT);
    out->tile_sort_ms = el(EV_EMIT, EV_SORT);
    out->ranges_ms = el(EV_SORT, EV_RANGES);
    out->blend_ms = el(EV_RANGES, EV_BLEND);
    out->total_ms = el(EV_START, EV_BLEND);
    return GS_OK;
}

gs_status gs_last_frame_id(const gs_context *ctx, uint64_t *out) {
    if (!ctx || !out) return GS_ERR_INVALID_ARG;
    *out = ctx->have_last ? ctx->frame_id : 0;
    return GS_OK;
}

gs_status gs_last_render_stats(gs_context *ctx, gs_render_stats *out) {
    if (!ctx || !out) return GS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    const gs_status st = drain_deferred(ctx, true, nullptr);
    *out = ctx->stats;
    return st;
}

}  // extern "C"
