/*
 * gs.h — C ABI of the GB300 3D Gaussian Splatting forward rasterizer.
 *
 * The library renders the standard 3DGS formulation that the paper
 * re-implements on an IPU (Sec. 3.1): cull and project every Gaussian,
 * order Gaussians by depth per screen tile, and alpha-composite each pixel
 * front to back with Eq. 1. Here the per-tile depth order comes from one
 * global radix sort of 64-bit (tile id, depth) keys, as in the original GPU
 * implementation the paper describes in Sec. 3.1, and each screen tile is
 * blended by one CUDA thread block.
 *
 * Conventions for every entry point:
 *  - Every array argument is a DEVICE pointer unless its comment says "host".
 *    The caller allocates and owns all input and output buffers; the library
 *    owns only the scratch workspace inside a gs_context.
 *  - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed
 *    as void*, NULL = legacy default stream) unless their comment says they
 *    synchronise. GS_OK means "validated and launched".
 *  - Errors are returned, never thrown or aborted on. Invalid arguments are
 *    detected on the host before any launch. Errors that only the device can
 *    see (a bounded wait that gave up, a count above a buffer's capacity) set
 *    an error word in the context; gs_sync_status() reports it, and so does
 *    the next synchronising call on the same context.
 *  - A context may be used from one host thread at a time.
 *  - Layouts: Gaussians are structure-of-arrays FP32; images are row-major
 *    height x width, colour images HWC (3 floats per pixel).
 *  - Pixel (i, j) covers [i, i+1) x [j, j+1) in image coordinates and is
 *    sampled at its centre (i + 0.5, j + 0.5). Camera frame: x right,
 *    y down, z forward.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1, /* a null pointer, a size or an option out of range  */
    GS_ERR_CUDA = 2,        /* a CUDA runtime call failed; see gs_last_error()    */
    GS_ERR_OOM = 3,         /* the workspace could not grow                        */
    GS_ERR_CAPACITY = 4,    /* an output buffer is smaller than the result         */
    GS_ERR_TIMEOUT = 5,     /* a device-side bounded wait gave up                  */
    GS_ERR_UNSUPPORTED = 6  /* a valid request this build does not implement       */
} gs_status;

typedef struct gs_context gs_context;

/* The scene: n Gaussians (Sec. 3.1: mean, covariance from a rotation and a
 * diagonal scale, opacity, SH colour). All pointers are device FP32.
 *   means          n x 3 world-space means
 *   log_scales     n x 3 per-axis log standard deviations (S = diag(exp(.)))
 *   quats          n x 4 rotation quaternions (w, x, y, z); normalised inside
 *   opacity_logits n     opacity = 1 / (1 + exp(-logit))
 *   sh             n x (sh_degree+1)^2 x 3 real SH coefficients (coefficient
 *                  k = l^2 + l + m, real basis with the Condon-Shortley
 *                  phase), colour = max(0, sum_k c_k Y_k(dir) + 0.5) with
 *                  dir the unit vector from the camera centre to the mean. */
typedef struct {
    const float *means;
    const float *log_scales;
    const float *quats;
    const float *opacity_logits;
    const float *sh;
    int64_t n;         /* 0 <= n < 2^31                                        */
    int32_t sh_degree; /* 0 .. 3                                               */
} gs_gaussians;

/* Pinhole camera (host struct). world_to_cam is the 3x4 row-major [R | t]
 * mapping world points to camera space. A point projects to
 * (fx x/z + cx, fy y/z + cy). Gaussians with camera z <= near_z are culled
 * (Sec. 4.5 step 1). */
typedef struct {
    float world_to_cam[12];
    float fx, fy, cx, cy;
    int32_t width, height; /* 1 .. 16384                                       */
    float near_z;          /* > 0; 0.2 in the standard formulation             */
} gs_camera;

/* Per-Gaussian projected record written by gs_project (48 bytes, 16-byte
 * aligned). Only records of visible Gaussians (tiles[i] > 0, see gs_project)
 * are written; the others keep whatever the buffer held. */
typedef struct {
    float mean2d[2];  /* projected mean in pixels                              */
    float conic[3];   /* (Q00, Q01, Q11) of the inverse 2D covariance          */
    float opacity;    /* sigmoid(logit)                                        */
    float rgb[3];     /* SH colour                                             */
    float depth;      /* camera-space z; the sort key uses its FP32 bits       */
    int32_t radius;   /* ceil(3 sqrt(lambda_max)) in pixels (clamped to 2^30)  */
    uint32_t tiles;   /* number of screen tiles in the record's tile rect      */
} gs_record;

/* Output images (device). rgb is required; the others may be NULL.
 *   rgb        height x width x 3  C + T_final * bg
 *   final_T    height x width      transmittance left after blending
 *   n_contrib  height x width      1-based position, in the pixel's tile
 *                                  list, of the last Gaussian blended (0: none)
 *   n_eval     height x width      list entries evaluated by the pixel,
 *                                  including the one that stopped it */
typedef struct {
    float *rgb;
    float *final_T;
    int32_t *n_contrib;
    int32_t *n_eval;
} gs_framebuffer;

/* Blend schedules; all produce identical outputs.
 *   GS_BLEND_CULLED       each warp owns a pixel block and skips records that
 *                         cannot reach alpha >= 1/255 in it (default):
 *                         gs_render uses 8x8 blocks (as GS_BLEND_CULLED_8X8;
 *                         with thread-block clusters, 8x4 blocks until a
 *                         frame averaged more than 1024 keys per list tile);
 *                         gs_blend on caller-provided gs_records 8x4 blocks
 *   GS_BLEND_BASIC        one thread per pixel evaluates every record of its
 *                         tile
 *   GS_BLEND_CULLED_WIDE  as CULLED with 16x8 blocks (16-wide tiles; 8x8
 *                         tiles use 8x4 blocks)
 *   GS_BLEND_CULLED_TILE  as CULLED with one warp per 16x16 tile (other
 *                         tiles use 8x4 blocks)
 *   GS_BLEND_CULLED_8X8   8x8 blocks, two pixels per lane: in gs_render
 *                         (and gs_render_batch) the two pixels go through
 *                         packed FP32 pair instructions (fma / mul / sub
 *                         .f32x2, each element rounded as the scalar
 *                         operation); gs_blend on gs_records computes them
 *                         one at a time
 *   GS_BLEND_TMA          gs_render only (gs_blend falls back to CULLED): the
 *                         records of the sorted lists are first gathered in
 *                         list order, then each tile's batches are staged in
 *                         shared memory with bulk copies (cp.async.bulk,
 *                         double-buffered, mbarrier completion) and blended as
 *                         CULLED */
enum { GS_BLEND_CULLED = 0, GS_BLEND_BASIC = 1, GS_BLEND_CULLED_WIDE = 2, GS_BLEND_CULLED_TILE = 3,
       GS_BLEND_CULLED_8X8 = 4, GS_BLEND_TMA = 5 };

/* Precision of the blend records gs_render, gs_render_backward and
 * gs_render_batch write during the projection and the blend reads. Every
 * record holds, in FP32, the 2D mean, the conic scaled to a base-2 exponent
 * and the alpha threshold log2(1 / (255 opacity)) of the FP32 opacity, so
 * every precision takes the same alpha >= 1/255 decisions (a 16-bit conic's
 * relative error, multiplied by |power| up to ln 255 at the 1/255 edge, would
 * exceed the image error bound on dense scenes). Opacity and colour:
 *   F32   FP32 (48-byte records)
 *   F16   FP16 opacity and colour (36 bytes)
 *   BF16  FP16 opacity and BF16 colour stored as colour - 1 (36 bytes): the
 *         offset keeps BF16's rounding error at or below 2^-9 on colours in
 *         [0, 2), and the opacity needs FP16's 11 significant bits.
 * With F16 and BF16 the image is within 4e-3 (max abs per channel) of the
 * exact result. Values are decoded to FP32 when staged; compositing and
 * transmittance stay FP32. Binning always uses the FP32 projection, so the
 * per-tile lists do not change. */
enum { GS_RECORD_F32 = 0, GS_RECORD_F16 = 1, GS_RECORD_BF16 = 2 };

/* Options. gs_default_options() fills the standard values. */
typedef struct {
    int32_t tile_w, tile_h; /* screen tile: 16x16 (default), 16x8 or 8x8      */
    float bg[3];            /* background colour added as T_final * bg         */
    int32_t record_dtype;   /* GS_RECORD_F32 (default), _F16 or _BF16          */
    int32_t blend_variant;  /* GS_BLEND_CULLED (default), _BASIC, _CULLED_WIDE,
                               _CULLED_TILE, _CULLED_8X8, _TMA                 */
    int32_t direct_launch;  /* gs_render and gs_render_batch: 0 = replay a
                               captured CUDA graph (default), 1 = launch the
                               kernels directly, see gs_render               */
    int32_t sync_mode;      /* gs_render: GS_SYNC_FRAME (default) or
                               GS_SYNC_DEFERRED, see gs_render                 */
    int32_t temporal;       /* gs_render: temporal re-binning, see gs_render
                               (needs GS_SYNC_FRAME): 0 off, 1 adaptive, 2
                               whenever possible                              */
    int32_t batch_mode;     /* gs_render_batch: GS_BATCH_AUTO (default),
                               GS_BATCH_JOINT or GS_BATCH_PER_VIEW             */
    int32_t batch_depth;    /* gs_render_batch, joint schedule: records staged
                               per shared-memory batch of the blend, 64, 128
                               or 256 (0 = 256)                                */
    int32_t cluster;        /* gs_render (and gs_render_batch, which then
                               renders view by view): thread-block clusters of
                               the blend, see GS_CLUSTER_*; 16x16 tiles only */
    int32_t list_tiles;     /* gs_render and gs_render_batch (jointly too;
                               not gs_render_batch_backward): lists of list
                               tiles without clusters, see GS_LISTS_*; 16x16
                               tiles only, not together with cluster         */
    int32_t tile_order;     /* gs_render: the order in which the blend's thread
                               blocks take tiles, see GS_ORDER_*             */
} gs_options;

/* Thread-block clusters of the blend (gs_options.cluster; Sec. 4.4 and 5.5
 * of the paper share Gaussians between neighbouring screen tiles instead of
 * routing them to each tile). With 2 or 4 the per-tile lists are built for
 * list tiles of 2 x 1 or 2 x 2 screen tiles (32 x 16 or 32 x 32 pixels, so a
 * splat spanning them is listed once instead of two or four times), and the
 * thread blocks of one list tile run as one cluster: each stages a share of
 * every batch of records into its shared memory and the others copy the
 * records that reach their tile from it (distributed shared memory), so a
 * record is read from L2 once per cluster. Colours and transmittance equal
 * those of 16x16 lists bit for bit; n_contrib and n_eval count positions in
 * the list tile's list (gs_render_backward accepts them). Not with temporal
 * re-binning. */
enum { GS_CLUSTER_NONE = 0, GS_CLUSTER_2X1 = 2, GS_CLUSTER_2X2 = 4 };

/* List tiles without clusters (gs_options.list_tiles = the number of screen
 * tiles per list tile): with GS_LISTS_2X1, _2X2, _4X4 or _8X8 the per-tile
 * lists are built for list tiles of 2 x 1, 2 x 2, 4 x 4 or 8 x 8 screen
 * tiles (so a splat spanning several screen tiles is listed fewer times),
 * and the thread block of every 16 x 16 screen tile reads its list tile's
 * list itself, keeps (compacted in list order) the records whose 16 x 16
 * tile rect holds its tile and whose conservative box meets it, and blends
 * them: no cluster barriers, at the price of each list entry being read by
 * every screen tile of its list tile. Outputs as with the clusters (colours
 * and transmittance equal the 16x16 lists' bit for bit, list positions are
 * the list tile's). gs_render_batch's joint schedule takes them too (one work
 * item per screen tile of a list tile); gs_render_batch_backward does not
 * (GS_ERR_UNSUPPORTED). Not with temporal re-binning. */
enum { GS_LISTS_1X1 = 0, GS_LISTS_2X1 = 2, GS_LISTS_2X2 = 4, GS_LISTS_4X4 = 16, GS_LISTS_8X8 = 64 };

/* Order of gs_render's blend blocks (gs_options.tile_order). LONGEST_FIRST
 * (default): one small kernel sorts the frame's (list) tiles by the bit
 * length of their list, longest first, and block b of the culled blends
 * (GS_BLEND_CULLED, _CULLED_WIDE, _CULLED_TILE, _CULLED_8X8) and of the
 * list-tile blend takes the b-th tile of that order, so the tiles with the
 * longest lists start first and the short ones fill the end of the launch
 * (on a clustered scene a few tiles hold twenty times the mean list). GRID:
 * block b takes tile b (row order). The images are identical. The basic,
 * TMA and cluster blends, and gs_render_backward, always run in grid order.
 * Measured on a 1M-Gaussian 1080p frame: one frame at a time longest first
 * is faster (0.34 against 0.37 ms); with eight frames in flight on eight
 * streams grid order is (their blends fill each other's ends, and the sort
 * kernel and the ordered start cost ~3 %). */
enum { GS_ORDER_LONGEST_FIRST = 0, GS_ORDER_GRID = 1 };

/* How gs_render_batch schedules the views. JOINT: one projection, one key
 * sort and one persistent blend over all views (pays off for many short
 * per-tile lists). PER_VIEW: the views one after another through the
 * single-view pipeline, whose depth-first sort needs fewer digit passes over
 * long key lists. AUTO: PER_VIEW after a batch that averaged more than 8M
 * keys per view, JOINT otherwise. */
enum { GS_BATCH_AUTO = 0, GS_BATCH_JOINT = 1, GS_BATCH_PER_VIEW = 2 };

/* When gs_render checks a frame's key count (see gs_render). */
enum { GS_SYNC_FRAME = 0, GS_SYNC_DEFERRED = 1 };

void gs_default_options(gs_options *opts /* host */);

/* Context: owns the scratch workspace (grown on demand) and the device error
 * word, bound to one CUDA device. *ctx is set to NULL on failure:
 * GS_ERR_INVALID_ARG for a null ctx or a device index that does not exist
 * (also when the machine has no CUDA device), GS_ERR_CUDA if the context's
 * small device and pinned host buffers or its events cannot be created.
 * gs_destroy(NULL) does nothing. */
gs_status gs_create(gs_context **ctx /* host out */, int device);
void gs_destroy(gs_context *ctx);
/* Message of the last failing call on this context (host string, valid until
 * the next call on the context). */
const char *gs_last_error(const gs_context *ctx);
/* Synchronises the given stream, then returns and clears the device error
 * word (GS_ERR_TIMEOUT / GS_ERR_CAPACITY) or a pending CUDA error. */
gs_status gs_sync_status(gs_context *ctx, void *stream);
/* Bytes of device workspace the context currently holds. */
size_t gs_workspace_bytes(const gs_context *ctx);

/* Stage 1 — projection (Sec. 3.1 stages 1-2; square 3-sigma bound of
 * Sec. 4.4; near-plane cull of Sec. 4.5 step 1).
 *   records  n x gs_record, 16-byte aligned: written for visible Gaussians
 *   tiles    n x u32: number of screen tiles the Gaussian's rect covers, 0 for
 *            a culled Gaussian (behind the near plane, degenerate, or with an
 *            empty rect); always written. */
gs_status gs_project(gs_context *ctx, const gs_gaussians *g, const gs_camera *cam,
                     const gs_options *opts, gs_record *records, uint32_t *tiles, void *stream);

/* Stage 2 — binning (Sec. 3.1 stage 3; Sec. 4.5 step 2). Every record i with
 * tiles[i] > 0 is listed once in each tile of its rect
 *   columns [floor((u - r) / tw), floor((u + r + tw - 1) / tw)),
 *   rows    [floor((v - r) / th), floor((v + r + th - 1) / th)),
 * clamped to the tile grid, and the lists are ordered by
 * (tile id, FP32 bits of depth, record index). tiles[i] must equal the
 * rect's area (as gs_project writes it); a record where it does not is
 * skipped and flagged (GS_ERR_INVALID_ARG from gs_sync_status).
 *   keys     capacity x u64   out: tile << 32 | bits(depth), ascending
 *   values   capacity x u32   out: record index
 *   ranges   tiles x 2 x u32  out: [first, last+1) per tile, (0, 0) if empty,
 *                             tiles = ceil(W / tw) * ceil(H / th), row-major
 *   n_keys   host out: the number of pairs K.
 * SYNCHRONISES the stream once to read K. If K > capacity nothing is
 * written past the buffers, *n_keys holds K and GS_ERR_CAPACITY is
 * returned. */
gs_status gs_bin(gs_context *ctx, const gs_record *records, const uint32_t *tiles, int64_t n,
                 const gs_camera *cam,
                 const gs_options *opts, uint64_t *keys, uint32_t *values, int64_t capacity,
                 uint32_t *ranges, int64_t *n_keys, void *stream);

/* Stable ascending sort of n (key, value) pairs on the low key_bits bits of
 * the keys (1 .. 64), in place. Least-significant-digit radix sort with
 * 8-bit digits, one pass per digit, each pass a single launch that chains
 * per-block digit counts by decoupled look-back (Onesweep, Adinets and
 * Merrill 2022). Bits above key_bits must be zero. */
gs_status gs_sort_pairs(gs_context *ctx, uint64_t *keys, uint32_t *values, int64_t n,
                        int32_t key_bits, void *stream);

/* Allocation-free variant of gs_sort_pairs, for callers that may not
 * allocate device memory (allocator or memory-pool callbacks, fixed-footprint
 * real-time loops, hosts that own all device memory): same sort, same
 * arguments, no gs_context. The paper has no counterpart; this is a library
 * service. Its scratch is one array built into libgs.so, about 4 MiB
 * (4,227,328 bytes), which every GPU that loads the library holds until the
 * process exits.
 *   n <= GS_NOALLOC_SORT_MAX_PAIRS, else GS_ERR_CAPACITY (nothing launched).
 *   All calls share that array: calls that overlap on the GPU corrupt each
 *   other; serialise them. The first call on a device looks the array up
 *   with that device current; the address is kept, so that device must not
 *   be reset after the first call.
 *   Device indices of 64 and above are not served (GS_ERR_CUDA).
 *   Returns after the sort has finished on `stream` (waits once on that
 *   stream to read the device error word); GS_ERR_TIMEOUT if a bounded wait
 *   gave up. Calls no cudaMalloc/cudaFree. */
#define GS_NOALLOC_SORT_MAX_PAIRS 262144
gs_status gs_sort_pairs_noalloc(uint64_t *keys, uint32_t *values, int64_t n, int32_t key_bits,
                                void *stream);

/* Per-tile [first, last+1) ranges of n sorted keys (tile id = key >> 32).
 * ranges: n_tiles x 2 x u32, fully overwritten ((0, 0) for empty tiles). */
gs_status gs_tile_ranges(gs_context *ctx, const uint64_t *keys, int64_t n, int32_t n_tiles,
                         uint32_t *ranges, void *stream);

/* Stage 3 — blending (Eq. 1; Sec. 4.5 step 3). For each pixel, front to back
 * over its tile's list values[ranges[2t] .. ranges[2t+1]):
 *   power = -(Q00 dx^2 + Q11 dy^2) / 2 - Q01 dx dy, d = pixel centre - mean2d;
 *   skip if power > 0; alpha = min(0.99, opacity * exp(power));
 *   skip if alpha < 1/255; T' = T (1 - alpha); stop if T' < 1e-4 (that
 *   Gaussian is not added); C += rgb alpha T; T = T'.
 * records/values/ranges as produced by gs_project / gs_bin. */
gs_status gs_blend(gs_context *ctx, const gs_record *records, const uint32_t *values,
                   const uint32_t *ranges, const gs_camera *cam, const gs_options *opts,
                   const gs_framebuffer *fb, void *stream);

/* Whole forward pass (Sec. 3.1: cull, project, depth-sort per tile,
 * composite) on workspace owned by the context, with the same results as
 * gs_project -> gs_bin -> gs_blend. Two kernels project the Gaussians,
 * reserve key slots and emit the keys with the sort's digit histograms; the
 * sort and the ranges read the key count on the device; the blend follows.
 * The key buffers are sized from earlier frames (with headroom); a frame that
 * needs more writes nothing past them and is detected by its count:
 *   GS_SYNC_FRAME     the call SYNCHRONISES once at the end to check the
 *                     count; if the frame needed more room it grows the
 *                     buffers and renders the frame again, so a returned
 *                     image is never truncated.
 *   GS_SYNC_DEFERRED  the call does not synchronise (up to 4 frames in
 *                     flight). The count and the error word of each frame
 *                     are read back asynchronously and checked by later calls
 *                     on the context (gs_render, gs_render_backward,
 *                     gs_sync_status, gs_last_render_stats). A frame that
 *                     overflowed makes that later call return
 *                     GS_ERR_CAPACITY without doing its own work: the buffers
 *                     have then grown and the caller renders again.
 *                     gs_render_backward waits for the frame it
 *                     differentiates and fails if that frame overflowed.
 * CUDA graph (opts->direct_launch = 0, default): the frame's launches (from
 * the key sort's scratch reset to the blend) are captured once into a CUDA
 * graph on a stream of the context's own, without running them, and
 * replayed on `stream` by later frames with the same scene arrays (pointers,
 * count, SH degree), image size, options (other than sync_mode),
 * framebuffer pointers, key capacity and blend schedule while the context's
 * buffers keep their addresses; each replay sets the frame's camera in the
 * projection's launch, so the host issues one graph launch where it would
 * issue about twenty calls. The context keeps eight such graphs (frames that
 * alternate framebuffers or scenes replay too; re-binned frames of temporal
 * mode have graphs of their own). Frames with stage timing on
 * (gs_set_stage_timing), with GS_BLEND_TMA, with direct_launch = 1 or on a
 * stream the caller is capturing launch the kernels directly, and so does a context after four captures in a row
 * (for its next 32 frames, doubling up to 1024 while captures keep missing,
 * e.g. a loop over more views than the context keeps graphs for). Results
 * are the same either way. */
/* Temporal re-binning (opts->temporal = 1 or 2; the paper's temporal-
 * locality idea, Sec. 5.4 and Sec. 6): when the previous frame on this
 * context was rendered the same way with the same Gaussian count and tile
 * grid, this frame's per-tile lists are rebuilt from that frame's: only
 * Gaussians whose tile rect changed ("moved", counted in
 * gs_render_stats.n_moved) leave and enter tiles, and each tile is put in
 * this frame's (depth, index) order by a merge or an in-tile sort. The
 * lists, and so the image, are identical to those of a full binning. The
 * frame is binned from scratch instead when there is no such state, when
 * more than 8 % of the visible Gaussians moved in the previous frame, or
 * when a tile list exceeds 4096 entries. With temporal = 1 the context also
 * times both kinds of frames (CUDA events around the binning, or around the
 * whole frame when it replays a CUDA graph) and bins in full while re-binned
 * frames measured slower, and re-bins only after a full
 * frame measured the churn; once re-binning is ruled out (by
 * that measurement or by the churn) the next 6 frames are rendered without
 * tracking tile rects (n_moved = 0 on them), the two after them measure the
 * churn again, and the gate tries one re-binned frame: one frame in 8
 * re-measures. temporal = 2 re-bins whenever it can and measures the churn
 * (n_moved) on every frame. */
gs_status gs_render(gs_context *ctx, const gs_gaussians *g, const gs_camera *cam,
                    const gs_options *opts, const gs_framebuffer *fb, void *stream);

/* Gradients of the Gaussian parameters (device, caller-owned, overwritten):
 * shapes as in gs_gaussians. d_records is optional: n x 9 floats receive
 * dL/d(u, v, Q00, Q01, Q11, opacity, r, g, b) of every projected record. */
typedef struct {
    float *d_means;
    float *d_log_scales;
    float *d_quats;
    float *d_opacity_logits;
    float *d_sh;
    float *d_records;
} gs_grads;

/* Backward of the last gs_render made on this context (the paper's Sec. 7
 * names the backward pass as the next step; Eq. 1 and the projection of
 * Sec. 3.1 differentiated). Given dL/dC for that image (d_rgb, height x
 * width x 3), writes dL/d(parameters) for a loss L of the image:
 *   blend: each tile walked back to front from each pixel's last
 *   contributor, transmittance recovered from the final T
 *   (T_k = T_{k+1} / (1 - alpha_k)); alpha = min(0.99, o G) has no
 *   derivative where it is clamped; skipped and stopped Gaussians none.
 *   projection: chain rule through the conic inverse, J W R S, the
 *   normalised quaternion, exp of the log-scales, the sigmoid and the SH
 *   colour (zero where a channel was clamped at 0). The rect and radius are
 *   discrete and have no derivative.
 * g, cam and opts must be those of that gs_render, and fb must hold the
 * final_T and n_contrib it wrote (both required here). Invisible Gaussians
 * get zero gradients. The call checks that the context's last frame is that
 * frame: the same five parameter pointers, count and SH degree, every camera
 * field, tile shape, background and record precision; otherwise (another
 * gs_render came in between, e.g. a second view rendered before the first
 * view's backward) it returns GS_ERR_INVALID_ARG and writes nothing. The
 * caller then renders that frame again (a render is deterministic, so its
 * final_T and n_contrib come out bit for bit the same) and calls again.
 * gs_bin and gs_sort_pairs reuse the buffers the lists live in, so after them
 * there is no frame to differentiate. */
gs_status gs_render_backward(gs_context *ctx, const gs_gaussians *g, const gs_camera *cam,
                             const gs_options *opts, const gs_framebuffer *fb, const float *d_rgb,
                             const gs_grads *out, void *stream);

/* Renders n_views cameras (of any sizes) of one scene in one call — the
 * batched form of gs_render with identical per-view results (same rules,
 * same per-tile order). One launch projects every (view, Gaussian) pair into
 * compact records; one sort orders all views' keys, whose tile ids are
 * numbered across the views; one persistent blend kernel takes the tiles of
 * all views from a queue ordered longest list first, which evens out the
 * imbalance between dense and empty screen regions (the paper's Sec. 6
 * load-imbalance finding). The whole sequence is captured once into a CUDA
 * graph and replayed while the scene arrays, the number and sizes of the
 * views, the options and the buffer sizes stay the same (cameras and
 * framebuffer pointers may change: they travel in a table copied at the
 * start of each replay). SYNCHRONISES once at the end; if the frame needed
 * larger buffers they grow and the batch is rendered again.
 *   cams, fbs: host arrays of n_views entries (1 .. 4096); fbs[v] as for
 *   gs_render (rgb required). tile size, bg and record_dtype from opts. */
gs_status gs_render_batch(gs_context *ctx, const gs_gaussians *g, const gs_camera *cams, int32_t n_views,
                          const gs_options *opts, const gs_framebuffer *fbs, void *stream);

/* Backward of the last gs_render_batch, which must have used the joint
 * schedule (GS_BATCH_JOINT, or AUTO on short lists) with the same Gaussians,
 * number of views and options: the gradients of sum over views v of
 * <d_rgb[v], rgb_v> with respect to the five parameter arrays, as the sum of
 * gs_render_backward over the views. One blend-gradient launch covers the
 * tiles of all views; one projection-gradient launch covers every visible
 * (view, Gaussian) pair and adds into the Gaussian's gradients (overwritten,
 * not accumulated across calls).
 *   fbs[v].final_T / n_contrib: the buffers the forward wrote (required);
 *   d_rgb: host array of n_views device pointers, each height x width x 3;
 *   out->d_records (optional): per visible (view, Gaussian) record, 9 floats. */
gs_status gs_render_batch_backward(gs_context *ctx, const gs_gaussians *g, const gs_camera *cams, int32_t n_views,
                                   const gs_options *opts, const gs_framebuffer *fbs, const float *const *d_rgb,
                                   const gs_grads *out, void *stream);

/* Autotuner of gs_render_batch: renders the batch with each screen-tile
 * shape and list form (16x16, 16x8, 8x8 with a list per tile; 16x16 with
 * GS_CLUSTER_2X1 and GS_CLUSTER_2X2, which render view by view; 16x16 with
 * GS_LISTS_2X1, GS_LISTS_2X2, GS_LISTS_4X4 and GS_LISTS_8X8) and, for the
 * joint schedule with a list per tile, each blend staging depth (256, 128,
 * 64 records), times three runs of each with CUDA events, and writes the
 * fastest into opts->tile_w / tile_h / cluster / list_tiles / batch_depth.
 * ms_out (host, 9 floats, optional) receives per candidate the mean time of
 * its best depth, in that order. */
gs_status gs_autotune_batch(gs_context *ctx, const gs_gaussians *g, const gs_camera *cams, int32_t n_views,
                            gs_options *opts, const gs_framebuffer *fbs, void *stream, float *ms_out);

/* Self-test of the library's failure detection (no counterpart in the
 * paper). Every wait of one thread block on another (the decoupled
 * look-backs of the scan and of the sort) gives up after a time limit, sets
 * the context's error word and stays in bounds, so a lost predecessor can
 * never hang the GPU. This entry point makes such a wait run out on purpose:
 * it runs the scan (kind 0) or one sort pass (kind 1) with partition 0 never
 * taken, so every block waits on a status word nothing sets, with the given
 * limit (1 us .. 5 s). Expected result: GS_ERR_TIMEOUT, after which the
 * context works normally. SYNCHRONISES; allocates and frees its scratch. */
gs_status gs_selftest_bounded_wait(gs_context *ctx, int32_t kind, int64_t timeout_ns, void *stream);

/* Sets the number of (tile, Gaussian) pairs gs_render's key buffers hold and
 * stops the context from shrinking it between frames (the buffers grow if a
 * frame needs more). */
gs_status gs_reserve_keys(gs_context *ctx, int64_t key_capacity);

/* Number of the last frame gs_render made on this context that a
 * gs_render_backward could still differentiate: 1 for the first frame, then
 * counting up; 0 when there is none (no frame yet, the frame overflowed its
 * key buffers, or gs_bin / gs_sort_pairs reused its buffers since). A caller
 * that keeps several frames alive saves the number after each gs_render and
 * compares it before a backward. */
gs_status gs_last_frame_id(const gs_context *ctx, uint64_t *out /* host */);

/* Statistics of the last gs_render on this context (host out). Waits for
 * deferred frames first and returns the first error among them (the
 * statistics are still filled in). */
typedef struct {
    int64_t n_visible; /* records with radius > 0                              */
    int64_t n_keys;    /* (tile, Gaussian) pairs K                             */
    int32_t key_bits;  /* significant key bits sorted                          */
    int32_t n_tiles;
    int64_t n_moved;   /* temporal re-binning: Gaussians whose tile rect
                          changed since the previous frame (0 otherwise)     */
    int32_t rebinned;  /* 1 if the lists were re-binned from the previous
                          frame's, 0 if binned from scratch                  */
    int32_t reserved;
} gs_render_stats;
gs_status gs_last_render_stats(gs_context *ctx, gs_render_stats *out);

/* Per-stage device times of gs_render, measured with CUDA events recorded on
 * the render stream between the stages (tracing; off by default). */
typedef struct {
    float project_ms;     /* projection + compact list of visible Gaussians     */
    float depth_sort_ms;  /* depth sort of the compact list                     */
    float entry_scan_ms;  /* scan of the tile counts in depth order             */
    float emit_ms;        /* key emission                                       */
    float tile_sort_ms;   /* tile-digit passes of the key sort                  */
    float ranges_ms;      /* per-tile ranges                                    */
    float blend_ms;       /* gs_blend kernel                                    */
    float total_ms;       /* first event to last                                */
} gs_stage_times;
/* enable != 0 turns per-stage events on for later gs_render calls. */
gs_status gs_set_stage_timing(gs_context *ctx, int enable);
/* Times of the last gs_render made with timing on; SYNCHRONISES on its last
 * event. GS_ERR_INVALID_ARG if no timed render happened yet. */
gs_status gs_last_stage_times(gs_context *ctx, gs_stage_times *out /* host */);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
