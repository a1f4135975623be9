// gs_blend.cu — per-tile front-to-back alpha compositing (Eq. 1; Sec. 4.5
// step 3). One thread block per screen tile, one thread per pixel. The
// tile's depth-ordered list is walked in batches: the block stages a batch
// of records in shared memory (each thread fetches one record), then every
// pixel composites the batch. A block stops as soon as every pixel in it
// has stopped (transmittance below 1e-4), counted with a barrier reduction.
#include "gs_internal.cuh"

namespace {

using namespace gs;

struct BlendArgs {
    const float4 *records;
    const uint32_t *values;
    const uint32_t *ranges;
    GsGrid grid;
    int width, height;
    float bg[3];
    float *rgb;
    float *final_T;
    int32_t *n_contrib;
    int32_t *n_eval;
};

template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) blend_kernel(const BlendArgs a) {
    constexpr int kN = TW * TH;
    __shared__ float4 s_r0[kN];   // (u, v, Q00, Q01)
    __shared__ float4 s_r1[kN];   // (Q11, opacity, red, green)
    __shared__ float s_blue[kN];

    const int tile = blockIdx.x;
    const int tx = tile % a.grid.tiles_x, ty = tile / a.grid.tiles_x;
    const int tid = threadIdx.x;
    const int px = tx * TW + tid % TW, py = ty * TH + tid / TW;
    const bool inside = px < a.width && py < a.height;
    const float fx = px + 0.5f, fy = py + 0.5f;
    const uint32_t first = a.ranges[2 * tile], last = a.ranges[2 * tile + 1];

    bool done = !inside;
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f;
    int32_t n_contrib = 0, n_eval = 0;
    int32_t pos = 0;  // list position of the next record

    for (uint32_t start = first; start < last; start += kN) {
        if (__syncthreads_count(done) == kN) break;
        const uint32_t k = start + tid;
        if (k < last) {
            const float4 *r = a.records + 3 * (size_t)a.values[k];
            s_r0[tid] = __ldg(r);
            s_r1[tid] = __ldg(r + 1);
            s_blue[tid] = __ldg(reinterpret_cast<const float *>(r + 2));
        }
        __syncthreads();
        const int cnt = min((uint32_t)kN, last - start);
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
                ++pos;
                const float4 q0 = s_r0[j];
                const float dx = fx - q0.x, dy = fy - q0.y;
                const float4 q1 = s_r1[j];
                const float power = -0.5f * (q0.z * dx * dx + q1.x * dy * dy) - q0.w * dx * dy;
                if (power > 0.f) continue;
                const float alpha = fminf(kAlphaMax, q1.y * __expf(power));
                if (alpha < kAlphaMin) continue;
                const float Tn = T * (1.f - alpha);
                if (Tn < kTMin) {
                    done = true;
                    break;
                }
                const float w = alpha * T;
                cr = fmaf(q1.z, w, cr);
                cg = fmaf(q1.w, w, cg);
                cb = fmaf(s_blue[j], w, cb);
                T = Tn;
                n_contrib = pos;
            }
            n_eval = pos;
        }
    }
    if (!inside) return;
    const size_t p = (size_t)py * a.width + px;
    a.rgb[3 * p + 0] = fmaf(T, a.bg[0], cr);
    a.rgb[3 * p + 1] = fmaf(T, a.bg[1], cg);
    a.rgb[3 * p + 2] = fmaf(T, a.bg[2], cb);
    if (a.final_T) a.final_T[p] = T;
    if (a.n_contrib) a.n_contrib[p] = n_contrib;
    if (a.n_eval) a.n_eval[p] = n_eval;
}

}  // namespace

cudaError_t gs_launch_blend(const gs_record *records, const uint32_t *values, const uint32_t *ranges,
                            const GsGrid &grid, int width, int height, const float bg[3],
                            const gs_framebuffer &fb, cudaStream_t s) {
    BlendArgs a{reinterpret_cast<const float4 *>(records), values, ranges, grid, width, height,
                {bg[0], bg[1], bg[2]}, fb.rgb, fb.final_T, fb.n_contrib, fb.n_eval};
    const unsigned blocks = (unsigned)(grid.tiles_x * grid.tiles_y);
    if (grid.tile_w == 16 && grid.tile_h == 16)
        blend_kernel<16, 16><<<blocks, 256, 0, s>>>(a);
    else if (grid.tile_w == 16 && grid.tile_h == 8)
        blend_kernel<16, 8><<<blocks, 128, 0, s>>>(a);
    else
        blend_kernel<8, 8><<<blocks, 64, 0, s>>>(a);
    return cudaGetLastError();
}
