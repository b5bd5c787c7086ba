// render.cu -- per-tile front-to-back compositing (camera and LiDAR).
//
// One CTA per screen tile, one thread per pixel (ray).  The tile's sorted
// list of records is walked in batches of `blockDim.x` records; each batch is
// staged into shared memory by bulk async copies (one 80-byte cp.async.bulk
// per record, completing on an mbarrier), double-buffered so the next batch
// lands while the current one is composited.  Every thread then solves
// Eq. 2 for its ray against each staged surfel in closed form (q = Q r,
// (u, v) = (q_0, q_1)/q_2, depth or distance = det/q_2; see
// gsr_internal.cuh), falls back to the 2DGS screen-space low-pass where it
// is larger, and composites with alpha = min(0.99, o G), skipping
// alpha < 1/255 and stopping before T (1 - alpha) < 1e-4.  A warp leaves a
// batch once all its rays are done (warp vote); the CTA leaves the list once
// all its rays are done (block vote).
#include "gsr_internal.cuh"

namespace gsr {

struct RayState {
    float T, A, B, D;
    float f0, f1, f2;
    float n0, n1, n2;
    uint32_t last;
    uint32_t walk;
    bool done;
};

// Composite one tile with the whole CTA.  Threads beyond the tile's rays only
// help staging.  `gb` counts the batches this CTA has staged so far (it picks
// the buffer and the mbarrier phase, so a persistent CTA can run many tiles).
template <int KIND>
__device__ __forceinline__ void render_tile(const SensorDev& sd, int tile_w, int tile_h, int local_tile,
                                            const uint2 range, const float4* __restrict__ rec,
                                            const uint32_t* __restrict__ pval, const FrameOut& out,
                                            uint32_t* counters, float4* buf, uint64_t* bars, uint32_t& gb)
{
    const int nthr = blockDim.x;
    const int tid = threadIdx.x;
    const int tx = local_tile % sd.tiles_x, ty = local_tile / sd.tiles_x;
    const int x = tx * tile_w + tid % tile_w;
    const int y = ty * tile_h + tid / tile_w;
    const bool inside = tid < tile_w * tile_h && x < sd.width && y < sd.height;

    float rx, ry, d0, d1, d2;
    ray_setup<KIND>(sd, x, y, rx, ry, d0, d1, d2);
    RayState s;
    s.T = 1.f; s.A = 0.f; s.B = 0.f; s.D = 0.f;
    s.f0 = s.f1 = s.f2 = 0.f;
    s.n0 = s.n1 = s.n2 = 0.f;
    s.last = 0;
    s.walk = (uint32_t)(range.y - range.x);
    s.done = !inside;

    const uint32_t start = range.x;
    const int n = (int)(range.y - range.x);
    const int nb = (n + nthr - 1) / nthr;
    const float columns = (float)sd.width;
    const float near_plane = sd.near_plane;

    // batch b of this tile is the CTA's batch g = gb + b: buffer and barrier
    // g & 1, phase parity (g >> 1) & 1
    auto issue = [&](int b) {
        const uint32_t g = gb + (uint32_t)b;
        const int first = b * nthr;
        const int cnt = min(nthr, n - first);
        uint64_t* bar = bars + (g & 1);
        float4* dst = buf + (size_t)(g & 1) * nthr * kRecordF4;
        if (tid == 0) mbar_arrive_expect_tx(bar, (uint32_t)cnt * kRecordBytes);
        if (tid < cnt) {
            const uint32_t slot = pval[start + first + tid];
            bulk_g2s(dst + tid * kRecordF4, rec + (size_t)slot * kRecordF4, kRecordBytes, bar);
        }
    };
    auto wait = [&](int b) {
        const uint32_t g = gb + (uint32_t)b;
        return mbar_wait_bounded(bars + (g & 1), (g >> 1) & 1, counters);
    };

    bool ok = true;
    int issued = 0;
    if (nb > 0) {
        issue(0);
        issued = 1;
    }
    for (int b = 0; b < nb; ++b) {
        if (b + 1 < nb) {
            issue(b + 1);
            issued = b + 2;
        }
        if (!wait(b)) ok = false;
        const float4* B = buf + (size_t)((gb + b) & 1) * nthr * kRecordF4;
        const int cnt = min(nthr, n - b * nthr);
        if (ok) {
            for (int j = 0; j < cnt; ++j) {
                if (__all_sync(0xffffffffu, s.done)) break;
                if (s.done) continue;
                const float4* Rj = B + j * kRecordF4;
                Splat sp;
                if (!splat_eval<KIND>(Rj, rx, ry, d0, d1, d2, near_plane, columns, sp)) continue;
                const float alpha = sp.alpha, z = sp.z;
                const float Tn = s.T * (1.f - alpha);
                if (Tn < kTMin) {
                    s.done = true;
                    s.walk = (uint32_t)(b * nthr + j + 1);
                    continue;
                }
                const float w = alpha * s.T;
                const float4 r3 = Rj[3];
                s.f0 = fmaf(w, r3.y, s.f0);
                if (KIND == GSR_SENSOR_PINHOLE) {
                    s.f1 = fmaf(w, r3.z, s.f1);
                    s.f2 = fmaf(w, r3.w, s.f2);
                    const float4 r4 = Rj[4];
                    s.n0 = fmaf(w, r4.x, s.n0);
                    s.n1 = fmaf(w, r4.y, s.n1);
                    s.n2 = fmaf(w, r4.z, s.n2);
                }
                s.A += w;
                const float wz = w * z;
                s.B += wz;
                s.D = fmaf(wz, z, s.D);
                s.T = Tn;
                s.last = (uint32_t)(b * nthr + j + 1);
            }
        }
        // one block-uniform vote: a thread whose bounded wait gave up counts
        // as done (it composites nothing more; every later wait is bounded too)
        if (__syncthreads_and(s.done || !ok)) {
            // no copy may still be landing in shared memory when the CTA
            // leaves or moves on to its next tile
            if (b + 1 < nb) wait(b + 1);
            break;
        }
    }
    gb += (uint32_t)issued;

    if (!inside) return;
    const size_t HW = (size_t)sd.width * sd.height;
    const size_t pix = (size_t)y * sd.width + x;
    if (KIND == GSR_SENSOR_PINHOLE) {
        if (out.color) {
            out.color[pix] = fmaf(s.T, sd.bg[0], s.f0);
            out.color[HW + pix] = fmaf(s.T, sd.bg[1], s.f1);
            out.color[2 * HW + pix] = fmaf(s.T, sd.bg[2], s.f2);
        }
        if (out.normal) {
            out.normal[pix] = s.n0;
            out.normal[HW + pix] = s.n1;
            out.normal[2 * HW + pix] = s.n2;
        }
    } else {
        if (out.color) out.color[pix] = s.f0;
    }
    if (out.depth) out.depth[pix] = s.A > 0.f ? s.B / s.A : 0.f;
    if (out.alpha) out.alpha[pix] = s.A;
    if (out.trans) out.trans[pix] = s.T;
    if (out.depth_acc) {
        out.depth_acc[pix] = s.B;
        out.depth_acc[HW + pix] = s.D;
    }
    if (out.n_contrib) out.n_contrib[pix] = s.last;
    if (out.n_walk) out.n_walk[pix] = s.walk;
}

template <int KIND>
__global__ void __launch_bounds__(256) k_render(SensorTable tab, int sensor, const float4* __restrict__ rec,
                                                const uint2* __restrict__ ranges, const uint32_t* __restrict__ pval,
                                                FrameOut out, uint32_t* counters)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    float4* buf = reinterpret_cast<float4*>(smem_raw + 128);
    const SensorDev& sd = tab.s[sensor];
    if (threadIdx.x == 0) {
        mbar_init(bars, 1);
        mbar_init(bars + 1, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int lt = blockIdx.x;
    uint32_t gb = 0;
    render_tile<KIND>(sd, sd.tile_w, sd.tile_h, lt, ranges[sd.tile_base + lt], rec, pval, out, counters, buf, bars,
                      gb);
}

// Outputs of every sensor of a plan, for the whole-rig kernel.
struct RigOut {
    FrameOut o[GSR_MAX_SENSORS];
};

// The whole rig in one persistent launch: each CTA takes the next tile from a
// global work queue that lists every sensor's tiles longest list first, so
// the long LiDAR and near-field tiles start early and the short ones fill in
// behind them; the sensor kind is uniform per tile, so the branch is too.
__global__ void __launch_bounds__(256) k_render_rig(SensorTable tab, const float4* __restrict__ rec,
                                                    const uint2* __restrict__ ranges,
                                                    const uint32_t* __restrict__ pval,
                                                    const uint32_t* __restrict__ order, RigOut outs,
                                                    uint32_t* counters)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    float4* buf = reinterpret_cast<float4*>(smem_raw + 128);
    __shared__ uint32_t item_s;
    if (threadIdx.x == 0) {
        mbar_init(bars, 1);
        mbar_init(bars + 1, 1);
        fence_mbar_init();
    }
    uint32_t gb = 0;
    const uint32_t T = (uint32_t)tab.total_tiles;
    for (;;) {
        __syncthreads();  // the previous item (and the barrier init) is done with
        if (threadIdx.x == 0) item_s = atomicAdd(&counters[C_QUEUE], 1u);
        __syncthreads();
        const uint32_t item = item_s;
        if (item >= T) break;
        const uint32_t tile = order[item];
        int s = 0;
        while (s + 1 < tab.n && (int)tile >= tab.s[s + 1].tile_base) ++s;
        const SensorDev& sd = tab.s[s];
        const int lt = (int)tile - sd.tile_base;
        if (sd.kind == GSR_SENSOR_PINHOLE)
            render_tile<GSR_SENSOR_PINHOLE>(sd, sd.tile_w, sd.tile_h, lt, ranges[tile], rec, pval, outs.o[s],
                                            counters, buf, bars, gb);
        else
            render_tile<GSR_SENSOR_LIDAR>(sd, sd.tile_w, sd.tile_h, lt, ranges[tile], rec, pval, outs.o[s],
                                          counters, buf, bars, gb);
    }
}

size_t render_smem_bytes(int threads) { return 128 + 2 * (size_t)threads * kRecordBytes; }

cudaError_t launch_render(const gsr_plan* p, const void* ws, int sensor, const FrameOut& out, cudaStream_t st)
{
    const SensorTable tab = make_sensor_table(p);
    const SensorDev& sd = tab.s[sensor];
    const int threads = sd.tile_w * sd.tile_h;
    const size_t smem = render_smem_bytes(threads);
    const int tiles = sd.tiles_x * sd.tiles_y;
    const float4* rec = region<float4>(p, ws, R_RECORDS);
    const uint2* ranges = region<uint2>(p, ws, R_RANGES);
    const int pb = sort_result_buffer(tile_sort_passes(p));
    const uint32_t* pval = region<uint32_t>(p, ws, pb ? R_PAIR_VAL_B : R_PAIR_VAL_A);
    uint32_t* counters = region<uint32_t>(p, ws, R_COUNTERS);
    if (sd.kind == GSR_SENSOR_PINHOLE)
        k_render<GSR_SENSOR_PINHOLE><<<tiles, threads, smem, st>>>(tab, sensor, rec, ranges, pval, out, counters);
    else
        k_render<GSR_SENSOR_LIDAR><<<tiles, threads, smem, st>>>(tab, sensor, rec, ranges, pval, out, counters);
    return cudaGetLastError();
}

// Persistent CTAs for the whole-rig kernel: resident CTAs per SM x SMs of the
// current device, for CTAs of `threads` threads (32..256, a power of two).
static int rig_grid(int threads, cudaError_t& err)
{
    static int cached[64][4] = {};
    int dev = 0;
    err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return 0;
    const int ti = threads <= 32 ? 0 : threads <= 64 ? 1 : threads <= 128 ? 2 : 3;
    if (dev >= 0 && dev < 64 && cached[dev][ti] > 0) return cached[dev][ti];
    int sms = 0, per_sm = 0;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_rig, threads, render_smem_bytes(threads));
    if (err != cudaSuccess) return 0;
    const int g = sms * (per_sm > 0 ? per_sm : 1);
    if (dev >= 0 && dev < 64) cached[dev][ti] = g;
    return g;
}

cudaError_t launch_render_rig(const gsr_plan* p, const void* ws, const FrameOut* outs, cudaStream_t st)
{
    const SensorTable tab = make_sensor_table(p);
    RigOut ro;
    for (int i = 0; i < GSR_MAX_SENSORS; ++i) ro.o[i] = i < p->n_sensors ? outs[i] : FrameOut{};
    uint32_t* counters = region<uint32_t>(p, ws, R_COUNTERS);
    cudaError_t e = cudaMemsetAsync(counters + C_QUEUE, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    // one CTA per tile in flight, as wide as the largest tile of the plan
    int threads = 32;
    for (int i = 0; i < p->n_sensors; ++i) threads = max(threads, tab.s[i].tile_w * tab.s[i].tile_h);
    const int grid = rig_grid(threads, e);
    if (e != cudaSuccess) return e;
    const int pb = sort_result_buffer(tile_sort_passes(p));
    k_render_rig<<<grid, threads, render_smem_bytes(threads), st>>>(
        tab, region<float4>(p, ws, R_RECORDS), region<uint2>(p, ws, R_RANGES),
        region<uint32_t>(p, ws, pb ? R_PAIR_VAL_B : R_PAIR_VAL_A), region<uint32_t>(p, ws, R_TILE_VAL_A), ro,
        counters);
    return cudaGetLastError();
}

}  // namespace gsr
