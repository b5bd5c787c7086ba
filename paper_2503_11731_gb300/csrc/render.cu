// render.cu -- per-tile front-to-back compositing (camera and LiDAR).
//
// One CTA per screen tile, one thread per pixel (ray).  The tile's sorted
// list of records is walked in batches of D records; each batch is staged
// into shared memory by bulk async copies (one 96-byte cp.async.bulk per
// record, completing on an mbarrier), double-buffered so the next batch
// lands while the current one is composited.  Each warp first drops the
// records whose support box misses all its rays (one lane per record, a
// ballot), then every thread solves
// Eq. 2 for its ray against each staged surfel in closed form (q = Q r,
// (u, v) = (q_0, q_1)/q_2, depth or distance = det/q_2; see
// gsr_internal.cuh), falls back to the 2DGS screen-space low-pass where it
// is larger, and composites with alpha = min(0.99, o G), skipping
// alpha < 1/255 and stopping before T (1 - alpha) < 1e-4.  A warp leaves a
// batch once all its rays are done (warp vote); the CTA leaves the list once
// all its rays are done (block vote).
#include "gsr_internal.cuh"

namespace gsr {

#ifndef GSR_ILP
#define GSR_ILP 4
#endif
constexpr int kIlp = GSR_ILP;  // records evaluated per step of a ray's walk (divides 32)

// Resident CTAs per SM the persistent compositing kernels are compiled for
// (256 threads each; 3 caps registers at 80 per thread, which measured
// faster than 64 with its spills, though fewer CTAs of a tile's threads fit).
#ifndef GSR_RIG_MIN_CTAS
#define GSR_RIG_MIN_CTAS 3
#endif

// One ray of a tile: its pixel / cell, whether it is inside the sensor, and
// the quantities of its two planes (ray_setup).
struct TileRay {
    int x, y;
    bool inside;
    float rx, ry, d0, d1, d2;
};

template <int KIND>
__device__ __forceinline__ TileRay tile_ray(const SensorDev& sd, const float2* dirs, int local_tile)
{
    TileRay t;
    const int tid = threadIdx.x;
    const int tx = local_tile % sd.tiles_x, ty = local_tile / sd.tiles_x;
    int lx, ly;
    tile_ray_xy(sd.tile_w, sd.tile_h, tid, lx, ly);
    t.x = tx * sd.tile_w + lx;
    t.y = ty * sd.tile_h + ly;
    t.inside = tid < sd.tile_w * sd.tile_h && t.x < sd.width && t.y < sd.height;
    ray_setup<KIND>(sd, dirs, t.x, t.y, t.rx, t.ry, t.d0, t.d1, t.d2);
    return t;
}

// Ray-index box (x0, x1, y0, y1) of the warp's rays still walking (empty if
// none): a record whose support box misses it cannot reach any of them.
__device__ __forceinline__ float4 warp_box(const TileRay& ray, bool done)
{
    const bool live = ray.inside && !done;
    const int x0 = __reduce_min_sync(0xffffffffu, live ? ray.x : 0x7fffffff);
    const int x1 = __reduce_max_sync(0xffffffffu, live ? ray.x : -1);
    const int y0 = __reduce_min_sync(0xffffffffu, live ? ray.y : 0x7fffffff);
    const int y1 = __reduce_max_sync(0xffffffffu, live ? ray.y : -1);
    return make_float4((float)x0, (float)x1, (float)y0, (float)y1);
}

// Walk list positions [lo, hi) of a tile (list starting at `start`) with the
// whole CTA, continuing each ray's state.  Batches of D records (a multiple
// of kIlp) are staged by bulk copies, double-buffered; `gb` counts the batches this CTA
// has staged so far (buffer and mbarrier phase), so a persistent CTA can walk
// many lists.  Every thread of the CTA must call it.
template <int KIND>
__device__ __forceinline__ void walk_list(const SensorDev& sd, const TileRay& ray, uint32_t start, int lo, int hi,
                                          const float4* __restrict__ rec, const uint32_t* __restrict__ pval,
                                          RayState& s, uint32_t* counters, float4* buf, uint64_t* bars,
                                          uint32_t& gb, int D)
{
    const int nthr = blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31;
    const int n = hi - lo;
    const int nb = n > 0 ? (n + D - 1) / D : 0;
    const float columns = (float)sd.width;
    const float near_plane = sd.near_plane;
    float4 wbox = warp_box(ray, s.done);

    // batch b is the CTA's batch g = gb + b: buffer and barrier g & 1, phase
    // parity (g >> 1) & 1
    auto issue = [&](int b) {
        const uint32_t g = gb + (uint32_t)b;
        const int first = b * D;
        const int cnt = min(D, n - first);
        uint64_t* bar = bars + (g & 1);
        float4* dst = buf + (size_t)(g & 1) * D * kRecordF4;
        if (tid == 0) mbar_arrive_expect_tx(bar, (uint32_t)cnt * kRecordBytes);
        for (int i = tid; i < cnt; i += nthr) {
            const uint32_t slot = pval[start + lo + first + i];
            bulk_g2s(dst + i * kRecordF4, rec + (size_t)slot * kRecordF4, kRecordBytes, bar);
        }
    };
    auto wait = [&](int b) {
        const uint32_t g = gb + (uint32_t)b;
        return mbar_wait_bounded(bars + (g & 1), (g >> 1) & 1, counters);
    };

    // nothing to do for this CTA: no batch is staged
    if (nb == 0 || __syncthreads_and(s.done)) return;
    bool ok = true;
    issue(0);
    int issued = 1;
    for (int b = 0; b < nb; ++b) {
        if (b + 1 < nb) {
            issue(b + 1);
            issued = b + 2;
        }
        if (!wait(b)) ok = false;
        const float4* B = buf + (size_t)((gb + b) & 1) * D * kRecordF4;
        const int cnt = min(D, n - b * D);
        const int pos0 = lo + b * D;  // list position of the batch's first record
        if (ok) {
            // the box of the rays still walking shrinks as rays saturate
            if (b > 0) wbox = warp_box(ray, s.done);
            for (int g0 = 0; g0 < cnt; g0 += 32) {
                if (__all_sync(0xffffffffu, s.done)) break;
                // one lane per record: does its support box meet any ray of
                // this warp?  Records that do not are skipped by the warp.
                const int jt = g0 + lane;
                bool meet = jt < cnt && box_meets<KIND>(B[jt * kRecordF4 + 5], wbox, columns);
                if (KIND == GSR_SENSOR_PINHOLE && meet) {
                    // and the footprint itself (support conic and low-pass
                    // disc, one pixel of margin) meets the box
                    const float4* Rj = B + jt * kRecordF4;
                    meet = footprint_meets_box(Rj[0], Rj[1], Rj[2], Rj[3].x, wbox.x, wbox.y, wbox.z, wbox.w);
                }
                uint32_t mask = __ballot_sync(0xffffffffu, meet);
                while (mask) {
                    if (__all_sync(0xffffffffu, s.done)) break;
                    // the next kIlp records of the mask, in list order: their
                    // evaluations are independent (the chains interleave), the
                    // compositing stays in list order
                    int idx[kIlp];
#pragma unroll
                    for (int e = 0; e < kIlp; ++e) {
                        idx[e] = mask ? __ffs(mask) - 1 : -1;
                        mask &= mask - 1u;
                    }
                    if (s.done) continue;
                    float al[kIlp], zz[kIlp];
#pragma unroll
                    for (int e = 0; e < kIlp; ++e) {
                        Splat sp;
                        const bool hit = splat_eval<KIND>(B + (g0 + max(idx[e], 0)) * kRecordF4, ray.rx, ray.ry,
                                                          ray.d0, ray.d1, ray.d2, near_plane, columns, sp);
                        al[e] = (hit && idx[e] >= 0) ? sp.alpha : 0.f;  // a hit has alpha >= 1/255
                        zz[e] = sp.z;
                    }
#pragma unroll
                    for (int e = 0; e < kIlp; ++e) {
                        if (s.done || al[e] == 0.f) continue;
                        const int j = g0 + idx[e];
                        const float alpha = al[e], z = zz[e];
                        const float Tn = s.T * (1.f - alpha);
                        if (Tn < kTMin) {
                            s.done = true;
                            s.walk = (uint32_t)(pos0 + j + 1);
                            continue;
                        }
                        const float4* Rj = B + j * kRecordF4;
                        const float w = alpha * s.T;
                        const float4 r3 = Rj[3];
                        s.f0 = fmaf(w, r3.y, s.f0);
                        s.f1 = fmaf(w, r3.z, s.f1);  // green, or the LiDAR ray-drop probability
                        if (KIND != GSR_SENSOR_LIDAR) {
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
                        s.last = (uint32_t)(pos0 + j + 1);
                    }
                }
            }
        }
        // one block-uniform vote: a thread whose bounded wait gave up counts
        // as done (it composites nothing more; every later wait is bounded too)
        if (__syncthreads_and(s.done || !ok)) {
            // no copy may still be landing in shared memory when the CTA
            // leaves or moves on: batch b if its wait gave up (a second
            // bounded wait), and batch b + 1 if it was issued
            if (!ok) wait(b);
            if (b + 1 < nb) wait(b + 1);
            break;
        }
    }
    gb += (uint32_t)issued;
    if (!ok) s.done = true;
}

template <int KIND>
__device__ __forceinline__ void write_ray(const SensorDev& sd, const TileRay& ray, const RayState& s,
                                          const FrameOut& out)
{
    if (!ray.inside) return;
    const size_t HW = (size_t)sd.width * sd.height;
    const size_t pix = (size_t)ray.y * sd.width + ray.x;
    if (KIND != GSR_SENSOR_LIDAR) {
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
        if (out.drop) out.drop[pix] = s.f1 + s.T;  // a beam that leaves the scene is dropped
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

// ------------------------------------------------------------- split tiles
// A tile whose list is longer than `first` positions is walked in chunks:
// chunk 0 = the first `first` positions, then chunks of `chunk` positions
// (gsr_tiling.split_first / split_chunk).  Chunk 0 is walked like any tile
// (with each ray's
// stop rule).  If rays are still alive after it, their state is stored
// (the carry) and chunks 1..C are walked in parallel by other CTAs, each
// from T = 1 with the same stop rule (a partial).  Exactness: with T_s the
// transmittance entering chunk c and P_c the partial's transmittance, no
// ray stops inside chunk c iff the partial did not stop and T_s P_c >= 1e-4
// (T only decreases); its weights are then T_s times the partial's, so the
// chunk merges as C += T_s C_c, T = T_s P_c.  A ray that stops inside chunk
// c walks that chunk again from T_s, record by record.  The CTA that
// finishes a tile's last chunk merges them in list order.
// Phase A: the tile's list (or its chunk 0).  Threads beyond the tile's rays
// only help staging.
template <int KIND>
__device__ __forceinline__ void render_tile(const SensorDev& sd, const float2* dirs, int local_tile, uint32_t tile,
                                            const uint2 range,
                                            const float4* __restrict__ rec, const uint32_t* __restrict__ pval,
                                            const FrameOut& out, uint32_t* counters, float4* buf, uint64_t* bars,
                                            uint32_t& gb, const SplitBufs& sp, int D)
{
    const TileRay ray = tile_ray<KIND>(sd, dirs, local_tile);
    const int n = (int)(range.y - range.x);
    RayState s;
    ray_init(s, !ray.inside, (uint32_t)n);
    const uint4 info = sp.info[tile];
    const bool split = info.x > 0;
    walk_list<KIND>(sd, ray, range.x, 0, split ? sd.split_first : n, rec, pval, s, counters, buf, bars, gb, D);
    if (split) {
        const int R = sd.tile_w * sd.tile_h;
        if (!__syncthreads_and(s.done)) {
            if ((int)threadIdx.x < R) store_ray(ray_block(sp, info.y, R, 0), R, threadIdx.x, s);
            if (threadIdx.x == 0) sp.state[tile] = make_uint2(1u, info.x);
            return;
        }
        if (threadIdx.x == 0) sp.state[tile] = make_uint2(2u, info.x);
    }
    write_ray<KIND>(sd, ray, s, out);
}

// Phase B: chunk c of a split tile; the CTA that walks the tile's last
// remaining chunk merges all of them and writes the tile's outputs.
template <int KIND>
__device__ __forceinline__ void render_chunk(const SensorDev& sd, const float2* dirs, int local_tile, uint32_t tile,
                                             int c,
                                             const uint2 range, const float4* __restrict__ rec,
                                             const uint32_t* __restrict__ pval, const FrameOut& out,
                                             uint32_t* counters, float4* buf, uint64_t* bars, uint32_t& gb,
                                             const SplitBufs& sp, uint32_t* flag_s, int D)
{
    const TileRay ray = tile_ray<KIND>(sd, dirs, local_tile);
    const int n = (int)(range.y - range.x);
    const int R = sd.tile_w * sd.tile_h;
    const int r = threadIdx.x;
    const uint4 info = sp.info[tile];
    const uint32_t st = __ldcg(&sp.state[tile].x);
    if (st == 1u) {
        RayState carry, s;
        bool done = true;
        if (r < R) {
            load_ray(ray_block(sp, info.y, R, 0), R, r, carry);
            done = carry.done;
        }
        ray_init(s, done, (uint32_t)n);
        walk_list<KIND>(sd, ray, range.x, chunk_begin(sd.split_first, sd.split_chunk, c),
                        min(n, chunk_begin(sd.split_first, sd.split_chunk, c + 1)), rec, pval, s, counters,
                        buf, bars, gb, D);
        if (r < R) store_ray(ray_block(sp, info.y, R, c), R, r, s);
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) *flag_s = atomicSub(&sp.state[tile].y, 1u) == 1u ? 1u : 0u;
    __syncthreads();
    if (!*flag_s || st != 1u) return;
    __threadfence();

    // merge chunks 1..C in list order onto the carry
    RayState S;
    ray_init(S, true, (uint32_t)n);
    if (r < R) load_ray(ray_block(sp, info.y, R, 0), R, r, S);
    const int C = (int)info.x;
    for (int k = 1; k <= C; ++k) {
        bool need = false;
        if (!S.done) {
            RayState p;
            load_ray(ray_block(sp, info.y, R, k), R, r, p);
            const float Tn = S.T * p.T;
            if (!p.done && Tn >= kTMin) {
                S.f0 = fmaf(S.T, p.f0, S.f0);
                S.f1 = fmaf(S.T, p.f1, S.f1);
                S.f2 = fmaf(S.T, p.f2, S.f2);
                S.n0 = fmaf(S.T, p.n0, S.n0);
                S.n1 = fmaf(S.T, p.n1, S.n1);
                S.n2 = fmaf(S.T, p.n2, S.n2);
                S.A = fmaf(S.T, p.A, S.A);
                S.B = fmaf(S.T, p.B, S.B);
                S.D = fmaf(S.T, p.D, S.D);
                if (p.last) S.last = p.last;
                S.T = Tn;
            } else {
                need = true;
            }
        }
        if (__syncthreads_or(need)) {
            // rays that stop inside chunk k walk it again from their state
            const bool was = S.done;
            S.done = S.done || !need;
            walk_list<KIND>(sd, ray, range.x, chunk_begin(sd.split_first, sd.split_chunk, k),
                            min(n, chunk_begin(sd.split_first, sd.split_chunk, k + 1)), rec, pval, S,
                            counters, buf, bars, gb, D);
            if (!need) S.done = was;
        }
        // block k now holds the state after chunk k (the backward starts its
        // walk of chunk k - 1 there); kept only by a render that writes the
        // final T, the backward's input
        if (out.trans != nullptr && r < R) store_ray(ray_block(sp, info.y, R, k), R, r, S);
    }
    write_ray<KIND>(sd, ray, S, out);
}

__device__ __forceinline__ void init_bars(uint64_t* bars)
{
    if (threadIdx.x == 0) {
        mbar_init(bars, 1);
        mbar_init(bars + 1, 1);
        fence_mbar_init();
    }
}

template <int KIND>
__global__ void __launch_bounds__(256) k_render(SensorTable tab, int sensor, const float4* __restrict__ rec,
                                                const uint2* __restrict__ ranges, const uint32_t* __restrict__ pval,
                                                FrameOut out, uint32_t* counters, SplitBufs sp)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    float4* buf = reinterpret_cast<float4*>(smem_raw + 128);
    const SensorDev& sd = tab.s[sensor];
    init_bars(bars);
    __syncthreads();
    const int lt = blockIdx.x;
    const uint32_t tile = (uint32_t)(sd.tile_base + lt);
    uint32_t gb = 0;
    render_tile<KIND>(sd, tab.dirs, lt, tile, ranges[tile], rec, pval, out, counters, buf, bars, gb, sp,
                      tab.batch > 0 ? tab.batch : (int)blockDim.x);
}

// Outputs of every sensor of a plan, for the whole-rig kernels.
struct RigOut {
    FrameOut o[GSR_MAX_SENSORS];
};

__device__ __forceinline__ int sensor_of_tile(const SensorTable& tab, uint32_t tile)
{
    int s = 0;
    while (s + 1 < tab.n && (int)tile >= tab.s[s + 1].tile_base) ++s;
    return s;
}

// The whole rig in one persistent launch: each CTA takes the next tile from a
// global work queue that lists every sensor's tiles longest list first, so
// the long LiDAR and near-field tiles start early and the short ones fill in
// behind them; the sensor kind is uniform per tile, so the branch is too.
__global__ void __launch_bounds__(256, GSR_RIG_MIN_CTAS) k_render_rig(SensorTable tab, const float4* __restrict__ rec,
                                                    const uint2* __restrict__ ranges,
                                                    const uint32_t* __restrict__ pval,
                                                    const uint32_t* __restrict__ order, RigOut outs,
                                                    uint32_t* counters, SplitBufs sp)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    float4* buf = reinterpret_cast<float4*>(smem_raw + 128);
    __shared__ uint32_t item_s;
    init_bars(bars);
    uint32_t gb = 0;
    const int D = tab.batch > 0 ? tab.batch : (int)blockDim.x;
    const uint32_t T = (uint32_t)tab.total_tiles;
    for (;;) {
        __syncthreads();  // the previous item (and the barrier init) is done with
        // after a bounded wait gave up anywhere, the frame is void: take no more work
        if (threadIdx.x == 0)
            item_s = __ldcg(&counters[C_STATUS]) == (uint32_t)GSR_ERR_TIMEOUT ? T : atomicAdd(&counters[C_QUEUE], 1u);
        __syncthreads();
        const uint32_t item = item_s;
        if (item >= T) break;
        const uint32_t tile = order[item];
        const int s = sensor_of_tile(tab, tile);
        const SensorDev& sd = tab.s[s];
        const int lt = (int)tile - sd.tile_base;
        if (sd.kind == GSR_SENSOR_PINHOLE)
            render_tile<GSR_SENSOR_PINHOLE>(sd, tab.dirs, lt, tile, ranges[tile], rec, pval, outs.o[s], counters,
                                            buf, bars, gb, sp, D);
        else if (sd.kind == GSR_SENSOR_CYLINDRICAL)
            render_tile<GSR_SENSOR_CYLINDRICAL>(sd, tab.dirs, lt, tile, ranges[tile], rec, pval, outs.o[s],
                                                counters, buf, bars, gb, sp, D);
        else
            render_tile<GSR_SENSOR_LIDAR>(sd, tab.dirs, lt, tile, ranges[tile], rec, pval, outs.o[s], counters, buf,
                                          bars, gb, sp, D);
    }
}

// Phase B over the split items of every sensor (only < 0) or of one sensor.
__global__ void __launch_bounds__(256, GSR_RIG_MIN_CTAS) k_render_split(SensorTable tab, const float4* __restrict__ rec,
                                                      const uint2* __restrict__ ranges,
                                                      const uint32_t* __restrict__ pval, RigOut outs,
                                                      uint32_t* counters, SplitBufs sp, int only)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
    float4* buf = reinterpret_cast<float4*>(smem_raw + 128);
    __shared__ uint32_t item_s, flag_s;
    init_bars(bars);
    const uint32_t n_items = counters[C_NITEMS];
    uint32_t begin = 0, end = n_items;
    if (only >= 0) {
        begin = sp.info[tab.s[only].tile_base].z;
        if (only + 1 < tab.n) end = sp.info[tab.s[only + 1].tile_base].z;
    }
    uint32_t gb = 0;
    const int D = tab.batch > 0 ? tab.batch : (int)blockDim.x;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0)
            item_s = __ldcg(&counters[C_STATUS]) == (uint32_t)GSR_ERR_TIMEOUT
                         ? end
                         : begin + atomicAdd(&counters[C_SPLIT_QUEUE], 1u);
        __syncthreads();
        const uint32_t item = item_s;
        if (item >= end) break;
        const uint2 it = sp.items[item];
        const uint32_t tile = it.x;
        const int s = sensor_of_tile(tab, tile);
        const SensorDev& sd = tab.s[s];
        const int lt = (int)tile - sd.tile_base;
        if (sd.kind == GSR_SENSOR_PINHOLE)
            render_chunk<GSR_SENSOR_PINHOLE>(sd, tab.dirs, lt, tile, (int)it.y, ranges[tile], rec, pval, outs.o[s],
                                             counters, buf, bars, gb, sp, &flag_s, D);
        else if (sd.kind == GSR_SENSOR_CYLINDRICAL)
            render_chunk<GSR_SENSOR_CYLINDRICAL>(sd, tab.dirs, lt, tile, (int)it.y, ranges[tile], rec, pval, outs.o[s],
                                                 counters, buf, bars, gb, sp, &flag_s, D);
        else
            render_chunk<GSR_SENSOR_LIDAR>(sd, tab.dirs, lt, tile, (int)it.y, ranges[tile], rec, pval, outs.o[s],
                                           counters, buf, bars, gb, sp, &flag_s, D);
    }
}

// Self-test of the bounded wait: an mbarrier armed for 16 bytes that no copy
// will deliver, waited on with `tries` tries by the same helper every staging
// wait of the library uses.  The wait gives up, records GSR_ERR_TIMEOUT in the
// status word and the kernel returns; no copy or tensor-core operation is
// outstanding at any point.
__global__ void __launch_bounds__(32) k_selftest_wait(uint32_t* counters, uint32_t tries)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16u);
    mbar_wait_bounded(&bar, 0u, counters, tries);
}

cudaError_t launch_selftest_wait(uint32_t* counters, uint32_t tries, cudaStream_t stream)
{
    k_selftest_wait<<<1, 32, 0, stream>>>(counters, tries);
    return cudaGetLastError();
}

// Dynamic shared memory of a compositing CTA staging D records per batch.
size_t render_smem_bytes(int D) { return 128 + 2 * (size_t)D * kRecordBytes; }

static int batch_of(const SensorTable& tab, int threads) { return tab.batch > 0 ? tab.batch : threads; }

// Opt in to more than 48 KB of dynamic shared memory where a batch needs it.
template <class K>
static cudaError_t smem_attr(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

SplitBufs split_bufs(const gsr_plan* p, const void* ws)
{
    SplitBufs sp;
    sp.info = region<uint4>(p, ws, R_SPLIT_INFO);
    sp.state = region<uint2>(p, ws, R_SPLIT_STATE);
    sp.items = region<uint2>(p, ws, R_SPLIT_ITEMS);
    sp.rays = region<float>(p, ws, R_SPLIT_RAYS);
    return sp;
}

// Persistent CTAs for the rig and split kernels: resident CTAs per SM x SMs
// of the current device, for CTAs of `threads` threads (32..256, a power of
// two) with `smem` bytes of dynamic shared memory (D = 32..512 records).
static int persistent_grid(int which, int threads, size_t smem, cudaError_t& err)
{
    static int cached[64][2][4][6] = {};
    int dev = 0;
    err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return 0;
    const int ti = threads <= 32 ? 0 : threads <= 64 ? 1 : threads <= 128 ? 2 : 3;
    int bi = 0;
    while (bi < 5 && render_smem_bytes(32 << bi) < smem) ++bi;
    if (dev >= 0 && dev < 64 && cached[dev][which][ti][bi] > 0) return cached[dev][which][ti][bi];
    int sms = 0, per_sm = 0;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return 0;
    if (which == 0)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_rig, threads, smem);
    else
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_split, threads, smem);
    if (err != cudaSuccess) return 0;
    const int g = sms * (per_sm > 0 ? per_sm : 1);
    if (dev >= 0 && dev < 64) cached[dev][which][ti][bi] = g;
    return g;
}

// Phase B (the chunks of split tiles) of one sensor (only >= 0) or of all.
static cudaError_t launch_split(const gsr_plan* p, const void* ws, const SensorTable& tab, const RigOut& ro,
                                int threads, int only, cudaStream_t st)
{
    uint32_t* counters = region<uint32_t>(p, ws, R_COUNTERS);
    cudaError_t e = cudaMemsetAsync(counters + C_SPLIT_QUEUE, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const size_t smem = render_smem_bytes(batch_of(tab, threads));
    if ((e = smem_attr(k_render_split, smem)) != cudaSuccess) return e;
    const int grid = persistent_grid(1, threads, smem, e);
    if (e != cudaSuccess) return e;
    const int pb = sort_result_buffer(tile_sort_passes(p));
    k_render_split<<<grid, threads, smem, st>>>(
        tab, region<float4>(p, ws, R_RECORDS), region<uint2>(p, ws, R_RANGES),
        region<uint32_t>(p, ws, pb ? R_PAIR_VAL_B : R_PAIR_VAL_A), ro, counters, split_bufs(p, ws), only);
    return cudaGetLastError();
}

cudaError_t launch_render(const gsr_plan* p, const void* ws, int sensor, const FrameOut& out, cudaStream_t st)
{
    const SensorTable tab = make_sensor_table(p, ws);
    const SensorDev& sd = tab.s[sensor];
    const int threads = sd.tile_w * sd.tile_h;
    const size_t smem = render_smem_bytes(batch_of(tab, threads));
    const int tiles = sd.tiles_x * sd.tiles_y;
    const float4* rec = region<float4>(p, ws, R_RECORDS);
    const uint2* ranges = region<uint2>(p, ws, R_RANGES);
    const int pb = sort_result_buffer(tile_sort_passes(p));
    const uint32_t* pval = region<uint32_t>(p, ws, pb ? R_PAIR_VAL_B : R_PAIR_VAL_A);
    uint32_t* counters = region<uint32_t>(p, ws, R_COUNTERS);
    const SplitBufs sp = split_bufs(p, ws);
    cudaError_t e;
    if (sd.kind == GSR_SENSOR_PINHOLE) {
        if ((e = smem_attr(k_render<GSR_SENSOR_PINHOLE>, smem)) != cudaSuccess) return e;
        k_render<GSR_SENSOR_PINHOLE><<<tiles, threads, smem, st>>>(tab, sensor, rec, ranges, pval, out, counters,
                                                                   sp);
    } else if (sd.kind == GSR_SENSOR_CYLINDRICAL) {
        if ((e = smem_attr(k_render<GSR_SENSOR_CYLINDRICAL>, smem)) != cudaSuccess) return e;
        k_render<GSR_SENSOR_CYLINDRICAL><<<tiles, threads, smem, st>>>(tab, sensor, rec, ranges, pval, out,
                                                                       counters, sp);
    } else {
        if ((e = smem_attr(k_render<GSR_SENSOR_LIDAR>, smem)) != cudaSuccess) return e;
        k_render<GSR_SENSOR_LIDAR><<<tiles, threads, smem, st>>>(tab, sensor, rec, ranges, pval, out, counters, sp);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    RigOut ro;
    for (int i = 0; i < GSR_MAX_SENSORS; ++i) ro.o[i] = FrameOut{};
    ro.o[sensor] = out;
    return launch_split(p, ws, tab, ro, threads, sensor, st);
}

cudaError_t launch_render_rig(const gsr_plan* p, const void* ws, const FrameOut* outs, cudaStream_t st)
{
    const SensorTable tab = make_sensor_table(p, ws);
    RigOut ro;
    for (int i = 0; i < GSR_MAX_SENSORS; ++i) ro.o[i] = i < p->n_sensors ? outs[i] : FrameOut{};
    uint32_t* counters = region<uint32_t>(p, ws, R_COUNTERS);
    cudaError_t e = cudaMemsetAsync(counters + C_QUEUE, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    // one CTA per tile in flight, as wide as the largest tile of the plan
    int threads = 32;
    for (int i = 0; i < p->n_sensors; ++i) threads = max(threads, tab.s[i].tile_w * tab.s[i].tile_h);
    const size_t smem = render_smem_bytes(batch_of(tab, threads));
    if ((e = smem_attr(k_render_rig, smem)) != cudaSuccess) return e;
    const int grid = persistent_grid(0, threads, smem, e);
    if (e != cudaSuccess) return e;
    const int pb = sort_result_buffer(tile_sort_passes(p));
    k_render_rig<<<grid, threads, smem, st>>>(
        tab, region<float4>(p, ws, R_RECORDS), region<uint2>(p, ws, R_RANGES),
        region<uint32_t>(p, ws, pb ? R_PAIR_VAL_B : R_PAIR_VAL_A), region<uint32_t>(p, ws, R_TILE_VAL_A), ro,
        counters, split_bufs(p, ws));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_split(p, ws, tab, ro, threads, -1, st);
}

}  // namespace gsr
