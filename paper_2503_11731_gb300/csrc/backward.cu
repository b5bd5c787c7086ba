// backward.cu -- reconstruction loss and the hand-written backward pass.
//
//  k_loss_pixel / k_loss_gather / k_loss_reduce
//      L1 + depth distortion + normal consistency (the 2DGS regularisers
//      of the representation the paper adopts, Sec. II / III-A) and the
//      per-pixel gradients w.r.t. the camera outputs.
//  k_render_backward
//      reverse-order walk of each tile list from every pixel's last
//      contributor; T_i is recovered as T_{i+1} / (1 - alpha_i) from the
//      final T, so no per-pixel list is stored.  Per-record gradients are
//      reduced over the warp before the FP32 atomics.
//  k_preprocess_backward
//      chains the record gradients to the raw surfel parameters (the
//      inverse of the preprocess of Eqs. 1-3), one thread per surfel,
//      summing over sensors without atomics.
#include <atomic>
#include <mutex>

#include "gsr_internal.cuh"

namespace gsr {

namespace {

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

}  // namespace

// ===================================================================== loss
struct LossArgs {
    const float* rgb;
    const float* alpha;
    const float* dacc;     // [2][H][W]
    const float* normal;
    const float* target;
    float* g_rgb;
    float* g_alpha;
    float* g_dacc;
    float* g_normal;
    float* scratch;        // [6][H][W]: dL/d(dX), dL/d(dY) per pixel
    float* partial;        // [blocks][3]
    int W, H;
    int cyl;               // 1: cylindrical camera (Eq. 4), 0: pinhole
    float fx, fy, cx, cy;
    float w_dist, w_norm, mask_alpha;
};

// Direction whose multiple by the rendered depth is the back-projected point
// of pixel (x, y): pinhole ((x + 1/2 - cx)/fx, (y + 1/2 - cy)/fy, 1);
// cylindrical (sin phi, y_n, cos phi), its depth being the horizontal distance.
__device__ __forceinline__ void backproject_dir(const LossArgs& a, int x, int y, float* d)
{
    const float u = (x + 0.5f - a.cx) / a.fx, v = (y + 0.5f - a.cy) / a.fy;
    if (a.cyl) {
        sincosf(u, &d[0], &d[2]);
        d[1] = v;
    } else {
        d[0] = u;
        d[1] = v;
        d[2] = 1.f;
    }
}

// Pass 1: per-pixel terms, the direct gradients, and the gradient of the
// normal term w.r.t. the two central differences of this pixel.
__global__ void __launch_bounds__(256) k_loss_pixel(LossArgs a)
{
    __shared__ float red[3][8];
    const int HW = a.W * a.H;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    float l1 = 0.f, dist = 0.f, nc = 0.f;
    if (p < HW) {
        const int x = p % a.W, y = p / a.W;
        const float inv3 = 1.f / (3.f * HW), inv = 1.f / HW;
        for (int c = 0; c < 3; ++c) {
            const float d = a.rgb[c * HW + p] - a.target[c * HW + p];
            l1 += fabsf(d);
            a.g_rgb[c * HW + p] = sgnf(d) * inv3;
        }
        const float A = a.alpha[p], B = a.dacc[p], D = a.dacc[HW + p];
        dist = fmaf(A, D, -B * B);
        a.g_alpha[p] = a.w_dist * D * inv;
        a.g_dacc[p] = -2.f * a.w_dist * B * inv;
        a.g_dacc[HW + p] = a.w_dist * A * inv;
        float gN0 = 0.f, gN1 = 0.f, gN2 = 0.f;
        float gdx[3] = {0.f, 0.f, 0.f}, gdy[3] = {0.f, 0.f, 0.f};
        if (x > 0 && x + 1 < a.W && y > 0 && y + 1 < a.H) {
            const int qs[4] = {p - 1, p + 1, p - a.W, p + a.W};
            const int qx[4] = {x - 1, x + 1, x, x};
            const int qy[4] = {y, y, y - 1, y + 1};
            float X[4][3];
            bool ok = true;
            for (int k = 0; k < 4; ++k) {
                const float Aq = a.alpha[qs[k]];
                ok = ok && (Aq >= a.mask_alpha);
                const float Db = Aq > 0.f ? a.dacc[qs[k]] / Aq : 0.f;
                float dir[3];
                backproject_dir(a, qx[k], qy[k], dir);
                X[k][0] = dir[0] * Db;
                X[k][1] = dir[1] * Db;
                X[k][2] = dir[2] * Db;
            }
            const float dX[3] = {X[1][0] - X[0][0], X[1][1] - X[0][1], X[1][2] - X[0][2]};
            const float dY[3] = {X[3][0] - X[2][0], X[3][1] - X[2][1], X[3][2] - X[2][2]};
            // cr = dY x dX
            const float cr[3] = {dY[1] * dX[2] - dY[2] * dX[1], dY[2] * dX[0] - dY[0] * dX[2],
                                 dY[0] * dX[1] - dY[1] * dX[0]};
            const float nrm = sqrtf(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
            if (ok && nrm > 0.f) {
                const float Nd[3] = {cr[0] / nrm, cr[1] / nrm, cr[2] / nrm};
                const float N[3] = {a.normal[p], a.normal[HW + p], a.normal[2 * HW + p]};
                nc = 1.f - (N[0] * Nd[0] + N[1] * Nd[1] + N[2] * Nd[2]);
                const float s = -a.w_norm * inv;
                gN0 = s * Nd[0];
                gN1 = s * Nd[1];
                gN2 = s * Nd[2];
                const float gNd[3] = {s * N[0], s * N[1], s * N[2]};
                const float dd = Nd[0] * gNd[0] + Nd[1] * gNd[1] + Nd[2] * gNd[2];
                const float gcr[3] = {(gNd[0] - Nd[0] * dd) / nrm, (gNd[1] - Nd[1] * dd) / nrm,
                                      (gNd[2] - Nd[2] * dd) / nrm};
                // cr = dY x dX: dL/d dY = dX x gcr, dL/d dX = gcr x dY
                gdy[0] = dX[1] * gcr[2] - dX[2] * gcr[1];
                gdy[1] = dX[2] * gcr[0] - dX[0] * gcr[2];
                gdy[2] = dX[0] * gcr[1] - dX[1] * gcr[0];
                gdx[0] = gcr[1] * dY[2] - gcr[2] * dY[1];
                gdx[1] = gcr[2] * dY[0] - gcr[0] * dY[2];
                gdx[2] = gcr[0] * dY[1] - gcr[1] * dY[0];
            }
        }
        a.g_normal[p] = gN0;
        a.g_normal[HW + p] = gN1;
        a.g_normal[2 * HW + p] = gN2;
        for (int k = 0; k < 3; ++k) {
            a.scratch[k * HW + p] = gdx[k];
            a.scratch[(3 + k) * HW + p] = gdy[k];
        }
    }
    // block partial sums (fixed order: deterministic)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    l1 = warp_sum(l1);
    dist = warp_sum(dist);
    nc = warp_sum(nc);
    if (lane == 0) {
        red[0][w] = l1;
        red[1][w] = dist;
        red[2][w] = nc;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        float s = 0.f;
        for (int k = 0; k < 8; ++k) s += red[threadIdx.x][k];
        a.partial[blockIdx.x * 3 + threadIdx.x] = s;
    }
}

// Pass 2: each pixel gathers dL/dX from the central differences of its four
// neighbours, then dL/d(expected depth) -> dL/dB, dL/dA.
__global__ void __launch_bounds__(256) k_loss_gather(LossArgs a)
{
    const int HW = a.W * a.H;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= HW) return;
    const int x = p % a.W, y = p / a.W;
    float gX[3] = {0.f, 0.f, 0.f};
    // dX(q) = X(q.x+1) - X(q.x-1): pixel p is q.x+1 for q = p-1 and q.x-1 for q = p+1
    for (int k = 0; k < 3; ++k) {
        if (x > 0) gX[k] += a.scratch[k * HW + p - 1];
        if (x + 1 < a.W) gX[k] -= a.scratch[k * HW + p + 1];
        if (y > 0) gX[k] += a.scratch[(3 + k) * HW + p - a.W];
        if (y + 1 < a.H) gX[k] -= a.scratch[(3 + k) * HW + p + a.W];
    }
    const float A = a.alpha[p];
    if (A > 0.f) {
        float dir[3];
        backproject_dir(a, x, y, dir);
        const float gD = gX[0] * dir[0] + gX[1] * dir[1] + gX[2] * dir[2];
        const float B = a.dacc[p];
        a.g_dacc[p] += gD / A;
        a.g_alpha[p] += -gD * B / (A * A);
    }
}

__global__ void k_loss_reduce(const float* __restrict__ partial, int nblocks, float w_dist, float w_norm, int HW,
                              float* __restrict__ loss)
{
    __shared__ double red[3][32];
    double s[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 3; ++k) s[k] += partial[b * 3 + k];
    for (int k = 0; k < 3; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 3; ++k)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t[k] += red[k][w];
        const double l1 = t[0] / (3.0 * HW), dist = t[1] / HW, nc = t[2] / HW;
        loss[1] = (float)l1;
        loss[2] = (float)(w_dist * dist);
        loss[3] = (float)(w_norm * nc);
        loss[0] = (float)(l1 + w_dist * dist + w_norm * nc);
    }
}

// ================================================================ LiDAR loss
// Per ray: m = 1 where the target has a return (target range > 0);
//   L = w_range mean_m |range - range*| + w_int mean_m |I - I*|
//     + w_drop mean_all BCE(clamp(drop, eps, 1 - eps), [range* <= 0]).
struct LidarLossArgs {
    const float* range;
    const float* alpha;
    const float* intensity;
    const float* drop;
    const float* t_range;
    const float* t_int;
    float* g_alpha;
    float* g_dacc;       // [2][B][C]
    float* g_int;
    float* g_drop;
    float* partial;      // [blocks][4]: returns, sum |dr|, sum |dI|, sum BCE
    float* inv;          // [2]: 1 / returns (0 if none), 1 / rays
    int n;
    float w_range, w_int, w_drop;
};
constexpr float kDropEps = 0x1p-20f;  // 1 - eps is exact in FP32

__global__ void __launch_bounds__(256) k_lidar_loss_terms(LidarLossArgs a)
{
    __shared__ float red[4][8];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (p < a.n) {
        const bool ret = a.t_range[p] > 0.f;
        if (ret) {
            v[0] = 1.f;
            v[1] = fabsf(a.range[p] - a.t_range[p]);
            v[2] = fabsf(a.intensity[p] - a.t_int[p]);
        }
        const float pc = fminf(fmaxf(a.drop[p], kDropEps), 1.f - kDropEps);
        v[3] = ret ? -logf(1.f - pc) : -logf(pc);
    }
    for (int k = 0; k < 4; ++k) {
        const float s = warp_sum(v[k]);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        a.partial[blockIdx.x * 4 + threadIdx.x] = s;
    }
}

__global__ void k_lidar_loss_reduce(LidarLossArgs a, int nblocks, float* __restrict__ loss)
{
    __shared__ double red[4][32];
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 4; ++k) s[k] += a.partial[b * 4 + k];
    for (int k = 0; k < 4; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k = 0; k < 4; ++k)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t[k] += red[k][w];
        const double im = t[0] > 0.0 ? 1.0 / t[0] : 0.0, ia = 1.0 / a.n;
        const double lr = a.w_range * t[1] * im, li = a.w_int * t[2] * im, ld = a.w_drop * t[3] * ia;
        loss[0] = (float)(lr + li + ld);
        loss[1] = (float)lr;
        loss[2] = (float)li;
        loss[3] = (float)ld;
        a.inv[0] = (float)im;
        a.inv[1] = (float)ia;
    }
}

__global__ void __launch_bounds__(256) k_lidar_loss_grad(LidarLossArgs a)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n) return;
    const float im = a.inv[0], ia = a.inv[1];
    const bool ret = a.t_range[p] > 0.f;
    // range = B / A where A > 0 (0 elsewhere, with no gradient)
    const float A = a.alpha[p], r = a.range[p];
    const float gr = ret ? a.w_range * im * sgnf(r - a.t_range[p]) : 0.f;
    const float gB = A > 0.f ? gr / A : 0.f;
    a.g_dacc[p] = gB;
    a.g_dacc[a.n + p] = 0.f;
    a.g_alpha[p] = -gB * r;
    a.g_int[p] = ret ? a.w_int * im * sgnf(a.intensity[p] - a.t_int[p]) : 0.f;
    const float d = a.drop[p];
    const float y = ret ? 0.f : 1.f;
    a.g_drop[p] = (d > kDropEps && d < 1.f - kDropEps) ? a.w_drop * ia * (d - y) / (d * (1.f - d)) : 0.f;
}

// ======================================================= backward rasteriser
constexpr int kGradComponents = 20;  // record-gradient floats written (r0..r4)

struct TileRayBox {
    int x, y;
    bool live;
};

// Ray-index box (x0, x1, y0, y1) of the warp's live rays (empty if none).
__device__ __forceinline__ float4 warp_ray_box(const TileRayBox& r)
{
    const int x0 = __reduce_min_sync(0xffffffffu, r.live ? r.x : 0x7fffffff);
    const int x1 = __reduce_max_sync(0xffffffffu, r.live ? r.x : -1);
    const int y0 = __reduce_min_sync(0xffffffffu, r.live ? r.y : 0x7fffffff);
    const int y1 = __reduce_max_sync(0xffffffffu, r.live ? r.y : -1);
    return make_float4((float)x0, (float)x1, (float)y0, (float)y1);
}

struct BwdArgs {
    const float* trans;
    const uint32_t* n_contrib;
    const float* g_rgb;     // [3][H][W] (LiDAR: the intensity, [H][W])
    const float* g_alpha;
    const float* g_dacc;    // [2][H][W]
    const float* g_normal;  // [3][H][W] (camera only)
    const float* g_drop;    // [H][W] (LiDAR only: d/d(sum w rho + T))
    float4* recgrad;        // [slots][5]
};

// The tiles of one sensor in the plan's schedule order (longest list first),
// by a stable compaction of the whole-rig tile order (one CTA).
__global__ void __launch_bounds__(1024) k_sensor_order(const uint32_t* __restrict__ order, uint32_t n_tiles,
                                                       uint32_t t0, uint32_t t1, uint32_t* __restrict__ out)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t base_s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) base_s = 0;
    __syncthreads();
    for (uint32_t i0 = 0; i0 < n_tiles; i0 += 1024) {
        const uint32_t i = i0 + threadIdx.x;
        const uint32_t t = i < n_tiles ? order[i] : 0xffffffffu;
        const bool mine = t >= t0 && t < t1;
        const uint32_t bal = __ballot_sync(0xffffffffu, mine);
        if (lane == 0) wsum[w] = __popc(bal);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int k = 0; k < 32; ++k) {
            if (k < w) before += wsum[k];
            total += wsum[k];
        }
        if (mine) out[base_s + before + __popc(bal & ((1u << lane) - 1u))] = t;
        __syncthreads();
        if (threadIdx.x == 0) base_s += total;
        __syncthreads();
    }
}

// Reverse walk of one tile (or of one chunk of a split tile) by the whole
// CTA: list positions [lo_pos, min(hi_pos, last)) of each ray, from the back.
// mode 0 starts at the ray's end (T = final transmittance, nothing behind);
// mode 1 starts at the end of chunk cc of a split tile from the state the
// forward merge stored there (block cc) and the final state (block C): the
// contributions behind are the final sums minus those in front.
template <int KIND>
__device__ __forceinline__ void bwd_tile(const SensorTable& tab, const SensorDev& sd, int lt, int lo_pos,
                                         int hi_pos, int mode, const SplitBufs& sp, int cc, const float4* __restrict__ rec,
                                         const uint2* __restrict__ ranges, const uint32_t* __restrict__ pval,
                                         const BwdArgs& a, uint32_t* counters, uint64_t* bars, uint32_t* sslot,
                                         float4* buf, uint32_t* wmax, uint32_t& gb)
{
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int tx = lt % sd.tiles_x, ty = lt / sd.tiles_x;
    int lx, ly;
    tile_ray_xy(sd.tile_w, sd.tile_h, tid, lx, ly);
    const int x = tx * sd.tile_w + lx;
    const int y = ty * sd.tile_h + ly;
    const bool inside = tid < sd.tile_w * sd.tile_h && x < sd.width && y < sd.height;
    const size_t HW = (size_t)sd.width * sd.height;
    const size_t pix = (size_t)y * sd.width + x;
    const uint32_t tile = (uint32_t)(sd.tile_base + lt);
    float rx, ry, d0, d1, d2;
    ray_setup<KIND>(sd, tab.dirs, x, y, rx, ry, d0, d1, d2);
    const uint2 range = ranges[tile];
    uint32_t last = 0;
    float T = 1.f;
    float gC[3] = {0.f, 0.f, 0.f}, gN[3] = {0.f, 0.f, 0.f}, gA = 0.f, gB = 0.f, gD = 0.f;
    // accumulated contributions of the surfels behind the current one
    float Ca[3] = {0.f, 0.f, 0.f};
    float Aa = 0.f, Ba = 0.f, Da = 0.f, Na[3] = {0.f, 0.f, 0.f};
    if (inside) {
        last = min(a.n_contrib[pix], (uint32_t)hi_pos);
        if (mode == 0) {
            T = a.trans[pix];
            if (KIND == GSR_SENSOR_LIDAR) {
                Ca[1] = T;  // a beam that leaves the scene is dropped: the drop's background is 1
            } else {
                Ca[0] = T * sd.bg[0];
                Ca[1] = T * sd.bg[1];
                Ca[2] = T * sd.bg[2];
            }
        } else {
            const int R = sd.tile_w * sd.tile_h;
            const uint4 info = sp.info[tile];
            RayState Sc, Sf;
            load_ray(ray_block(sp, info.y, R, cc), R, tid, Sc);
            load_ray(ray_block(sp, info.y, R, (int)info.x), R, tid, Sf);
            T = Sc.T;
            if (KIND == GSR_SENSOR_LIDAR) {
                Ca[0] = Sf.f0 - Sc.f0;
                Ca[1] = (Sf.f1 - Sc.f1) + Sf.T;
            } else {
                Ca[0] = (Sf.f0 - Sc.f0) + Sf.T * sd.bg[0];
                Ca[1] = (Sf.f1 - Sc.f1) + Sf.T * sd.bg[1];
                Ca[2] = (Sf.f2 - Sc.f2) + Sf.T * sd.bg[2];
            }
            Aa = Sf.A - Sc.A;
            Ba = Sf.B - Sc.B;
            Da = Sf.D - Sc.D;
            Na[0] = Sf.n0 - Sc.n0;
            Na[1] = Sf.n1 - Sc.n1;
            Na[2] = Sf.n2 - Sc.n2;
        }
        if (last <= (uint32_t)lo_pos) last = 0;  // nothing of this ray in [lo_pos, hi_pos)
        if (KIND == GSR_SENSOR_LIDAR) {
            if (a.g_rgb) gC[0] = a.g_rgb[pix];
            if (a.g_drop) gC[1] = a.g_drop[pix];
        } else if (a.g_rgb) {
            gC[0] = a.g_rgb[pix];
            gC[1] = a.g_rgb[HW + pix];
            gC[2] = a.g_rgb[2 * HW + pix];
        }
        if (a.g_normal) {
            gN[0] = a.g_normal[pix];
            gN[1] = a.g_normal[HW + pix];
            gN[2] = a.g_normal[2 * HW + pix];
        }
        if (a.g_alpha) gA = a.g_alpha[pix];
        if (a.g_dacc) {
            gB = a.g_dacc[pix];
            gD = a.g_dacc[HW + pix];
        }
    }

    uint32_t m = __reduce_max_sync(0xffffffffu, last);
    const uint32_t wlast = m;  // this warp's rays look at positions < wlast only
    const int lane = tid & 31;
    TileRayBox trb;
    trb.x = x; trb.y = y; trb.live = inside && last > 0;
    const float4 wbox = warp_ray_box(trb);
    __syncthreads();  // the previous walk's readers of wmax and the buffers are done
    if ((tid & 31) == 0) wmax[tid >> 5] = m;
    __syncthreads();
    uint32_t maxlast = 0;
    for (int k = 0; k < (nthr >> 5); ++k) maxlast = max(maxlast, wmax[k]);
    const int span = maxlast > (uint32_t)lo_pos ? (int)maxlast - lo_pos : 0;
    const int nb = (span + nthr - 1) / nthr;
    const float columns = (float)sd.width;

    // batch b covers list positions [lo, hi) counted from the end; it is the
    // CTA's batch g = gb + b (buffer and barrier g & 1, phase (g >> 1) & 1)
    auto issue = [&](int b) {
        const uint32_t g = gb + (uint32_t)b;
        const int hi = (int)maxlast - b * nthr;
        const int lo = max(lo_pos, hi - nthr);
        const int cnt = hi - lo;
        uint64_t* bar = bars + (g & 1);
        float4* dst = buf + (size_t)(g & 1) * nthr * kRecordF4;
        if (tid == 0) mbar_arrive_expect_tx(bar, (uint32_t)cnt * kRecordBytes);
        if (tid < cnt) {
            const uint32_t slot = pval[range.x + lo + tid];
            sslot[(g & 1) * nthr + tid] = slot;
            bulk_g2s(dst + tid * kRecordF4, rec + (size_t)slot * kRecordF4, kRecordBytes, bar);
        }
    };
    bool ok = true;
    if (nb > 0) issue(0);
    for (int b = 0; b < nb; ++b) {
        const uint32_t g = gb + (uint32_t)b;
        if (b + 1 < nb) issue(b + 1);
        if (!mbar_wait_bounded(bars + (g & 1), (g >> 1) & 1, counters)) ok = false;
        ok = __syncthreads_and(ok);  // block-uniform; slot ids of this batch are visible
        const int hi = (int)maxlast - b * nthr;
        const int lo = max(lo_pos, hi - nthr);
        const float4* Bf = buf + (size_t)(g & 1) * nthr * kRecordF4;
        const uint32_t* Sl = sslot + (g & 1) * nthr;
        // groups of 32 positions from the back; a lane per position tests the
        // record's support box against the box of the warp's active rays
        for (int g1 = hi; g1 > lo && ok; g1 -= 32) {
            const int g0 = max(lo, g1 - 32);
            const int jt = g0 + lane;
            bool meet = jt < g1 && box_meets<KIND>(Bf[(jt - lo) * kRecordF4 + 5], wbox, columns) &&
                        (uint32_t)jt < wlast;
            if (KIND == GSR_SENSOR_PINHOLE && meet) {  // and the footprint itself meets the box
                const float4* Rt = Bf + (jt - lo) * kRecordF4;
                meet = footprint_meets_box(Rt[0], Rt[1], Rt[2], Rt[3].x, wbox.x, wbox.y, wbox.z, wbox.w);
            }
            uint32_t mask = __ballot_sync(0xffffffffu, meet);
            // the records of the mask from the highest position, two at a time:
            // both evaluations are independent (their chains interleave), the
            // transmittance recovery and gradients stay in reverse order
            auto apply = [&](const int j, const Splat& sp, const bool contrib) {
                if (!__any_sync(0xffffffffu, contrib)) return;
                const float4* Rj = Bf + (j - lo) * kRecordF4;
                    float g[32];
    #pragma unroll
                    for (int k = 0; k < 32; ++k) g[k] = 0.f;
                    if (contrib) {
                        const float al = sp.alpha, z = sp.z;
                        const float om = 1.f - al;
                        T = T / om;  // transmittance in front of this surfel
                        const float w = al * T;
                        const float4 r3 = Rj[3], r4 = Rj[4];
                        const float io = 1.f / om;
                        float dal = gA * (T - Aa * io) + gB * (T * z - Ba * io) + gD * (T * z * z - Da * io);
                        float c[3] = {r3.y, r3.z, r3.w};
                        if (KIND != GSR_SENSOR_LIDAR) {  // camera: colour and normal
                            const float n[3] = {r4.x, r4.y, r4.z};
    #pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                dal += gC[k] * (T * c[k] - Ca[k] * io) + gN[k] * (T * n[k] - Na[k] * io);
                                Ca[k] = fmaf(w, c[k], Ca[k]);
                                Na[k] = fmaf(w, n[k], Na[k]);
                                g[13 + k] = w * gC[k];   // colour
                                g[16 + k] = w * gN[k];   // normal
                            }
                        } else {  // LiDAR: intensity and ray-drop probability
    #pragma unroll
                            for (int k = 0; k < 2; ++k) {
                                dal += gC[k] * (T * c[k] - Ca[k] * io);
                                Ca[k] = fmaf(w, c[k], Ca[k]);
                                g[13 + k] = w * gC[k];
                            }
                        }
                        Aa += w;
                        Ba = fmaf(w, z, Ba);
                        Da = fmaf(w * z, z, Da);
                        const float dz = w * (gB + 2.f * z * gD);
                        const float o = r3.x;
                        float dG = 0.f;
                        if (o * sp.G < kAlphaMax) {
                            g[12] = dal * sp.G;  // opacity
                            dG = dal * o;
                        }
                        const float drho = -0.5f * sp.G * dG;
                        if (sp.use3) {
                            const float iq = 1.f / sp.q2;
                            const float dq0 = 2.f * sp.u * iq * drho;
                            const float dq1 = 2.f * sp.v * iq * drho;
                            const float dq2 = -2.f * sp.rho * iq * drho - sp.z * iq * dz;
                            g[11] = dz * iq;  // det
                            float r0, r1, r2;
                            if (KIND == GSR_SENSOR_PINHOLE) {
                                r0 = sp.dx; r1 = sp.dy; r2 = 1.f;
                                const float4 q0 = Rj[0], q1 = Rj[1], q2 = Rj[2];
                                g[3] = -(dq0 * q0.x + dq1 * q1.x + dq2 * q2.x);  // centre x
                                g[7] = -(dq0 * q0.y + dq1 * q1.y + dq2 * q2.y);  // centre y
                            } else {
                                r0 = d0; r1 = d1; r2 = d2;
                            }
                            g[0] = dq0 * r0; g[1] = dq0 * r1; g[2] = dq0 * r2;
                            g[4] = dq1 * r0; g[5] = dq1 * r1; g[6] = dq1 * r2;
                            g[8] = dq2 * r0; g[9] = dq2 * r1; g[10] = dq2 * r2;
                        } else {
                            g[3] = -2.f * kLowPassInvVar * sp.dx * drho;
                            g[7] = -2.f * kLowPassInvVar * sp.dy * drho;
                            g[19] = dz;  // centre depth
                        }
                    }
                    // reduce-scatter over the warp: after it lane l holds the sum of
                    // component l over the 32 rays (5 halving exchanges, 31 shuffles)
    #pragma unroll
                    for (int o = 16; o >= 1; o >>= 1) {
                        const bool up = (lane & o) != 0;
    #pragma unroll
                        for (int k = 0; k < o; ++k) {
                            const float send = up ? g[k] : g[k + o];
                            const float keep = up ? g[k + o] : g[k];
                            g[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                        }
                    }
                    if (lane < kGradComponents && g[0] != 0.f)
                        atomicAdd(reinterpret_cast<float*>(a.recgrad + (size_t)Sl[j - lo] * kRecordF4) + lane, g[0]);
            };
            while (mask) {
                const int bit = 31 - __clz(mask);
                mask &= ~(1u << bit);
                const int bit2 = mask ? 31 - __clz(mask) : -1;
                if (bit2 >= 0) mask &= ~(1u << bit2);
                const int j = g0 + bit, j2 = g0 + (bit2 >= 0 ? bit2 : bit);
                Splat sp, sp2;
                const bool h = splat_eval<KIND>(Bf + (j - lo) * kRecordF4, rx, ry, d0, d1, d2, sd.near_plane, columns, sp);
                const bool h2 = splat_eval<KIND>(Bf + (j2 - lo) * kRecordF4, rx, ry, d0, d1, d2, sd.near_plane, columns,
                                                 sp2);
                apply(j, sp, h && (uint32_t)j < last);
                if (bit2 >= 0) apply(j2, sp2, h2 && (uint32_t)j2 < last);
            }
        }
        __syncthreads();  // buffer g&1 is free for batch g+2
        if (!ok) {
            if (b + 1 < nb) mbar_wait_bounded(bars + ((g + 1) & 1), ((g + 1) >> 1) & 1, counters);
            gb += (uint32_t)min(nb, b + 2);
            return;
        }
    }
    gb += (uint32_t)nb;
}

// Shared-memory layout of the backward kernels: mbarriers, slot ids, records.
struct BwdSmem {
    uint64_t* bars;
    uint32_t* sslot;
    float4* buf;
};

__device__ __forceinline__ BwdSmem bwd_smem(unsigned char* raw)
{
    BwdSmem m;
    m.bars = reinterpret_cast<uint64_t*>(raw);
    m.sslot = reinterpret_cast<uint32_t*>(raw + 128);          // [2][nthr]
    m.buf = reinterpret_cast<float4*>(raw + 128 + 2 * 256 * 4);  // [2][nthr][kRecordF4]
    if (threadIdx.x == 0) {
        mbar_init(m.bars, 1);
        mbar_init(m.bars + 1, 1);
        fence_mbar_init();
    }
    return m;
}

// One CTA per tile of the camera, longest list first.  A split tile (its
// forward merge stored per-chunk states) walks only its last chunk here; its
// other chunks are walked by k_render_backward_chunks.
template <int KIND>
__global__ void __launch_bounds__(256) k_render_backward(SensorTable tab, int sensor,
                                                         const float4* __restrict__ rec,
                                                         const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ pval, BwdArgs a,
                                                         uint32_t* counters, const uint32_t* __restrict__ sorder,
                                                         SplitBufs sp)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint32_t wmax[8];
    const BwdSmem sm = bwd_smem(smem_raw);
    const SensorDev& sd = tab.s[sensor];
    const uint32_t tile = sorder[blockIdx.x];  // longest lists first
    const uint4 info = sp.info[tile];
    const bool split = info.x > 0 && sp.state[tile].x == 1u;
    const int lo_pos = split ? chunk_begin(sd.split_first, sd.split_chunk, (int)info.x) : 0;
    uint32_t gb = 0;
    bwd_tile<KIND>(tab, sd, (int)tile - sd.tile_base, lo_pos, 0x7fffffff, 0, sp, 0, rec, ranges, pval, a, counters,
                   sm.bars, sm.sslot, sm.buf, wmax, gb);
}

// Chunks 0..C-1 of the camera's split tiles (persistent; item (tile, c) of
// the forward's split list walks chunk c - 1 backwards from the state after it).
template <int KIND>
__global__ void __launch_bounds__(256) k_render_backward_chunks(SensorTable tab, int sensor,
                                                                const float4* __restrict__ rec,
                                                                const uint2* __restrict__ ranges,
                                                                const uint32_t* __restrict__ pval, BwdArgs a,
                                                                uint32_t* counters, SplitBufs sp)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint32_t wmax[8], item_s;
    const BwdSmem sm = bwd_smem(smem_raw);
    const SensorDev& sd = tab.s[sensor];
    const uint32_t begin = sp.info[sd.tile_base].z;
    const uint32_t end = sensor + 1 < tab.n ? sp.info[tab.s[sensor + 1].tile_base].z : counters[C_NITEMS];
    uint32_t gb = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item_s = begin + atomicAdd(&counters[C_SPLIT_QUEUE], 1u);
        __syncthreads();
        const uint32_t item = item_s;
        if (item >= end) break;
        const uint2 it = sp.items[item];
        if (sp.state[it.x].x != 1u) continue;  // finished in chunk 0: walked whole by k_render_backward
        const int cc = (int)it.y - 1;
        bwd_tile<KIND>(tab, sd, (int)it.x - sd.tile_base, chunk_begin(sd.split_first, sd.split_chunk, cc),
                       chunk_begin(sd.split_first, sd.split_chunk, cc + 1), 1, sp, cc, rec, ranges, pval, a, counters, sm.bars,
                       sm.sslot, sm.buf, wmax, gb);
    }
}

// ================================================== preprocess backward
namespace {

struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 mul(const float* M, V3 v)
{
    return v3(M[0] * v.x + M[1] * v.y + M[2] * v.z, M[3] * v.x + M[4] * v.y + M[5] * v.z,
              M[6] * v.x + M[7] * v.y + M[8] * v.z);
}
__device__ __forceinline__ V3 mulT(const float* M, V3 v)
{
    return v3(M[0] * v.x + M[3] * v.y + M[6] * v.z, M[1] * v.x + M[4] * v.y + M[7] * v.z,
              M[2] * v.x + M[5] * v.y + M[8] * v.z);
}

// SH basis (deg <= 3, the same functions as the preprocess) and its gradient
// w.r.t. the (unnormalised) direction components.
__device__ __forceinline__ void sh_basis_grad(int deg, V3 d, float* b, V3* gb)
{
    const float x = d.x, y = d.y, z = d.z;
    const float C0 = 0.28209479177387814f, C1 = 0.4886025119029199f;
    const float C2a = 1.0925484305920792f, C2b = 0.31539156525252005f, C2c = 0.5462742152960396f;
    const float C3a = -0.5900435899266435f, C3b = 2.890611442640554f, C3c = -0.4570457994644658f;
    const float C3d = 0.3731763325901154f, C3e = 1.445305721320277f;
    b[0] = C0;
    gb[0] = v3(0.f, 0.f, 0.f);
    if (deg < 1) return;
    b[1] = -C1 * y; gb[1] = v3(0.f, -C1, 0.f);
    b[2] = C1 * z;  gb[2] = v3(0.f, 0.f, C1);
    b[3] = -C1 * x; gb[3] = v3(-C1, 0.f, 0.f);
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    b[4] = C2a * x * y;                b[5] = -C2a * y * z;
    b[6] = C2b * (2.f * zz - xx - yy); b[7] = -C2a * x * z;
    b[8] = C2c * (xx - yy);
    gb[4] = v3(C2a * y, C2a * x, 0.f);
    gb[5] = v3(0.f, -C2a * z, -C2a * y);
    gb[6] = v3(-2.f * C2b * x, -2.f * C2b * y, 4.f * C2b * z);
    gb[7] = v3(-C2a * z, 0.f, -C2a * x);
    gb[8] = v3(2.f * C2c * x, -2.f * C2c * y, 0.f);
    if (deg < 3) return;
    b[9] = C3a * y * (3.f * xx - yy);
    b[10] = C3b * x * y * z;
    b[11] = C3c * y * (4.f * zz - xx - yy);
    b[12] = C3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    b[13] = C3c * x * (4.f * zz - xx - yy);
    b[14] = C3e * z * (xx - yy);
    b[15] = C3a * x * (xx - 3.f * yy);
    gb[9] = v3(6.f * C3a * x * y, C3a * (3.f * xx - 3.f * yy), 0.f);
    gb[10] = v3(C3b * y * z, C3b * x * z, C3b * x * y);
    gb[11] = v3(-2.f * C3c * x * y, C3c * (4.f * zz - xx - 3.f * yy), 8.f * C3c * y * z);
    gb[12] = v3(-6.f * C3d * x * z, -6.f * C3d * y * z, C3d * (6.f * zz - 3.f * xx - 3.f * yy));
    gb[13] = v3(C3c * (4.f * zz - 3.f * xx - yy), -2.f * C3c * x * y, 8.f * C3c * x * z);
    gb[14] = v3(2.f * C3e * x * z, -2.f * C3e * y * z, C3e * (xx - yy));
    gb[15] = v3(C3a * (3.f * xx - 3.f * yy), -6.f * C3a * x * y, 0.f);
}

// Backward of the ray-direction record (LiDAR and cylindrical camera):
// M = [a b ms] (columns), Q = adj(M) (the record's rows r0..r2 .xyz), det(M)
// (r2.w).  Each entry of the adjugate is a 2x2 minor of M, and the
// derivative of det(M) w.r.t. m_ij is its cofactor, adj(M)_ji.
__device__ __forceinline__ void adjugate_backward(V3 a, V3 b, V3 ms, float4 G0, float4 G1, float4 G2, V3& gA,
                                                  V3& gB, V3& g_ms)
{
    const float m00 = a.x, m01 = b.x, m02 = ms.x;
    const float m10 = a.y, m11 = b.y, m12 = ms.y;
    const float m20 = a.z, m21 = b.z, m22 = ms.z;
    const float gq00 = G0.x, gq01 = G0.y, gq02 = G0.z, gq10 = G1.x, gq11 = G1.y, gq12 = G1.z;
    const float gq20 = G2.x, gq21 = G2.y, gq22 = G2.z, g_det = G2.w;
    float g00 = 0.f, g01 = 0.f, g02 = 0.f, g10 = 0.f, g11 = 0.f, g12 = 0.f, g20 = 0.f, g21 = 0.f, g22 = 0.f;
    g11 += gq00 * m22; g22 += gq00 * m11; g12 -= gq00 * m21; g21 -= gq00 * m12;  // q00 = m11 m22 - m12 m21
    g02 += gq01 * m21; g21 += gq01 * m02; g01 -= gq01 * m22; g22 -= gq01 * m01;  // q01 = m02 m21 - m01 m22
    g01 += gq02 * m12; g12 += gq02 * m01; g02 -= gq02 * m11; g11 -= gq02 * m02;  // q02 = m01 m12 - m02 m11
    g12 += gq10 * m20; g20 += gq10 * m12; g10 -= gq10 * m22; g22 -= gq10 * m10;  // q10 = m12 m20 - m10 m22
    g00 += gq11 * m22; g22 += gq11 * m00; g02 -= gq11 * m20; g20 -= gq11 * m02;  // q11 = m00 m22 - m02 m20
    g02 += gq12 * m10; g10 += gq12 * m02; g00 -= gq12 * m12; g12 -= gq12 * m00;  // q12 = m02 m10 - m00 m12
    g10 += gq20 * m21; g21 += gq20 * m10; g11 -= gq20 * m20; g20 -= gq20 * m11;  // q20 = m10 m21 - m11 m20
    g01 += gq21 * m20; g20 += gq21 * m01; g00 -= gq21 * m21; g21 -= gq21 * m00;  // q21 = m01 m20 - m00 m21
    g00 += gq22 * m11; g11 += gq22 * m00; g01 -= gq22 * m10; g10 -= gq22 * m01;  // q22 = m00 m11 - m01 m10
    g00 += g_det * fmaf(m11, m22, -m12 * m21);
    g01 += g_det * fmaf(m12, m20, -m10 * m22);
    g02 += g_det * fmaf(m10, m21, -m11 * m20);
    g10 += g_det * fmaf(m02, m21, -m01 * m22);
    g11 += g_det * fmaf(m00, m22, -m02 * m20);
    g12 += g_det * fmaf(m01, m20, -m00 * m21);
    g20 += g_det * fmaf(m01, m12, -m02 * m11);
    g21 += g_det * fmaf(m02, m10, -m00 * m12);
    g22 += g_det * fmaf(m00, m11, -m01 * m10);
    gA = v3(g00, g10, g20);
    gB = v3(g01, g11, g21);
    g_ms = v3(g02, g12, g22);
}

}  // namespace

struct PreBwdArgs {
    gsr_surfels S;
    const float* poses;
    int n_obj;
    const float4* recgrad;
    const uint32_t* counts;
    gsr_surfel_grads G;
};

__global__ void __launch_bounds__(128) k_preprocess_backward(SensorTable tab, PreBwdArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const gsr_surfels& S = a.S;
    if (i >= S.n) return;
    // ---- forward quantities independent of the sensor
    V3 mu = v3(S.pos[3 * i], S.pos[3 * i + 1], S.pos[3 * i + 2]);
    const float4 qr = reinterpret_cast<const float4*>(S.quat)[i];
    const float qn = sqrtf(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z + qr.w * qr.w);
    const float w = qr.x / qn, x = qr.y / qn, y = qr.z / qn, z = qr.w / qn;
    V3 tu = v3(1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y));
    V3 tv = v3(2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x));
    V3 nw = v3(2.f * (x * z + w * y), 2.f * (y * z - w * x), 1.f - 2.f * (x * x + y * y));
    float Ro[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    bool has_obj = false;
    if (S.obj_id) {
        const int k = S.obj_id[i];
        if (k >= 0 && k < a.n_obj) {
            const float* P = a.poses + 12 * k;
            const float R9[9] = {P[0], P[1], P[2], P[4], P[5], P[6], P[8], P[9], P[10]};
            for (int t = 0; t < 9; ++t) Ro[t] = R9[t];
            mu = mul(Ro, mu) + v3(P[3], P[7], P[11]);
            tu = mul(Ro, tu);
            tv = mul(Ro, tv);
            nw = mul(Ro, nw);
            has_obj = true;
        }
    }
    const float2 ls = reinterpret_cast<const float2*>(S.log_scale)[i];
    const float su = __expf(ls.x), sv = __expf(ls.y);
    const float logit = S.opacity[i];
    const float o = 1.f / (1.f + __expf(-logit));
    const int deg = S.sh_degree;
    const int K = (deg + 1) * (deg + 1);
    const float* sh = S.sh + (size_t)i * K * 3;

    // accumulated gradients (world, after the object pose)
    V3 g_mu = v3(0, 0, 0), g_tu = v3(0, 0, 0), g_tv = v3(0, 0, 0), g_nw = v3(0, 0, 0);
    float g_su = 0.f, g_sv = 0.f, g_o = 0.f, g_int = 0.f, g_rd = 0.f;
    float g_sh[48];
    for (int k = 0; k < 3 * K; ++k) g_sh[k] = 0.f;
    bool any = false;

    for (int si = 0; si < tab.n; ++si) {
        const SensorDev& sd = tab.s[si];
        const size_t slot = (size_t)si * S.n + i;
        if (a.counts[slot] == 0) continue;
        const float4* RG = a.recgrad + slot * kRecordF4;
        const float4 G0 = RG[0], G1 = RG[1], G2 = RG[2], G3 = RG[3], G4 = RG[4];
        any = true;
        g_o += G3.x;
        const V3 org = v3(sd.origin[0], sd.origin[1], sd.origin[2]);
        V3 vd = mu - org;
        const float flip = dot(nw, vd) > 0.f ? -1.f : 1.f;
        // normal: n_s = R (flip nw)
        g_nw = g_nw + flip * mulT(sd.R, v3(G4.x, G4.y, G4.z));
        const V3 ms = mul(sd.R, mu) + v3(sd.t[0], sd.t[1], sd.t[2]);
        const V3 Rtu = mul(sd.R, tu), Rtv = mul(sd.R, tv);
        const V3 A = su * Rtu, B = sv * Rtv;
        V3 gA, gB, g_ms;
        if (sd.kind == GSR_SENSOR_PINHOLE) {
            const float iz = 1.f / ms.z;
            const float ex = ms.x * iz, ey = ms.y * iz;
            const float m00 = sd.fx * (A.x - ex * A.z), m01 = sd.fx * (B.x - ex * B.z);
            const float m10 = sd.fy * (A.y - ey * A.z), m11 = sd.fy * (B.y - ey * B.z);
            const float m20 = A.z, m21 = B.z;
            const float det = m00 * m11 - m01 * m10;
            // record: Q0 = (m11, -m01, 0), Q1 = (-m10, m00, 0),
            // Q2 = ((m10 m21 - m11 m20) iz, (m01 m20 - m00 m21) iz, det iz), det, c = (fx ex + cx, fy ey + cy)
            float g00 = G1.y, g01 = -G0.y, g10 = -G1.x, g11 = G0.x, g20 = 0.f, g21 = 0.f;
            float g_det = G2.w + G2.z * iz;
            float g_iz = G2.x * (m10 * m21 - m11 * m20) + G2.y * (m01 * m20 - m00 * m21) + G2.z * det;
            g10 += G2.x * m21 * iz; g21 += G2.x * m10 * iz; g11 -= G2.x * m20 * iz; g20 -= G2.x * m11 * iz;
            g01 += G2.y * m20 * iz; g20 += G2.y * m01 * iz; g00 -= G2.y * m21 * iz; g21 -= G2.y * m00 * iz;
            g00 += g_det * m11; g11 += g_det * m00; g01 -= g_det * m10; g10 -= g_det * m01;
            float g_ex = sd.fx * G0.w, g_ey = sd.fy * G1.w;
            gA = v3(sd.fx * g00, sd.fy * g10, -sd.fx * ex * g00 - sd.fy * ey * g10 + g20);
            gB = v3(sd.fx * g01, sd.fy * g11, -sd.fx * ex * g01 - sd.fy * ey * g11 + g21);
            g_ex -= sd.fx * (A.z * g00 + B.z * g01);
            g_ey -= sd.fy * (A.z * g10 + B.z * g11);
            g_ms = v3(g_ex * iz, g_ey * iz, G4.w);
            g_iz += g_ex * ms.x + g_ey * ms.y;
            g_ms.z += -g_iz * iz * iz;
        } else if (sd.kind == GSR_SENSOR_LIDAR || sd.kind == GSR_SENSOR_CYLINDRICAL) {
            // record: M = [a b ms] (columns), Q = adj(M) (rows r0..r2 .xyz),
            // det(M), low-pass centre, order key
            adjugate_backward(A, B, ms, G0, G1, G2, gA, gB, g_ms);
            if (sd.kind == GSR_SENSOR_LIDAR) {
                // centre column = (azimuth - az0) / d_az - 1/2, row = (el_max - elevation) / d_el,
                // key |ms|
                const float rxy2 = ms.x * ms.x + ms.y * ms.y;
                const float rxy = sqrtf(rxy2);
                const float rc2 = rxy2 + ms.z * ms.z;
                const float rc = sqrtf(rc2);
                const float gcol = G0.w * sd.inv_d_az, gel = -G1.w * sd.inv_d_el;
                if (rxy2 > 0.f) {  // straight above or below the sensor the centre's angles have no gradient
                    g_ms.x += gcol * (-ms.y / rxy2) - gel * ms.z * ms.x / (rxy * rc2);
                    g_ms.y += gcol * (ms.x / rxy2) - gel * ms.z * ms.y / (rxy * rc2);
                    g_ms.z += gel * rxy / rc2;
                }
                g_ms = g_ms + (G4.w / rc) * ms;
            } else {
                // centre (cx + fx atan2(x, z), cy + fy y / r_h), key r_h = |(x, z)|
                const float rh2 = ms.x * ms.x + ms.z * ms.z;
                const float rh = sqrtf(rh2);
                const float gcx = G0.w * sd.fx, gcy = G1.w * sd.fy;
                const float yr3 = ms.y / (rh2 * rh);
                g_ms.x += gcx * ms.z / rh2 - gcy * yr3 * ms.x + G4.w * ms.x / rh;
                g_ms.y += gcy / rh;
                g_ms.z += -gcx * ms.x / rh2 - gcy * yr3 * ms.z + G4.w * ms.z / rh;
            }
        } else {
            continue;
        }
        g_mu = g_mu + mulT(sd.R, g_ms);
        g_su += dot(Rtu, gA);
        g_sv += dot(Rtv, gB);
        g_tu = g_tu + su * mulT(sd.R, gA);
        g_tv = g_tv + sv * mulT(sd.R, gB);
        if (sd.kind == GSR_SENSOR_LIDAR) {
            g_int += G3.y;  // intensity
            g_rd += G3.z;   // ray-drop probability
            continue;
        }
        // colour: max(0, sum Y(d) c + 0.5), d = normalise(mu - origin) (object frame)
        const float vlen = sqrtf(dot(vd, vd));
        const V3 dw = (1.f / vlen) * vd;
        const V3 dl = has_obj ? mulT(Ro, dw) : dw;
        float b[16];
        V3 gb[16];
        sh_basis_grad(deg, dl, b, gb);
        float raw[3] = {0.5f, 0.5f, 0.5f};
        for (int k = 0; k < K; ++k)
            for (int c = 0; c < 3; ++c) raw[c] += b[k] * sh[3 * k + c];
        const float gcol[3] = {raw[0] > 0.f ? G3.y : 0.f, raw[1] > 0.f ? G3.z : 0.f, raw[2] > 0.f ? G3.w : 0.f};
        V3 g_dl = v3(0, 0, 0);
        for (int k = 0; k < K; ++k) {
            float sk = 0.f;
            for (int c = 0; c < 3; ++c) {
                g_sh[3 * k + c] += b[k] * gcol[c];
                sk += sh[3 * k + c] * gcol[c];
            }
            g_dl = g_dl + sk * gb[k];
        }
        const V3 g_dw = has_obj ? mul(Ro, g_dl) : g_dl;
        g_mu = g_mu + (1.f / vlen) * (g_dw - dot(dw, g_dw) * dw);
    }
    if (!any) return;
    // opacity logit
    a.G.opacity[i] += g_o * o * (1.f - o);
    // scales
    a.G.log_scale[2 * i] += g_su * su;
    a.G.log_scale[2 * i + 1] += g_sv * sv;
    if (a.G.intensity) a.G.intensity[i] += g_int;
    if (a.G.ray_drop && S.ray_drop) {  // rho = sigmoid(ray-drop logit)
        const float rho = 1.f / (1.f + __expf(-S.ray_drop[i]));
        a.G.ray_drop[i] += g_rd * rho * (1.f - rho);
    }
    // undo the object rotation
    if (has_obj) {
        g_mu = mulT(Ro, g_mu);
        g_tu = mulT(Ro, g_tu);
        g_tv = mulT(Ro, g_tv);
        g_nw = mulT(Ro, g_nw);
    }
    a.G.pos[3 * i] += g_mu.x;
    a.G.pos[3 * i + 1] += g_mu.y;
    a.G.pos[3 * i + 2] += g_mu.z;
    // rotation columns -> normalised quaternion -> raw quaternion
    const float gw = 2.f * (z * g_tu.y - y * g_tu.z - z * g_tv.x + x * g_tv.z + y * g_nw.x - x * g_nw.y);
    const float gx = 2.f * (y * g_tu.y + z * g_tu.z + y * g_tv.x - 2.f * x * g_tv.y + w * g_tv.z + z * g_nw.x -
                            w * g_nw.y - 2.f * x * g_nw.z);
    const float gy = 2.f * (-2.f * y * g_tu.x + x * g_tu.y - w * g_tu.z + x * g_tv.x + z * g_tv.z + w * g_nw.x +
                            z * g_nw.y - 2.f * y * g_nw.z);
    const float gz = 2.f * (-2.f * z * g_tu.x + w * g_tu.y + x * g_tu.z - w * g_tv.x - 2.f * z * g_tv.y + y * g_tv.z +
                            x * g_nw.x + y * g_nw.y);
    const float dq = w * gw + x * gx + y * gy + z * gz;
    a.G.quat[4 * i] += (gw - w * dq) / qn;
    a.G.quat[4 * i + 1] += (gx - x * dq) / qn;
    a.G.quat[4 * i + 2] += (gy - y * dq) / qn;
    a.G.quat[4 * i + 3] += (gz - z * dq) / qn;
    for (int k = 0; k < 3 * K; ++k) a.G.sh[(size_t)i * K * 3 + k] += g_sh[k];
}

// ================================================================= host side
size_t backward_smem_bytes(int threads) { return 128 + 2 * 256 * 4 + 2 * (size_t)threads * kRecordBytes; }

cudaError_t launch_loss(const gsr_plan* p, void* ws, int sensor, const gsr_camera_out* fwd, const float* target,
                        const gsr_loss_weights* wt, float* loss, const gsr_camera_grad* g, cudaStream_t st)
{
    const gsr_sensor& s = p->sensors[sensor];
    LossArgs a;
    a.rgb = fwd->rgb;
    a.alpha = fwd->alpha;
    a.dacc = fwd->depth_acc;
    a.normal = fwd->normal;
    a.target = target;
    a.g_rgb = g->rgb;
    a.g_alpha = g->alpha;
    a.g_dacc = g->depth_acc;
    a.g_normal = g->normal;
    a.W = s.width;
    a.H = s.height;
    a.cyl = s.kind == GSR_SENSOR_CYLINDRICAL;
    a.fx = s.fx; a.fy = s.fy; a.cx = s.cx; a.cy = s.cy;
    a.w_dist = wt->w_dist;
    a.w_norm = wt->w_normal;
    a.mask_alpha = wt->mask_alpha;
    const int HW = s.width * s.height;
    const int blocks = (HW + 255) / 256;
    a.scratch = region<float>(p, ws, R_LOSS_SCRATCH);
    a.partial = a.scratch + (size_t)6 * HW;
    k_loss_pixel<<<blocks, 256, 0, st>>>(a);
    k_loss_gather<<<blocks, 256, 0, st>>>(a);
    k_loss_reduce<<<1, 1024, 0, st>>>(a.partial, blocks, a.w_dist, a.w_norm, HW, loss);
    return cudaGetLastError();
}

cudaError_t launch_lidar_loss(const gsr_plan* p, void* ws, int sensor, const gsr_lidar_out* fwd,
                              const float* t_range, const float* t_int, const gsr_lidar_loss_weights* wt,
                              float* loss, const gsr_lidar_grad* g, cudaStream_t st)
{
    const gsr_sensor& s = p->sensors[sensor];
    LidarLossArgs a;
    a.range = fwd->range;
    a.alpha = fwd->alpha;
    a.intensity = fwd->intensity;
    a.drop = fwd->ray_drop;
    a.t_range = t_range;
    a.t_int = t_int;
    a.g_alpha = g->alpha;
    a.g_dacc = g->depth_acc;
    a.g_int = g->intensity;
    a.g_drop = g->ray_drop;
    a.n = s.width * s.height;
    a.w_range = wt->w_range;
    a.w_int = wt->w_intensity;
    a.w_drop = wt->w_drop;
    const int blocks = (a.n + 255) / 256;
    a.partial = region<float>(p, ws, R_LOSS_SCRATCH);
    a.inv = a.partial + (size_t)4 * blocks;
    k_lidar_loss_terms<<<blocks, 256, 0, st>>>(a);
    k_lidar_loss_reduce<<<1, 1024, 0, st>>>(a, blocks, loss);
    k_lidar_loss_grad<<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

SplitBufs split_bufs(const gsr_plan* p, const void* ws);

template <int KIND>
static cudaError_t render_backward_kind(const gsr_plan* p, void* ws, int sensor, const BwdArgs& a, cudaStream_t st)
{
    const SensorTable tab = make_sensor_table(p, ws);
    const SensorDev& sd = tab.s[sensor];
    const int threads = sd.tile_w * sd.tile_h;
    const int tiles = sd.tiles_x * sd.tiles_y;
    const int pb = sort_result_buffer(tile_sort_passes(p));
    const uint32_t* pval = region<uint32_t>(p, ws, pb ? R_PAIR_VAL_B : R_PAIR_VAL_A);
    const size_t smem = backward_smem_bytes(threads);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_render_backward<KIND>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    // this sensor's tiles in schedule order (the tile-key scratch of the sort is free)
    uint32_t* sorder = region<uint32_t>(p, ws, R_TILE_KEY_A);
    k_sensor_order<<<1, 1024, 0, st>>>(region<uint32_t>(p, ws, R_TILE_VAL_A), (uint32_t)p->tile_base[p->n_sensors],
                                       (uint32_t)sd.tile_base, (uint32_t)(sd.tile_base + tiles), sorder);
    const SplitBufs sp = split_bufs(p, ws);
    uint32_t* counters = region<uint32_t>(p, ws, R_COUNTERS);
    k_render_backward<KIND><<<tiles, threads, smem, st>>>(tab, sensor, region<float4>(p, ws, R_RECORDS),
                                                          region<uint2>(p, ws, R_RANGES), pval, a, counters,
                                                          sorder, sp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the other chunks of split tiles, persistent over the sensor's split items
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_render_backward_chunks<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_backward_chunks<KIND>, threads,
                                                           smem)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(counters + C_SPLIT_QUEUE, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
    k_render_backward_chunks<KIND><<<sms * (per_sm > 0 ? per_sm : 1), threads, smem, st>>>(
        tab, sensor, region<float4>(p, ws, R_RECORDS), region<uint2>(p, ws, R_RANGES), pval, a, counters, sp);
    return cudaGetLastError();
}

static cudaError_t zero_recgrad(const gsr_plan* p, void* ws, int accumulate, cudaStream_t st)
{
    if (accumulate) return cudaSuccess;
    const uint64_t slots = (uint64_t)p->n_surfels * p->n_sensors;
    return cudaMemsetAsync(region<float4>(p, ws, R_RECGRAD), 0, slots * kRecordBytes, st);
}

cudaError_t launch_render_backward(const gsr_plan* p, void* ws, int sensor, const gsr_camera_out* fwd,
                                   const gsr_camera_grad* g, int accumulate, cudaStream_t st)
{
    cudaError_t e = zero_recgrad(p, ws, accumulate, st);
    if (e != cudaSuccess) return e;
    BwdArgs a;
    a.trans = fwd->trans;
    a.n_contrib = fwd->n_contrib;
    a.g_rgb = g->rgb;
    a.g_alpha = g->alpha;
    a.g_dacc = g->depth_acc;
    a.g_normal = g->normal;
    a.g_drop = nullptr;
    a.recgrad = region<float4>(p, ws, R_RECGRAD);
    if (p->sensors[sensor].kind == GSR_SENSOR_CYLINDRICAL)
        return render_backward_kind<GSR_SENSOR_CYLINDRICAL>(p, ws, sensor, a, st);
    return render_backward_kind<GSR_SENSOR_PINHOLE>(p, ws, sensor, a, st);
}

cudaError_t launch_render_backward_lidar(const gsr_plan* p, void* ws, int sensor, const gsr_lidar_out* fwd,
                                         const gsr_lidar_grad* g, int accumulate, cudaStream_t st)
{
    cudaError_t e = zero_recgrad(p, ws, accumulate, st);
    if (e != cudaSuccess) return e;
    BwdArgs a;
    a.trans = fwd->trans;
    a.n_contrib = fwd->n_contrib;
    a.g_rgb = g->intensity;
    a.g_alpha = g->alpha;
    a.g_dacc = g->depth_acc;
    a.g_normal = nullptr;
    a.g_drop = g->ray_drop;
    a.recgrad = region<float4>(p, ws, R_RECGRAD);
    return render_backward_kind<GSR_SENSOR_LIDAR>(p, ws, sensor, a, st);
}

cudaError_t launch_preprocess_backward(const gsr_plan* p, const void* ws, const gsr_surfels* s,
                                       const gsr_objects* obj, const gsr_surfel_grads* out, cudaStream_t st)
{
    const SensorTable tab = make_sensor_table(p, ws);
    PreBwdArgs a;
    a.S = *s;
    a.poses = (obj && obj->n_objects > 0) ? obj->pose : nullptr;
    a.n_obj = (obj && obj->n_objects > 0) ? obj->n_objects : 0;
    a.recgrad = region<float4>(p, ws, R_RECGRAD);
    a.counts = region<uint32_t>(p, ws, R_COUNTS);
    a.G = *out;
    if (s->n > 0) k_preprocess_backward<<<(s->n + 127) / 128, 128, 0, st>>>(tab, a);
    return cudaGetLastError();
}

}  // namespace gsr

// ===================================================== allocation-free loss
// Scratch of gsr_loss_noalloc: a fixed file-scope device array, so callers
// that cannot allocate device memory still get the loss.  Host code only
// ever passes its device address (looked up once per device below) to the
// kernels; the symbol itself is a host-side stand-in.
static constexpr size_t kNoAllocScratchFloats =
    6ull * GSR_NOALLOC_MAX_PIXELS + 3ull * (GSR_NOALLOC_MAX_PIXELS / 256) + 64;
static __device__ __align__(256) float g_noalloc_loss_scratch[kNoAllocScratchFloats];

namespace gsr {

gsr_status cuda_status(cudaError_t e);

// Device address of g_noalloc_loss_scratch on the current device `dev`,
// looked up on the first call for that device and cached.
static float* noalloc_scratch(int dev, cudaError_t* err)
{
    constexpr int kMaxDevices = 64;
    static std::atomic<float*> cache[kMaxDevices];
    static std::mutex mu;
    if (dev < 0 || dev >= kMaxDevices) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    float* p = cache[dev].load(std::memory_order_acquire);
    if (p) return p;
    std::lock_guard<std::mutex> lock(mu);
    p = cache[dev].load(std::memory_order_relaxed);
    if (p) return p;
    void* addr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_loss_scratch);
    if (e != cudaSuccess || addr == nullptr) {
        *err = e != cudaSuccess ? e : cudaErrorInvalidSymbol;
        return nullptr;
    }
    p = static_cast<float*>(addr);
    cache[dev].store(p, std::memory_order_release);
    return p;
}

}  // namespace gsr

extern "C" gsr_status gsr_loss_noalloc(const gsr_sensor* camera, const gsr_camera_out* fwd, const float* target_rgb,
                                       const gsr_loss_weights* weights, float* loss, const gsr_camera_grad* grad,
                                       void* stream)
{
    using namespace gsr;
    if (!camera || !fwd || !target_rgb || !weights || !loss || !grad) return GSR_ERR_INVALID_ARG;
    if (camera->kind != GSR_SENSOR_PINHOLE && camera->kind != GSR_SENSOR_CYLINDRICAL) return GSR_ERR_UNSUPPORTED;
    if (camera->width <= 0 || camera->height <= 0 || !(camera->fx > 0.f && camera->fy > 0.f))
        return GSR_ERR_INVALID_ARG;
    if ((int64_t)camera->width * camera->height > GSR_NOALLOC_MAX_PIXELS) return GSR_ERR_TOO_LARGE;
    if (!fwd->rgb || !fwd->alpha || !fwd->depth_acc || !fwd->normal) return GSR_ERR_INVALID_ARG;
    if (!grad->rgb || !grad->alpha || !grad->depth_acc || !grad->normal) return GSR_ERR_INVALID_ARG;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e);
    float* scratch = noalloc_scratch(dev, &e);
    if (!scratch) return cuda_status(e);
    LossArgs a;
    a.rgb = fwd->rgb;
    a.alpha = fwd->alpha;
    a.dacc = fwd->depth_acc;
    a.normal = fwd->normal;
    a.target = target_rgb;
    a.g_rgb = grad->rgb;
    a.g_alpha = grad->alpha;
    a.g_dacc = grad->depth_acc;
    a.g_normal = grad->normal;
    a.W = camera->width;
    a.H = camera->height;
    a.cyl = camera->kind == GSR_SENSOR_CYLINDRICAL;
    a.fx = camera->fx; a.fy = camera->fy; a.cx = camera->cx; a.cy = camera->cy;
    a.w_dist = weights->w_dist;
    a.w_norm = weights->w_normal;
    a.mask_alpha = weights->mask_alpha;
    const int HW = camera->width * camera->height;
    const int blocks = (HW + 255) / 256;
    a.scratch = scratch;
    a.partial = scratch + (size_t)6 * HW;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    k_loss_pixel<<<blocks, 256, 0, st>>>(a);
    k_loss_gather<<<blocks, 256, 0, st>>>(a);
    k_loss_reduce<<<1, 1024, 0, st>>>(a.partial, blocks, a.w_dist, a.w_norm, HW, loss);
    return cuda_status(cudaGetLastError());
}
