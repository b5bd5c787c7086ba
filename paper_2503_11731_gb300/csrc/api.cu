// api.cu -- the extern "C" entry points declared in include/gsr.h.
//
// Argument checking, the workspace layout of a plan, and the launches of the
// preprocess, binning and compositing kernels.  No device allocation.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>

#include "gsr_internal.cuh"

namespace gsr {

cudaError_t launch_preprocess(const SensorTable& tab, const gsr_surfels& S, const float* poses, int n_obj,
                              float4* rec, ushort4* rects, uint32_t* counts, uint32_t* keys, uint4* spans,
                              int first, int n_plan, cudaStream_t st);
cudaError_t bin_sort(const gsr_plan* p, void* ws, cudaStream_t st);
cudaError_t launch_render(const gsr_plan* p, const void* ws, int sensor, const FrameOut& out, cudaStream_t st);
cudaError_t launch_loss(const gsr_plan* p, void* ws, int sensor, const gsr_camera_out* fwd, const float* target,
                        const gsr_loss_weights* wt, float* loss, const gsr_camera_grad* g, cudaStream_t st);
cudaError_t launch_render_backward(const gsr_plan* p, void* ws, int sensor, const gsr_camera_out* fwd,
                                   const gsr_camera_grad* g, int accumulate, cudaStream_t st);
cudaError_t launch_render_backward_lidar(const gsr_plan* p, void* ws, int sensor, const gsr_lidar_out* fwd,
                                         const gsr_lidar_grad* g, int accumulate, cudaStream_t st);
cudaError_t launch_lidar_loss(const gsr_plan* p, void* ws, int sensor, const gsr_lidar_out* fwd,
                              const float* t_range, const float* t_int, const gsr_lidar_loss_weights* wt,
                              float* loss, const gsr_lidar_grad* g, cudaStream_t st);
cudaError_t launch_preprocess_backward(const gsr_plan* p, const void* ws, const gsr_surfels* s,
                                       const gsr_objects* obj, const gsr_surfel_grads* out, cudaStream_t st);
cudaError_t launch_selftest_wait(uint32_t* counters, uint32_t tries, cudaStream_t stream);

static thread_local char g_cuda_err[256] = "";

static gsr_status cuda_fail(cudaError_t e)
{
    if (e == cudaSuccess) return GSR_OK;
    std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return GSR_ERR_CUDA;
}

// Status of a CUDA result for entry points in other translation units
// (records the error string like the entry points here).
gsr_status cuda_status(cudaError_t e) { return cuda_fail(e); }

int ray_dir_entries(const gsr_plan* p)
{
    int n = 0;
    for (int i = 0; i < p->n_sensors; ++i)
        if (p->sensors[i].kind != GSR_SENSOR_PINHOLE) n += p->sensors[i].width + p->sensors[i].height;
    return n;
}

SensorTable make_sensor_table(const gsr_plan* p, const void* ws)
{
    SensorTable t;
    std::memset(&t, 0, sizeof(t));
    t.n = p->n_sensors;
    t.tile_w = p->tiling.tile_w;
    t.tile_h = p->tiling.tile_h;
    t.total_tiles = p->tile_base[p->n_sensors];
    t.batch = p->tiling.batch_depth;
    const double deg = 3.14159265358979323846 / 180.0;
    int dir_off = 0;
    for (int i = 0; i < p->n_sensors; ++i) {
        const gsr_sensor& s = p->sensors[i];
        SensorDev& d = t.s[i];
        d.kind = s.kind;
        d.width = s.width;
        d.height = s.height;
        d.tiles_x = p->tiles_x[i];
        d.tiles_y = p->tiles_y[i];
        d.tile_base = p->tile_base[i];
        d.tile_w = s.tile_w;
        d.tile_h = s.tile_h;
        double R[9], tt[3];
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b) R[a * 3 + b] = s.world_to_sensor[a * 4 + b];
            tt[a] = s.world_to_sensor[a * 4 + 3];
        }
        for (int k = 0; k < 9; ++k) d.R[k] = (float)R[k];
        for (int a = 0; a < 3; ++a) d.t[a] = (float)tt[a];
        for (int b = 0; b < 3; ++b) d.origin[b] = (float)-(R[0 * 3 + b] * tt[0] + R[1 * 3 + b] * tt[1] + R[2 * 3 + b] * tt[2]);
        d.fx = s.fx; d.fy = s.fy; d.cx = s.cx; d.cy = s.cy;
        if (s.kind == GSR_SENSOR_LIDAR) {
            const double del = (double)(s.el_max_deg - s.el_min_deg) * deg / (s.height - 1);
            const double daz = 2.0 * 3.14159265358979323846 / s.width;
            d.el_max = (float)(s.el_max_deg * deg);
            d.d_el = (float)del;
            d.inv_d_el = (float)(1.0 / del);
            d.az0 = (float)(s.az0_deg * deg);
            d.d_az = (float)daz;
            d.inv_d_az = (float)(1.0 / daz);
        }
        d.near_plane = s.near_plane;
        for (int c = 0; c < 3; ++c) d.bg[c] = s.bg[c];
        // list split: the sensor's, else the plan's, else the defaults
        const int sf = s.split_first > 0 ? s.split_first : p->tiling.split_first;
        const int sc = s.split_chunk > 0 ? s.split_chunk : p->tiling.split_chunk;
        d.split_first = sf > 0 ? sf : kSplitFirstDefault;
        d.split_chunk = sc > 0 ? sc : kSplitChunkDefault;
        d.dir_off = dir_off;
        if (s.kind != GSR_SENSOR_PINHOLE) dir_off += s.width + s.height;
    }
    t.dirs = ws != nullptr ? region<float2>(p, const_cast<void*>(ws), R_RAY_DIRS) : nullptr;
    return t;
}

}  // namespace gsr

using namespace gsr;

static bool tile_ok(int w, int h)
{
    auto pow2 = [](int v) { return v >= 1 && v <= 256 && (v & (v - 1)) == 0; };
    const int n = w * h;
    return pow2(w) && pow2(h) && (n == 32 || n == 64 || n == 128 || n == 256);
}

extern "C" gsr_status gsr_plan_init(gsr_plan* plan, int32_t n_surfels, const gsr_sensor* sensors,
                                    int32_t n_sensors, const gsr_tiling* tiling, int64_t max_dup)
{
    if (!plan || !sensors || !tiling) return GSR_ERR_INVALID_ARG;
    if (n_surfels < 0 || n_sensors < 1 || n_sensors > GSR_MAX_SENSORS) return GSR_ERR_INVALID_ARG;
    if (!tile_ok(tiling->tile_w, tiling->tile_h)) return GSR_ERR_UNSUPPORTED;
    const int bd = tiling->batch_depth;
    if (!(bd == 0 || bd == 32 || bd == 64 || bd == 128 || bd == 256 || bd == 512)) return GSR_ERR_UNSUPPORTED;
    const int sf = tiling->split_first, sc = tiling->split_chunk;
    if (sf != 0 && (sf < 256 || sf > (1 << 24))) return GSR_ERR_UNSUPPORTED;
    if (sc != 0 && (sc < 64 || sc > (1 << 24))) return GSR_ERR_UNSUPPORTED;
    std::memset(plan, 0, sizeof(*plan));
    plan->n_surfels = n_surfels;
    plan->n_sensors = n_sensors;
    plan->tiling = *tiling;
    const uint64_t slots = (uint64_t)n_surfels * (uint64_t)n_sensors;
    if (slots >= (1ull << 32)) return GSR_ERR_INVALID_ARG;
    int64_t base = 0;
    for (int i = 0; i < n_sensors; ++i) {
        const gsr_sensor& s = sensors[i];
        if (s.kind != GSR_SENSOR_PINHOLE && s.kind != GSR_SENSOR_LIDAR && s.kind != GSR_SENSOR_CYLINDRICAL)
            return GSR_ERR_UNSUPPORTED;
        if (s.width <= 0 || s.height <= 0 || s.width > 65535 || s.height > 65535) return GSR_ERR_INVALID_ARG;
        if (!(s.near_plane > 0.f)) return GSR_ERR_INVALID_ARG;
        if (s.kind != GSR_SENSOR_LIDAR && !(s.fx > 0.f && s.fy > 0.f)) return GSR_ERR_INVALID_ARG;
        if (s.kind == GSR_SENSOR_CYLINDRICAL &&
            !(s.cx / s.fx <= 3.1415960f && ((float)s.width - s.cx) / s.fx <= 3.1415960f))
            return GSR_ERR_INVALID_ARG;
        if (s.kind == GSR_SENSOR_LIDAR && (s.height < 2 || !(s.el_max_deg > s.el_min_deg))) return GSR_ERR_INVALID_ARG;
        if (s.split_first != 0 && (s.split_first < 256 || s.split_first > (1 << 24))) return GSR_ERR_UNSUPPORTED;
        if (s.split_chunk != 0 && (s.split_chunk < 64 || s.split_chunk > (1 << 24))) return GSR_ERR_UNSUPPORTED;
        plan->sensors[i] = s;
        if (s.tile_w == 0 && s.tile_h == 0) {
            plan->sensors[i].tile_w = tiling->tile_w;
            plan->sensors[i].tile_h = tiling->tile_h;
        }
        const int tw = plan->sensors[i].tile_w, th = plan->sensors[i].tile_h;
        if (!tile_ok(tw, th)) return GSR_ERR_UNSUPPORTED;
        plan->tiles_x[i] = (s.width + tw - 1) / tw;
        plan->tiles_y[i] = (s.height + th - 1) / th;
        plan->tile_base[i] = (int32_t)base;
        base += (int64_t)plan->tiles_x[i] * plan->tiles_y[i];
    }
    if (base >= (1ll << 31)) return GSR_ERR_INVALID_ARG;
    plan->tile_base[n_sensors] = (int32_t)base;
    if (max_dup <= 0) {
        long double d = 64.0L * (long double)slots;
        max_dup = d > 2147483647.0L ? 2147483647LL : (int64_t)d;
        if (max_dup < 4096) max_dup = 4096;
    }
    if (max_dup > 2147483647LL) return GSR_ERR_INVALID_ARG;
    plan->max_dup = max_dup;
    // the fixed sort grid: 4 CTAs on each of the 152 SMs (3 measured the same
    // on the rig frame, 5 slower)
    plan->sort_ctas = kSortCtasPerSm * 152;

    uint64_t sz[R_END];
    const uint64_t G = (uint64_t)plan->sort_ctas;
    sz[R_RECORDS] = slots * kRecordBytes;
    sz[R_RECTS] = slots * 8;
    sz[R_COUNTS] = slots * 4;
    sz[R_DEPTHKEY] = slots * 4;
    sz[R_PAIR_KEY_A] = sz[R_PAIR_VAL_A] = sz[R_PAIR_KEY_B] = sz[R_PAIR_VAL_B] = (uint64_t)max_dup * 4;
    sz[R_RANGES] = (uint64_t)base * 8;
    sz[R_VIS_KEY_A] = sz[R_VIS_VAL_A] = sz[R_VIS_KEY_B] = sz[R_VIS_VAL_B] = slots * 4;
    sz[R_CNT_SORTED] = slots * 4;
    sz[R_OFFSETS] = slots * 4;
    sz[R_HIST] = ((uint64_t)(1 << kRadixBitsWide) * G + G + 64) * 4;  // digit-major histogram + block sums
    sz[R_PARTIAL] = G * 12 + 64;  // 64-bit partials, then 32-bit ones (the split plan)
    sz[R_COUNTERS] = C_WORDS * 4;
    sz[R_SENSOR_OF_TILE] = 64;
    sz[R_RECGRAD] = slots * kRecordBytes;
    sz[R_RAY_DIRS] = (uint64_t)ray_dir_entries(plan) * 8 + 64;
    uint64_t max_hw = 0, max_rays = 0;
    for (int i = 0; i < n_sensors; ++i) {
        const uint64_t hw = (uint64_t)sensors[i].width * sensors[i].height;
        if (sensors[i].kind != GSR_SENSOR_LIDAR) max_hw = std::max<uint64_t>(max_hw, hw);
        else max_rays = std::max<uint64_t>(max_rays, hw);
    }
    sz[R_LOSS_SCRATCH] =
        (std::max<uint64_t>(6 * max_hw + 3 * ((max_hw + 255) / 256), 4 * ((max_rays + 255) / 256)) + 64) * 4;
    sz[R_TILE_KEY_A] = sz[R_TILE_VAL_A] = sz[R_TILE_KEY_B] = sz[R_TILE_VAL_B] = (uint64_t)base * 4;
    sz[R_SPLIT_INFO] = (uint64_t)base * 16;
    sz[R_SPLIT_STATE] = (uint64_t)base * 8;
    sz[R_SPLIT_ITEMS] = split_item_capacity(plan) * 8;
    sz[R_SPLIT_RAYS] = split_ray_capacity(plan) * kRayWords * 4;
    sz[R_SPANS] = slots * 16;
    static_assert(R_END <= 32, "gsr_plan::off has 32 entries");
    uint64_t off = 0;
    for (int r = 0; r < R_END; ++r) {
        plan->off[r] = off;
        off += (sz[r] + 255) & ~uint64_t(255);
    }
    plan->workspace_bytes = off;
    return GSR_OK;
}

extern "C" gsr_status gsr_workspace_size(const gsr_plan* plan, size_t* bytes)
{
    if (!plan || !bytes) return GSR_ERR_INVALID_ARG;
    *bytes = (size_t)plan->workspace_bytes;
    return GSR_OK;
}

static gsr_status check_ws(const gsr_plan* plan, const void* ws, size_t bytes)
{
    if (!plan || !ws) return GSR_ERR_INVALID_ARG;
    if (bytes < plan->workspace_bytes || (reinterpret_cast<uintptr_t>(ws) & 255)) return GSR_ERR_WORKSPACE;
    return GSR_OK;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

extern "C" gsr_status gsr_preprocess(const gsr_plan* plan, const gsr_surfels* surfels, const gsr_objects* objects,
                                     void* workspace, size_t workspace_bytes, void* stream)
{
    if (!plan || !surfels || surfels->n != plan->n_surfels) return GSR_ERR_INVALID_ARG;
    return gsr_preprocess_part(plan, surfels, objects, 0, workspace, workspace_bytes, stream);
}

extern "C" gsr_status gsr_preprocess_part(const gsr_plan* plan, const gsr_surfels* surfels,
                                          const gsr_objects* objects, int first, void* workspace,
                                          size_t workspace_bytes, void* stream)
{
    gsr_status st = check_ws(plan, workspace, workspace_bytes);
    if (st != GSR_OK) return st;
    if (!surfels || surfels->n < 0 || first < 0 || (int64_t)first + surfels->n > plan->n_surfels)
        return GSR_ERR_INVALID_ARG;
    if (surfels->sh_degree < 0 || surfels->sh_degree > 3) return GSR_ERR_UNSUPPORTED;
    if (surfels->n > 0 && (!surfels->pos || !surfels->log_scale || !surfels->quat || !surfels->opacity || !surfels->sh))
        return GSR_ERR_INVALID_ARG;
    if (!aligned16(surfels->quat) || !aligned16(surfels->sh) || !aligned16(surfels->log_scale))
        return GSR_ERR_INVALID_ARG;
    const float* poses = nullptr;
    int n_obj = 0;
    if (objects && objects->n_objects > 0) {
        if (!objects->pose) return GSR_ERR_INVALID_ARG;
        poses = objects->pose;
        n_obj = objects->n_objects;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (first == 0) {
        uint32_t* counters = region<uint32_t>(plan, workspace, R_COUNTERS);
        e = cudaMemsetAsync(counters, 0, C_WORDS * 4, s);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (surfels->n > 0) {
        const SensorTable tab = make_sensor_table(plan);
        e = launch_preprocess(tab, *surfels, poses, n_obj, region<float4>(plan, workspace, R_RECORDS),
                              region<ushort4>(plan, workspace, R_RECTS), region<uint32_t>(plan, workspace, R_COUNTS),
                              region<uint32_t>(plan, workspace, R_DEPTHKEY), region<uint4>(plan, workspace, R_SPANS),
                              first, plan->n_surfels, s);
    }
    return cuda_fail(e);
}

extern "C" gsr_status gsr_bin_sort(const gsr_plan* plan, void* workspace, size_t workspace_bytes, void* stream)
{
    gsr_status st = check_ws(plan, workspace, workspace_bytes);
    if (st != GSR_OK) return st;
    return cuda_fail(bin_sort(plan, workspace, reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" gsr_status gsr_render_camera(const gsr_plan* plan, const void* workspace, size_t workspace_bytes,
                                        int32_t sensor, const gsr_camera_out* out, void* stream)
{
    gsr_status st = check_ws(plan, workspace, workspace_bytes);
    if (st != GSR_OK) return st;
    if (!out || sensor < 0 || sensor >= plan->n_sensors) return GSR_ERR_INVALID_ARG;
    if (plan->sensors[sensor].kind == GSR_SENSOR_LIDAR) return GSR_ERR_INVALID_ARG;
    FrameOut o{out->rgb, out->depth, out->normal, out->alpha, out->trans, out->depth_acc, out->n_contrib,
               out->n_walk, nullptr};
    return cuda_fail(launch_render(plan, workspace, sensor, o, reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" gsr_status gsr_render_lidar(const gsr_plan* plan, const void* workspace, size_t workspace_bytes,
                                       int32_t sensor, const gsr_lidar_out* out, void* stream)
{
    gsr_status st = check_ws(plan, workspace, workspace_bytes);
    if (st != GSR_OK) return st;
    if (!out || sensor < 0 || sensor >= plan->n_sensors) return GSR_ERR_INVALID_ARG;
    if (plan->sensors[sensor].kind != GSR_SENSOR_LIDAR) return GSR_ERR_INVALID_ARG;
    FrameOut o{out->intensity, out->range, nullptr, out->alpha, out->trans, nullptr, out->n_contrib,
               out->n_walk, out->ray_drop};
    return cuda_fail(launch_render(plan, workspace, sensor, o, reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" gsr_status gsr_read_status(const gsr_plan* plan, const void* workspace, int32_t* device_status,
                                      int64_t* n_visible, int64_t* n_pairs, void* stream)
{
    if (!plan || !workspace || !device_status) return GSR_ERR_INVALID_ARG;
    uint32_t h[C_WORDS];
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(h, region<uint32_t>(plan, workspace, R_COUNTERS), sizeof(h),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    *device_status = (int32_t)h[C_STATUS];
    if (n_visible) *n_visible = h[C_NVIS];
    if (n_pairs) {
        unsigned long long want;
        std::memcpy(&want, &h[C_NDUP_WANT], sizeof(want));
        *n_pairs = (int64_t)want;
    }
    return GSR_OK;
}

extern "C" gsr_status gsr_selftest_wait_timeout(const gsr_plan* plan, void* workspace, size_t workspace_bytes,
                                                uint32_t tries, void* stream)
{
    if (!plan || !workspace || tries == 0 || tries > (1u << 20)) return GSR_ERR_INVALID_ARG;
    size_t need = 0;
    gsr_status st = gsr_workspace_size(plan, &need);
    if (st != GSR_OK) return st;
    if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return GSR_ERR_WORKSPACE;
    return cuda_fail(launch_selftest_wait(region<uint32_t>(plan, workspace, R_COUNTERS), tries,
                                          reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" const char* gsr_status_string(gsr_status s)
{
    switch (s) {
    case GSR_OK: return "GSR_OK";
    case GSR_ERR_INVALID_ARG: return "GSR_ERR_INVALID_ARG";
    case GSR_ERR_CUDA: return "GSR_ERR_CUDA";
    case GSR_ERR_WORKSPACE: return "GSR_ERR_WORKSPACE";
    case GSR_ERR_CAPACITY: return "GSR_ERR_CAPACITY";
    case GSR_ERR_TIMEOUT: return "GSR_ERR_TIMEOUT";
    case GSR_ERR_UNSUPPORTED: return "GSR_ERR_UNSUPPORTED";
    case GSR_ERR_TOO_LARGE: return "GSR_ERR_TOO_LARGE";
    }
    return "GSR_ERR_UNKNOWN";
}

extern "C" const char* gsr_last_cuda_error(void) { return g_cuda_err; }

extern "C" gsr_status gsr_workspace_region(const gsr_plan* plan, const void* workspace, int32_t which, void** ptr,
                                           size_t* bytes)
{
    if (!plan || !workspace || !ptr) return GSR_ERR_INVALID_ARG;
    const uint64_t slots = (uint64_t)plan->n_surfels * plan->n_sensors;
    const int pb = sort_result_buffer(tile_sort_passes(plan));
    const int vb = sort_result_buffer(kDepthSortPasses);
    int r;
    uint64_t n;
    switch (which) {
    case 0: r = R_RECORDS; n = slots * kRecordBytes; break;
    case 1: r = R_RECTS; n = slots * 8; break;
    case 2: r = R_COUNTS; n = slots * 4; break;
    case 3: r = R_DEPTHKEY; n = slots * 4; break;
    case 4: r = pb ? R_PAIR_KEY_B : R_PAIR_KEY_A; n = (uint64_t)plan->max_dup * 4; break;
    case 5: r = pb ? R_PAIR_VAL_B : R_PAIR_VAL_A; n = (uint64_t)plan->max_dup * 4; break;
    case 6: r = R_RANGES; n = (uint64_t)plan->tile_base[plan->n_sensors] * 8; break;
    case 7: r = vb ? R_VIS_VAL_B : R_VIS_VAL_A; n = slots * 4; break;
    case 8: r = R_SPLIT_INFO; n = (uint64_t)plan->tile_base[plan->n_sensors] * 16; break;
    default: return GSR_ERR_INVALID_ARG;
    }
    *ptr = region<void>(plan, workspace, r);
    if (bytes) *bytes = (size_t)n;
    return GSR_OK;
}

extern "C" size_t gsr_struct_size(int32_t which)
{
    switch (which) {
    case 0: return sizeof(gsr_plan);
    case 1: return sizeof(gsr_sensor);
    case 2: return sizeof(gsr_surfels);
    case 3: return sizeof(gsr_objects);
    case 4: return sizeof(gsr_camera_out);
    case 5: return sizeof(gsr_lidar_out);
    case 6: return sizeof(gsr_tiling);
    case 7: return sizeof(gsr_camera_grad);
    case 8: return sizeof(gsr_surfel_grads);
    case 9: return sizeof(gsr_loss_weights);
    case 10: return sizeof(gsr_anchors);
    case 11: return sizeof(gsr_mlp);
    case 12: return sizeof(gsr_mlp_grads);
    case 13: return sizeof(gsr_surfel_table);
    case 14: return sizeof(gsr_autotune_space);
    case 15: return sizeof(gsr_autotune_result);
    case 16: return sizeof(gsr_zone_grid);
    case 17: return sizeof(gsr_streamer);
    case 18: return sizeof(gsr_lidar_grad);
    case 19: return sizeof(gsr_lidar_loss_weights);
    default: return 0;
    }
}

// ------------------------------------------------------------------ training
static gsr_status check_camera(const gsr_plan* plan, int32_t sensor)
{
    if (sensor < 0 || sensor >= plan->n_sensors) return GSR_ERR_INVALID_ARG;
    const int32_t kind = plan->sensors[sensor].kind;
    if (kind != GSR_SENSOR_PINHOLE && kind != GSR_SENSOR_CYLINDRICAL) return GSR_ERR_UNSUPPORTED;
    return GSR_OK;
}

extern "C" gsr_status gsr_loss(const gsr_plan* plan, void* workspace, size_t workspace_bytes, int32_t sensor,
                               const gsr_camera_out* fwd, const float* target_rgb, const gsr_loss_weights* weights,
                               float* loss, const gsr_camera_grad* grad, void* stream)
{
    gsr_status st = check_ws(plan, workspace, workspace_bytes);
    if (st != GSR_OK) return st;
    if ((st = check_camera(plan, sensor)) != GSR_OK) return st;
    if (!fwd || !target_rgb || !weights || !loss || !grad) return GSR_ERR_INVALID_ARG;
    if (!fwd->rgb || !fwd->alpha || !fwd->depth_acc || !fwd->normal) return GSR_ERR_INVALID_ARG;
    if (!grad->rgb || !grad->alpha || !grad->depth_acc || !grad->normal) return GSR_ERR_INVALID_ARG;
    return cuda_fail(launch_loss(plan, workspace, sensor, fwd, target_rgb, weights, loss, grad,
                                 reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" gsr_status gsr_backward_render(const gsr_plan* plan, void* workspace, size_t workspace_bytes,
                                          int32_t sensor, const gsr_camera_out* fwd, const gsr_camera_grad* grad,
                                          int32_t accumulate, void* stream)
{
    gsr_status st = check_ws(plan, workspace, workspace_bytes);
    if (st != GSR_OK) return st;
    if ((st = check_camera(plan, sensor)) != GSR_OK) return st;
    if (!fwd || !grad || !fwd->trans || !fwd->n_contrib) return GSR_ERR_INVALID_ARG;
    return cuda_fail(launch_render_backward(plan, workspace, sensor, fwd, grad, accumulate,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

static gsr_status check_lidar(const gsr_plan* plan, int32_t sensor)
{
    if (sensor < 0 || sensor >= plan->n_sensors) return GSR_ERR_INVALID_ARG;
    if (plan->sensors[sensor].kind != GSR_SENSOR_LIDAR) return GSR_ERR_UNSUPPORTED;
    return GSR_OK;
}

extern "C" gsr_status gsr_lidar_loss(const gsr_plan* plan, void* workspace, size_t workspace_bytes, int32_t sensor,
                                     const gsr_lidar_out* fwd, const float* target_range,
                                     const float* target_intensity, const gsr_lidar_loss_weights* weights,
                                     float* loss, const gsr_lidar_grad* grad, void* stream)
{
    gsr_status st = check_ws(plan, workspace, workspace_bytes);
    if (st != GSR_OK) return st;
    if ((st = check_lidar(plan, sensor)) != GSR_OK) return st;
    if (!fwd || !target_range || !target_intensity || !weights || !loss || !grad) return GSR_ERR_INVALID_ARG;
    if (!fwd->range || !fwd->alpha || !fwd->intensity || !fwd->ray_drop) return GSR_ERR_INVALID_ARG;
    if (!grad->intensity || !grad->alpha || !grad->depth_acc || !grad->ray_drop) return GSR_ERR_INVALID_ARG;
    return cuda_fail(launch_lidar_loss(plan, workspace, sensor, fwd, target_range, target_intensity, weights, loss,
                                       grad, reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" gsr_status gsr_backward_render_lidar(const gsr_plan* plan, void* workspace, size_t workspace_bytes,
                                                int32_t sensor, const gsr_lidar_out* fwd, const gsr_lidar_grad* grad,
                                                int32_t accumulate, void* stream)
{
    gsr_status st = check_ws(plan, workspace, workspace_bytes);
    if (st != GSR_OK) return st;
    if ((st = check_lidar(plan, sensor)) != GSR_OK) return st;
    if (!fwd || !grad || !fwd->trans || !fwd->n_contrib) return GSR_ERR_INVALID_ARG;
    return cuda_fail(launch_render_backward_lidar(plan, workspace, sensor, fwd, grad, accumulate,
                                                  reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" gsr_status gsr_backward_preprocess(const gsr_plan* plan, const void* workspace, size_t workspace_bytes,
                                              const gsr_surfels* surfels, const gsr_objects* objects,
                                              const gsr_surfel_grads* out, void* stream)
{
    gsr_status st = check_ws(plan, workspace, workspace_bytes);
    if (st != GSR_OK) return st;
    if (!surfels || surfels->n != plan->n_surfels || !out) return GSR_ERR_INVALID_ARG;
    if (surfels->sh_degree < 0 || surfels->sh_degree > 3) return GSR_ERR_UNSUPPORTED;
    if (surfels->n > 0 && (!out->pos || !out->log_scale || !out->quat || !out->opacity || !out->sh))
        return GSR_ERR_INVALID_ARG;
    if (objects && objects->n_objects > 0 && !objects->pose) return GSR_ERR_INVALID_ARG;
    return cuda_fail(launch_preprocess_backward(plan, workspace, surfels, objects, out,
                                                reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" gsr_status gsr_backward(const gsr_plan* plan, void* workspace, size_t workspace_bytes, int32_t sensor,
                                   const gsr_camera_out* fwd, const gsr_camera_grad* grad,
                                   const gsr_surfels* surfels, const gsr_objects* objects,
                                   const gsr_surfel_grads* out, void* stream)
{
    gsr_status st = gsr_backward_render(plan, workspace, workspace_bytes, sensor, fwd, grad, 0, stream);
    if (st != GSR_OK) return st;
    return gsr_backward_preprocess(plan, workspace, workspace_bytes, surfels, objects, out, stream);
}

// ------------------------------------------------------------------ whole rig
namespace gsr {
cudaError_t launch_render_rig(const gsr_plan* p, const void* ws, const FrameOut* outs, cudaStream_t st);
}

static gsr_status rig_outputs(const gsr_plan* plan, const gsr_camera_out* cam, const gsr_lidar_out* lid,
                              FrameOut* outs)
{
    for (int i = 0; i < plan->n_sensors; ++i) {
        if (plan->sensors[i].kind != GSR_SENSOR_LIDAR) {
            if (!cam) return GSR_ERR_INVALID_ARG;
            const gsr_camera_out& o = cam[i];
            outs[i] = FrameOut{o.rgb, o.depth, o.normal, o.alpha, o.trans, o.depth_acc, o.n_contrib, o.n_walk,
                               nullptr};
        } else {
            if (!lid) return GSR_ERR_INVALID_ARG;
            const gsr_lidar_out& o = lid[i];
            outs[i] = FrameOut{o.intensity, o.range, nullptr, o.alpha, o.trans, nullptr, o.n_contrib, o.n_walk,
                               o.ray_drop};
        }
    }
    return GSR_OK;
}

extern "C" gsr_status gsr_render_rig(const gsr_plan* plan, const void* workspace, size_t workspace_bytes,
                                     const gsr_camera_out* camera_outs, const gsr_lidar_out* lidar_outs, void* stream)
{
    gsr_status st = check_ws(plan, workspace, workspace_bytes);
    if (st != GSR_OK) return st;
    FrameOut outs[GSR_MAX_SENSORS];
    if ((st = rig_outputs(plan, camera_outs, lidar_outs, outs)) != GSR_OK) return st;
    return cuda_fail(launch_render_rig(plan, workspace, outs, reinterpret_cast<cudaStream_t>(stream)));
}

struct gsr_frame_graph_s {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" gsr_status gsr_frame_graph_create(const gsr_plan* plan, const gsr_surfels* surfels,
                                             const gsr_objects* objects, void* workspace, size_t workspace_bytes,
                                             const gsr_camera_out* camera_outs, const gsr_lidar_out* lidar_outs,
                                             int32_t stages, void* stream, gsr_frame_graph** graph)
{
    if (!graph || !stream || stages <= 0 || stages > 7) return GSR_ERR_INVALID_ARG;
    *graph = nullptr;
    gsr_status st = check_ws(plan, workspace, workspace_bytes);
    if (st != GSR_OK) return st;
    if (stages & GSR_STAGE_RENDER_RIG) {
        FrameOut outs[GSR_MAX_SENSORS];
        if ((st = rig_outputs(plan, camera_outs, lidar_outs, outs)) != GSR_OK) return st;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e);
    gsr_status rs = GSR_OK;
    if (stages & GSR_STAGE_PREPROCESS) rs = gsr_preprocess(plan, surfels, objects, workspace, workspace_bytes, stream);
    if (rs == GSR_OK && (stages & GSR_STAGE_BIN_SORT)) rs = gsr_bin_sort(plan, workspace, workspace_bytes, stream);
    if (rs == GSR_OK && (stages & GSR_STAGE_RENDER_RIG))
        rs = gsr_render_rig(plan, workspace, workspace_bytes, camera_outs, lidar_outs, stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (rs != GSR_OK) {
        if (g) cudaGraphDestroy(g);
        return rs;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e);
    }
    gsr_frame_graph* h = new (std::nothrow) gsr_frame_graph{g, x};
    if (!h) {
        cudaGraphExecDestroy(x);
        cudaGraphDestroy(g);
        return GSR_ERR_INVALID_ARG;
    }
    *graph = h;
    return GSR_OK;
}

extern "C" gsr_status gsr_frame_graph_launch(gsr_frame_graph* graph, void* stream)
{
    if (!graph) return GSR_ERR_INVALID_ARG;
    return cuda_fail(cudaGraphLaunch(graph->exec, reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" gsr_status gsr_frame_graph_destroy(gsr_frame_graph* graph)
{
    if (!graph) return GSR_OK;
    cudaError_t e1 = cudaGraphExecDestroy(graph->exec);
    cudaError_t e2 = cudaGraphDestroy(graph->graph);
    delete graph;
    return cuda_fail(e1 != cudaSuccess ? e1 : e2);
}
