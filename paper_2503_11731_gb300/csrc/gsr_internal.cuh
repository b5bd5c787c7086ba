// gsr_internal.cuh -- device-side layout and helpers shared by the kernels.
//
// Record (one per (sensor, surfel) slot, 5 x float4 = 80 B, written by the
// preprocess and staged into shared memory by the compositing kernels):
//   r0 = (Q00, Q01, Q02, c_x)   r1 = (Q10, Q11, Q12, c_y)
//   r2 = (Q20, Q21, Q22, det)   r3 = (opacity, f0, f1, f2)
//   r4 = (n_x, n_y, n_z, z_c)
// Q is the adjugate of the surfel's 3x3 ray-space matrix M (Eq. 1: the
// distinct rows of W H), so for a ray r (camera: (p - c, 1) in pixel-
// homogeneous coordinates about the projected centre c; LiDAR: the unit ray
// direction) the solution of Eq. 2 is (u, v, 1) ~ q = Q r, and the depth /
// distance of the intersection is det / q_2.  f = colour (camera) or
// (intensity, 0, 0) (LiDAR); n = facing normal in the sensor frame; z_c =
// centre depth (camera) or centre range (LiDAR), the composite-order key.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gsr.h"

namespace gsr {

constexpr int kRecordF4 = 5;
constexpr int kRecordBytes = kRecordF4 * 16;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kSupport = 9.0f;          // (3 sigma)^2 in units of sigma^2
constexpr float kLowPassInvVar = 2.0f;    // 1 / sigma_lp^2, sigma_lp^2 = 1/2 (px or cells)
constexpr float kLowPassRadius = 2.12132034f; // 3 sigma_lp
constexpr int kSortThreads = 256;
constexpr int kSortIPT = 8;               // items per thread per sort tile
constexpr int kSortTile = kSortThreads * kSortIPT;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

// Workspace regions (indices into gsr_plan::off).
enum Region : int {
    R_RECORDS = 0, R_RECTS, R_COUNTS, R_DEPTHKEY,
    R_PAIR_KEY_A, R_PAIR_VAL_A, R_PAIR_KEY_B, R_PAIR_VAL_B,
    R_RANGES,
    R_VIS_KEY_A, R_VIS_VAL_A, R_VIS_KEY_B, R_VIS_VAL_B,
    R_CNT_SORTED, R_OFFSETS,
    R_HIST, R_PARTIAL,
    R_COUNTERS,
    R_SENSOR_OF_TILE,
    R_RECGRAD,       // d(loss)/d(record), same layout as R_RECORDS
    R_LOSS_SCRATCH,  // loss: [6][H][W] central-difference gradients + block partials
    R_END
};

// Counter words (uint32 unless noted) at R_COUNTERS.
enum Counter : int {
    C_NVIS = 0,      // visible slots after compaction
    C_NDUP = 1,      // pairs kept (<= max_dup)
    C_STATUS = 2,    // gsr_status of device-side conditions
    C_QUEUE = 3,     // work-queue head of the persistent rig kernel
    C_NDUP_WANT = 4, // uint64 at words 4..5: pairs requested
    C_TIMEOUT_AT = 6,
    C_WORDS = 16
};

struct SensorDev {
    int kind;            // gsr_sensor_kind
    int width, height;
    int tiles_x, tiles_y;
    int tile_base;
    float R[9];          // world -> sensor rotation, row-major
    float t[3];
    float origin[3];     // sensor origin in world
    float fx, fy, cx, cy;
    float el_max, d_el, az0, d_az;   // radians (LiDAR)
    float inv_d_el, inv_d_az;
    float near_plane;
    float bg[3];
};

struct SensorTable {
    int n;
    int tile_w, tile_h;
    int total_tiles;
    SensorDev s[GSR_MAX_SENSORS];
};

// Host helper: the workspace region pointer.
template <class T>
inline T* region(const gsr_plan* p, const void* ws, int r)
{
    return reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(ws) + p->off[r]);
}

// Unified per-pixel outputs of a sensor (camera or LiDAR).
struct FrameOut {
    float* color;      // [C][H][W] (camera rgb, LiDAR intensity)
    float* depth;      // expected depth / range
    float* normal;     // [3][H][W]
    float* alpha;
    float* trans;
    float* depth_acc;  // [2][H][W]
    uint32_t* n_contrib;
    uint32_t* n_walk;
};

SensorTable make_sensor_table(const gsr_plan* p);

// Which buffer (0 = A, 1 = B) holds the result of a sort of `passes` passes that started in A.
inline int sort_result_buffer(int passes) { return passes & 1; }
int tile_sort_passes(const gsr_plan* p);
constexpr int kDepthSortPasses = 4;

// --------------------------------------------------------------- device helpers
__device__ __forceinline__ void set_status(uint32_t* counters, int code)
{
    atomicCAS(&counters[C_STATUS], 0u, (uint32_t)code);
}

// Shared-memory address for PTX.
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One bulk async copy global -> shared completing on `bar` (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on a phase of `bar`.  Each try_wait suspends for a
// hardware-chosen interval; after `limit` tries the wait gives up, records
// GSR_ERR_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* counters,
                                                  uint32_t limit = 1u << 22)
{
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    set_status(counters, GSR_ERR_TIMEOUT);
    return false;
}

// ------------------------------------------------------------ splat evaluation
// One ray against one staged record (Eqs. 2-3 / 2,5 in closed form plus the
// 2DGS low-pass fallback).  Shared by the forward and backward rasterisers
// so that both take bit-identical decisions.
struct Splat {
    float alpha;   // min(0.99, o G)
    float z;       // contribution depth / distance
    float G;       // Gaussian value of the chosen branch
    float q0, q1, q2, u, v, rho;
    float dx, dy;  // ray minus projected centre (pixels, or wrapped cells)
    bool use3;     // ray-splat intersection (true) or low-pass (false)
};

template <int KIND>
__device__ __forceinline__ bool splat_eval(const float4* __restrict__ R, float rx, float ry, float d0, float d1,
                                           float d2, float near_plane, float columns, Splat& sp)
{
    const float4 r0 = R[0], r1 = R[1], r2 = R[2];
    float dx = rx - r0.w, dy = ry - r1.w;
    float q0, q1, q2;
    if (KIND == GSR_SENSOR_PINHOLE) {
        q0 = fmaf(r0.x, dx, r0.y * dy);
        q1 = fmaf(r1.x, dx, r1.y * dy);
        q2 = fmaf(r2.x, dx, fmaf(r2.y, dy, r2.z));
    } else {
        q0 = fmaf(r0.x, d0, fmaf(r0.y, d1, r0.z * d2));
        q1 = fmaf(r1.x, d0, fmaf(r1.y, d1, r1.z * d2));
        q2 = fmaf(r2.x, d0, fmaf(r2.y, d1, r2.z * d2));
        const float half = 0.5f * columns;
        if (dx >= half) dx -= columns;
        if (dx < -half) dx += columns;
    }
    const float rq = __fdividef(1.f, q2);
    const float u = q0 * rq, v = q1 * rq;
    const float zi = r2.w * rq;
    const float rho3 = fmaf(u, u, v * v);
    const float rholp = kLowPassInvVar * fmaf(dx, dx, dy * dy);
    const bool v3 = (zi > near_plane) && (rho3 <= kSupport);
    const bool vlp = rholp <= kSupport;
    if (!(v3 || vlp)) return false;
    const bool use3 = v3 && (!vlp || rho3 <= rholp);
    const float rho = use3 ? rho3 : rholp;
    const float G = __expf(-0.5f * rho);
    const float alpha = fminf(kAlphaMax, R[3].x * G);
    if (alpha < kAlphaMin) return false;
    sp.alpha = alpha;
    sp.z = use3 ? zi : R[4].w;
    sp.G = G;
    sp.q0 = q0; sp.q1 = q1; sp.q2 = q2;
    sp.u = u; sp.v = v; sp.rho = rho;
    sp.dx = dx; sp.dy = dy;
    sp.use3 = use3;
    return true;
}

// Per-ray setup shared by the forward and backward rasterisers.
template <int KIND>
__device__ __forceinline__ void ray_setup(const SensorDev& sd, int x, int y, float& rx, float& ry, float& d0,
                                          float& d1, float& d2)
{
    if (KIND == GSR_SENSOR_PINHOLE) {
        rx = x + 0.5f;
        ry = y + 0.5f;
        d0 = d1 = d2 = 0.f;
    } else {
        rx = (float)x;
        ry = (float)y;
        float se, ce, sa, ca;
        sincosf(sd.el_max - y * sd.d_el, &se, &ce);
        sincosf(sd.az0 + (x + 0.5f) * sd.d_az, &sa, &ca);
        d0 = ce * ca;
        d1 = ce * sa;
        d2 = se;
    }
}

}  // namespace gsr
