// gsr_internal.cuh -- device-side layout and helpers shared by the kernels.
//
// Record (one per (sensor, surfel) slot, 6 x float4 = 96 B, written by the
// preprocess and staged into shared memory by the compositing kernels):
//   r0 = (Q00, Q01, Q02, c_x)   r1 = (Q10, Q11, Q12, c_y)
//   r2 = (Q20, Q21, Q22, det)   r3 = (opacity, f0, f1, f2)
//   r4 = (n_x, n_y, n_z, z_c)   r5 = (x0, x1, y0, y1) support box in ray indices
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

// Records are 6 float4; r5 = the ray-index box of the support (LiDAR
// columns x0..x1 on the azimuth circle, x0 in [0, columns)), used to skip
// records that miss every ray of a warp.
constexpr int kRecordF4 = 6;
constexpr int kRecordBytes = kRecordF4 * 16;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;
constexpr float kSupport = 9.0f;          // (3 sigma)^2 in units of sigma^2
constexpr float kLowPassInvVar = 2.0f;    // 1 / sigma_lp^2, sigma_lp^2 = 1/2 (px or cells)
constexpr float kLowPassRadius = 2.12132034f; // 3 sigma_lp
constexpr int kSortThreads = 256;
constexpr int kRadixBits = 8;
constexpr int kRadixBitsWide = 9;         // the widest digit of a pass (a key of 8k + 1 bits)
constexpr int kSortCtasPerSm = 4;         // the plan's sort grid: 4 CTAs on each SM
constexpr int kRadixIPT = 16;             // items per thread per radix scatter tile
constexpr int kRadixTile = kSortThreads * kRadixIPT;
constexpr int kRadixCtasPerSm = 2;        // resident radix scatter CTAs per SM (73-82 KB of shared memory each)
// Default split of long tile lists (gsr_tiling.split_first / split_chunk = 0).
constexpr int kSplitFirstDefault = 16384;  // positions walked before a tile's list is split
constexpr int kSplitChunkDefault = 384;    // positions per later chunk
constexpr int kRayWords = 13;             // words of a stored per-ray compositing state
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
    R_TILE_KEY_A, R_TILE_VAL_A, R_TILE_KEY_B, R_TILE_VAL_B,  // tiles by descending list length
    R_SPLIT_INFO,    // per tile uint4: chunks after the first, ray-record base, first item
    R_SPLIT_STATE,   // per tile uint2: phase-A outcome, chunks not yet walked
    R_SPLIT_ITEMS,   // (tile, chunk) of every split tile's chunks 1..C
    R_SPLIT_RAYS,    // ray records of split tiles (carry + one block per chunk)
    R_SPANS,         // per slot: the exact footprint's tile-row spans when short (SpanTable)
    R_RAY_DIRS,      // per cylinder / LiDAR sensor: its columns' then its rows' ray-direction terms (float2)
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
    C_NTILES = 7,    // total tiles of the plan (item count of the tile-order sort)
    C_NITEMS = 8,    // split-tile chunks of this frame
    C_SPLIT_QUEUE = 9, // work-queue head of the split-chunk kernel
    C_WORDS = 16
};

struct SensorDev {
    int kind;            // gsr_sensor_kind
    int width, height;
    int tiles_x, tiles_y;
    int tile_w, tile_h;  // screen tile of this sensor (rays)
    int tile_base;
    float R[9];          // world -> sensor rotation, row-major
    float t[3];
    float origin[3];     // sensor origin in world
    float fx, fy, cx, cy;
    float el_max, d_el, az0, d_az;   // radians (LiDAR)
    float inv_d_el, inv_d_az;
    float near_plane;
    float bg[3];
    int split_first, split_chunk;  // long lists: chunk 0 = split_first positions, then split_chunk each
    int dir_off;                   // first entry of this sensor's ray-direction table (cylinder, LiDAR)
};

struct SensorTable {
    int n;
    int tile_w, tile_h;
    int total_tiles;
    int batch;  // records staged per step of a walk; 0 = the CTA's thread count
    SensorDev s[GSR_MAX_SENSORS];
    const float2* dirs;  // ray-direction tables (R_RAY_DIRS), null where no render reads them
};

// The plan's sensors of one model (kernels instantiated per model).
struct SensorIds {
    int n;
    uint8_t id[GSR_MAX_SENSORS];
};

// First list position of chunk c of a split tile.
__host__ __device__ __forceinline__ int chunk_begin(int first, int chunk, int c)
{
    return c == 0 ? 0 : first + (c - 1) * chunk;
}

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
    float* drop;       // LiDAR ray-drop probability
};

SensorTable make_sensor_table(const gsr_plan* p, const void* ws = nullptr);
// Entries of the ray-direction tables: width + height per cylinder / LiDAR sensor.
int ray_dir_entries(const gsr_plan* p);
// Fill the tables (once per frame, by gsr_bin_sort).
cudaError_t launch_ray_dirs(const gsr_plan* p, void* ws, cudaStream_t st);

// Which buffer (0 = A, 1 = B) holds the result of a sort of `passes` passes that started in A.
inline int sort_result_buffer(int passes) { return passes & 1; }

// Capacity of the split-tile ray records (a fixed share of the pair
// capacity: one 52-byte record per 16 pairs) and of the split items (each
// item holds >= 32 ray records).  Tiles beyond it are walked unsplit.
inline uint64_t split_ray_capacity(const gsr_plan* p)
{
    const uint64_t c = (uint64_t)p->max_dup / 16;
    return c < 65536 ? 65536 : c;
}
inline uint64_t split_item_capacity(const gsr_plan* p) { return split_ray_capacity(p) / 32 + 1; }
int tile_sort_passes(const gsr_plan* p);
// Digit widths of the tile-key passes, low digit first; returns the count.
int tile_sort_widths(const gsr_plan* p, int widths[4]);
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

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
        // the ray direction d (LiDAR: unit; cylinder: (sin phi, y_n, cos phi))
        q0 = fmaf(r0.x, d0, fmaf(r0.y, d1, r0.z * d2));
        q1 = fmaf(r1.x, d0, fmaf(r1.y, d1, r1.z * d2));
        q2 = fmaf(r2.x, d0, fmaf(r2.y, d1, r2.z * d2));
        if (KIND == GSR_SENSOR_LIDAR) {  // the azimuth wraps around the spin
            const float half = 0.5f * columns;
            if (dx >= half) dx -= columns;
            if (dx < -half) dx += columns;
        }
    }
    // straight-line code (no early return): callers evaluate several
    // records at once and the independent chains interleave
    const float rq = __fdividef(1.f, q2);
    const float u = q0 * rq, v = q1 * rq;
    const float zi = r2.w * rq;
    const float rho3 = fmaf(u, u, v * v);
    const float rholp = kLowPassInvVar * fmaf(dx, dx, dy * dy);
    // G = max(G_3, G_lp) belongs to the smaller of the two radii; an
    // intersection at or behind the near plane takes no part, and a NaN
    // radius compares false and loses to the low-pass.  Ties take the
    // intersection.  Either branch counts only within the support.
    const float rho3f = zi > near_plane ? rho3 : __int_as_float(0x7f800000);
    const bool use3 = rho3f <= rholp;
    const float rho = fminf(rho3f, rholp);
    const bool inside = rho <= kSupport;
    // G = exp(-rho / 2) = 2^(-rho log2(e) / 2): one multiply by the folded
    // constant -log2(e) / 2 and the hardware base-2 exponential (rho <= 9 on
    // every hit, so the result is far from the flush-to-zero range)
    float G;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(G) : "f"(rho * -0.72134752f));
    const float alpha = fminf(kAlphaMax, R[3].x * G);
    sp.alpha = alpha;
    sp.z = use3 ? zi : R[4].w;
    sp.G = G;
    sp.q0 = q0; sp.q1 = q1; sp.q2 = q2;
    sp.u = u; sp.v = v; sp.rho = rho;
    sp.dx = dx; sp.dy = dy;
    sp.use3 = use3;
    return inside && alpha >= kAlphaMin;
}

// ------------------------------------------------------------ tile culling
// Support threshold of a surfel of opacity o: alpha = min(0.99, o G) >= 1/255
// needs rho <= 2 ln(255 o) (capped at the 3-sigma support), plus a margin.
__device__ __forceinline__ float support_rho(float o)
{
    return fminf(kSupport, __fadd_rn(__fmul_rn(2.f, __logf(__fmul_rn(255.f, o))), 1e-3f));
}

// Screen footprint of a camera record whose support disc lies in front of
// the camera: E(d) = q0^2 + q1^2 - rho q2^2 <= 0 with q = Q (d, 1), d = p - c.
// E(d) = d^T M d + 2 n^T d + k (M positive definite for such an ellipse).
// All arithmetic uses explicit _rn intrinsics so that every kernel that
// evaluates it takes bit-identical decisions.
struct Footprint {
    float m00, m01, m11, n0, n1, k;
    float cx, cy;
    float rlp2;   // squared low-pass radius (px^2)
    bool conic;   // M is safely positive definite
};

__device__ __forceinline__ Footprint make_footprint(float4 r0, float4 r1, float4 r2, float o)
{
    Footprint f;
    const float rho = support_rho(o);
    const float a0 = r0.x, a1 = r0.y, b0 = r1.x, b1 = r1.y, c0 = r2.x, c1 = r2.y, c2 = r2.z;
    f.m00 = __fsub_rn(__fadd_rn(__fmul_rn(a0, a0), __fmul_rn(b0, b0)), __fmul_rn(rho, __fmul_rn(c0, c0)));
    f.m01 = __fsub_rn(__fadd_rn(__fmul_rn(a0, a1), __fmul_rn(b0, b1)), __fmul_rn(rho, __fmul_rn(c0, c1)));
    f.m11 = __fsub_rn(__fadd_rn(__fmul_rn(a1, a1), __fmul_rn(b1, b1)), __fmul_rn(rho, __fmul_rn(c1, c1)));
    f.n0 = -__fmul_rn(rho, __fmul_rn(c2, c0));
    f.n1 = -__fmul_rn(rho, __fmul_rn(c2, c1));
    f.k = -__fmul_rn(rho, __fmul_rn(c2, c2));
    f.cx = r0.w;
    f.cy = r1.w;
    f.rlp2 = fmaxf(__fmul_rn(0.5f, rho), 0.f);
    const float dm = __fsub_rn(__fmul_rn(f.m00, f.m11), __fmul_rn(f.m01, f.m01));
    f.conic = f.m00 > 0.f && f.m11 > 0.f && dm > __fmul_rn(1e-4f, __fmul_rn(f.m00, f.m11));
    return f;
}

__device__ __forceinline__ float fp_eval(const Footprint& f, float dx, float dy)
{
    const float qx = __fadd_rn(__fadd_rn(__fmul_rn(f.m00, dx), __fmul_rn(f.m01, dy)), __fmul_rn(2.f, f.n0));
    const float qy = __fadd_rn(__fadd_rn(__fmul_rn(f.m01, dx), __fmul_rn(f.m11, dy)), __fmul_rn(2.f, f.n1));
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, qx), __fmul_rn(dy, qy)), f.k);
}

// min of E along d_y in [lo, hi] at fixed d_x (and the symmetric case).
__device__ __forceinline__ float fp_edge_y(const Footprint& f, float dx, float lo, float hi)
{
    const float t = -__fdiv_rn(__fadd_rn(__fmul_rn(f.m01, dx), f.n1), f.m11);
    return fp_eval(f, dx, fminf(fmaxf(t, lo), hi));
}
__device__ __forceinline__ float fp_edge_x(const Footprint& f, float dy, float lo, float hi)
{
    const float t = -__fdiv_rn(__fadd_rn(__fmul_rn(f.m01, dy), f.n0), f.m00);
    return fp_eval(f, fminf(fmaxf(t, lo), hi), dy);
}

// Can any pixel centre of the tile [x0, x1) x [y0, y1) (pixel units) see
// the surfel?  The rectangle of centres is widened by one pixel on each side
// to absorb FP32 rounding of the per-pixel evaluation.
__device__ __forceinline__ bool footprint_hits(const Footprint& f, float x0, float y0, float x1, float y1)
{
    const float lx = __fsub_rn(__fsub_rn(x0, 0.5f), f.cx), hx = __fsub_rn(__fadd_rn(x1, 0.5f), f.cx);
    const float ly = __fsub_rn(__fsub_rn(y0, 0.5f), f.cy), hy = __fsub_rn(__fadd_rn(y1, 0.5f), f.cy);
    // low-pass disc around the centre
    const float ex = fminf(fmaxf(0.f, lx), hx), ey = fminf(fmaxf(0.f, ly), hy);
    const float r = __fadd_rn(sqrtf(f.rlp2), 1.f);
    if (__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)) <= __fmul_rn(r, r)) return true;
    if (!f.conic) return true;
    // unconstrained minimiser of the convex quadratic
    const float det = __fsub_rn(__fmul_rn(f.m00, f.m11), __fmul_rn(f.m01, f.m01));
    const float sx = __fdiv_rn(__fsub_rn(__fmul_rn(f.m01, f.n1), __fmul_rn(f.m11, f.n0)), det);
    const float sy = __fdiv_rn(__fsub_rn(__fmul_rn(f.m01, f.n0), __fmul_rn(f.m00, f.n1)), det);
    if (sx >= lx && sx <= hx && sy >= ly && sy <= hy) return fp_eval(f, sx, sy) <= 0.f;
    if (fp_edge_y(f, lx, ly, hy) <= 0.f || fp_edge_y(f, hx, ly, hy) <= 0.f) return true;
    return fp_edge_x(f, ly, lx, hx) <= 0.f || fp_edge_x(f, hy, lx, hx) <= 0.f;
}

// The same question for culling inside the compositing walk, in fast FP32
// (fused operations, approximate reciprocals): the one-pixel margin is far
// larger than their error, so a record it rejects cannot reach a pixel
// centre of the box.  Box = pixels [x0, x1] x [y0, y1] (inclusive).
__device__ __forceinline__ bool footprint_meets_box(const float4 r0, const float4 r1, const float4 r2, float o,
                                                    float x0, float x1, float y0, float y1)
{
    const float rho = fminf(kSupport, 2.f * __logf(255.f * o) + 1e-3f);
    const float a0 = r0.x, a1 = r0.y, b0 = r1.x, b1 = r1.y, c0 = r2.x, c1 = r2.y, c2 = r2.z;
    const float m00 = a0 * a0 + b0 * b0 - rho * c0 * c0;
    const float m01 = a0 * a1 + b0 * b1 - rho * c0 * c1;
    const float m11 = a1 * a1 + b1 * b1 - rho * c1 * c1;
    const float n0 = -rho * c2 * c0, n1 = -rho * c2 * c1, k = -rho * c2 * c2;
    // pixel centres x + 1/2 of the box, widened by one pixel, relative to the centre
    const float lx = x0 - 0.5f - r0.w, hx = x1 + 1.5f - r0.w;
    const float ly = y0 - 0.5f - r1.w, hy = y1 + 1.5f - r1.w;
    const float ex = fminf(fmaxf(0.f, lx), hx), ey = fminf(fmaxf(0.f, ly), hy);
    const float r = sqrtf(fmaxf(0.5f * rho, 0.f)) + 1.f;
    if (ex * ex + ey * ey <= r * r) return true;  // the low-pass disc
    const float dm = m00 * m11 - m01 * m01;
    if (!(m00 > 0.f && m11 > 0.f && dm > 1e-4f * m00 * m11)) return true;  // no usable conic
    auto E = [&](float dx, float dy) {
        return dx * (m00 * dx + m01 * dy + 2.f * n0) + dy * (m01 * dx + m11 * dy + 2.f * n1) + k;
    };
    const float id = __fdividef(1.f, dm);
    const float sx = (m01 * n1 - m11 * n0) * id, sy = (m01 * n0 - m00 * n1) * id;
    if (sx >= lx && sx <= hx && sy >= ly && sy <= hy) return E(sx, sy) <= 0.f;
    const float i00 = __fdividef(1.f, m00), i11 = __fdividef(1.f, m11);
    const float ty0 = fminf(fmaxf(-(m01 * lx + n1) * i11, ly), hy), ty1 = fminf(fmaxf(-(m01 * hx + n1) * i11, ly), hy);
    const float tx0 = fminf(fmaxf(-(m01 * ly + n0) * i00, lx), hx), tx1 = fminf(fmaxf(-(m01 * hy + n0) * i00, lx), hx);
    return E(lx, ty0) <= 0.f || E(hx, ty1) <= 0.f || E(tx0, ly) <= 0.f || E(tx1, hy) <= 0.f;
}

// Bit 15 of rect.w marks a camera slot whose tile set is footprint-tested.
constexpr uint16_t kRectExact = 0x8000;

// Roots of a dx^2 + 2 b dx + e = 0 (a > 0); false if none.
__device__ __forceinline__ bool fp_roots(float a, float b, float e, float& lo, float& hi)
{
    const float disc = __fsub_rn(__fmul_rn(b, b), __fmul_rn(a, e));
    if (!(disc >= 0.f)) return false;
    const float s = sqrtf(disc);
    lo = __fdiv_rn(__fsub_rn(-b, s), a);
    hi = __fdiv_rn(__fadd_rn(-b, s), a);
    return true;
}

// x-extent (relative to the centre) of the footprint inside the horizontal
// band dy in [ly, hy]: the conic part is convex, so its extremes over the
// band are at the band edges or at its own leftmost / rightmost points; the
// low-pass disc (radius r) adds [-w, w].  Returns false if the band misses both.
__device__ __forceinline__ bool footprint_row(const Footprint& f, float ly, float hy, float& xlo, float& xhi)
{
    bool any = false;
    xlo = 3.0e38f;
    xhi = -3.0e38f;
    const float r = __fadd_rn(sqrtf(f.rlp2), 1.f);
    const float yc = fminf(fmaxf(0.f, ly), hy);
    const float w2 = __fsub_rn(__fmul_rn(r, r), __fmul_rn(yc, yc));
    if (w2 >= 0.f) {
        const float w = sqrtf(w2);
        xlo = -w;
        xhi = w;
        any = true;
    }
    if (!f.conic) {  // no usable conic: the whole row band is kept
        xlo = -3.0e38f;
        xhi = 3.0e38f;
        return true;
    }
    // the conic's own leftmost / rightmost points satisfy m01 dx + m11 dy + n1 = 0,
    // i.e. dy = g dx + h, where E(dx, g dx + h) = A dx^2 + 2 B dx + C vanishes
    const float g = -__fdiv_rn(f.m01, f.m11), h = -__fdiv_rn(f.n1, f.m11);
    const float A = __fadd_rn(__fadd_rn(f.m00, __fmul_rn(2.f, __fmul_rn(f.m01, g))), __fmul_rn(f.m11, __fmul_rn(g, g)));
    const float B = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(f.m01, h), __fmul_rn(f.m11, __fmul_rn(g, h))), f.n0),
                              __fmul_rn(f.n1, g));
    const float C = __fadd_rn(__fadd_rn(__fmul_rn(f.m11, __fmul_rn(h, h)), __fmul_rn(2.f, __fmul_rn(f.n1, h))), f.k);
    float x0, x1;
    // the conic contains the centre (E(0) = k <= 0), so both extreme points
    // exist; if rounding says otherwise, keep the whole band
    if (!(A > 0.f) || !fp_roots(A, B, C, x0, x1)) {
        xlo = -3.0e38f;
        xhi = 3.0e38f;
        return true;
    }
    {
        const float y0 = __fadd_rn(__fmul_rn(g, x0), h), y1 = __fadd_rn(__fmul_rn(g, x1), h);
        if (y0 >= ly && y0 <= hy) {
            xlo = fminf(xlo, x0);
            xhi = fmaxf(xhi, x0);
            any = true;
        }
        if (y1 >= ly && y1 <= hy) {
            xlo = fminf(xlo, x1);
            xhi = fmaxf(xhi, x1);
            any = true;
        }
    }
    // and the band edges
    const float cand[2] = {ly, hy};
    for (int k = 0; k < 2; ++k) {
        const float dy = cand[k];
        const float b = __fadd_rn(__fmul_rn(f.m01, dy), f.n0);
        const float e = __fadd_rn(__fadd_rn(__fmul_rn(f.m11, __fmul_rn(dy, dy)), __fmul_rn(2.f, __fmul_rn(f.n1, dy))), f.k);
        float lo, hi;
        if (fp_roots(f.m00, b, e, lo, hi)) {
            xlo = fminf(xlo, lo);
            xhi = fmaxf(xhi, hi);
            any = true;
        }
    }
    return any;
}

// Tile columns [t0, t1] of tile row ty that the footprint reaches, widened by
// one pixel on each side for FP32 rounding (clamped to [tx0, tx1]).
__device__ __forceinline__ bool footprint_span(const Footprint& f, int ty, int TW, int TH, int tx0, int tx1, int& t0,
                                               int& t1)
{
    const float ly = __fsub_rn(__fsub_rn((float)(ty * TH), 0.5f), f.cy);
    const float hy = __fsub_rn(__fadd_rn((float)((ty + 1) * TH), 0.5f), f.cy);
    float xlo, xhi;
    if (!footprint_row(f, ly, hy, xlo, xhi)) return false;
    const float X0 = __fadd_rn(xlo, f.cx), X1 = __fadd_rn(xhi, f.cx);
    // tile tx covers [tx TW - 0.5, (tx+1) TW + 0.5]
    const float a = fmaxf(__fdiv_rn(__fsub_rn(__fsub_rn(X0, 0.5f), (float)TW), (float)TW), -1.f);
    const float b = fminf(__fdiv_rn(__fadd_rn(X1, 0.5f), (float)TW), 65536.f);
    t0 = max(tx0, (int)ceilf(a));
    t1 = min(tx1, (int)floorf(b));
    return t0 <= t1;
}

// Tile-row spans of an exact camera footprint, cached by the preprocess for
// the duplication when the rectangle has at most kSpanRows rows and fewer
// than 255 columns (a uint4 per slot, little-endian bytes): byte 0 = rows
// cached (0 = none), then per row of the rectangle (from its first row) the
// first tile column minus the rectangle's and the span length (0 = the
// footprint misses the row).
constexpr int kSpanRows = 7;

// Does a record's support box r5 meet the warp box?  LiDAR columns are
// intervals on the azimuth circle of `columns` cells (the warp's never wraps).
template <int KIND>
__device__ __forceinline__ bool box_meets(const float4 r5, const float4 w, float columns)
{
    const bool rows = r5.w >= w.z && r5.z <= w.w;
    if (KIND != GSR_SENSOR_LIDAR) return rows && r5.y >= w.x && r5.x <= w.y;
    float d = w.x - r5.x;  // warp start inside the record's interval?
    if (d < 0.f) d += columns;
    float e = r5.x - w.x;  // record start inside the warp's interval?
    if (e < 0.f) e += columns;
    return rows && w.x <= w.y && (d <= r5.y - r5.x || e <= w.y - w.x);
}

// Per-ray compositing state.  Stored ray records (split tiles, below) keep
// its 13 fields in this order, one word each.
struct RayState {
    float T, A, B, D;
    float f0, f1, f2;
    float n0, n1, n2;
    uint32_t last;
    uint32_t walk;
    bool done;
};

// Ray of thread `tid` within a tile of tw x th rays.  A warp takes an 8 x 4
// block of the tile where the tile is wider than 8 and divides into such
// blocks (a compact block keeps the warp's ray box, against which the walks
// cull records, small), else the tile's rays in row-major order.  The
// forward and the backward walks, and the ray records of split tiles, all
// use this map.
__device__ __forceinline__ void tile_ray_xy(int tw, int th, int tid, int& lx, int& ly)
{
    if (tw > 8 && (tw & 7) == 0 && (th & 3) == 0) {
        const int lane = tid & 31, w = tid >> 5, wpr = tw >> 3;
        lx = (w % wpr) * 8 + (lane & 7);
        ly = (w / wpr) * 4 + (lane >> 3);
    } else {
        lx = tid % tw;
        ly = tid / tw;
    }
}

__device__ __forceinline__ void ray_init(RayState& s, bool done, uint32_t n)
{
    s.T = 1.f; s.A = 0.f; s.B = 0.f; s.D = 0.f;
    s.f0 = s.f1 = s.f2 = 0.f;
    s.n0 = s.n1 = s.n2 = 0.f;
    s.last = 0;
    s.walk = n;
    s.done = done;
}

// Ray record block: field f of ray r at blk[f * R + r] (coalesced per field).
__device__ __forceinline__ void store_ray(float* blk, int R, int r, const RayState& s)
{
    blk[0 * R + r] = s.T; blk[1 * R + r] = s.A; blk[2 * R + r] = s.B; blk[3 * R + r] = s.D;
    blk[4 * R + r] = s.f0; blk[5 * R + r] = s.f1; blk[6 * R + r] = s.f2;
    blk[7 * R + r] = s.n0; blk[8 * R + r] = s.n1; blk[9 * R + r] = s.n2;
    blk[10 * R + r] = __uint_as_float(s.last);
    blk[11 * R + r] = __uint_as_float(s.walk);
    blk[12 * R + r] = __uint_as_float(s.done ? 1u : 0u);
}

// Loads bypass L1: the block was written by another CTA of this grid.
__device__ __forceinline__ void load_ray(const float* blk, int R, int r, RayState& s)
{
    s.T = __ldcg(blk + 0 * R + r); s.A = __ldcg(blk + 1 * R + r);
    s.B = __ldcg(blk + 2 * R + r); s.D = __ldcg(blk + 3 * R + r);
    s.f0 = __ldcg(blk + 4 * R + r); s.f1 = __ldcg(blk + 5 * R + r); s.f2 = __ldcg(blk + 6 * R + r);
    s.n0 = __ldcg(blk + 7 * R + r); s.n1 = __ldcg(blk + 8 * R + r); s.n2 = __ldcg(blk + 9 * R + r);
    s.last = __float_as_uint(__ldcg(blk + 10 * R + r));
    s.walk = __float_as_uint(__ldcg(blk + 11 * R + r));
    s.done = __float_as_uint(__ldcg(blk + 12 * R + r)) != 0u;
}

struct SplitBufs {
    const uint4* info;  // per tile: x = chunks after the first (0: not split), y = ray-record base, z = first item
    uint2* state;       // per tile: x = 1 carry stored / 2 finished in chunk 0, y = chunks not yet walked
    const uint2* items; // (tile, chunk)
    float* rays;        // ray records, kRayWords words each
};

__device__ __forceinline__ float* ray_block(const SplitBufs& sp, uint32_t base, int R, int k)
{
    return sp.rays + ((size_t)base + (size_t)k * R) * kRayWords;
}

// Per-ray setup shared by the forward and backward rasterisers.  A cylinder
// or LiDAR ray's direction comes from its sensor's tables (the sine and
// cosine of each column's and row's angle, evaluated in FP64 and rounded to
// FP32 once per frame), so every direction is within a few FP32 roundings of
// the exact one wherever the angle lies; rays outside the sensor (ragged
// tiles) read its last column or row, and their results are never used.
template <int KIND>
__device__ __forceinline__ void ray_setup(const SensorDev& sd, const float2* __restrict__ dirs, int x, int y,
                                          float& rx, float& ry, float& d0, float& d1, float& d2)
{
    const int cx = min(max(x, 0), sd.width - 1), cy = min(max(y, 0), sd.height - 1);
    if (KIND == GSR_SENSOR_PINHOLE) {
        rx = x + 0.5f;
        ry = y + 0.5f;
        d0 = d1 = d2 = 0.f;
    } else if (KIND == GSR_SENSOR_CYLINDRICAL) {
        // Eq. 4: azimuth about the camera's y axis, height on the unit cylinder
        rx = x + 0.5f;
        ry = y + 0.5f;
        const float2 c = dirs[sd.dir_off + cx];              // (sin phi, cos phi)
        d0 = c.x;
        d1 = dirs[sd.dir_off + sd.width + cy].x;            // (y + 1/2 - cy) / fy
        d2 = c.y;
    } else {
        rx = (float)x;
        ry = (float)y;
        const float2 a = dirs[sd.dir_off + cx];              // (cos az, sin az)
        const float2 e = dirs[sd.dir_off + sd.width + cy];   // (cos el, sin el)
        d0 = e.x * a.x;
        d1 = e.x * a.y;
        d2 = e.y;
    }
}

}  // namespace gsr
