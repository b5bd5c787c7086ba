// mlp.cu -- anchor MLP decode (neural Gaussians) and its training kernels.
//
// The paper infers each surfel's attributes by passing anchor features
// through an MLP (Sec. III-A, "Scene Reconstruction", anchors as in
// Scaffold-GS).  Per anchor a and view origin o:
//   X = [f_a (32), (x_a - o)/|x_a - o| (3), |x_a - o| (1)]      (36 inputs)
//   H = ReLU(X W1 + b1)                                         (64 hidden)
//   Y = H W2 + b2 = 10 offsets x {opacity logit, colour logits (3),
//       log-scales (2), raw quaternion (4)}                     (100 outputs)
// and offset j becomes a surfel at x_a + l_a o_{a,j} with log-scale y + ln l_a,
// colour sigmoid(y) (stored as a degree-0 SH coefficient), and the anchor's
// LiDAR intensity.  The LiDAR scene's head (the paper reconstructs a
// separate LiDAR scene whose MLP infers rho and r as well) reads the three
// colour logits as intensity logit, ray-drop logit and an unused value.  Anchors whose bounding sphere (l_a max|o| + 3 m) lies
// outside a given camera frustum are culled (their surfels get opacity
// logit -1e4, which the preprocess discards).
//
//  k_decode_tc   BF16 inputs/weights on tcgen05 tensor cores with FP32
//                accumulators in tensor memory: one CTA = 128 anchors =
//                one M=128 tile; layer 1 (K=48 padded, N=64), bias+ReLU in
//                registers, layer 2 (K=64, N=112 padded) into the same
//                TMEM columns, epilogue writes the surfel table.
//  k_decode_f32  the same decode in FP32 on the SIMT cores (reference path).
//  k_decode_backward  recomputes the forward in FP32 and back-propagates
//                d(loss)/d(surfel table) to W1, b1, W2, b2 and the features.
//  k_adam        Adam update of FP32 master parameters.
#include "gsr_internal.cuh"
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "tcgen05.cuh"

namespace gsr {

namespace {

constexpr int kFeat = 32, kIn = 36, kInPad = 48, kHid = 64, kOff = 10, kOut = 100, kOutPad = 112;
constexpr int kTileA = 128;  // anchors per CTA (the MMA M)
constexpr float kY00 = 0.28209479177387814f;
constexpr float kCulledLogit = -1.0e4f;

struct DecodeArgs {
    int n;                    // anchors
    const float* pos;         // [n][3]
    const float* feature;     // [n][32]
    const float* scale;       // [n]
    const float* offsets;     // [n][10][3]
    const float* intensity;   // [n][10] or null
    const float* w1;          // [36][64]
    const float* b1;          // [64]
    const float* w2;          // [64][100]
    const float* b2;          // [100]
    int head;                 // GSR_HEAD_CAMERA or GSR_HEAD_LIDAR
    float ox, oy, oz;         // view origin
    int cull;                 // 1: test the camera frustum below
    float R[9], t[3];         // world -> camera
    float plane[4][3];        // unit inward normals of the side planes (camera frame)
    float near_plane;
    float* out_pos;           // [n*10][3]
    float* out_log_scale;     // [n*10][2]
    float* out_quat;          // [n*10][4]
    float* out_opacity;       // [n*10]
    float* out_sh;            // [n*10][1][3]
    float* out_intensity;     // [n*10] or null
    float* out_ray_drop;      // [n*10] or null (LiDAR head)
    uint32_t* status;         // device status word (timeouts), or null
};

__device__ __forceinline__ bool culled(const DecodeArgs& a, int i)
{
    if (!a.cull) return false;
    const float x = a.pos[3 * i], y = a.pos[3 * i + 1], z = a.pos[3 * i + 2];
    const float px = fmaf(a.R[0], x, fmaf(a.R[1], y, a.R[2] * z)) + a.t[0];
    const float py = fmaf(a.R[3], x, fmaf(a.R[4], y, a.R[5] * z)) + a.t[1];
    const float pz = fmaf(a.R[6], x, fmaf(a.R[7], y, a.R[8] * z)) + a.t[2];
    float omax = 0.f;
    for (int j = 0; j < kOff; ++j) {
        const float* o = a.offsets + ((size_t)i * kOff + j) * 3;
        omax = fmaxf(omax, sqrtf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]));
    }
    const float r = a.scale[i] * omax + 3.f;
    if (pz < a.near_plane - r) return true;
    for (int k = 0; k < 4; ++k)
        if (a.plane[k][0] * px + a.plane[k][1] * py + a.plane[k][2] * pz < -r) return true;
    return false;
}

__device__ __forceinline__ void input_row(const DecodeArgs& a, int i, float* X)
{
    for (int k = 0; k < kFeat; ++k) X[k] = a.feature[(size_t)i * kFeat + k];
    const float vx = a.pos[3 * i] - a.ox, vy = a.pos[3 * i + 1] - a.oy, vz = a.pos[3 * i + 2] - a.oz;
    const float d = sqrtf(vx * vx + vy * vy + vz * vz);
    const float id = 1.f / d;
    X[32] = vx * id;
    X[33] = vy * id;
    X[34] = vz * id;
    X[35] = d;
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + __expf(-x)); }

// Surfels of anchor i from its 100 outputs y (bias included).
__device__ __forceinline__ void write_surfels(const DecodeArgs& a, int i, const float* y, bool cull)
{
    const float l = a.scale[i];
    const float ll = __logf(l);
    const float x0 = a.pos[3 * i], x1 = a.pos[3 * i + 1], x2 = a.pos[3 * i + 2];
    for (int j = 0; j < kOff; ++j) {
        const size_t s = (size_t)i * kOff + j;
        const float* yj = y + kOff * j;
        const float* o = a.offsets + s * 3;
        a.out_pos[3 * s] = fmaf(l, o[0], x0);
        a.out_pos[3 * s + 1] = fmaf(l, o[1], x1);
        a.out_pos[3 * s + 2] = fmaf(l, o[2], x2);
        a.out_opacity[s] = cull ? kCulledLogit : yj[0];
        a.out_log_scale[2 * s] = yj[4] + ll;
        a.out_log_scale[2 * s + 1] = yj[5] + ll;
        reinterpret_cast<float4*>(a.out_quat)[s] = make_float4(yj[6], yj[7], yj[8], yj[9]);
        if (a.head == GSR_HEAD_LIDAR) {
            if (a.out_sh)
                for (int c = 0; c < 3; ++c) a.out_sh[3 * s + c] = 0.f;
            if (a.out_intensity) a.out_intensity[s] = sigmoidf_(yj[1]);
            if (a.out_ray_drop) a.out_ray_drop[s] = yj[2];
        } else {
            for (int c = 0; c < 3; ++c) a.out_sh[3 * s + c] = (sigmoidf_(yj[1 + c]) - 0.5f) * (1.f / kY00);
            if (a.out_intensity) a.out_intensity[s] = a.intensity ? a.intensity[s] : 0.f;
        }
    }
}

__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, uint32_t* status)
{
    for (uint32_t it = 0; it < (1u << 24); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    if (status) atomicCAS(status, 0u, (uint32_t)GSR_ERR_TIMEOUT);
    return false;
}

__device__ __forceinline__ void store_bf16x8(unsigned char* dst, const float* v)
{
    __nv_bfloat162 p[4];
    for (int q = 0; q < 4; ++q) p[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<uint4*>(p);
}

}  // namespace

// ------------------------------------------------------------ tcgen05 decode
constexpr int kSmemW1 = kHid * kInPad * 2;      // B of layer 1: [64 n][48 k]
constexpr int kSmemW2 = kOutPad * kHid * 2;     // B of layer 2: [112 n][64 k]
constexpr int kSmemX = kTileA * kInPad * 2;     // A of layer 1: [128 m][48 k]
constexpr int kSmemH = kTileA * kHid * 2;       // A of layer 2: [128 m][64 k]
constexpr int kOffW1 = 0, kOffW2 = kOffW1 + kSmemW1, kOffX = kOffW2 + kSmemW2, kOffH = kOffX + kSmemX;
constexpr int kOffB1 = kOffH + kSmemH, kOffB2 = kOffB1 + kHid * 4, kOffBar = kOffB2 + kOutPad * 4;
constexpr int kDecodeSmem = kOffBar + 64;

// The surfels of tile `tile` (anchor i = tile * 128 + thread), staged array
// by array in `stg` (the free input and hidden buffers, 7168 floats) and
// written with consecutive threads on consecutive words; the same values as
// write_surfels.  Every branch is uniform over the CTA (each flush holds
// barriers).  The caller has made every tensor-core operation of the tile
// complete, so the buffers are free.
__device__ __forceinline__ void write_surfels_staged(const DecodeArgs& a, int tile, const float* y, bool valid,
                                                     bool cull, float* stg)
{
    const int tid = threadIdx.x;
    const int i = tile * kTileA + tid;
    const int ns = min(kTileA, a.n - tile * kTileA) * kOff;  // surfels of the tile
    const size_t s0 = (size_t)tile * kTileA * kOff;          // its first surfel
    auto flush = [&](float* dst, int width) {
        __syncthreads();
        const int cnt = ns * width;
        float* d = dst + s0 * width;
        for (int e = tid; e < cnt; e += kTileA) d[e] = stg[e];
        __syncthreads();
    };
    if (valid) {
        const float l = a.scale[i];
        const float x0 = a.pos[3 * i], x1 = a.pos[3 * i + 1], x2 = a.pos[3 * i + 2];
#pragma unroll
        for (int j = 0; j < kOff; ++j) {
            const float* o = a.offsets + ((size_t)i * kOff + j) * 3;
            float* p = stg + (tid * kOff + j) * 3;
            p[0] = fmaf(l, o[0], x0);
            p[1] = fmaf(l, o[1], x1);
            p[2] = fmaf(l, o[2], x2);
        }
    }
    flush(a.out_pos, 3);
    if (valid) {
#pragma unroll
        for (int j = 0; j < kOff; ++j) stg[tid * kOff + j] = cull ? kCulledLogit : y[kOff * j];
    }
    flush(a.out_opacity, 1);
    if (valid) {
        const float ll = __logf(a.scale[i]);
#pragma unroll
        for (int j = 0; j < kOff; ++j) {
            stg[(tid * kOff + j) * 2] = y[kOff * j + 4] + ll;
            stg[(tid * kOff + j) * 2 + 1] = y[kOff * j + 5] + ll;
        }
    }
    flush(a.out_log_scale, 2);
    if (valid) {
#pragma unroll
        for (int j = 0; j < kOff; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) stg[(tid * kOff + j) * 4 + q] = y[kOff * j + 6 + q];
    }
    flush(a.out_quat, 4);
    if (a.head == GSR_HEAD_LIDAR) {
        if (a.out_sh) {
            if (valid)
                for (int e = 0; e < 3 * kOff; ++e) stg[tid * kOff * 3 + e] = 0.f;
            flush(a.out_sh, 3);
        }
        if (a.out_intensity) {
            if (valid)
#pragma unroll
                for (int j = 0; j < kOff; ++j) stg[tid * kOff + j] = sigmoidf_(y[kOff * j + 1]);
            flush(a.out_intensity, 1);
        }
        if (a.out_ray_drop) {
            if (valid)
#pragma unroll
                for (int j = 0; j < kOff; ++j) stg[tid * kOff + j] = y[kOff * j + 2];
            flush(a.out_ray_drop, 1);
        }
    } else {
        if (valid) {
#pragma unroll
            for (int j = 0; j < kOff; ++j)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    stg[(tid * kOff + j) * 3 + c] = (sigmoidf_(y[kOff * j + 1 + c]) - 0.5f) * (1.f / kY00);
        }
        flush(a.out_sh, 3);
        if (a.out_intensity) {
            if (valid)
#pragma unroll
                for (int j = 0; j < kOff; ++j)
                    stg[tid * kOff + j] = a.intensity ? a.intensity[(size_t)i * kOff + j] : 0.f;
            flush(a.out_intensity, 1);
        }
    }
}

// Persistent CTAs: the weights are converted once per CTA and TMEM is
// allocated once; each CTA then takes tiles of 128 anchors in turn.  Per
// tile: the input rows (BF16, K-major canonical layout), layer 1 by one
// tcgen05.mma chain into TMEM, bias + ReLU to the BF16 hidden rows, layer 2
// into the same TMEM columns, and the tile's surfels staged array by array
// in the (then free) input and hidden buffers and written with coalesced
// stores.  Each tile commits twice, so its two waits take parities 0 and 1.
__global__ void __launch_bounds__(kTileA) k_decode_tc(DecodeArgs a)
{
    extern __shared__ __align__(128) unsigned char sm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kOffBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kOffBar + 8);
    float* sb1 = reinterpret_cast<float*>(sm + kOffB1);
    float* sb2 = reinterpret_cast<float*>(sm + kOffB2);
    float* stg = reinterpret_cast<float*>(sm + kOffX);  // output staging: the X and H buffers
    const int tid = threadIdx.x, warp = tid >> 5;
    const int ntiles = (a.n + kTileA - 1) / kTileA;

    // weights -> BF16 in the K-major canonical layout (B operands), biases
    for (int e = tid; e < kHid * kInPad; e += kTileA) {
        const int n = e / kInPad, k = e % kInPad;
        const float v = k < kIn ? a.w1[k * kHid + n] : 0.f;
        *reinterpret_cast<__nv_bfloat16*>(sm + kOffW1 + tc::canon_offset(n, k, kInPad)) = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < kOutPad * kHid; e += kTileA) {
        const int n = e / kHid, k = e % kHid;
        const float v = n < kOut ? a.w2[k * kOut + n] : 0.f;
        *reinterpret_cast<__nv_bfloat16*>(sm + kOffW2 + tc::canon_offset(n, k, kHid)) = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < kHid; e += kTileA) sb1[e] = a.b1[e];
    for (int e = tid; e < kOutPad; e += kTileA) sb2[e] = e < kOut ? a.b2[e] : 0.f;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 128);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // input row of this thread's anchor
        const int i = tile * kTileA + tid;
        const bool valid = i < a.n;
        float X[kInPad];
#pragma unroll
        for (int k = 0; k < kInPad; ++k) X[k] = 0.f;
        bool cull = false;
        if (valid) {
            input_row(a, i, X);
            cull = culled(a, i);
        }
        // the previous tile's staged outputs are written (the loop's last barrier)
#pragma unroll
        for (int c = 0; c < kInPad / 8; ++c)
            store_bf16x8(sm + kOffX + tc::canon_offset(tid, 8 * c, kInPad), X + 8 * c);
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();

        // layer 1: D[128 x 64] = X[128 x 48] W1t[48 x 64]
        if (tid == 0) {
            constexpr uint32_t id1 = tc::idesc_bf16_f32(kTileA, kHid);
            const uint32_t xa = smem_u32(sm + kOffX), wa = smem_u32(sm + kOffW1);
            for (int s = 0; s < kInPad / 16; ++s)
                tc::mma_bf16(tmem, tc::smem_desc(xa + 256 * s, 128, (kInPad / 8) * 128),
                             tc::smem_desc(wa + 256 * s, 128, (kInPad / 8) * 128), id1, s > 0);
            tc::commit(bar);
        }
        bool ok = wait_phase(bar, 0, a.status);
        tc::fence_after_sync();
        // epilogue 1: bias + ReLU -> BF16 hidden row (A operand of layer 2)
#pragma unroll
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float v[16];
            tc::ld16(trow + c0, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = fmaxf(v[q] + sb1[c0 + q], 0.f);
            store_bf16x8(sm + kOffH + tc::canon_offset(tid, c0, kHid), v);
            store_bf16x8(sm + kOffH + tc::canon_offset(tid, c0 + 8, kHid), v + 8);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        ok = __syncthreads_and(ok);
        tc::fence_after_sync();
        // layer 2: D[128 x 112] = H[128 x 64] W2t[64 x 112] (into the same columns)
        if (tid == 0 && ok) {
            constexpr uint32_t id2 = tc::idesc_bf16_f32(kTileA, kOutPad);
            const uint32_t ha = smem_u32(sm + kOffH), wb = smem_u32(sm + kOffW2);
            for (int s = 0; s < kHid / 16; ++s)
                tc::mma_bf16(tmem, tc::smem_desc(ha + 256 * s, 128, (kHid / 8) * 128),
                             tc::smem_desc(wb + 256 * s, 128, (kHid / 8) * 128), id2, s > 0);
            tc::commit(bar);
        }
        if (ok) ok = wait_phase(bar, 1, a.status);
        ok = __syncthreads_and(ok);  // block-uniform: tcgen05.ld below is warp-collective
        tc::fence_after_sync();
        if (!ok) break;  // no MMA of this CTA is outstanding past its wait
        float y[kOutPad];
#pragma unroll
        for (int c0 = 0; c0 < kOutPad; c0 += 16) tc::ld16(trow + c0, y + c0);
#pragma unroll
        for (int q = 0; q < kOut; ++q) y[q] += sb2[q];
        tc::fence_before_sync();
        write_surfels_staged(a, tile, y, valid, cull, stg);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

// ------------------------------------------------------------ FP32 decode
__global__ void __launch_bounds__(128) k_decode_f32(DecodeArgs a)
{
    __shared__ float w1[kIn * kHid];
    __shared__ float w2[kHid * kOut];
    __shared__ float b1[kHid], b2[kOut];
    for (int e = threadIdx.x; e < kIn * kHid; e += blockDim.x) w1[e] = a.w1[e];
    for (int e = threadIdx.x; e < kHid * kOut; e += blockDim.x) w2[e] = a.w2[e];
    for (int e = threadIdx.x; e < kHid; e += blockDim.x) b1[e] = a.b1[e];
    for (int e = threadIdx.x; e < kOut; e += blockDim.x) b2[e] = a.b2[e];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    float X[kIn];
    input_row(a, i, X);
    float H[kHid];
    for (int h = 0; h < kHid; ++h) {
        float s = b1[h];
        for (int k = 0; k < kIn; ++k) s = fmaf(X[k], w1[k * kHid + h], s);
        H[h] = fmaxf(s, 0.f);
    }
    float y[kOut];
    for (int o = 0; o < kOut; ++o) {
        float s = b2[o];
        for (int h = 0; h < kHid; ++h) s = fmaf(H[h], w2[h * kOut + o], s);
        y[o] = s;
    }
    write_surfels(a, i, y, culled(a, i));
}

// ------------------------------------------------------------ backward
struct DecodeGradArgs {
    DecodeArgs f;
    const float* g_opacity;    // [n*10]
    const float* g_sh;         // [n*10][1][3]
    const float* g_log_scale;  // [n*10][2]
    const float* g_quat;       // [n*10][4]
    const float* g_intensity;  // [n*10] or null (LiDAR head)
    const float* g_ray_drop;   // [n*10] or null (LiDAR head)
    float* g_w1;               // [36][64]   (accumulated)
    float* g_b1;               // [64]
    float* g_w2;               // [64][100]
    float* g_b2;               // [100]
    float* g_feature;          // [n][32] or null (accumulated)
};

constexpr int kBwdTile = 64;

// One thread per anchor recomputes X, H, Y in FP32 and forms dY, dH, dX;
// the CTA then reduces the weight gradients over its anchors in shared
// memory (deterministically, in anchor order) before one atomic per weight.
__global__ void __launch_bounds__(kBwdTile) k_decode_backward(DecodeGradArgs g)
{
    extern __shared__ float sb[];
    float* sX = sb;                        // [64][36]
    float* sH = sX + kBwdTile * kIn;       // [64][64]
    float* sdY = sH + kBwdTile * kHid;     // [64][100]
    float* sdP = sdY + kBwdTile * kOut;    // [64][64] d(pre-activation)
    const DecodeArgs& a = g.f;
    const int t = threadIdx.x;
    const int i = blockIdx.x * kBwdTile + t;
    const bool valid = i < a.n;
    float X[kIn], H[kHid], pre[kHid], dY[kOut];
    for (int k = 0; k < kIn; ++k) X[k] = 0.f;
    for (int h = 0; h < kHid; ++h) H[h] = pre[h] = 0.f;
    for (int o = 0; o < kOut; ++o) dY[o] = 0.f;
    if (valid) {
        input_row(a, i, X);
        for (int h = 0; h < kHid; ++h) {
            float s = a.b1[h];
            for (int k = 0; k < kIn; ++k) s = fmaf(X[k], a.w1[k * kHid + h], s);
            pre[h] = s;
            H[h] = fmaxf(s, 0.f);
        }
        const bool cull = culled(a, i);
        for (int j = 0; j < kOff; ++j) {
            const size_t s = (size_t)i * kOff + j;
            float y[4];
            for (int c = 0; c < 3; ++c) {
                float v = a.b2[kOff * j + 1 + c];
                for (int h = 0; h < kHid; ++h) v = fmaf(H[h], a.w2[h * kOut + kOff * j + 1 + c], v);
                y[c] = v;
            }
            float* d = dY + kOff * j;
            d[0] = cull ? 0.f : g.g_opacity[s];
            if (a.head == GSR_HEAD_LIDAR) {
                const float sg = sigmoidf_(y[0]);
                d[1] = g.g_intensity ? g.g_intensity[s] * sg * (1.f - sg) : 0.f;
                d[2] = g.g_ray_drop ? g.g_ray_drop[s] : 0.f;
                d[3] = 0.f;
            } else {
                for (int c = 0; c < 3; ++c) {
                    const float sg = sigmoidf_(y[c]);
                    d[1 + c] = g.g_sh[3 * s + c] * sg * (1.f - sg) * (1.f / kY00);
                }
            }
            d[4] = g.g_log_scale[2 * s];
            d[5] = g.g_log_scale[2 * s + 1];
            for (int q = 0; q < 4; ++q) d[6 + q] = g.g_quat[4 * s + q];
        }
    }
    // dH = W2 dY, dP = dH * relu'(pre), dX = W1 dP
    float dP[kHid];
    for (int h = 0; h < kHid; ++h) {
        float s = 0.f;
        for (int o = 0; o < kOut; ++o) s = fmaf(a.w2[h * kOut + o], dY[o], s);
        dP[h] = pre[h] > 0.f ? s : 0.f;
    }
    if (valid && g.g_feature) {
        for (int k = 0; k < kFeat; ++k) {
            float s = 0.f;
            for (int h = 0; h < kHid; ++h) s = fmaf(a.w1[k * kHid + h], dP[h], s);
            g.g_feature[(size_t)i * kFeat + k] += s;
        }
    }
    for (int k = 0; k < kIn; ++k) sX[t * kIn + k] = X[k];
    for (int h = 0; h < kHid; ++h) {
        sH[t * kHid + h] = H[h];
        sdP[t * kHid + h] = dP[h];
    }
    for (int o = 0; o < kOut; ++o) sdY[t * kOut + o] = dY[o];
    __syncthreads();
    // weight gradients summed over the CTA's anchors
    for (int e = t; e < kHid * kOut; e += kBwdTile) {
        const int h = e / kOut, o = e % kOut;
        float s = 0.f;
        for (int m = 0; m < kBwdTile; ++m) s = fmaf(sH[m * kHid + h], sdY[m * kOut + o], s);
        if (s != 0.f) atomicAdd(g.g_w2 + e, s);
    }
    for (int o = t; o < kOut; o += kBwdTile) {
        float s = 0.f;
        for (int m = 0; m < kBwdTile; ++m) s += sdY[m * kOut + o];
        if (s != 0.f) atomicAdd(g.g_b2 + o, s);
    }
    for (int e = t; e < kIn * kHid; e += kBwdTile) {
        const int k = e / kHid, h = e % kHid;
        float s = 0.f;
        for (int m = 0; m < kBwdTile; ++m) s = fmaf(sX[m * kIn + k], sdP[m * kHid + h], s);
        if (s != 0.f) atomicAdd(g.g_w1 + e, s);
    }
    for (int h = t; h < kHid; h += kBwdTile) {
        float s = 0.f;
        for (int m = 0; m < kBwdTile; ++m) s += sdP[m * kHid + h];
        if (s != 0.f) atomicAdd(g.g_b1 + h, s);
    }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// ------------------------------------------------------------ host side
static gsr_status fill_decode_args(const gsr_anchors* an, const gsr_mlp* mlp, const float* origin,
                                   const gsr_sensor* cam, const gsr_surfel_table* out, uint32_t* status,
                                   DecodeArgs& a)
{
    if (!an || !mlp || !origin) return GSR_ERR_INVALID_ARG;
    if (an->k != kOff || an->feat_dim != kFeat || mlp->hidden != kHid) return GSR_ERR_UNSUPPORTED;
    if (an->n < 0 || (an->n > 0 && (!an->pos || !an->feature || !an->scale || !an->offsets))) return GSR_ERR_INVALID_ARG;
    if (!mlp->w1 || !mlp->b1 || !mlp->w2 || !mlp->b2) return GSR_ERR_INVALID_ARG;
    if (mlp->head != GSR_HEAD_CAMERA && mlp->head != GSR_HEAD_LIDAR) return GSR_ERR_INVALID_ARG;
    a = DecodeArgs{};
    a.head = mlp->head;
    a.n = an->n;
    a.pos = an->pos;
    a.feature = an->feature;
    a.scale = an->scale;
    a.offsets = an->offsets;
    a.intensity = an->intensity;
    a.w1 = mlp->w1;
    a.b1 = mlp->b1;
    a.w2 = mlp->w2;
    a.b2 = mlp->b2;
    a.ox = origin[0];
    a.oy = origin[1];
    a.oz = origin[2];
    a.status = status;
    if (cam) {
        if (cam->kind != GSR_SENSOR_PINHOLE) return GSR_ERR_UNSUPPORTED;
        a.cull = 1;
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) a.R[3 * r + c] = cam->world_to_sensor[4 * r + c];
            a.t[r] = cam->world_to_sensor[4 * r + 3];
        }
        const double P[4][3] = {{cam->fx, 0.0, cam->cx},
                                {-cam->fx, 0.0, cam->width - cam->cx},
                                {0.0, cam->fy, cam->cy},
                                {0.0, -cam->fy, cam->height - cam->cy}};
        for (int k = 0; k < 4; ++k) {
            const double nn = std::sqrt(P[k][0] * P[k][0] + P[k][1] * P[k][1] + P[k][2] * P[k][2]);
            for (int c = 0; c < 3; ++c) a.plane[k][c] = (float)(P[k][c] / nn);
        }
        a.near_plane = cam->near_plane;
    }
    if (out) {
        if (an->n > 0 && (!out->pos || !out->log_scale || !out->quat || !out->opacity ||
                          (!out->sh && mlp->head == GSR_HEAD_CAMERA)))
            return GSR_ERR_INVALID_ARG;
        a.out_pos = out->pos;
        a.out_log_scale = out->log_scale;
        a.out_quat = out->quat;
        a.out_opacity = out->opacity;
        a.out_sh = out->sh;
        a.out_intensity = out->intensity;
        a.out_ray_drop = out->ray_drop;
    }
    return GSR_OK;
}

gsr_status cuda_status(cudaError_t e);

}  // namespace gsr

using namespace gsr;

// Persistent decode CTAs: resident CTAs per SM x SMs of the current device.
static int decode_grid(cudaError_t& err)
{
    static int cached[64] = {};
    int dev = 0;
    err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return 0;
    if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
    int sms = 0, per_sm = 0;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_decode_tc, kTileA, kDecodeSmem);
    if (err != cudaSuccess) return 0;
    const int g = sms * (per_sm > 0 ? per_sm : 1);
    if (dev >= 0 && dev < 64) cached[dev] = g;
    return g;
}

extern "C" gsr_status gsr_decode_anchors(const gsr_anchors* anchors, const gsr_mlp* mlp, const float* origin,
                                         const gsr_sensor* cull_camera, int32_t precision,
                                         const gsr_surfel_table* out, uint32_t* device_status, void* stream)
{
    DecodeArgs a;
    gsr_status st = fill_decode_args(anchors, mlp, origin, cull_camera, out, device_status, a);
    if (st != GSR_OK) return st;
    if (!out) return GSR_ERR_INVALID_ARG;
    if (a.n == 0) return GSR_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (precision == GSR_DECODE_BF16_TENSOR) {
        cudaError_t e = cudaFuncSetAttribute(k_decode_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kDecodeSmem);
        if (e != cudaSuccess) return cuda_status(e);
        const int tiles = (a.n + kTileA - 1) / kTileA;
        int grid = decode_grid(e);
        if (e != cudaSuccess) return cuda_status(e);
        k_decode_tc<<<grid < tiles ? grid : tiles, kTileA, kDecodeSmem, s>>>(a);
    } else if (precision == GSR_DECODE_F32) {
        k_decode_f32<<<(a.n + 127) / 128, 128, 0, s>>>(a);
    } else {
        return GSR_ERR_INVALID_ARG;
    }
    return cuda_status(cudaGetLastError());
}

extern "C" gsr_status gsr_decode_backward(const gsr_anchors* anchors, const gsr_mlp* mlp, const float* origin,
                                          const gsr_sensor* cull_camera, const gsr_surfel_grads* d_surfels,
                                          const gsr_mlp_grads* out, void* stream)
{
    DecodeGradArgs g;
    gsr_status st = fill_decode_args(anchors, mlp, origin, cull_camera, nullptr, nullptr, g.f);
    if (st != GSR_OK) return st;
    if (!d_surfels || !out) return GSR_ERR_INVALID_ARG;
    if (!d_surfels->opacity || !d_surfels->log_scale || !d_surfels->quat) return GSR_ERR_INVALID_ARG;
    if (!d_surfels->sh && mlp->head == GSR_HEAD_CAMERA) return GSR_ERR_INVALID_ARG;
    if (!out->w1 || !out->b1 || !out->w2 || !out->b2) return GSR_ERR_INVALID_ARG;
    g.g_opacity = d_surfels->opacity;
    g.g_sh = d_surfels->sh;
    g.g_log_scale = d_surfels->log_scale;
    g.g_quat = d_surfels->quat;
    g.g_intensity = d_surfels->intensity;
    g.g_ray_drop = d_surfels->ray_drop;
    g.g_w1 = out->w1;
    g.g_b1 = out->b1;
    g.g_w2 = out->w2;
    g.g_b2 = out->b2;
    g.g_feature = out->feature;
    if (g.f.n == 0) return GSR_OK;
    const size_t smem = (size_t)kBwdTile * (kIn + kHid + kOut + kHid) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_decode_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_status(e);
    k_decode_backward<<<(g.f.n + kBwdTile - 1) / kBwdTile, kBwdTile, smem, reinterpret_cast<cudaStream_t>(stream)>>>(g);
    return cuda_status(cudaGetLastError());
}

extern "C" gsr_status gsr_adam(float* param, const float* grad, float* m, float* v, int64_t n, float lr, float beta1,
                               float beta2, float eps, int32_t step, void* stream)
{
    if (n < 0 || step < 1 || (n > 0 && (!param || !grad || !m || !v))) return GSR_ERR_INVALID_ARG;
    if (n == 0) return GSR_OK;
    const float c1 = 1.f / (1.f - powf(beta1, (float)step));
    const float c2 = 1.f / (1.f - powf(beta2, (float)step));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_adam<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(param, grad, m, v, n, lr, beta1, beta2, eps, c1, c2);
    return cuda_status(cudaGetLastError());
}
