// preprocess.cu -- per-(sensor, surfel) projection, culling and bounding.
//
// Implements the surfel side of Eqs. 1-3 and 5 (arXiv 2503.11731 Sec. III-A)
// for every (sensor, surfel) slot: the world -> sensor transform of
// H = [s_u t_u, s_v t_v, mu] (Eq. 1), the closed-form solution operator of
// Eq. 2 (the adjugate Q of the ray-space matrix, see gsr_internal.cuh), the
// 3-sigma screen bound of the surfel united with the low-pass disc of the
// 2DGS fallback, the tile rectangle and count, the SH colour and the normal.
// One thread per slot; the sensors of a surfel block are adjacent in the
// grid.  HBM-bound: 40 B of geometry per surfel and sensor, + the SH
// coefficients of visible camera slots.
#include "gsr_internal.cuh"

namespace gsr {

namespace {

struct F3 {
    float x, y, z;
};
__device__ __forceinline__ F3 f3(float x, float y, float z) { return F3{x, y, z}; }
__device__ __forceinline__ F3 operator+(F3 a, F3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ F3 operator*(float s, F3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(F3 a, F3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ F3 mat3(const float* M, F3 v)
{
    return f3(fmaf(M[0], v.x, fmaf(M[1], v.y, M[2] * v.z)), fmaf(M[3], v.x, fmaf(M[4], v.y, M[5] * v.z)),
              fmaf(M[6], v.x, fmaf(M[7], v.y, M[8] * v.z)));
}
__device__ __forceinline__ F3 mat3T(const float* M, F3 v)
{
    return f3(fmaf(M[0], v.x, fmaf(M[3], v.y, M[6] * v.z)), fmaf(M[1], v.x, fmaf(M[4], v.y, M[7] * v.z)),
              fmaf(M[2], v.x, fmaf(M[5], v.y, M[8] * v.z)));
}

// Columns t_u, t_v, n of the rotation of quaternion (w, x, y, z) (normalised here).
__device__ __forceinline__ void quat_frame(float4 q, F3& tu, F3& tv, F3& n)
{
    float inv = rsqrtf(fmaf(q.x, q.x, fmaf(q.y, q.y, fmaf(q.z, q.z, q.w * q.w))));
    float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
    tu = f3(1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y));
    tv = f3(2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x));
    n = f3(2.f * (x * z + w * y), 2.f * (y * z - w * x), 1.f - 2.f * (x * x + y * y));
}

// Real spherical harmonics to degree 3 (Condon-Shortley phase) at unit d,
// accumulated against coefficients c[K][3]; returns max(0, sum + 0.5).
__device__ __forceinline__ F3 sh_colour(int deg, const float* __restrict__ c, F3 d)
{
    const float x = d.x, y = d.y, z = d.z;
    float b[16];
    b[0] = 0.28209479177387814f;
    int K = 1;
    if (deg >= 1) {
        b[1] = -0.4886025119029199f * y;
        b[2] = 0.4886025119029199f * z;
        b[3] = -0.4886025119029199f * x;
        K = 4;
    }
    if (deg >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        b[4] = 1.0925484305920792f * x * y;
        b[5] = -1.0925484305920792f * y * z;
        b[6] = 0.31539156525252005f * (2.f * zz - xx - yy);
        b[7] = -1.0925484305920792f * x * z;
        b[8] = 0.5462742152960396f * (xx - yy);
        K = 9;
        if (deg >= 3) {
            b[9] = -0.5900435899266435f * y * (3.f * xx - yy);
            b[10] = 2.890611442640554f * x * y * z;
            b[11] = -0.4570457994644658f * y * (4.f * zz - xx - yy);
            b[12] = 0.3731763325901154f * z * (2.f * zz - 3.f * xx - 3.f * yy);
            b[13] = -0.4570457994644658f * x * (4.f * zz - xx - yy);
            b[14] = 1.445305721320277f * z * (xx - yy);
            b[15] = -0.5900435899266435f * x * (xx - 3.f * yy);
            K = 16;
        }
    }
    float r = 0.5f, g = 0.5f, bl = 0.5f;
    if (K == 16) {
        // 48 coefficients = 12 aligned float4 loads
        const float4* c4 = reinterpret_cast<const float4*>(c);
        float cf[48];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float4 v = __ldg(c4 + k);
            cf[4 * k] = v.x; cf[4 * k + 1] = v.y; cf[4 * k + 2] = v.z; cf[4 * k + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            r = fmaf(b[k], cf[3 * k], r);
            g = fmaf(b[k], cf[3 * k + 1], g);
            bl = fmaf(b[k], cf[3 * k + 2], bl);
        }
    } else {
        for (int k = 0; k < K; ++k) {
            r = fmaf(b[k], __ldg(c + 3 * k), r);
            g = fmaf(b[k], __ldg(c + 3 * k + 1), g);
            bl = fmaf(b[k], __ldg(c + 3 * k + 2), bl);
        }
    }
    return f3(fmaxf(r, 0.f), fmaxf(g, 0.f), fmaxf(bl, 0.f));
}

__device__ __forceinline__ void project(const SensorDev& s, F3 p, float& x, float& y, float& xmin, float& xmax,
                                        float& ymin, float& ymax)
{
    float iz = 1.f / p.z;
    x = fmaf(s.fx, p.x * iz, s.cx);
    y = fmaf(s.fy, p.y * iz, s.cy);
    xmin = fminf(xmin, x); xmax = fmaxf(xmax, x);
    ymin = fminf(ymin, y); ymax = fmaxf(ymax, y);
}

// Distance from the origin to the 2D segment p -> q.
__device__ __forceinline__ float seg_dist(float px, float py, float qx, float qy)
{
    const float ex = qx - px, ey = qy - py;
    const float ee = fmaf(ex, ex, ey * ey);
    float t = ee > 0.f ? -(px * ex + py * ey) / ee : 0.f;
    t = fminf(fmaxf(t, 0.f), 1.f);
    const float dx = fmaf(t, ex, px), dy = fmaf(t, ey, py);
    return sqrtf(fmaf(dx, dx, dy * dy));
}

// Pixel/cell index range [i0, i1] whose centres (index + off) can fall in [lo, hi].
__device__ __forceinline__ void index_range(float lo, float hi, float off, int n, int& i0, int& i1)
{
    lo = fmaxf(lo - off, -2.f);
    hi = fminf(hi - off, (float)n + 1.f);
    i0 = max(0, (int)ceilf(lo));
    i1 = min(n - 1, (int)floorf(hi));
}

}  // namespace

// Surfel i of the table S is surfel `first + i` of the plan (n_plan surfels),
// so several tables (e.g. a decoded background and posed objects) can share
// one plan.  Composite ties break by plan index, as in a single table.  One
// instantiation per sensor model keeps each one's registers to its own
// bound; the grid walks the plan's sensors of that model (ids) fastest.
// Resident 256-thread CTAs per SM the preprocess is compiled for: 4 caps it
// at 64 registers (a few bytes of spills), which measured faster on the rig
// frame than 3 (80 registers) or 2 (96): more resident warps hide its
// latencies better than the spared registers would.
#ifndef GSR_PRE_MIN_CTAS
#define GSR_PRE_MIN_CTAS 4
#endif
template <int KIND>
__global__ void __launch_bounds__(256, GSR_PRE_MIN_CTAS) k_preprocess(SensorTable tab, SensorIds ids, gsr_surfels S,
                                                    const float* __restrict__ poses, int n_obj,
                                                    float4* __restrict__ rec, ushort4* __restrict__ rects,
                                                    uint32_t* __restrict__ counts, uint32_t* __restrict__ keys,
                                                    uint4* __restrict__ spans, int first, int n_plan)
{
    // the sensors of a surfel block run back to back (sensor fastest), so
    // the block's surfel data is read from DRAM once and from L2 after
    const int i = (int)(blockIdx.x / (unsigned)ids.n) * blockDim.x + threadIdx.x;
    const int si = ids.id[blockIdx.x % (unsigned)ids.n];
    if (i >= S.n) return;
    const SensorDev& sd = tab.s[si];
    const size_t slot = (size_t)si * n_plan + first + i;

    // ---- surfel in world (optional rigid object pose)
    F3 mu = f3(__ldg(S.pos + 3 * i), __ldg(S.pos + 3 * i + 1), __ldg(S.pos + 3 * i + 2));
    float4 q = __ldg(reinterpret_cast<const float4*>(S.quat) + i);
    float2 ls = __ldg(reinterpret_cast<const float2*>(S.log_scale) + i);
    F3 tu, tv, nw;
    quat_frame(q, tu, tv, nw);
    const float* Ro = nullptr;
    if (S.obj_id != nullptr) {
        int k = __ldg(S.obj_id + i);
        if (k >= 0 && k < n_obj) {
            Ro = poses + 12 * k;
            float Rm[9] = {__ldg(Ro), __ldg(Ro + 1), __ldg(Ro + 2), __ldg(Ro + 4), __ldg(Ro + 5),
                           __ldg(Ro + 6), __ldg(Ro + 8), __ldg(Ro + 9), __ldg(Ro + 10)};
            mu = mat3(Rm, mu) + f3(__ldg(Ro + 3), __ldg(Ro + 7), __ldg(Ro + 11));
            tu = mat3(Rm, tu);
            tv = mat3(Rm, tv);
            nw = mat3(Rm, nw);
        }
    }
    const float su = __expf(ls.x), sv = __expf(ls.y);
    const F3 ms = mat3(sd.R, mu) + f3(sd.t[0], sd.t[1], sd.t[2]);
    const F3 a = su * mat3(sd.R, tu);
    const F3 b = sv * mat3(sd.R, tv);

    uint32_t cnt = 0;
    ushort4 rect = make_ushort4(0, 0, 0, 0);
    float zkey;
    float4 r0, r1, r2;
    float4 r5 = make_float4(0.f, -1.f, 0.f, -1.f);  // ray-index bounding box of the support
    const int TW = sd.tile_w, TH = sd.tile_h;

    // Opacity-aware support: alpha = min(0.99, o G) reaches 1/255 only where
    // G >= 1/(255 o), i.e. rho <= 2 ln(255 o); a surfel with o < 1/255 never
    // contributes.  rho_cut (with a margin for FP32 rounding) bounds both the
    // ray-splat support (radius sqrt(rho_cut) sigma) and the low-pass disc
    // (radius sqrt(rho_cut / 2) px or cells).
    const float o = 1.f / (1.f + __expf(-__ldg(S.opacity + i)));
    const float rho_cut = fminf(kSupport, 2.f * __logf(255.f * o) + 1e-3f);
    const float ksig = sqrtf(fmaxf(rho_cut, 0.f));
    const float rlp = sqrtf(fmaxf(0.5f * rho_cut, 0.f));
    const bool never = !(rho_cut > 0.f);

    if (KIND == GSR_SENSOR_PINHOLE) {
        zkey = ms.z;
        if (!(ms.z > sd.near_plane) || never) {
            counts[slot] = 0;
            keys[slot] = __float_as_uint(fmaxf(zkey, 0.f));
            rects[slot] = rect;
            return;
        }
        const float iz = 1.f / ms.z;
        const float ex = ms.x * iz, ey = ms.y * iz;
        const float ccx = fmaf(sd.fx, ex, sd.cx), ccy = fmaf(sd.fy, ey, sd.cy);
        // ray-space matrix about the projected centre (rows: x - c_x z, y - c_y z, z in pixels)
        const float m00 = sd.fx * fmaf(-ex, a.z, a.x), m01 = sd.fx * fmaf(-ex, b.z, b.x);
        const float m10 = sd.fy * fmaf(-ey, a.z, a.y), m11 = sd.fy * fmaf(-ey, b.z, b.y);
        const float m20 = a.z, m21 = b.z;
        const float det = fmaf(m00, m11, -m01 * m10);
        // adjugate / z_c (the third column of M is (0, 0, z_c))
        r0 = make_float4(m11, -m01, 0.f, ccx);
        r1 = make_float4(-m10, m00, 0.f, ccy);
        r2 = make_float4(fmaf(m10, m21, -m11 * m20) * iz, fmaf(m01, m20, -m00 * m21) * iz, det * iz, det);

        // support bound: the square mu +- k a +- k b clipped to z >= near, projected
        float xmin = ccx - rlp, xmax = ccx + rlp;
        float ymin = ccy - rlp, ymax = ccy + rlp;
        const F3 ka = ksig * a, kb = ksig * b;
        F3 P[4] = {ms + ka + kb, ms + ka - kb, ms - ka - kb, ms - ka + kb};
        const float zn = sd.near_plane;
        float px, py;
        bool front = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const F3 A = P[k], B = P[(k + 1) & 3];
            const bool ia = A.z >= zn, ib = B.z >= zn;
            front = front && ia;
            if (ia) project(sd, A, px, py, xmin, xmax, ymin, ymax);
            if (ia != ib) {
                const float t = (zn - A.z) / (B.z - A.z);
                F3 C = A + t * (B - A);
                C.z = zn;
                project(sd, C, px, py, xmin, xmax, ymin, ymax);
            }
        }
        // one pixel of margin for FP32 rounding
        int x0, x1, y0, y1;
        index_range(xmin - 1.f, xmax + 1.f, 0.5f, sd.width, x0, x1);
        index_range(ymin - 1.f, ymax + 1.f, 0.5f, sd.height, y0, y1);
        if (x0 <= x1 && y0 <= y1) {
            r5 = make_float4((float)x0, (float)x1, (float)y0, (float)y1);
            rect = make_ushort4(x0 / TW, x1 / TW, y0 / TH, y1 / TH);
            cnt = (uint32_t)(rect.y - rect.x + 1) * (uint32_t)(rect.w - rect.z + 1);
            if (front && cnt > 1) {
                // support disc entirely in front: keep only the tiles its
                // footprint (or the low-pass disc) reaches
                const Footprint fp = make_footprint(r0, r1, r2, o);
                const bool cache = rect.w - rect.z < kSpanRows && rect.y - rect.x < 255;
                // the span table as two 64-bit words (byte b at bits 8 (b % 8))
                unsigned long long lo = cache ? (unsigned long long)(rect.w - rect.z + 1) : 0ull, hi = 0ull;
                uint32_t c = 0;
                for (int ty = rect.z; ty <= rect.w; ++ty) {
                    int t0, t1;
                    if (footprint_span(fp, ty, TW, TH, rect.x, rect.y, t0, t1)) {
                        c += (uint32_t)(t1 - t0 + 1);
                        if (cache) {
                            const int b = 1 + 2 * (ty - rect.z);
                            const unsigned long long v =
                                (unsigned long long)(t0 - rect.x) | ((unsigned long long)(t1 - t0 + 1) << 8);
                            if (b < 7) lo |= v << (8 * b);
                            else if (b == 7) { lo |= (v & 0xffull) << 56; hi |= v >> 8; }
                            else hi |= v << (8 * (b - 8));
                        }
                    }
                }
                spans[slot] = make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
                cnt = c;
                rect.w |= kRectExact;
            }
        }
    } else if (KIND == GSR_SENSOR_CYLINDRICAL) {
        // Eq. 4: pixel (x, y) looks along (sin phi, y_n, cos phi) with
        // phi = (x + 1/2 - c_x) / f_x and y_n = (y + 1/2 - c_y) / f_y; depth
        // and order key are the horizontal distance sqrt(x^2 + z^2)
        const float rh = sqrtf(fmaf(ms.x, ms.x, ms.z * ms.z));
        zkey = rh;
        if (!(rh > sd.near_plane) || never) {
            counts[slot] = 0;
            keys[slot] = __float_as_uint(fmaxf(zkey, 0.f));
            rects[slot] = rect;
            return;
        }
        // M = [a b ms] (columns), Q = adj(M), det(M): q = Q d gives
        // (u, v) = (q0, q1) / q2 and the distance det / q2 along d
        const float m00 = a.x, m01 = b.x, m02 = ms.x;
        const float m10 = a.y, m11 = b.y, m12 = ms.y;
        const float m20 = a.z, m21 = b.z, m22 = ms.z;
        const float q00 = fmaf(m11, m22, -m12 * m21), q01 = fmaf(m02, m21, -m01 * m22), q02 = fmaf(m01, m12, -m02 * m11);
        const float q10 = fmaf(m12, m20, -m10 * m22), q11 = fmaf(m00, m22, -m02 * m20), q12 = fmaf(m02, m10, -m00 * m12);
        const float q20 = fmaf(m10, m21, -m11 * m20), q21 = fmaf(m01, m20, -m00 * m21), q22 = fmaf(m00, m11, -m01 * m10);
        const float det = fmaf(m00, q00, fmaf(m01, q10, m02 * q20));
        // low-pass centre in pixels
        const float phc = atan2f(ms.x, ms.z);
        const float ccx = fmaf(sd.fx, phc, sd.cx), ccy = fmaf(sd.fy, ms.y / rh, sd.cy);
        r0 = make_float4(q00, q01, q02, ccx);
        r1 = make_float4(q10, q11, q12, ccy);
        r2 = make_float4(q20, q21, q22, det);

        // Bound of the support ellipse, inside the circumscribed octagon (as
        // for the LiDAR), united with the low-pass disc.  When every vertex's
        // horizontal position lies in the open half-plane facing the centre's
        // azimuth, the octagon's xz-projection misses the y axis: the azimuth
        // phi = atan2(x, z) takes its extremes at vertices, where the offset
        // from the centre's azimuth is atan(cross / dot) with dot > 0; and
        // y_n = y / sqrt(x^2 + z^2), whose gradient is orthogonal to the
        // position, has no interior extremum on a plane that misses the camera
        // centre, so per-edge bounds (max y over the edge's least horizontal
        // distance, ...) cover it.  Otherwise every column is taken, and when
        // all vertices lie on one side of the camera's horizontal plane y_n
        // keeps that sign with |y_n| >= min |y| / (largest horizontal distance,
        // reached at a vertex).  A plane through (nearly) the camera centre
        // takes the elevation range of the bounding sphere.  Azimuth ranges
        // that leave [-pi, pi] take every column.
        const float kk = ksig * 1.0823922f;
        const float rad = kk * fmaxf(su, sv);
        const float r3d = sqrtf(dot(ms, ms));
        F3 nrm = f3(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x));
        const float plane_off = fabsf(dot(nrm, ms)) * rsqrtf(fmaxf(dot(nrm, nrm), 1e-30f));
        float ph_lo = -4.f, ph_hi = 4.f;        // azimuth (full columns outside [-pi, pi])
        float yn_lo = -1e30f, yn_hi = 1e30f;    // y_n (full rows when unbounded)
        if (plane_off > 1e-3f * r3d) {
            const float cs[8] = {0.92387953f, 0.38268343f, -0.38268343f, -0.92387953f,
                                 -0.92387953f, -0.38268343f, 0.38268343f, 0.92387953f};
            const float sn[8] = {0.38268343f, 0.92387953f, 0.92387953f, 0.38268343f,
                                 -0.38268343f, -0.92387953f, -0.92387953f, -0.38268343f};
            const float ux = ms.x / rh, uz = ms.z / rh;
            F3 V[8];
            float rv[8];
            float t_lo = 0.f, t_hi = 0.f, dmin = 1e30f, vy_lo = 1e30f, vy_hi = -1e30f, r_far = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                V[j] = ms + kk * (cs[j] * a + sn[j] * b);
                rv[j] = sqrtf(fmaf(V[j].x, V[j].x, V[j].z * V[j].z));
                const float cr = fmaf(uz, V[j].x, -ux * V[j].z), dt = fmaf(ux, V[j].x, uz * V[j].z);
                dmin = fminf(dmin, dt);
                const float t = cr / dt;
                t_lo = fminf(t_lo, t);
                t_hi = fmaxf(t_hi, t);
                vy_lo = fminf(vy_lo, V[j].y);
                vy_hi = fmaxf(vy_hi, V[j].y);
                r_far = fmaxf(r_far, rv[j]);
            }
            if (dmin > 1e-6f * rh) {
                ph_lo = phc + atanf(t_lo);
                ph_hi = phc + atanf(t_hi);
                float s_lo = 1e30f, s_hi = -1e30f;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const F3 P0 = V[j], P1 = V[(j + 1) & 7];
                    const float rmin = seg_dist(P0.x, P0.z, P1.x, P1.z);
                    const float rmax = fmaxf(rv[j], rv[(j + 1) & 7]);
                    const float ymax = fmaxf(P0.y, P1.y), ymin = fminf(P0.y, P1.y);
                    s_hi = fmaxf(s_hi, ymax / (ymax >= 0.f ? rmin : rmax));
                    s_lo = fminf(s_lo, ymin / (ymin <= 0.f ? rmin : rmax));
                }
                yn_lo = s_lo;
                yn_hi = s_hi;
            } else {
                if (vy_lo > 0.f) yn_lo = vy_lo / r_far;
                if (vy_hi < 0.f) yn_hi = vy_hi / r_far;
            }
        } else if (r3d > rad * 1.0001f + 1e-6f) {
            const float beta = asinf(fminf(rad / r3d, 1.f));
            const float el = atan2f(ms.y, rh);
            if (el + beta < 1.5f) yn_hi = tanf(el + beta);
            if (el - beta > -1.5f) yn_lo = tanf(el - beta);
            if (rh > rad * 1.0001f + 1e-6f) {
                const float gam = asinf(fminf(rad / rh, 1.f));
                ph_lo = phc - gam;
                ph_hi = phc + gam;
            }
        }
        float xmin = ccx - rlp, xmax = ccx + rlp;
        float ymin = ccy - rlp, ymax = ccy + rlp;
        if (ph_lo >= -3.14159265f && ph_hi <= 3.14159265f) {
            xmin = fminf(xmin, fmaf(sd.fx, ph_lo, sd.cx));
            xmax = fmaxf(xmax, fmaf(sd.fx, ph_hi, sd.cx));
        } else {
            xmin = -2.f;
            xmax = (float)sd.width + 2.f;
        }
        ymin = yn_lo > -1e29f ? fminf(ymin, fmaf(sd.fy, yn_lo, sd.cy)) : -2.f;
        ymax = yn_hi < 1e29f ? fmaxf(ymax, fmaf(sd.fy, yn_hi, sd.cy)) : (float)sd.height + 2.f;
        // one pixel of margin for FP32 rounding
        int x0, x1, y0, y1;
        index_range(xmin - 1.f, xmax + 1.f, 0.5f, sd.width, x0, x1);
        index_range(ymin - 1.f, ymax + 1.f, 0.5f, sd.height, y0, y1);
        if (x0 <= x1 && y0 <= y1) {
            r5 = make_float4((float)x0, (float)x1, (float)y0, (float)y1);
            rect = make_ushort4(x0 / TW, x1 / TW, y0 / TH, y1 / TH);
            cnt = (uint32_t)(rect.y - rect.x + 1) * (uint32_t)(rect.w - rect.z + 1);
        }
    } else {
        const float rc = sqrtf(dot(ms, ms));
        zkey = rc;
        if (!(rc > sd.near_plane) || never) {
            counts[slot] = 0;
            keys[slot] = __float_as_uint(fmaxf(zkey, 0.f));
            rects[slot] = rect;
            return;
        }
        // M = [a b ms] (columns), Q = adj(M), det(M)
        const float m00 = a.x, m01 = b.x, m02 = ms.x;
        const float m10 = a.y, m11 = b.y, m12 = ms.y;
        const float m20 = a.z, m21 = b.z, m22 = ms.z;
        const float q00 = fmaf(m11, m22, -m12 * m21), q01 = fmaf(m02, m21, -m01 * m22), q02 = fmaf(m01, m12, -m02 * m11);
        const float q10 = fmaf(m12, m20, -m10 * m22), q11 = fmaf(m00, m22, -m02 * m20), q12 = fmaf(m02, m10, -m00 * m12);
        const float q20 = fmaf(m10, m21, -m11 * m20), q21 = fmaf(m01, m20, -m00 * m21), q22 = fmaf(m00, m11, -m01 * m10);
        const float det = fmaf(m00, q00, fmaf(m01, q10, m02 * q20));
        // low-pass centre in cell coordinates (ray (i, j) sits at (j, i))
        const float rxy = sqrtf(fmaf(ms.x, ms.x, ms.y * ms.y));
        const float az = atan2f(ms.y, ms.x);
        const float el = atan2f(ms.z, rxy);
        float daz = az - sd.az0;
        daz -= 6.283185307179586f * floorf(daz * 0.15915494309189535f);
        const float ccol = daz * sd.inv_d_az - 0.5f;
        const float crow = (sd.el_max - el) * sd.inv_d_el;
        r0 = make_float4(q00, q01, q02, ccol);
        r1 = make_float4(q10, q11, q12, crow);
        r2 = make_float4(q20, q21, q22, det);

        // Angular bound of the support ellipse, united with the low-pass disc.
        // The ellipse {mu + k(c a + s b)} lies inside the circumscribed octagon
        // with vertices mu + (k / cos 22.5deg)(cos t_j a + sin t_j b),
        // t_j = 22.5 + 45 j deg.  For a convex planar polygon whose plane misses
        // the sensor and whose xy-projection misses the z axis, azimuth is
        // monotonic along each edge (extremes at vertices) and elevation has no
        // interior extremum (its gradient is orthogonal to the position, so it
        // cannot be parallel to a plane normal n with n.x != 0), so per-edge
        // bounds on atan(z / rho) cover it: max z over min rho (z >= 0) or over
        // max rho (z < 0), and symmetrically for the minimum.  Other cases fall
        // back to the bounding sphere of the octagon.
        const float kk = ksig * 1.0823922f;
        const float rad = kk * fmaxf(su, sv);
        int i0, i1, tx0, tx1;
        const int A = sd.width;
        const int tiles_x = sd.tiles_x;
        const bool full_rows = !(rc > rad * 1.0001f + 1e-6f);
        const bool full_cols = full_rows || !(rxy > rad * 1.0001f + 1e-6f);
        F3 nrm = f3(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x));
        const float plane_off = fabsf(dot(nrm, ms)) * rsqrtf(fmaxf(dot(nrm, nrm), 1e-30f));
        const bool octagon = !full_cols && plane_off > 1e-3f * rc;
        float el_lo = el, el_hi = el, az_lo = 0.f, az_hi = 0.f;
        if (octagon) {
            const float cs[8] = {0.92387953f, 0.38268343f, -0.38268343f, -0.92387953f,
                                 -0.92387953f, -0.38268343f, 0.38268343f, 0.92387953f};
            const float sn[8] = {0.38268343f, 0.92387953f, 0.92387953f, 0.38268343f,
                                 -0.38268343f, -0.92387953f, -0.92387953f, -0.38268343f};
            // Every vertex lies within rad of the centre while rxy > rad, so
            // its xy direction is within 90 deg of the centre's: its azimuth
            // offset atan2(cross, dot) is increasing in cross / dot (dot > 0),
            // and elevations atan2(z, r) (r > 0) are increasing in z / r, so
            // the extremes take four arctangents of extreme ratios.
            const float ux = ms.x / rxy, uy = ms.y / rxy;
            F3 V[8];
            float rv[8];
            float t_lo = 0.f, t_hi = 0.f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                V[j] = ms + kk * (cs[j] * a + sn[j] * b);
                rv[j] = sqrtf(fmaf(V[j].x, V[j].x, V[j].y * V[j].y));
                const float cr = fmaf(ux, V[j].y, -uy * V[j].x), dt = fmaf(ux, V[j].x, uy * V[j].y);
                const float t = cr / dt;
                t_lo = fminf(t_lo, t);
                t_hi = fmaxf(t_hi, t);
            }
            az_lo = atanf(t_lo);
            az_hi = atanf(t_hi);
            float s_lo = 1e30f, s_hi = -1e30f;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const F3 P0 = V[j], P1 = V[(j + 1) & 7];
                const float rmin = seg_dist(P0.x, P0.y, P1.x, P1.y);
                const float rmax = fmaxf(rv[j], rv[(j + 1) & 7]);
                const float zmax = fmaxf(P0.z, P1.z), zmin = fminf(P0.z, P1.z);
                s_hi = fmaxf(s_hi, zmax / (zmax >= 0.f ? rmin : rmax));
                s_lo = fminf(s_lo, zmin / (zmin <= 0.f ? rmin : rmax));
            }
            el_hi = atanf(s_hi);
            el_lo = atanf(s_lo);
        } else if (!full_rows) {
            const float beta = asinf(fminf(rad / rc, 1.f));
            el_lo = el - beta;
            el_hi = el + beta;
            if (!full_cols) {
                const float gam = asinf(fminf(rad / rxy, 1.f));
                az_lo = -gam;
                az_hi = gam;
            }
        }
        if (full_rows) {
            i0 = 0;
            i1 = sd.height - 1;
        } else {
            float lo = fminf((sd.el_max - el_hi) * sd.inv_d_el, crow - rlp) - 1.f;
            float hi = fmaxf((sd.el_max - el_lo) * sd.inv_d_el, crow + rlp) + 1.f;
            index_range(lo, hi, 0.f, sd.height, i0, i1);
        }
        if (full_cols) {
            tx0 = 0;
            tx1 = tiles_x - 1;
        } else {
            const float clo = fminf(az_lo * sd.inv_d_az, -rlp) - 1.f;
            const float chi = fmaxf(az_hi * sd.inv_d_az, rlp) + 1.f;
            const int j0 = (int)ceilf(ccol + clo), j1 = (int)floorf(ccol + chi);
            if (j1 - j0 + 1 >= A) {
                tx0 = 0;
                tx1 = tiles_x - 1;
            } else {
                int j0m = j0 % A;
                if (j0m < 0) j0m += A;
                const int j1m = j0m + (j1 - j0);
                tx0 = j0m / TW;
                if (j1m < A) {
                    tx1 = j1m / TW;
                } else {
                    const int txw = (j1m - A) / TW;
                    if (txw >= tx0) { tx0 = 0; tx1 = tiles_x - 1; }
                    else tx1 = tiles_x + txw;
                }
            }
        }
        if (i0 <= i1) {
            // columns [c0, c0 + cw) on the azimuth circle, c0 in [0, A)
            int c0 = 0, cw = A;
            if (!full_cols) {
                const float clo = fminf(az_lo * sd.inv_d_az, -rlp) - 1.f;
                const float chi = fmaxf(az_hi * sd.inv_d_az, rlp) + 1.f;
                const int j0 = (int)ceilf(ccol + clo), j1 = (int)floorf(ccol + chi);
                if (j1 - j0 + 1 < A) {
                    c0 = j0 % A;
                    if (c0 < 0) c0 += A;
                    cw = j1 - j0 + 1;
                }
            }
            r5 = make_float4((float)c0, (float)(c0 + cw - 1), (float)i0, (float)i1);
            rect = make_ushort4(tx0, tx1, i0 / TH, i1 / TH);
            cnt = (uint32_t)(rect.y - rect.x + 1) * (uint32_t)(rect.w - rect.z + 1);
        }
    }
    counts[slot] = cnt;
    keys[slot] = __float_as_uint(zkey);
    rects[slot] = rect;
    if (cnt == 0) return;

    // ---- appearance
    const F3 org = f3(sd.origin[0], sd.origin[1], sd.origin[2]);
    F3 vd = mu - org;
    const float vlen2 = dot(vd, vd);
    if (dot(nw, vd) > 0.f) nw = -1.f * nw;
    const F3 ns = mat3(sd.R, nw);
    float4 r3;
    if (KIND != GSR_SENSOR_LIDAR) {
        vd = rsqrtf(vlen2) * vd;
        if (Ro != nullptr) {
            float Rm[9] = {__ldg(Ro), __ldg(Ro + 1), __ldg(Ro + 2), __ldg(Ro + 4), __ldg(Ro + 5),
                           __ldg(Ro + 6), __ldg(Ro + 8), __ldg(Ro + 9), __ldg(Ro + 10)};
            vd = mat3T(Rm, vd);
        }
        const int K = (S.sh_degree + 1) * (S.sh_degree + 1);
        const F3 col = sh_colour(S.sh_degree, S.sh + (size_t)i * K * 3, vd);
        r3 = make_float4(o, col.x, col.y, col.z);
    } else {
        // LiDAR: intensity r and ray-drop probability rho, composited alike
        const float rho = S.ray_drop ? 1.f / (1.f + __expf(-__ldg(S.ray_drop + i))) : 0.f;
        r3 = make_float4(o, S.intensity ? __ldg(S.intensity + i) : 0.f, rho, 0.f);
    }
    float4* R = rec + slot * kRecordF4;
    R[0] = r0;
    R[1] = r1;
    R[2] = r2;
    R[3] = r3;
    R[4] = make_float4(ns.x, ns.y, ns.z, zkey);
    R[5] = r5;
}


// One launch per sensor model present in the plan.  Sensors the table is
// not for (gsr_surfels.sees) get empty slots for its surfels.
cudaError_t launch_preprocess(const SensorTable& tab, const gsr_surfels& S, const float* poses, int n_obj,
                              float4* rec, ushort4* rects, uint32_t* counts, uint32_t* keys, uint4* spans,
                              int first, int n_plan, cudaStream_t st)
{
    for (int kind = 0; kind < 3; ++kind) {
        const int bit = kind == GSR_SENSOR_LIDAR ? GSR_SEES_LIDARS : GSR_SEES_CAMERAS;
        const bool seen = S.sees == 0 || (S.sees & bit) != 0;
        SensorIds ids;
        ids.n = 0;
        for (int i = 0; i < tab.n; ++i) {
            if (tab.s[i].kind != kind) continue;
            if (seen) {
                ids.id[ids.n++] = (uint8_t)i;
            } else {
                const cudaError_t e =
                    cudaMemsetAsync(counts + (size_t)i * n_plan + first, 0, sizeof(uint32_t) * (size_t)S.n, st);
                if (e != cudaSuccess) return e;
            }
        }
        if (ids.n == 0) continue;
        const dim3 grid((unsigned)(((S.n + 255) / 256) * ids.n));
        if (kind == GSR_SENSOR_PINHOLE)
            k_preprocess<GSR_SENSOR_PINHOLE><<<grid, 256, 0, st>>>(tab, ids, S, poses, n_obj, rec, rects, counts,
                                                                   keys, spans, first, n_plan);
        else if (kind == GSR_SENSOR_LIDAR)
            k_preprocess<GSR_SENSOR_LIDAR><<<grid, 256, 0, st>>>(tab, ids, S, poses, n_obj, rec, rects, counts, keys,
                                                                 spans, first, n_plan);
        else
            k_preprocess<GSR_SENSOR_CYLINDRICAL><<<grid, 256, 0, st>>>(tab, ids, S, poses, n_obj, rec, rects,
                                                                       counts, keys, spans, first, n_plan);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace gsr
