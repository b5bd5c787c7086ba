// zones.cu -- large scenes: zone partition and the double-buffered zone streamer.
//
// Sec. III-A ("Support Large-scale Scenes"): frames are clustered by their
// XY location into 40 x 40 m zones with 25 % relative padding, and while
// rendering two threads double-buffer the zones, swapping in the Gaussians
// of the next block as the vehicle moves between blocks.  Here the zone
// membership and packing run on the host (C++), and the swap is a stream
// pair: the next zone's packed arrays go host -> device on a copy stream
// (plain cudaMemcpyAsync per array, from pinned memory) while the render
// stream keeps drawing from the front buffer; acquiring the new zone makes
// the render stream wait on the copy's event, and the buffer given up is
// only overwritten once the render stream has released it.
#include <cstring>

#include "gsr_internal.cuh"

namespace gsr {
gsr_status cuda_status(cudaError_t e);

namespace {

constexpr float kCulledLogit = -1.0e4f;

bool grid_ok(const gsr_zone_grid* g)
{
    return g && g->nx > 0 && g->ny > 0 && (int64_t)g->nx * g->ny < (1ll << 30) && g->zone_size > 0.f &&
           g->padding >= 0.f && g->padding <= 0.5f;
}

// Zones whose padded square holds (x, y): the ranges [i0, i1] x [j0, j1].
// Zone i spans [x0 + (i - p) s, x0 + (i + 1 + p) s) in double precision.
void zone_span(const gsr_zone_grid* g, double v, double o, int n, int& a0, int& a1)
{
    const double s = g->zone_size, p = g->padding;
    // candidates i with i - p <= (v - o)/s < i + 1 + p, checked exactly below
    const double u = (v - o) / s;
    int lo = (int)std::floor(u - 1.0 - p) - 1, hi = (int)std::floor(u + p) + 1;
    lo = lo < 0 ? 0 : lo;
    hi = hi > n - 1 ? n - 1 : hi;
    a0 = n;
    a1 = -1;
    for (int i = lo; i <= hi; ++i) {
        const double b0 = o + ((double)i - p) * s, b1 = o + ((double)i + 1.0 + p) * s;
        if (v >= b0 && v < b1) {
            a0 = i < a0 ? i : a0;
            a1 = i > a1 ? i : a1;
        }
    }
}

__global__ void k_fill(float* __restrict__ a, int64_t n, float v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

}  // namespace
}  // namespace gsr

using namespace gsr;

extern "C" int32_t gsr_zone_of(const gsr_zone_grid* grid, float x, float y)
{
    if (!grid_ok(grid)) return -1;
    const double s = grid->zone_size;
    const double i = std::floor(((double)x - grid->x0) / s), j = std::floor(((double)y - grid->y0) / s);
    if (i < 0.0 || j < 0.0 || i >= grid->nx || j >= grid->ny) return -1;
    return (int32_t)j * grid->nx + (int32_t)i;
}

extern "C" gsr_status gsr_zone_count(const gsr_zone_grid* grid, const float* pos, int64_t n, int64_t* counts)
{
    if (!grid_ok(grid) || n < 0 || (n > 0 && !pos) || !counts) return GSR_ERR_INVALID_ARG;
    const int nz = grid->nx * grid->ny;
    std::memset(counts, 0, sizeof(int64_t) * (size_t)nz);
    for (int64_t k = 0; k < n; ++k) {
        int i0, i1, j0, j1;
        zone_span(grid, pos[3 * k], grid->x0, grid->nx, i0, i1);
        zone_span(grid, pos[3 * k + 1], grid->y0, grid->ny, j0, j1);
        for (int j = j0; j <= j1; ++j)
            for (int i = i0; i <= i1; ++i) ++counts[j * grid->nx + i];
    }
    return GSR_OK;
}

extern "C" gsr_status gsr_zone_members(const gsr_zone_grid* grid, const float* pos, int64_t n, const int64_t* offsets,
                                       int64_t* members)
{
    if (!grid_ok(grid) || n < 0 || (n > 0 && !pos) || !offsets || !members) return GSR_ERR_INVALID_ARG;
    const int nz = grid->nx * grid->ny;
    for (int z = 0; z < nz; ++z)
        if (offsets[z + 1] < offsets[z]) return GSR_ERR_INVALID_ARG;
    int64_t* fill = new int64_t[(size_t)nz];
    for (int z = 0; z < nz; ++z) fill[z] = offsets[z];
    gsr_status st = GSR_OK;
    for (int64_t k = 0; k < n && st == GSR_OK; ++k) {
        int i0, i1, j0, j1;
        zone_span(grid, pos[3 * k], grid->x0, grid->nx, i0, i1);
        zone_span(grid, pos[3 * k + 1], grid->y0, grid->ny, j0, j1);
        for (int j = j0; j <= j1; ++j)
            for (int i = i0; i <= i1; ++i) {
                const int z = j * grid->nx + i;
                if (fill[z] >= offsets[z + 1]) {
                    st = GSR_ERR_INVALID_ARG;  // offsets not from gsr_zone_count of the same table
                    break;
                }
                members[fill[z]++] = k;
            }
    }
    delete[] fill;
    return st;
}

extern "C" gsr_status gsr_zone_pack(const gsr_surfels* table, const int64_t* members, int64_t count,
                                    const gsr_surfel_table* out)
{
    if (!table || !out || count < 0 || (count > 0 && !members)) return GSR_ERR_INVALID_ARG;
    if (table->sh_degree < 0 || table->sh_degree > 3) return GSR_ERR_UNSUPPORTED;
    if (count > 0 && (!table->pos || !table->log_scale || !table->quat || !table->opacity || !table->sh ||
                      !out->pos || !out->log_scale || !out->quat || !out->opacity || !out->sh))
        return GSR_ERR_INVALID_ARG;
    const int K3 = (table->sh_degree + 1) * (table->sh_degree + 1) * 3;
    for (int64_t q = 0; q < count; ++q) {
        const int64_t k = members[q];
        if (k < 0 || k >= table->n) return GSR_ERR_INVALID_ARG;
        std::memcpy(out->pos + 3 * q, table->pos + 3 * k, 12);
        std::memcpy(out->log_scale + 2 * q, table->log_scale + 2 * k, 8);
        std::memcpy(out->quat + 4 * q, table->quat + 4 * k, 16);
        out->opacity[q] = table->opacity[k];
        std::memcpy(out->sh + (size_t)K3 * q, table->sh + (size_t)K3 * k, sizeof(float) * K3);
        if (out->intensity) out->intensity[q] = table->intensity ? table->intensity[k] : 0.f;
        if (out->ray_drop) out->ray_drop[q] = table->ray_drop ? table->ray_drop[k] : kCulledLogit;
    }
    return GSR_OK;
}

// ------------------------------------------------------------- streamer
extern "C" gsr_status gsr_streamer_init(gsr_streamer* s, int32_t capacity, int32_t sh_degree,
                                        const gsr_surfel_table* buffers, void* copy_stream)
{
    if (!s || !buffers || capacity < 0 || sh_degree < 0 || sh_degree > 3) return GSR_ERR_INVALID_ARG;
    for (int b = 0; b < 2; ++b) {
        const gsr_surfel_table& t = buffers[b];
        if (capacity > 0 && (!t.pos || !t.log_scale || !t.quat || !t.opacity || !t.sh)) return GSR_ERR_INVALID_ARG;
    }
    std::memset(s, 0, sizeof(*s));
    s->capacity = capacity;
    s->sh_degree = sh_degree;
    s->copy_stream = copy_stream;
    s->front = 0;
    for (int b = 0; b < 2; ++b) {
        s->buf[b] = buffers[b];
        s->zone[b] = -1;
        s->count[b] = 0;
        cudaEvent_t e1, e2;
        cudaError_t e = cudaEventCreateWithFlags(&e1, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaEventCreateWithFlags(&e2, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaEventDestroy(e1);
            return cuda_status(e);
        }
        s->ready[b] = e1;
        s->released[b] = e2;
        s->released_valid[b] = 0;
    }
    return GSR_OK;
}

extern "C" gsr_status gsr_streamer_destroy(gsr_streamer* s)
{
    if (!s) return GSR_ERR_INVALID_ARG;
    for (int b = 0; b < 2; ++b) {
        if (s->ready[b]) cudaEventDestroy(reinterpret_cast<cudaEvent_t>(s->ready[b]));
        if (s->released[b]) cudaEventDestroy(reinterpret_cast<cudaEvent_t>(s->released[b]));
        s->ready[b] = s->released[b] = nullptr;
    }
    return GSR_OK;
}

extern "C" gsr_status gsr_streamer_prefetch(gsr_streamer* s, int32_t zone, const gsr_surfels* host_zone)
{
    if (!s || !host_zone || zone < 0) return GSR_ERR_INVALID_ARG;
    if (s->zone[0] == zone || s->zone[1] == zone) return GSR_OK;  // resident or on its way
    const int32_t n = host_zone->n;
    if (n < 0 || n > s->capacity) return GSR_ERR_CAPACITY;
    if (host_zone->sh_degree != s->sh_degree) return GSR_ERR_INVALID_ARG;
    if (n > 0 && (!host_zone->pos || !host_zone->log_scale || !host_zone->quat || !host_zone->opacity ||
                  !host_zone->sh))
        return GSR_ERR_INVALID_ARG;
    const int b = 1 - s->front;
    const gsr_surfel_table& d = s->buf[b];
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(s->copy_stream);
    cudaError_t e = cudaSuccess;
    // the buffer may still be drawn from by frames enqueued before it was given up
    if (s->released_valid[b])
        e = cudaStreamWaitEvent(cs, reinterpret_cast<cudaEvent_t>(s->released[b]), 0);
    const size_t K3 = (size_t)(s->sh_degree + 1) * (s->sh_degree + 1) * 3;
    auto copy = [&](float* dst, const float* src, size_t floats) {
        if (e == cudaSuccess && floats > 0)
            e = cudaMemcpyAsync(dst, src, floats * sizeof(float), cudaMemcpyHostToDevice, cs);
    };
    copy(d.pos, host_zone->pos, 3 * (size_t)n);
    copy(d.log_scale, host_zone->log_scale, 2 * (size_t)n);
    copy(d.quat, host_zone->quat, 4 * (size_t)n);
    copy(d.opacity, host_zone->opacity, (size_t)n);
    copy(d.sh, host_zone->sh, K3 * (size_t)n);
    if (d.intensity && host_zone->intensity) copy(d.intensity, host_zone->intensity, (size_t)n);
    if (d.ray_drop && host_zone->ray_drop) copy(d.ray_drop, host_zone->ray_drop, (size_t)n);
    // slots beyond the zone's surfels render nothing
    if (e == cudaSuccess && n < s->capacity) {
        const int64_t tail = (int64_t)s->capacity - n;
        const int blocks = (int)((tail + 255) / 256 < 1024 ? (tail + 255) / 256 : 1024);
        k_fill<<<blocks, 256, 0, cs>>>(d.opacity + n, tail, kCulledLogit);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(reinterpret_cast<cudaEvent_t>(s->ready[b]), cs);
    if (e != cudaSuccess) {
        s->zone[b] = -1;
        return cuda_status(e);
    }
    s->zone[b] = zone;
    s->count[b] = n;
    return GSR_OK;
}

extern "C" gsr_status gsr_streamer_acquire(gsr_streamer* s, int32_t zone, void* render_stream, gsr_surfels* out)
{
    if (!s || !out || zone < 0) return GSR_ERR_INVALID_ARG;
    int b = -1;
    if (s->zone[s->front] == zone) b = s->front;
    else if (s->zone[1 - s->front] == zone) b = 1 - s->front;
    if (b < 0) return GSR_ERR_INVALID_ARG;  // neither resident nor prefetched
    cudaStream_t rs = reinterpret_cast<cudaStream_t>(render_stream);
    cudaError_t e = cudaSuccess;
    if (b != s->front) {
        // give up the old front once the frames already enqueued are done with it
        e = cudaEventRecord(reinterpret_cast<cudaEvent_t>(s->released[s->front]), rs);
        if (e != cudaSuccess) return cuda_status(e);
        s->released_valid[s->front] = 1;
        s->front = b;
    }
    e = cudaStreamWaitEvent(rs, reinterpret_cast<cudaEvent_t>(s->ready[b]), 0);
    if (e != cudaSuccess) return cuda_status(e);
    const gsr_surfel_table& d = s->buf[b];
    std::memset(out, 0, sizeof(*out));
    out->n = s->capacity;
    out->sh_degree = s->sh_degree;
    out->pos = d.pos;
    out->log_scale = d.log_scale;
    out->quat = d.quat;
    out->opacity = d.opacity;
    out->sh = d.sh;
    out->intensity = d.intensity;
    out->ray_drop = d.ray_drop;
    return GSR_OK;
}
