// sort.cu -- binning of (sensor, surfel) records into screen tiles.
//
// The order every tile needs is the stable order of the 64-bit keys
// (global tile id << 32 | float bits of the centre depth) over the pairs
// emitted in slot order (the tile-splatting order of 3DGS, which the paper
// cites for splatting surfels onto sensor frames, Sec. II).  It is produced
// as one LSD radix sort whose depth digits are sorted before duplication:
//   1. compact the visible slots (tile count > 0), in slot order;
//   2. LSD radix sort of their 32-bit depth keys (4 passes of 8 bits);
//   3. exclusive prefix sum of their tile counts in that order;
//   4. duplication: each visible slot writes (tile id, slot) for every tile
//      of its rectangle at its offset -- the pairs come out depth-sorted;
//   5. LSD radix sort of the pairs by tile id (stable: keeps depth order);
//   6. [start, end) of every tile.
// Duplication preserves the relative order of the depth-sorted slots, so
// applying the depth passes before it gives exactly the 64-bit stable sort.
//
// All kernels read their item counts from device memory (no host sync);
// they run on a fixed grid of `sort_ctas` CTAs (the radix scatter, whose
// tiles need more shared memory, on half of it), each owning a contiguous
// chunk of the items, which keeps every pass stable and the scan small.
#include "gsr_internal.cuh"

namespace gsr {

namespace {

template <typename T, int NT>
__device__ __forceinline__ T block_exclusive_scan(T v, T& total, T* sm /* NT/32 + 1 */)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[w] = x;
    __syncthreads();
    if (w == 0) {
        T s = lane < NT / 32 ? sm[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NT / 32) sm[lane] = s;
    }
    __syncthreads();
    const T wp = w > 0 ? sm[w - 1] : T(0);
    total = sm[NT / 32 - 1];
    __syncthreads();
    return wp + x - v;
}

// Contiguous chunk [b, e) of n items owned by CTA `cta` of `G` (warp-aligned).
__device__ __forceinline__ void chunk_of(uint64_t n, int cta, int G, uint64_t& b, uint64_t& e)
{
    uint64_t per = (n + G - 1) / G;
    per = (per + 31) & ~uint64_t(31);
    b = min(n, per * (uint64_t)cta);
    e = min(n, b + per);
}

}  // namespace

// ------------------------------------------------------------------ compaction
// Visible slots (count > 0), in slot order.  A CTA owns a contiguous chunk
// of slots (a multiple of 32, so its loads are 16-byte aligned) and walks
// it 2048 slots at a time, eight consecutive slots per thread (two 16-byte
// loads of the counts), with one block scan per step.
constexpr int kCompactPer = 8;

__device__ __forceinline__ uint32_t compact_flags(const uint32_t* __restrict__ counts, uint64_t i, uint64_t e)
{
    uint32_t f = 0;
    if (i + kCompactPer <= e) {
        const uint4 a = __ldg(reinterpret_cast<const uint4*>(counts + i));
        const uint4 b = __ldg(reinterpret_cast<const uint4*>(counts + i + 4));
        f = (a.x > 0) | (a.y > 0) << 1 | (a.z > 0) << 2 | (a.w > 0) << 3 | (b.x > 0) << 4 | (b.y > 0) << 5 |
            (b.z > 0) << 6 | (b.w > 0) << 7;
    } else {
        for (int k = 0; k < kCompactPer; ++k)
            if (i + k < e && __ldg(counts + i + k) > 0) f |= 1u << k;
    }
    return f;
}

__global__ void __launch_bounds__(256) k_compact_count(const uint32_t* __restrict__ counts, uint64_t n_slots,
                                                       uint32_t* __restrict__ partial)
{
    __shared__ uint32_t sm[9];
    uint64_t b, e;
    chunk_of(n_slots, blockIdx.x, gridDim.x, b, e);
    uint32_t c = 0;
    for (uint64_t i = b + (uint64_t)threadIdx.x * kCompactPer; i < e; i += (uint64_t)blockDim.x * kCompactPer)
        c += __popc(compact_flags(counts, i, e));
    uint32_t tot;
    block_exclusive_scan<uint32_t, 256>(c, tot, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Exclusive scan of G partials in place (one CTA); the total goes to *total_out
// and, if cap_word != nullptr, min(total, cap) to *cap_word (capacity check).
template <typename T>
__global__ void __launch_bounds__(1024) k_scan_partials(T* __restrict__ partial, int G, T* __restrict__ total_out,
                                                        uint32_t* __restrict__ counters, int64_t cap, int cap_word)
{
    __shared__ T sm[33];
    const int per = (G + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(G, b + per);
    T s = 0;
    for (int i = b; i < e; ++i) s += partial[i];
    T tot;
    T off = block_exclusive_scan<T, 1024>(s, tot, sm);
    for (int i = b; i < e; ++i) {
        T v = partial[i];
        partial[i] = off;
        off += v;
    }
    if (threadIdx.x == 0) {
        if (total_out) *total_out = tot;
        if (cap_word >= 0) {
            uint64_t t = (uint64_t)tot;
            counters[cap_word] = (uint32_t)(t < (uint64_t)cap ? t : (uint64_t)cap);
            if (t > (uint64_t)cap) set_status(counters, GSR_ERR_CAPACITY);
        }
    }
}

// Counts and depth keys of slots [i, i + 8) (two 16-byte loads each; the
// chunks are 32-slot aligned), with zero counts past e.
__device__ __forceinline__ void compact_load(const uint32_t* __restrict__ counts, const uint32_t* __restrict__ depthkey,
                                             uint64_t i, uint64_t e, uint4 (&c)[2], uint4 (&d)[2])
{
    if (i + kCompactPer <= e) {
        c[0] = __ldg(reinterpret_cast<const uint4*>(counts + i));
        c[1] = __ldg(reinterpret_cast<const uint4*>(counts + i + 4));
        d[0] = __ldg(reinterpret_cast<const uint4*>(depthkey + i));
        d[1] = __ldg(reinterpret_cast<const uint4*>(depthkey + i + 4));
    } else {
        uint32_t cc[8], dd[8];
        for (int k = 0; k < kCompactPer; ++k) {
            cc[k] = i + k < e ? __ldg(counts + i + k) : 0u;
            dd[k] = i + k < e ? __ldg(depthkey + i + k) : 0u;
        }
        c[0] = make_uint4(cc[0], cc[1], cc[2], cc[3]);
        c[1] = make_uint4(cc[4], cc[5], cc[6], cc[7]);
        d[0] = make_uint4(dd[0], dd[1], dd[2], dd[3]);
        d[1] = make_uint4(dd[4], dd[5], dd[6], dd[7]);
    }
}

// The visible slots' depth keys and slot ids, in slot order: every slot's
// count and key arrive in one step (no load waits on another), and the next
// step's loads are in flight while this step is scanned and written.
__global__ void __launch_bounds__(256) k_compact_write(const uint32_t* __restrict__ counts,
                                                       const uint32_t* __restrict__ depthkey, uint64_t n_slots,
                                                       const uint32_t* __restrict__ partial,
                                                       uint32_t* __restrict__ vis_key, uint32_t* __restrict__ vis_val)
{
    __shared__ uint32_t sm[9];
    uint64_t b, e;
    chunk_of(n_slots, blockIdx.x, gridDim.x, b, e);
    uint32_t base = partial[blockIdx.x];
    const uint64_t step = (uint64_t)blockDim.x * kCompactPer;
    uint4 c[2] = {}, d[2] = {};
    uint64_t i = b + (uint64_t)threadIdx.x * kCompactPer;
    if (b < e && i < e) compact_load(counts, depthkey, i, e, c, d);
    for (uint64_t t0 = b; t0 < e; t0 += step) {
        const uint32_t cc[8] = {c[0].x, c[0].y, c[0].z, c[0].w, c[1].x, c[1].y, c[1].z, c[1].w};
        const uint32_t dd[8] = {d[0].x, d[0].y, d[0].z, d[0].w, d[1].x, d[1].y, d[1].z, d[1].w};
        const uint64_t icur = i;
        i += step;
        if (i < e) {
            compact_load(counts, depthkey, i, e, c, d);
        } else {
            c[0] = c[1] = d[0] = d[1] = make_uint4(0u, 0u, 0u, 0u);
        }
        uint32_t f = 0;
#pragma unroll
        for (int k = 0; k < kCompactPer; ++k) f |= (cc[k] > 0 ? 1u : 0u) << k;
        uint32_t tot;
        uint32_t r = base + block_exclusive_scan<uint32_t, 256>(__popc(f), tot, sm);
#pragma unroll
        for (int k = 0; k < kCompactPer; ++k) {
            if (cc[k] > 0) {
                vis_key[r] = dd[k];
                vis_val[r] = (uint32_t)(icur + k);
                ++r;
            }
        }
        base += tot;
    }
}

// ------------------------------------------------------------------ radix sort
// Per-CTA digit histogram of its chunk for a digit of BITS bits at `shift`;
// hist is digit-major: hist[d * G + cta].
template <int BITS>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                             const uint32_t* __restrict__ n_ptr, int shift,
                                                             uint32_t* __restrict__ hist)
{
    constexpr int R = 1 << BITS;
    __shared__ uint32_t h[kSortThreads / 32][R];
    const int w = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < (kSortThreads / 32) * R; k += kSortThreads) (&h[0][0])[k] = 0;
    __syncthreads();
    uint64_t b, e;
    chunk_of(*n_ptr, blockIdx.x, gridDim.x, b, e);
    for (uint64_t i = b + threadIdx.x; i < e; i += kSortThreads) atomicAdd(&h[w][(keys[i] >> shift) & (R - 1)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < R; d += kSortThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int k = 0; k < kSortThreads / 32; ++k) s += h[k][d];
        hist[(size_t)d * gridDim.x + blockIdx.x] = s;
    }
}

// Exclusive scan of the whole digit-major histogram (n a multiple of 8) in
// three steps: per-CTA sums of 2048-entry blocks, a scan of those sums, and
// the in-block scan plus the block's base.
constexpr int kScanBlock = 2048;

__global__ void __launch_bounds__(256) k_hist_block_sums(const uint32_t* __restrict__ hist, int n,
                                                         uint32_t* __restrict__ sums)
{
    __shared__ uint32_t sm[9];
    const int i = blockIdx.x * kScanBlock + threadIdx.x * 8;
    uint32_t s = 0;
    if (i < n) {
        const uint4 a = *reinterpret_cast<const uint4*>(hist + i);
        const uint4 b = *reinterpret_cast<const uint4*>(hist + i + 4);
        s = a.x + a.y + a.z + a.w + b.x + b.y + b.z + b.w;
    }
    uint32_t tot;
    block_exclusive_scan<uint32_t, 256>(s, tot, sm);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_hist_block_apply(uint32_t* __restrict__ hist, int n,
                                                          const uint32_t* __restrict__ bases)
{
    __shared__ uint32_t sm[9];
    const int i = blockIdx.x * kScanBlock + threadIdx.x * 8;
    uint32_t v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (i < n) {
        const uint4 a = *reinterpret_cast<const uint4*>(hist + i);
        const uint4 b = *reinterpret_cast<const uint4*>(hist + i + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
    uint32_t tot;
    uint32_t off = bases[blockIdx.x] + block_exclusive_scan<uint32_t, 256>(s, tot, sm);
    if (i < n) {
        uint32_t o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            o[k] = off;
            off += v[k];
        }
        *reinterpret_cast<uint4*>(hist + i) = make_uint4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<uint4*>(hist + i + 4) = make_uint4(o[4], o[5], o[6], o[7]);
    }
}

// Stable scatter of one digit pass (BITS = 8, or 9 for the top digit of a
// key of 8k + 1 bits).  CTA g owns the contiguous chunk [b, e) of the input
// (the same chunk k_radix_hist counted) and walks it in tiles of
// kRadixTile items, two CTAs per SM.  Per tile:
//   1. the keys and values arrive by two bulk copies (one mbarrier);
//   2. warp w ranks its items [w*SEG, w*SEG+SEG) in rounds of 32: the lanes
//      holding the same digit are found by one ballot per digit bit, and the
//      round's first such lane adds their count to the warp's counter of
//      that digit (match_any measured 1.6x slower on this GPU);
//   3. the input buffer is free again: the next tile's copies are issued and
//      land while this one is ordered and written;
//   4. a block scan over digits gives each (warp, digit) its offset in the
//      tile, and each digit the distance from its tile position to its
//      output position (the CTA's running digit bases stay in registers);
//   5. the tile is placed in digit order in a second buffer and written out,
//      consecutive threads writing consecutive positions of each digit run.
template <int BITS>
__device__ __forceinline__ uint32_t lanes_with_digit(uint32_t d)
{
    uint32_t m = 0xffffffffu;
#pragma unroll
    for (int bit = 0; bit < BITS; ++bit) {
        const bool on = (d >> bit) & 1u;
        const uint32_t v = __ballot_sync(0xffffffffu, on);
        m &= on ? v : ~v;
    }
    return m;
}

template <int BITS>
constexpr size_t radix_scatter_smem()
{
    return (size_t)(4 * kRadixTile + (kSortThreads / 32 + 1) * (1 << BITS) + kSortThreads / 32 + 2) * 4 + 16;
}

template <int BITS>
__global__ void __launch_bounds__(kSortThreads, kRadixCtasPerSm)
    k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
                    uint32_t* __restrict__ vout, const uint32_t* __restrict__ n_ptr, int shift,
                    const uint32_t* __restrict__ hist, uint32_t* __restrict__ counters)
{
    constexpr int R = 1 << BITS;
    constexpr int NT = kSortThreads;
    constexpr int NW = NT / 32;
    constexpr int IPT = kRadixIPT;
    constexpr int TILE = kRadixTile;
    constexpr int SEG = 32 * IPT;  // items per warp per tile
    constexpr int DPT = R / NT;    // digits per thread in the digit scan
    static_assert(R % NT == 0 && TILE == NT * IPT, "digit and tile shapes");
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* kb = smem;         // [TILE] input keys (bulk copy)
    uint32_t* vb = kb + TILE;    // [TILE] input values
    uint32_t* ko = vb + TILE;    // [TILE] keys in digit order
    uint32_t* vo = ko + TILE;    // [TILE] values in digit order
    uint32_t* wh = vo + TILE;    // [NW][R] warp digit counts, then offsets in the tile
    uint32_t* gd = wh + NW * R;  // [R] output position minus tile position
    uint32_t* sm = gd + R;       // [NW + 1] block scan
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + NW + 2);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t b, e;
    chunk_of(*n_ptr, blockIdx.x, gridDim.x, b, e);
    const int ntiles = e > b ? (int)((e - b + TILE - 1) / TILE) : 0;
    uint32_t base[DPT];  // output position of the CTA's next item of digit threadIdx.x * DPT + j
#pragma unroll
    for (int j = 0; j < DPT; ++j) base[j] = hist[(size_t)(threadIdx.x * DPT + j) * gridDim.x + blockIdx.x];
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    // tile t: whole 16-byte groups by bulk copy (a chunk starts 128-byte
    // aligned), a ragged end of < 4 items by plain loads
    auto tile_items = [&](int t) {
        const uint64_t s0 = b + (uint64_t)t * TILE;
        return (int)((e - s0) < (uint64_t)TILE ? (e - s0) : (uint64_t)TILE);
    };
    auto issue = [&](int t) {
        const uint64_t s0 = b + (uint64_t)t * TILE;
        const uint32_t nbulk = (uint32_t)tile_items(t) & ~3u;
        mbar_arrive_expect_tx(bar, nbulk * 8u);
        if (nbulk > 0) {
            bulk_g2s(kb, kin + s0, nbulk * 4u, bar);
            bulk_g2s(vb, vin + s0, nbulk * 4u, bar);
        }
    };
    if (threadIdx.x == 0 && ntiles > 0) issue(0);
    for (int t = 0; t < ntiles; ++t) {
        const uint64_t t0 = b + (uint64_t)t * TILE;
        const int nt = tile_items(t);
        const bool full = nt == TILE;
        const int nbulk = nt & ~3;
        for (int k = threadIdx.x; k < NW * R; k += NT) wh[k] = 0;
        const bool got = mbar_wait_bounded(bar, (uint32_t)t & 1u, counters);
        if (!__syncthreads_and(got)) {
            // give up: let the one copy in flight land (bounded) before leaving
            if (threadIdx.x == 0) mbar_wait_bounded(bar, (uint32_t)t & 1u, counters);
            __syncthreads();
            return;
        }
        uint32_t key[IPT], val[IPT], rank[IPT];
        const int li0 = w * SEG + lane;
#pragma unroll
        for (int r = 0; r < IPT; ++r) {
            const int li = li0 + r * 32;
            if (full) {
                key[r] = kb[li];
                val[r] = vb[li];
            } else {
                const bool ok = li < nt;
                key[r] = li < nbulk ? kb[li] : ok ? kin[t0 + li] : 0u;
                val[r] = li < nbulk ? vb[li] : ok ? vin[t0 + li] : 0u;
            }
        }
        fence_proxy_async_smem();  // these reads precede the next bulk copy into the buffer
        uint32_t* wc = wh + w * R;
#pragma unroll
        for (int r = 0; r < IPT; ++r) {
            const bool ok = full || li0 + r * 32 < nt;
            const uint32_t d = (key[r] >> shift) & (R - 1);
            uint32_t peers = lanes_with_digit<BITS>(d);
            if (!full) peers &= __ballot_sync(0xffffffffu, ok);
            const int leader = ok ? __ffs(peers) - 1 : lane;
            uint32_t old = 0;
            if (ok && lane == leader) {
                old = wc[d];
                wc[d] = old + __popc(peers);
            }
            old = __shfl_sync(0xffffffffu, old, leader);
            rank[r] = old + __popc(peers & lt);
            __syncwarp();
        }
        __syncthreads();
        if (threadIdx.x == 0 && t + 1 < ntiles) issue(t + 1);
        // per digit: the warps' counts, the tile's count and a block scan
        // over digits (thread k holds digits [k DPT, k DPT + DPT))
        uint32_t c[DPT][NW], tc[DPT], csum = 0;
#pragma unroll
        for (int j = 0; j < DPT; ++j) {
            const int d = threadIdx.x * DPT + j;
            tc[j] = 0;
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                c[j][k] = wh[k * R + d];
                tc[j] += c[j][k];
            }
            csum += tc[j];
        }
        uint32_t tot;
        uint32_t off = block_exclusive_scan<uint32_t, NT>(csum, tot, sm);
#pragma unroll
        for (int j = 0; j < DPT; ++j) {
            const int d = threadIdx.x * DPT + j;
            uint32_t run = off;
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                wh[k * R + d] = run;
                run += c[j][k];
            }
            gd[d] = base[j] - off;
            base[j] += tc[j];
            off += tc[j];
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < IPT; ++r) {
            if (full || li0 + r * 32 < nt) {
                const uint32_t pos = wc[(key[r] >> shift) & (R - 1)] + rank[r];
                ko[pos] = key[r];
                vo[pos] = val[r];
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const int k = i * NT + threadIdx.x;
            if (full || k < nt) {
                const uint32_t kk = ko[k];
                const uint32_t g = gd[(kk >> shift) & (R - 1)] + (uint32_t)k;
                kout[g] = kk;
                vout[g] = vo[k];
            }
        }
        // the next tile's counter reset and digit-order writes follow this
        // tile's reads of wh, ko and vo behind the next tile's first barriers
    }
}

// ------------------------------------------------------------ duplication
// Gather the tile counts of the visible slots in depth order; per-CTA sums.
__global__ void __launch_bounds__(256) k_dup_count(const uint32_t* __restrict__ vis_val,
                                                   const uint32_t* __restrict__ counts,
                                                   const uint32_t* __restrict__ n_ptr,
                                                   uint32_t* __restrict__ cnt_sorted,
                                                   unsigned long long* __restrict__ partial)
{
    __shared__ unsigned long long sm[9];
    uint64_t b, e;
    chunk_of(*n_ptr, blockIdx.x, gridDim.x, b, e);
    unsigned long long s = 0;
    for (uint64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        const uint32_t c = counts[vis_val[i]];
        cnt_sorted[i] = c;
        s += c;
    }
    unsigned long long tot;
    block_exclusive_scan<unsigned long long, 256>(s, tot, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Exclusive pair offset of every visible slot in depth order, saturated at
// the pair capacity (pairs at or beyond it are dropped).
__global__ void __launch_bounds__(256) k_dup_offsets(const uint32_t* __restrict__ cnt_sorted,
                                                     const uint32_t* __restrict__ n_ptr,
                                                     const unsigned long long* __restrict__ partial, uint64_t cap,
                                                     uint32_t* __restrict__ offs)
{
    // eight consecutive slots per thread, one block scan per 2048 slots
    constexpr int kPer = 8;
    __shared__ unsigned long long sm[9];
    uint64_t b, e;
    chunk_of(*n_ptr, blockIdx.x, gridDim.x, b, e);
    unsigned long long base = partial[blockIdx.x];
    for (uint64_t t0 = b; t0 < e; t0 += (uint64_t)blockDim.x * kPer) {
        const uint64_t i = t0 + (uint64_t)threadIdx.x * kPer;
        uint32_t c[kPer];
        unsigned long long s = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            c[k] = i + k < e ? cnt_sorted[i + k] : 0u;
            s += c[k];
        }
        unsigned long long tot;
        unsigned long long off = base + block_exclusive_scan<unsigned long long, 256>(s, tot, sm);
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            if (i + k < e) offs[i + k] = (uint32_t)(off < cap ? off : cap);
            off += c[k];
        }
        base += tot;
    }
}

// First index in [0, n) whose offset exceeds v (offsets are non-decreasing).
__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t* __restrict__ a, uint32_t n, uint32_t v)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (a[mid] <= v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Each visible slot writes (global tile id, slot) for every tile its bound
// keeps, row by row, at its pair offset; pairs beyond max_dup are dropped.
// Camera slots marked kRectExact keep only the tiles of each row that their
// footprint reaches, with the same test the preprocess counted with (or the
// spans it cached).  Work is split by PAIRS: CTA g writes the pairs
// [P g / G, P (g + 1) / G) of the P kept.  A CTA takes its slots 256 at a
// time and lists their tile rows, kDupRowsRound at a time: one thread per
// row finds the row's span, a block scan gives every row its first pair,
// and each warp then takes 128 consecutive pairs at a time, lane l walking
// the four pairs 4 l .. 4 l + 3 through the rows, and writes them out from
// shared memory in pair order (coalesced stores).  The cost per
// pair no longer depends on how the pairs fall into slots and rows.
constexpr int kDupRowsRound = 512;
constexpr int kPairsPerLane = 4;   // pairs a lane walks per warp chunk
constexpr int kStageStride = 40;  // = 8 mod 32: conflict-free staging both ways
constexpr int kDupCtasPerSortCta = 8;
constexpr int kDupRowsPerThread = kDupRowsRound / 256;

// Compiled for 4 resident CTAs per SM: 64 registers without spills (left to
// itself the compiler also took 64 but spilled); 3 (72) and 2 (90) measured
// slower.
__global__ void __launch_bounds__(256, 4) k_dup_write(SensorTable tab, int n_surfels,
                                                   const uint32_t* __restrict__ vis_val,
                                                   const uint32_t* __restrict__ cnt_sorted,
                                                   const uint32_t* __restrict__ offs,
                                                   const uint32_t* __restrict__ counters,
                                                   const ushort4* __restrict__ rects,
                                                   const float4* __restrict__ rec, const uint4* __restrict__ spans,
                                                   uint32_t* __restrict__ pkey, uint32_t* __restrict__ pval)
{
    // per slot of the batch
    __shared__ uint32_t s_off[256], s_cnt[256], s_slot[256], s_start[256], s_rowpre[257];
    __shared__ ushort4 s_rect[256];
    __shared__ uint4 s_span[256];
    __shared__ uint8_t s_sen[256];
    // per row of the round
    __shared__ uint32_t r_pre[kDupRowsRound + 1];  // first pair of the row within the round
    __shared__ uint32_t r_q0[kDupRowsRound];       // global position of the row's first pair
    __shared__ uint32_t r_key0[kDupRowsRound];     // tile id of column 0 of the row
    __shared__ uint16_t r_t0[kDupRowsRound], r_len[kDupRowsRound], r_lim[kDupRowsRound], r_tx[kDupRowsRound];
    __shared__ uint8_t r_slot[kDupRowsRound];
    // per warp: 32 kPairsPerLane staged pairs, [pair % kPairsPerLane][pair /
    // kPairsPerLane] with a row stride of kStageStride words
    __shared__ uint32_t st_key[8][kPairsPerLane * kStageStride], st_val[8][kPairsPerLane * kStageStride],
        st_q[8][kPairsPerLane * kStageStride];
    __shared__ uint32_t scan_s[9];
    __shared__ uint32_t rb_s, re_s;
    const uint32_t n_vis = counters[C_NVIS];
    const uint32_t P = counters[C_NDUP];
    const int G = gridDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t p0 = (uint32_t)((uint64_t)P * blockIdx.x / G), p1 = (uint32_t)((uint64_t)P * (blockIdx.x + 1) / G);
    if (p0 >= p1) return;
    if (tid == 0) {
        rb_s = upper_bound_u32(offs, n_vis, p0) - 1u;
        re_s = upper_bound_u32(offs, n_vis, p1 - 1u);
    }
    __syncthreads();
    const uint32_t rb = rb_s, re = re_s;
    for (uint32_t base = rb; base < re; base += 256) {
        // 1. the batch's slots and their tile-row counts
        const uint32_t i = base + tid;
        uint32_t nrows = 0;
        s_cnt[tid] = 0;
        if (i < re) {
            const uint32_t c = cnt_sorted[i];
            s_cnt[tid] = c;
            s_off[tid] = offs[i];
            if (c > 0) {
                const uint32_t slot = vis_val[i];
                const ushort4 rc = rects[slot];
                const bool exact = (rc.w & kRectExact) != 0;
                s_slot[tid] = slot;
                s_rect[tid] = rc;
                s_sen[tid] = (uint8_t)(slot / (uint32_t)n_surfels);
                s_span[tid] = exact ? spans[slot] : make_uint4(0u, 0u, 0u, 0u);
                nrows = (uint32_t)((rc.w & ~kRectExact) - rc.z + 1);
            }
        }
        uint32_t tot_rows;
        const uint32_t rp = block_exclusive_scan<uint32_t, 256>(nrows, tot_rows, scan_s);
        s_rowpre[tid] = rp;
        if (tid == 0) s_rowpre[256] = tot_rows;
        __syncthreads();
        uint32_t carry = 0;  // pairs of the batch's earlier rounds
        for (uint32_t R0 = 0; R0 < tot_rows; R0 += kDupRowsRound) {
            const uint32_t nr = min(tot_rows - R0, (uint32_t)kDupRowsRound);
            // 2. spans of rows R0 + 4 tid .. + 3
            const uint32_t rl0 = (uint32_t)tid * kDupRowsPerThread;
            uint32_t lens[kDupRowsPerThread];
            uint32_t own = 0;
            int sl = 0;
            if (rl0 < nr) {
                // the slot of the first row: the last with s_rowpre <= row
                const uint32_t r = R0 + rl0;
                int lo = 0, hi = 256;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (s_rowpre[mid] <= r) lo = mid;
                    else hi = mid;
                }
                sl = lo;
            }
#pragma unroll
            for (int k = 0; k < kDupRowsPerThread; ++k) {
                const uint32_t rl = rl0 + k;
                lens[k] = 0;
                if (rl >= nr) continue;
                const uint32_t r = R0 + rl;
                while (s_rowpre[sl + 1] <= r) ++sl;
                const ushort4 rc = s_rect[sl];
                const SensorDev& sd = tab.s[s_sen[sl]];
                const int ty = rc.z + (int)(r - s_rowpre[sl]);
                int t0 = rc.x, t1 = rc.y;
                if (rc.w & kRectExact) {
                    const uint4 tb = s_span[sl];
                    const int cached = (int)(tb.x & 0xffu);
                    if (cached > 0) {
                        const int kr = ty - rc.z;  // bytes 1 + 2 kr (first column) and 2 + 2 kr (length)
                        const int b0 = 1 + 2 * kr, b1 = 2 + 2 * kr;
                        const uint32_t w0 = b0 < 4 ? tb.x : b0 < 8 ? tb.y : b0 < 12 ? tb.z : tb.w;
                        const uint32_t w1 = b1 < 4 ? tb.x : b1 < 8 ? tb.y : b1 < 12 ? tb.z : tb.w;
                        t0 = rc.x + (int)((w0 >> (8 * (b0 & 3))) & 0xffu);
                        t1 = t0 + (int)((w1 >> (8 * (b1 & 3))) & 0xffu) - 1;
                    } else {
                        const float4* R = rec + (size_t)s_slot[sl] * kRecordF4;
                        const Footprint fp = make_footprint(R[0], R[1], R[2], R[3].x);
                        if (!footprint_span(fp, ty, sd.tile_w, sd.tile_h, rc.x, rc.y, t0, t1)) t1 = t0 - 1;
                    }
                }
                const uint32_t len = t1 >= t0 ? (uint32_t)(t1 - t0 + 1) : 0u;
                lens[k] = len;
                own += len;
                r_key0[rl] = (uint32_t)(sd.tile_base + ty * sd.tiles_x);
                r_t0[rl] = (uint16_t)t0;
                r_len[rl] = (uint16_t)len;
                r_tx[rl] = (uint16_t)sd.tiles_x;
                r_slot[rl] = (uint8_t)sl;
            }
            // 3. first pair of every row (block scan), the slot's first row
            // sets its start, then each row's global position and the
            // columns it may write (never past its slot's count)
            uint32_t tot;
            uint32_t pre = block_exclusive_scan<uint32_t, 256>(own, tot, scan_s);
#pragma unroll
            for (int k = 0; k < kDupRowsPerThread; ++k) {
                const uint32_t rl = rl0 + k;
                if (rl < nr) {
                    r_pre[rl] = pre;
                    const int s2 = r_slot[rl];
                    if (R0 + rl == s_rowpre[s2]) s_start[s2] = carry + pre;
                }
                pre += lens[k];
            }
            if (tid == 0) r_pre[nr] = tot;
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kDupRowsPerThread; ++k) {
                const uint32_t rl = rl0 + k;
                if (rl < nr) {
                    const int s2 = r_slot[rl];
                    const uint32_t in_slot = carry + r_pre[rl] - s_start[s2];
                    const uint32_t c = s_cnt[s2];
                    r_q0[rl] = s_off[s2] + in_slot;
                    r_lim[rl] = (uint16_t)(c > in_slot ? min(c - in_slot, (uint32_t)r_len[rl]) : 0u);
                }
            }
            __syncthreads();
            // 4. the round's pairs: warp chunks of 32 kPairsPerLane, lane l
            // the consecutive pairs kPairsPerLane l .. + kPairsPerLane - 1 (a
            // row changes at most a few times), staged in the warp's buffer
            // and written out in pair order (consecutive lanes, consecutive
            // addresses)
            uint32_t* sk = st_key[warp];
            uint32_t* sv = st_val[warp];
            uint32_t* sq = st_q[warp];
            constexpr uint32_t kChunk = 32u * kPairsPerLane;
            for (uint32_t w0 = (uint32_t)warp * kChunk; w0 < tot; w0 += 8u * kChunk) {
                const uint32_t pa = w0 + (uint32_t)(kPairsPerLane * lane);
                int rl = 0;
                uint32_t col = 0;
                if (pa < tot) {
                    int lo = 0, hi = (int)nr;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (r_pre[mid] <= pa) lo = mid;
                        else hi = mid;
                    }
                    rl = lo;
                    col = pa - r_pre[rl];
                }
#pragma unroll
                for (int e = 0; e < kPairsPerLane; ++e) {
                    uint32_t q = 0xffffffffu, key = 0u, val = 0u;
                    if (pa + (uint32_t)e < tot) {
                        while (col >= r_len[rl] && rl + 1 < (int)nr) {
                            col -= r_len[rl];
                            ++rl;
                        }
                        if (col < r_lim[rl]) {
                            const uint32_t qq = r_q0[rl] + col;
                            if (qq >= p0 && qq < p1) {
                                const uint32_t tx = r_t0[rl] + col, nx = r_tx[rl];
                                q = qq;
                                key = r_key0[rl] + (tx < nx ? tx : tx - nx);  // LiDAR azimuth wrap
                                val = s_slot[r_slot[rl]];
                            }
                        }
                        ++col;
                    }
                    sk[e * kStageStride + lane] = key;
                    sv[e * kStageStride + lane] = val;
                    sq[e * kStageStride + lane] = q;
                }
                __syncwarp();
#pragma unroll
                for (int i = 0; i < kPairsPerLane; ++i) {
                    const int m = i * 32 + lane, at = (m % kPairsPerLane) * kStageStride + m / kPairsPerLane;
                    const uint32_t q = sq[at];
                    if (q != 0xffffffffu) {
                        pkey[q] = sk[at];
                        pval[q] = sv[at];
                    }
                }
                __syncwarp();
            }
            carry += tot;
            __syncthreads();
        }
        __syncthreads();
    }
}

// Split plan of the frame (tiles in id order): a tile whose list is longer
// than F = split_first gets C = ceil((len - F) / split_chunk) chunks after
// its first and (C + 1) x rays ray records (its carry and one block per
// chunk), while the running total fits the capacity; items (tile, c),
// c = 1..C, are listed in tile order.
__device__ __forceinline__ uint32_t split_chunks(const SensorTable& tab, const uint2* __restrict__ ranges,
                                                 uint32_t t, unsigned long long& need)
{
    const uint32_t len = ranges[t].y - ranges[t].x;
    int s = 0;
    while (s + 1 < tab.n && (int)t >= tab.s[s + 1].tile_base) ++s;
    const SensorDev& sd = tab.s[s];
    need = 0;
    if (len <= (uint32_t)sd.split_first) return 0u;
    const uint32_t C = (len - (uint32_t)sd.split_first - 1) / (uint32_t)sd.split_chunk + 1;
    need = (unsigned long long)(C + 1) * (unsigned long long)(sd.tile_w * sd.tile_h);
    return C;
}

// The plan over all CTAs of the sort grid, in three passes around two scans
// of per-CTA partials (tiles in id order, as one sequential walk would take
// them): CTA g owns the tiles chunk_of(g) and its thread k a contiguous run
// of them.  (1) each CTA sums its tiles' ray blocks; (2) after the scan
// every tile has its ray offset (tiles in order, whether or not their split
// fits the capacity), the chunks of the tiles whose split fits are summed
// per CTA; (3) after the second scan every tile has its first item, and its
// plan and items are written.  Deterministic: the outcome depends only on
// the tile ranges.
__device__ __forceinline__ void split_run(uint32_t n_tiles, uint32_t& t0, uint32_t& t1)
{
    uint64_t b, e;
    chunk_of(n_tiles, blockIdx.x, gridDim.x, b, e);
    const uint32_t per = (uint32_t)((e - b + blockDim.x - 1) / blockDim.x);
    t0 = (uint32_t)min(e, b + (uint64_t)threadIdx.x * per);
    t1 = (uint32_t)min(e, (uint64_t)t0 + per);
}

__global__ void __launch_bounds__(256) k_split_rays(SensorTable tab, const uint2* __restrict__ ranges,
                                                    uint32_t n_tiles, unsigned long long* __restrict__ p64)
{
    __shared__ unsigned long long sm[9];
    uint32_t t0, t1;
    split_run(n_tiles, t0, t1);
    unsigned long long rays = 0;
    for (uint32_t t = t0; t < t1; ++t) {
        unsigned long long need;
        split_chunks(tab, ranges, t, need);
        rays += need;
    }
    unsigned long long tot;
    block_exclusive_scan<unsigned long long, 256>(rays, tot, sm);
    if (threadIdx.x == 0) p64[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_split_count(SensorTable tab, const uint2* __restrict__ ranges,
                                                     uint32_t n_tiles, unsigned long long cap_rays,
                                                     const unsigned long long* __restrict__ p64,
                                                     uint32_t* __restrict__ p32)
{
    __shared__ unsigned long long sm64[9];
    __shared__ uint32_t sm32[9];
    uint32_t t0, t1;
    split_run(n_tiles, t0, t1);
    unsigned long long rays = 0;
    for (uint32_t t = t0; t < t1; ++t) {
        unsigned long long need;
        split_chunks(tab, ranges, t, need);
        rays += need;
    }
    unsigned long long tot;
    unsigned long long off = p64[blockIdx.x] + block_exclusive_scan<unsigned long long, 256>(rays, tot, sm64);
    uint32_t nitems = 0;
    for (uint32_t t = t0; t < t1; ++t) {
        unsigned long long need;
        const uint32_t C = split_chunks(tab, ranges, t, need);
        if (C > 0 && off + need <= cap_rays) nitems += C;
        off += need;
    }
    uint32_t tot32;
    block_exclusive_scan<uint32_t, 256>(nitems, tot32, sm32);
    if (threadIdx.x == 0) p32[blockIdx.x] = tot32;
}

__global__ void __launch_bounds__(256) k_split_write(SensorTable tab, const uint2* __restrict__ ranges,
                                                     uint32_t n_tiles, unsigned long long cap_rays,
                                                     unsigned long long cap_items,
                                                     const unsigned long long* __restrict__ p64,
                                                     const uint32_t* __restrict__ p32, uint4* __restrict__ info,
                                                     uint2* __restrict__ items)
{
    __shared__ unsigned long long sm64[9];
    __shared__ uint32_t sm32[9];
    uint32_t t0, t1;
    split_run(n_tiles, t0, t1);
    unsigned long long rays = 0;
    for (uint32_t t = t0; t < t1; ++t) {
        unsigned long long need;
        split_chunks(tab, ranges, t, need);
        rays += need;
    }
    unsigned long long tot;
    const unsigned long long roff =
        p64[blockIdx.x] + block_exclusive_scan<unsigned long long, 256>(rays, tot, sm64);
    uint32_t nitems = 0;
    unsigned long long off = roff;
    for (uint32_t t = t0; t < t1; ++t) {
        unsigned long long need;
        const uint32_t C = split_chunks(tab, ranges, t, need);
        if (C > 0 && off + need <= cap_rays) nitems += C;
        off += need;
    }
    uint32_t tot32;
    uint32_t ioff = p32[blockIdx.x] + block_exclusive_scan<uint32_t, 256>(nitems, tot32, sm32);
    off = roff;
    for (uint32_t t = t0; t < t1; ++t) {
        unsigned long long need;
        uint32_t C = split_chunks(tab, ranges, t, need);
        if (C > 0 && off + need > cap_rays) C = 0;
        if (C > 0 && (unsigned long long)ioff + C > cap_items) C = 0;  // cannot happen: items <= rays / 32
        info[t] = make_uint4(C, C > 0 ? (uint32_t)off : 0u, ioff, 0u);
        for (uint32_t c = 1; c <= C; ++c) items[ioff + c - 1] = make_uint2(t, c);
        ioff += C;
        off += need;
    }
}

// Scheduling keys of the tiles: longest list first (ascending sort of
// 0xffff - min(len, 0xffff)), for the persistent whole-rig compositing kernel.
__global__ void __launch_bounds__(256) k_tile_keys(const uint2* __restrict__ ranges, uint32_t n_tiles,
                                                   uint32_t* __restrict__ key, uint32_t* __restrict__ val,
                                                   uint32_t* __restrict__ counters)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) counters[C_NTILES] = n_tiles;
    if (t >= n_tiles) return;
    const uint2 r = ranges[t];
    const uint32_t len = r.y - r.x;
    key[t] = 0xffffu - min(len, 0xffffu);
    val[t] = t;
}

// [start, end) of each tile in the sorted pair list (ranges pre-zeroed).
__global__ void __launch_bounds__(256) k_tile_ranges(const uint32_t* __restrict__ key,
                                                     const uint32_t* __restrict__ n_ptr, uint2* __restrict__ ranges)
{
    // four consecutive keys per step (one 16-byte load; the region is
    // 256-byte aligned), their neighbours from plain loads
    const uint32_t n = *n_ptr;
    const uint32_t n4 = (n + 3) / 4;
    const uint4* key4 = reinterpret_cast<const uint4*>(key);
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n4; v += gridDim.x * blockDim.x) {
        const uint32_t i0 = 4 * v;
        uint32_t k[6];
        k[0] = i0 > 0 ? __ldg(key + i0 - 1) : 0xffffffffu;
        if (i0 + 4 <= n) {
            const uint4 q = __ldg(key4 + v);
            k[1] = q.x; k[2] = q.y; k[3] = q.z; k[4] = q.w;
        } else {
            for (int j = 0; j < 4; ++j) k[1 + j] = i0 + j < n ? __ldg(key + i0 + j) : 0xffffffffu;
        }
        k[5] = i0 + 4 < n ? __ldg(key + i0 + 4) : 0xffffffffu;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t i = i0 + j;
            if (i >= n) break;
            const uint32_t t = k[1 + j];
            if (i == 0 || k[j] != t) ranges[t].x = i;
            if (i + 1 == n || k[2 + j] != t) ranges[t].y = i + 1;
        }
    }
}

// --------------------------------------------------------------- host side
// LSD radix sort of (key, value) pairs, n_ptr = item count on the device,
// with G CTAs (G <= the plan's sort_ctas); pass ps sorts the digit of
// widths[ps] bits (8 or 9) above the previous passes' bits.
static void radix_sort(const gsr_plan* p, void* ws, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                       const uint32_t* n_ptr, int first_shift, const int* widths, int passes, cudaStream_t st, int G)
{
    uint32_t* counters = region<uint32_t>(p, ws, R_COUNTERS);
    uint32_t* hist = region<uint32_t>(p, ws, R_HIST);
    uint32_t* sums = hist + (size_t)(1 << kRadixBitsWide) * p->sort_ctas;
    // the scatter's tiles need 2 CTAs per SM, half the plan's sort grid;
    // the histogram counts the same chunks
    G = G < p->sort_ctas * kRadixCtasPerSm / kSortCtasPerSm ? G : p->sort_ctas * kRadixCtasPerSm / kSortCtasPerSm;
    for (int bits = kRadixBits; bits <= kRadixBitsWide; ++bits) {
        const cudaError_t e = cudaFuncSetAttribute(bits > 8 ? k_radix_scatter<9> : k_radix_scatter<8>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)(bits > 8 ? radix_scatter_smem<9>() : radix_scatter_smem<8>()));
        if (e != cudaSuccess) return;
    }
    int shift = first_shift;
    for (int ps = 0; ps < passes; ++ps) {
        const int bits = widths[ps];
        const int nh = (1 << bits) * G, nb = (nh + kScanBlock - 1) / kScanBlock;
        const uint32_t* ki = (ps & 1) ? k1 : k0;
        const uint32_t* vi = (ps & 1) ? v1 : v0;
        uint32_t* ko = (ps & 1) ? k0 : k1;
        uint32_t* vo = (ps & 1) ? v0 : v1;
        if (bits > 8)
            k_radix_hist<9><<<G, kSortThreads, 0, st>>>(ki, n_ptr, shift, hist);
        else
            k_radix_hist<8><<<G, kSortThreads, 0, st>>>(ki, n_ptr, shift, hist);
        k_hist_block_sums<<<nb, 256, 0, st>>>(hist, nh, sums);
        k_scan_partials<uint32_t><<<1, 1024, 0, st>>>(sums, nb, nullptr, nullptr, 0, -1);
        k_hist_block_apply<<<nb, 256, 0, st>>>(hist, nh, sums);
        if (bits > 8)
            k_radix_scatter<9><<<G, kSortThreads, radix_scatter_smem<9>(), st>>>(ki, vi, ko, vo, n_ptr, shift, hist,
                                                                                counters);
        else
            k_radix_scatter<8><<<G, kSortThreads, radix_scatter_smem<8>(), st>>>(ki, vi, ko, vo, n_ptr, shift, hist,
                                                                                counters);
        shift += bits;
    }
}

static void radix_sort(const gsr_plan* p, void* ws, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                       const uint32_t* n_ptr, int first_shift, int passes, cudaStream_t st, int G)
{
    const int w[4] = {8, 8, 8, 8};
    radix_sort(p, ws, k0, v0, k1, v1, n_ptr, first_shift, w, passes, st, G);
}

// The tile key's passes: 8-bit digits, except that a key of 8k + 1 bits
// (k >= 1) takes a 9-bit top digit instead of a pass over one bit.
int tile_sort_widths(const gsr_plan* p, int widths[4])
{
    int bits = 1;
    while ((1ll << bits) < (long long)p->tile_base[p->n_sensors]) ++bits;
    int n = 0;
    while (bits > 0 && n < 4) {
        const int take = (bits == kRadixBitsWide) ? kRadixBitsWide : (bits < kRadixBits ? bits : kRadixBits);
        widths[n++] = take < kRadixBits ? kRadixBits : take;
        bits -= take;
    }
    return n;
}

int tile_sort_passes(const gsr_plan* p)
{
    int w[4];
    return tile_sort_widths(p, w);
}

// ------------------------------------------------------- ray directions
// The angles of a cylinder's columns (phi = (x + 1/2 - cx) / fx) and rows
// (the unit-cylinder height (y + 1/2 - cy) / fy), and of a LiDAR's columns
// (azimuth az0 + (x + 1/2) d_az) and beams (elevation el_max - y d_el), in
// FP64 from the sensor's own parameters, their sine and cosine rounded to
// FP32 once: a ray's direction is then within a few FP32 roundings of the
// exact one at any angle (an angle summed in FP32 near +-pi would carry
// several times more).
struct RayDirParams {
    int n;
    int kind[GSR_MAX_SENSORS], width[GSR_MAX_SENSORS], height[GSR_MAX_SENSORS], off[GSR_MAX_SENSORS];
    double a0[GSR_MAX_SENSORS], da[GSR_MAX_SENSORS], b0[GSR_MAX_SENSORS], db[GSR_MAX_SENSORS];
};

__global__ void __launch_bounds__(256) k_ray_dirs(RayDirParams q, int total, float2* __restrict__ dirs)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    int s = 0;
    while (s + 1 < q.n && (q.kind[s] == GSR_SENSOR_PINHOLE || e >= q.off[s] + q.width[s] + q.height[s])) ++s;
    const int k = e - q.off[s];
    const bool col = k < q.width[s];
    // a LiDAR's beams sit at whole multiples of d_el from el_max, a cylinder's rows at half-pixel centres
    const double row = k - q.width[s] + (q.kind[s] == GSR_SENSOR_LIDAR ? 0.0 : 0.5);
    const double v = col ? q.a0[s] + (k + 0.5) * q.da[s] : q.b0[s] + row * q.db[s];
    if (q.kind[s] == GSR_SENSOR_CYLINDRICAL) {
        dirs[e] = col ? make_float2((float)sin(v), (float)cos(v)) : make_float2((float)v, 0.f);
    } else {
        dirs[e] = make_float2((float)cos(v), (float)sin(v));
    }
}

cudaError_t launch_ray_dirs(const gsr_plan* p, void* ws, cudaStream_t st)
{
    const int total = ray_dir_entries(p);
    if (total == 0) return cudaSuccess;
    const SensorTable tab = make_sensor_table(p);
    const double deg = 3.14159265358979323846 / 180.0;
    RayDirParams q;
    memset(&q, 0, sizeof(q));
    q.n = p->n_sensors;
    for (int i = 0; i < p->n_sensors; ++i) {
        const gsr_sensor& s = p->sensors[i];
        q.kind[i] = s.kind;
        q.width[i] = s.width;
        q.height[i] = s.height;
        q.off[i] = tab.s[i].dir_off;
        if (s.kind == GSR_SENSOR_LIDAR) {
            q.a0[i] = (double)s.az0_deg * deg;
            q.da[i] = 2.0 * 3.14159265358979323846 / s.width;
            q.b0[i] = (double)s.el_max_deg * deg;
            q.db[i] = -((double)s.el_max_deg - (double)s.el_min_deg) * deg / (s.height - 1);
        } else if (s.kind == GSR_SENSOR_CYLINDRICAL) {
            // phi = (x + 1/2 - cx) / fx = -cx / fx + (x + 1/2) / fx; height likewise
            q.a0[i] = -(double)s.cx / (double)s.fx;
            q.da[i] = 1.0 / (double)s.fx;
            q.b0[i] = -(double)s.cy / (double)s.fy;
            q.db[i] = 1.0 / (double)s.fy;
        }
    }
    k_ray_dirs<<<(total + 255) / 256, 256, 0, st>>>(q, total, region<float2>(p, ws, R_RAY_DIRS));
    return cudaGetLastError();
}

cudaError_t bin_sort(const gsr_plan* p, void* ws, cudaStream_t st)
{
    // the frame's ray-direction tables, read by every render that follows
    const cudaError_t de = launch_ray_dirs(p, ws, st);
    if (de != cudaSuccess) return de;
    const SensorTable tab = make_sensor_table(p);
    const int G = p->sort_ctas;
    const uint64_t n_slots = (uint64_t)p->n_surfels * p->n_sensors;
    uint32_t* counters = region<uint32_t>(p, ws, R_COUNTERS);
    uint32_t* partial = region<uint32_t>(p, ws, R_PARTIAL);
    uint32_t* vk[2] = {region<uint32_t>(p, ws, R_VIS_KEY_A), region<uint32_t>(p, ws, R_VIS_KEY_B)};
    uint32_t* vv[2] = {region<uint32_t>(p, ws, R_VIS_VAL_A), region<uint32_t>(p, ws, R_VIS_VAL_B)};
    uint32_t* pk[2] = {region<uint32_t>(p, ws, R_PAIR_KEY_A), region<uint32_t>(p, ws, R_PAIR_KEY_B)};
    uint32_t* pv[2] = {region<uint32_t>(p, ws, R_PAIR_VAL_A), region<uint32_t>(p, ws, R_PAIR_VAL_B)};
    const uint32_t* counts = region<uint32_t>(p, ws, R_COUNTS);

    // 1. compaction
    k_compact_count<<<G, 256, 0, st>>>(counts, n_slots, partial);
    k_scan_partials<uint32_t><<<1, 1024, 0, st>>>(partial, G, counters + C_NVIS, counters, 0, -1);
    k_compact_write<<<G, 256, 0, st>>>(counts, region<uint32_t>(p, ws, R_DEPTHKEY), n_slots, partial, vk[0], vv[0]);
    // 2. depth passes
    radix_sort(p, ws, vk[0], vv[0], vk[1], vv[1], counters + C_NVIS, 0, kDepthSortPasses, st, G);
    const int vb = sort_result_buffer(kDepthSortPasses);
    // 3. offsets (64-bit partials), capacity check
    unsigned long long* p64 = reinterpret_cast<unsigned long long*>(partial);
    uint32_t* cnt_sorted = region<uint32_t>(p, ws, R_CNT_SORTED);
    k_dup_count<<<G, 256, 0, st>>>(vv[vb], counts, counters + C_NVIS, cnt_sorted, p64);
    k_scan_partials<unsigned long long><<<1, 1024, 0, st>>>(
        p64, G, reinterpret_cast<unsigned long long*>(counters + C_NDUP_WANT), counters, p->max_dup, C_NDUP);
    // 4. duplication, balanced by pairs
    uint32_t* offs = region<uint32_t>(p, ws, R_OFFSETS);
    k_dup_offsets<<<G, 256, 0, st>>>(cnt_sorted, counters + C_NVIS, p64, (uint64_t)p->max_dup, offs);
    // many more CTAs than fit at once: the windows are equal in pairs, not
    // in slots, and CTAs that finish early make room for the slow ones
    k_dup_write<<<kDupCtasPerSortCta * G, 256, 0, st>>>(tab, p->n_surfels, vv[vb], cnt_sorted, offs, counters,
                                   region<ushort4>(p, ws, R_RECTS), region<float4>(p, ws, R_RECORDS),
                                   region<uint4>(p, ws, R_SPANS), pk[0], pv[0]);
    // 5. tile passes
    int tw[4];
    const int tp = tile_sort_widths(p, tw);
    radix_sort(p, ws, pk[0], pv[0], pk[1], pv[1], counters + C_NDUP, 0, tw, tp, st, G);
    const int pb = sort_result_buffer(tp);
    // 6. tile ranges
    uint2* ranges = region<uint2>(p, ws, R_RANGES);
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)p->tile_base[p->n_sensors], st);
    k_tile_ranges<<<4 * G, 256, 0, st>>>(pk[pb], counters + C_NDUP, ranges);
    {
        const uint32_t nt = (uint32_t)p->tile_base[p->n_sensors];
        const uint64_t cap_rays = split_ray_capacity(p), cap_items = split_item_capacity(p);
        unsigned long long* sp64 = reinterpret_cast<unsigned long long*>(partial);
        uint32_t* sp32 = reinterpret_cast<uint32_t*>(sp64 + G);
        k_split_rays<<<G, 256, 0, st>>>(tab, ranges, nt, sp64);
        k_scan_partials<unsigned long long><<<1, 1024, 0, st>>>(sp64, G, nullptr, counters, 0, -1);
        k_split_count<<<G, 256, 0, st>>>(tab, ranges, nt, cap_rays, sp64, sp32);
        k_scan_partials<uint32_t><<<1, 1024, 0, st>>>(sp32, G, counters + C_NITEMS, counters, 0, -1);
        k_split_write<<<G, 256, 0, st>>>(tab, ranges, nt, cap_rays, cap_items, sp64, sp32,
                                         region<uint4>(p, ws, R_SPLIT_INFO), region<uint2>(p, ws, R_SPLIT_ITEMS));
    }
    // 7. tile schedule for the whole-rig kernel (2 passes over 16-bit keys)
    const uint32_t T = (uint32_t)p->tile_base[p->n_sensors];
    uint32_t* tk[2] = {region<uint32_t>(p, ws, R_TILE_KEY_A), region<uint32_t>(p, ws, R_TILE_KEY_B)};
    uint32_t* tv[2] = {region<uint32_t>(p, ws, R_TILE_VAL_A), region<uint32_t>(p, ws, R_TILE_VAL_B)};
    k_tile_keys<<<(T + 255) / 256, 256, 0, st>>>(ranges, T, tk[0], tv[0], counters);
    const uint32_t gt = (T + kRadixTile - 1) / kRadixTile;
    const int GT = gt < (uint32_t)G ? (int)gt : G;
    radix_sort(p, ws, tk[0], tv[0], tk[1], tv[1], counters + C_NTILES, 0, 2, st, GT < 1 ? 1 : GT);
    return cudaGetLastError();
}

}  // namespace gsr
