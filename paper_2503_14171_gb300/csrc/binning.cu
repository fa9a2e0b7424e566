// Tile binning (the front-to-back ordering of Sec. 4, per tile).
//
// Gaussians are first sorted by the FP32 bits of their view depth (a stable
// radix sort of n keys, ids ascending).  Each Gaussian then emits
// (tile mask << 48 | super-tile << 32 | id) for every super-tile of ks x ks
// tiles (ks = 1, 2 or 4, chosen per frame by super_side) its tile rect
// touches, in depth order; the mask marks which of the super-tile's ks^2 tiles
// the rect covers.  A stable radix sort on the super-tile bits alone yields
// per-super-tile lists ordered by (depth, id).  The blend filters a
// super-tile's list by the masks, which reproduces every tile's own
// front-to-back list exactly while sorting up to 3-5x fewer pairs than
// per-tile binning at ks = 4 (and 8 B instead of 12 B per pair and pass).
//
// The per-tile lists themselves (keys tile << 32 | depth bits, ids, ranges)
// are materialised only on request (gs_read_bins), by the same filter.
#include "gs_internal.cuh"
#include "tile_order.cuh"

namespace gs {
namespace {

// One thread per position of the depth order loads its Gaussian (sorted id,
// first pair slot, pair count, rect); the warp then emits the pairs of its 32
// Gaussians together, 32 at a time: lane l takes pair p = base + l of the
// warp's run, finds the Gaussian that owns it (a binary search over the
// lanes' run starts by shuffles), and forms the pair from that Gaussian's
// rect.  A Gaussian's pairs keep the per-Gaussian order (super-tile rows,
// then columns); a lane no longer loops over a large Gaussian's pairs while
// the rest of its warp idles.
// COUNT: also accumulate per-super-tile pair counts (shared memory, then one
// atomic per touched super-tile and block).  KS: the super-tile side (1, 2, 4).
template <bool COUNT, int KS>
__global__ void __launch_bounds__(256) k_emit(const uint32_t* __restrict__ ids, const uint32_t* __restrict__ offsets,
                                              const ushort4* __restrict__ rect, uint32_t n, int stiles_x,
                                              uint64_t* __restrict__ pairs, uint32_t* __restrict__ counts,
                                              uint32_t Ts, uint32_t cap, uint32_t id_base, bool rebase)
{
    __shared__ uint32_t s_cnt[COUNT ? kMaxSupersForCounts : 1];
    if (COUNT) {
        for (uint32_t t = threadIdx.x; t < Ts; t += blockDim.x) s_cnt[t] = 0;
        __syncthreads();
    }
    constexpr int ks = KS, ksh = KS == 4 ? 2 : KS == 2 ? 1 : 0;
    const int lane = threadIdx.x & 31;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    // this lane's Gaussian: pair count c (0 when it has none or k >= n),
    // first slot off, its super-tile columns nsx, first super-tile (sx0, sy0)
    uint32_t c = 0, off = 0, id = 0, r01 = 0, r23 = 0;
    if (k < n) {
        const uint32_t base = rebase ? offsets[0] : 0u;
        off = offsets[k] - base;
        const uint32_t end = offsets[k + 1] - base;
        id = ids[k] - id_base;
        if (off < end && id < n) {   // id >= n only after an expired bounded wait in the sort
            const ushort4 r = rect[id];
            r01 = (uint32_t)r.x | ((uint32_t)r.y << 16);
            r23 = (uint32_t)r.z | ((uint32_t)r.w << 16);
            c = end - off;
        }
    }
    // run start of each lane's pairs within the warp (exclusive scan) and the total
    uint32_t st = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, st, o);
        if (lane >= o) st += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, st, 31);
    st -= c;
    for (uint32_t pb = 0; pb < total; pb += 32) {
        const uint32_t p = pb + lane;
        // owner: the largest lane whose run starts at or before p (lanes
        // without pairs share their start with the next lane, so the largest
        // such lane owns p whenever p < total)
        int L = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t sc = __shfl_sync(0xffffffffu, st, L + step);
            if (sc <= p) L += step;
        }
        const uint32_t q = p - __shfl_sync(0xffffffffu, st, L);
        const uint32_t o_off = __shfl_sync(0xffffffffu, off, L);
        const uint32_t o_id = __shfl_sync(0xffffffffu, id, L);
        const uint32_t o01 = __shfl_sync(0xffffffffu, r01, L);
        const uint32_t o23 = __shfl_sync(0xffffffffu, r23, L);
        if (p < total) {
            const int rx = (int)(o01 & 0xFFFFu), ry = (int)(o01 >> 16);
            const int rz = (int)(o23 & 0xFFFFu), rw = (int)(o23 >> 16);
            const int sx0 = rx >> ksh, sy0 = ry >> ksh;
            const uint32_t nsx = (uint32_t)((rz >> ksh) - sx0 + 1);
            // q = (sy - sy0) nsx + (sx - sx0): below 2^21 the FP32 quotient
            // (q + 1/2) / nsx is within 2^-22 (q + 1/2) / nsx of its value, which
            // lies at least 1 / (2 nsx) from an integer, so it floors exactly
            const uint32_t dy = q < (1u << 21) ? (uint32_t)(((float)q + 0.5f) * __frcp_rn((float)nsx)) : q / nsx;
            const int sy = sy0 + (int)dy, sx = sx0 + (int)(q - dy * nsx);
            // rows and columns of the super-tile's ks x ks tiles inside the rect
            const int ly0 = max(ry - (sy << ksh), 0), ly1 = min(rw - (sy << ksh), ks - 1);
            const int lx0 = max(rx - (sx << ksh), 0), lx1 = min(rz - (sx << ksh), ks - 1);
            const uint32_t cols = ((2u << lx1) - 1u) & ~((1u << lx0) - 1u);
            uint32_t mask = 0;
#pragma unroll
            for (int ly = 0; ly < ks; ++ly)
                if (ly >= ly0 && ly <= ly1) mask |= cols << (ly << ksh);
            const uint32_t s = (uint32_t)(sy * stiles_x + sx);
            const uint32_t slot = o_off + q;
            if (slot < cap) pairs[slot] = ((uint64_t)mask << 48) | ((uint64_t)s << 32) | o_id;
            if (COUNT && s < Ts) atomicAdd(&s_cnt[s], 1u);
        }
    }
    if (COUNT) {
        __syncthreads();
        uint32_t* dst = counts + (size_t)(blockIdx.x % kCountCopies) * Ts;
        for (uint32_t t = threadIdx.x; t < Ts; t += blockDim.x) {
            const uint32_t v = s_cnt[t];
            if (v) atomicAdd(&dst[t], v);
        }
    }
}

// The emission of every view of a batch in one launch.  Position k of the
// batched (view, depth, id) order belongs to the view v whose stretch
// [start_v, start_v + n_v) holds it; its Gaussian is sorted[k] - start_v of
// that view, its pairs start at offsets[k] - offsets[start_v] of the view's own
// pair buffer, and they are emitted exactly as k_emit emits a single view's
// (same super-tile side, masks and order).  Per-super-tile counts go through
// shared memory for the block's first view and straight to global memory for
// the (rare) positions of a later view in the same block.
__global__ void __launch_bounds__(256) k_emit_views(const __grid_constant__ EmitViews b,
                                                    const uint32_t* __restrict__ sorted,
                                                    const uint32_t* __restrict__ offsets,
                                                    const ushort4* __restrict__ rect, uint32_t total,
                                                    uint32_t idx_mask)
{
    __shared__ uint32_t s_cnt[kMaxSupersForCounts];
    const uint32_t k0 = blockIdx.x * blockDim.x;
    int v0 = 0;
    while (v0 + 1 < b.V && k0 >= b.v[v0 + 1].start) ++v0;
    const EmitView& f = b.v[v0];
    const bool shared_counts = f.Ts <= (uint32_t)kMaxSupersForCounts;
    if (shared_counts) {
        for (uint32_t t = threadIdx.x; t < f.Ts; t += blockDim.x) s_cnt[t] = 0;
        __syncthreads();
    }
    const uint32_t k = k0 + threadIdx.x;
    if (k < total) {
        int v = v0;
        while (v + 1 < b.V && k >= b.v[v + 1].start) ++v;
        const EmitView& e = b.v[v];
        const uint32_t base = offsets[e.start];
        uint32_t off = offsets[k] - base;
        const uint32_t end = offsets[k + 1] - base;
        const uint32_t g = sorted[k] & idx_mask;   // a packed count in the top bits is not needed here
        const uint32_t id = g - e.start;
        if (off < end && id < e.n) {   // id >= n only after an expired bounded wait in the sort
            const ushort4 r = rect[g];
            const int ks = e.ks, ksh = __ffs(ks) - 1;
            const int sx0 = r.x >> ksh, sx1 = r.z >> ksh, sy0 = r.y >> ksh, sy1 = r.w >> ksh;
            uint32_t* gcnt = e.counts + (size_t)(blockIdx.x % kCountCopies) * e.Ts;
            for (int sy = sy0; sy <= sy1; ++sy) {
                const int ly0 = max((int)r.y - (sy << ksh), 0), ly1 = min((int)r.w - (sy << ksh), ks - 1);
                for (int sx = sx0; sx <= sx1 && off < end; ++sx) {
                    const int lx0 = max((int)r.x - (sx << ksh), 0), lx1 = min((int)r.z - (sx << ksh), ks - 1);
                    const uint32_t cols = ((2u << lx1) - 1u) & ~((1u << lx0) - 1u);
                    uint32_t mask = 0;
                    for (int ly = ly0; ly <= ly1; ++ly) mask |= cols << (ly << ksh);
                    const uint32_t st = (uint32_t)(sy * e.stiles_x + sx);
                    if (off < e.cap) e.pairs[off] = ((uint64_t)mask << 48) | ((uint64_t)st << 32) | id;
                    ++off;
                    if (st < e.Ts) {
                        if (v == v0 && shared_counts)
                            atomicAdd(&s_cnt[st], 1u);
                        else
                            atomicAdd(&gcnt[st], 1u);
                    }
                }
            }
        }
    }
    if (shared_counts) {
        __syncthreads();
        uint32_t* dst = f.counts + (size_t)(blockIdx.x % kCountCopies) * f.Ts;
        for (uint32_t t = threadIdx.x; t < f.Ts; t += blockDim.x) {
            const uint32_t c = s_cnt[t];
            if (c) atomicAdd(&dst[t], c);
        }
    }
}

__global__ void __launch_bounds__(256) k_ranges(const uint64_t* __restrict__ pairs, uint32_t P, uint32_t T,
                                                uint2* __restrict__ ranges)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    // super-tile field of the pair (bits 32..47; the tile mask sits above)
    const uint32_t t = (uint32_t)(pairs[i] >> 32) & 0xFFFFu;
    if (t >= T) return;   // only after an expired bounded wait in the sort
    if (i == 0 || ((uint32_t)(pairs[i - 1] >> 32) & 0xFFFFu) != t) ranges[t].x = i;
    if (i == P - 1 || ((uint32_t)(pairs[i + 1] >> 32) & 0xFFFFu) != t) ranges[t].y = i + 1;
}

__device__ __forceinline__ bool covers(ushort4 r, int tx, int ty)
{
    return (int)r.x <= tx && tx <= (int)r.z && (int)r.y <= ty && ty <= (int)r.w;
}

// Per-tile list materialisation: one block per tile walks its super-tile's list.
// WRITE = false: count the tile's Gaussians; WRITE = true: write them, in
// order, at tile_start[t].
template <bool WRITE>
__global__ void __launch_bounds__(256) k_tile_lists(const uint64_t* __restrict__ spairs, const uint2* __restrict__ sranges,
                                                    const ushort4* __restrict__ rect, const float* __restrict__ depth,
                                                    uint32_t n, int tiles_x, int ks, int stiles_x,
                                                    uint32_t* __restrict__ count,
                                                    const uint32_t* __restrict__ tile_start, uint64_t* __restrict__ keys,
                                                    uint32_t* __restrict__ vals)
{
    __shared__ int s_wcnt[8];
    const int t = blockIdx.x;
    const int tx = t % tiles_x, ty = t / tiles_x;
    const int ksh = __ffs(ks) - 1;
    const uint2 sr = sranges[(ty >> ksh) * stiles_x + (tx >> ksh)];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t base = WRITE ? tile_start[t] : 0u;
    for (uint32_t c0 = sr.x; c0 < sr.y; c0 += 256) {
        const uint32_t c = c0 + threadIdx.x;
        uint32_t id = 0xFFFFFFFFu;
        bool hit = false;
        if (c < sr.y) {
            id = (uint32_t)spairs[c];
            hit = id < n && covers(rect[id], tx, ty);
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) s_wcnt[warp] = __popc(ball);
        __syncthreads();
        int wbase = 0, tot = 0;
        for (int w = 0; w < 8; ++w) {
            wbase += w < warp ? s_wcnt[w] : 0;
            tot += s_wcnt[w];
        }
        if (WRITE && hit) {
            const uint32_t pos = base + wbase + __popc(ball & ((1u << lane) - 1u));
            if (keys) keys[pos] = ((uint64_t)t << 32) | (uint64_t)__float_as_uint(depth[id]);
            if (vals) vals[pos] = id;
        }
        base += tot;
        __syncthreads();
    }
    if (!WRITE && threadIdx.x == 0) count[t] = base;
}

// single-block exclusive scan of the per-tile counts -> starts and [start, end) ranges
__global__ void __launch_bounds__(1024) k_tile_starts(const uint32_t* __restrict__ count, uint32_t T,
                                                      uint32_t* __restrict__ start, uint2* __restrict__ ranges)
{
    __shared__ uint32_t s_warp[32];
    uint32_t carry = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t b0 = 0; b0 < T; b0 += 1024) {
        const uint32_t i = b0 + threadIdx.x;
        const uint32_t v = i < T ? count[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t wb = 0, tot = 0;
        for (int w = 0; w < 32; ++w) {
            wb += w < warp ? s_warp[w] : 0u;
            tot += s_warp[w];
        }
        if (i < T) {
            const uint32_t st = carry + wb + x - v;
            start[i] = st;
            if (ranges) ranges[i] = v ? make_uint2(st, st + v) : make_uint2(0u, 0u);
        }
        carry += tot;
        __syncthreads();
    }
}

// One block per view of a batch: view v's tiles (start[v] .. start[v + 1] - 1
// of the batch) heaviest first, in its own stretch of the order, so that the
// blend takes the views one after another.
struct ViewStarts {
    int start[kMaxViews + 1];
};
__global__ void __launch_bounds__(1024) k_tile_order_views(const uint32_t* __restrict__ work,
                                                            const __grid_constant__ ViewStarts vs,
                                                            uint32_t* __restrict__ order)
{
    const int v = blockIdx.x;
    const uint32_t b = (uint32_t)vs.start[v], T = (uint32_t)(vs.start[v + 1] - vs.start[v]);
    tile_order_block(work + b, T, order + b, b);
}

// One block: the tiles heaviest first (tile_order.cuh).
__global__ void __launch_bounds__(1024) k_tile_order(const uint32_t* __restrict__ work, uint32_t T,
                                                      uint32_t* __restrict__ order)
{
    tile_order_block(work, T, order);
}

}  // namespace

__global__ void k_iota(uint32_t* __restrict__ ids, uint32_t n)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ids[i] = i;
}

cudaError_t launch_iota(cudaStream_t s, uint32_t* ids, uint32_t n)
{
    if (n == 0) return cudaSuccess;
    k_iota<<<(n + 255) / 256, 256, 0, s>>>(ids, n); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tile_order_views(cudaStream_t s, const uint32_t* work, const int* start, int V, uint32_t* order)
{
    if (V < 1 || V > kMaxViews) return cudaErrorInvalidValue;
    ViewStarts vs{};
    for (int v = 0; v <= V; ++v) vs.start[v] = start[v];
    k_tile_order_views<<<V, 1024, 0, s>>>(work, vs, order); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tile_order(cudaStream_t s, const uint32_t* work, uint32_t T, uint32_t* order)
{
    if (T == 0) return cudaSuccess;
    k_tile_order<<<1, 1024, 0, s>>>(work, T, order); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_emit_pairs(cudaStream_t s, const uint32_t* ids, const uint32_t* offsets, const ushort4* rect,
                              uint32_t n, int ks, int stiles_x, uint64_t* pairs, uint32_t* counts, uint32_t Ts,
                              uint32_t cap, uint32_t id_base, bool rebase)
{
    if (n == 0) return cudaSuccess;
    const bool cnt = counts && Ts <= (uint32_t)kMaxSupersForCounts;
#define GS_EMIT(C, K)                                                                                         \
    k_emit<C, K><<<(n + 255) / 256, 256, 0, s>>>(ids, offsets, rect, n, stiles_x, pairs, C ? counts : nullptr, \
                                                 C ? Ts : 0u, cap, id_base, rebase)
    if (ks == 1) {
        if (cnt) GS_EMIT(true, 1); else GS_EMIT(false, 1);
    } else if (ks == 2) {
        if (cnt) GS_EMIT(true, 2); else GS_EMIT(false, 2);
    } else {
        if (cnt) GS_EMIT(true, 4); else GS_EMIT(false, 4);
    }
#undef GS_EMIT
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_emit_views(cudaStream_t s, const EmitViews& b, const uint32_t* sorted, const uint32_t* offsets,
                              const ushort4* rect, uint32_t total, bool packed)
{
    if (total == 0 || b.V <= 0) return cudaSuccess;
    k_emit_views<<<(total + 255) / 256, 256, 0, s>>>(b, sorted, offsets, rect, total,
                                                   packed ? kPackedIdxMask : 0xFFFFFFFFu);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ranges(cudaStream_t s, const uint64_t* pairs, uint32_t P, uint32_t T, uint2* ranges)
{
    if (P == 0) return cudaSuccess;
    k_ranges<<<(P + 255) / 256, 256, 0, s>>>(pairs, P, T, ranges); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tile_lists(cudaStream_t s, const uint64_t* spairs, const uint2* sranges, const ushort4* rect,
                              const float* depth, uint32_t n, int tiles_x, int tiles_y, int ks, int stiles_x,
                              uint32_t* count, uint32_t* start, uint64_t* keys, uint32_t* vals, uint2* ranges)
{
    const int T = tiles_x * tiles_y;
    k_tile_lists<false><<<T, 256, 0, s>>>(spairs, sranges, rect, depth, n, tiles_x, ks, stiles_x, count, nullptr,
                                          nullptr, nullptr); note_launch();
    k_tile_starts<<<1, 1024, 0, s>>>(count, (uint32_t)T, start, ranges); note_launch();
    if (keys || vals) {
        k_tile_lists<true><<<T, 256, 0, s>>>(spairs, sranges, rect, depth, n, tiles_x, ks, stiles_x, count, start,
                                             keys, vals); note_launch();
    }
    return cudaGetLastError();
}

}  // namespace gs
