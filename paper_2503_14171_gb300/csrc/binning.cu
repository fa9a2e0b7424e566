// Tile binning (the front-to-back ordering of Sec. 4, per tile).
//
// Gaussians are first sorted by the FP32 bits of their view depth (a stable
// radix sort of n keys, ids ascending), then each one emits (tile << 32 | id)
// for every tile of its rect, in depth order.  A stable radix sort on the tile
// bits alone then yields the pairs ordered by (tile, depth, id): the per-tile
// lists the blend walks front to back.  Sorting n depths once and only the
// tile bits of the P pairs moves ~4x fewer bytes than sorting P 64-bit
// (tile, depth) keys with values.
#include "gs_internal.cuh"

namespace gs {
namespace {

__global__ void __launch_bounds__(256) k_emit(const uint32_t* __restrict__ ids, const uint32_t* __restrict__ offsets,
                                              const int4* __restrict__ rect, uint32_t n, int tiles_x,
                                              uint64_t* __restrict__ pairs)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    uint32_t off = offsets[k];
    const uint32_t end = offsets[k + 1];
    if (off == end) return;
    const uint32_t id = ids[k];
    if (id >= n) return;   // only after an expired bounded wait in the sort
    const int4 r = rect[id];
    for (int ty = r.y; ty <= r.w; ++ty)
        for (int tx = r.x; tx <= r.z && off < end; ++tx) {
            const uint64_t t = (uint64_t)(ty * tiles_x + tx);
            pairs[off++] = (t << 32) | id;
        }
}

__global__ void __launch_bounds__(256) k_ranges(const uint64_t* __restrict__ pairs, uint32_t P, uint32_t T,
                                                uint2* __restrict__ ranges)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const uint32_t t = (uint32_t)(pairs[i] >> 32);
    if (t >= T) return;   // only after an expired bounded wait in the sort
    if (i == 0 || (uint32_t)(pairs[i - 1] >> 32) != t) ranges[t].x = i;
    if (i == P - 1 || (uint32_t)(pairs[i + 1] >> 32) != t) ranges[t].y = i + 1;
}

__global__ void __launch_bounds__(256) k_finalize(const uint64_t* __restrict__ pairs, uint32_t P, uint32_t n,
                                                  const float* __restrict__ depth, uint64_t* __restrict__ keys,
                                                  uint32_t* __restrict__ vals)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const uint64_t p = pairs[i];
    const uint32_t id = (uint32_t)p;
    const uint32_t dbits = id < n ? __float_as_uint(depth[id]) : 0xFFFFFFFFu;
    if (keys) keys[i] = (p & 0xFFFFFFFF00000000ull) | (uint64_t)dbits;
    if (vals) vals[i] = id;
}

}  // namespace

cudaError_t launch_emit_pairs(cudaStream_t s, const uint32_t* ids, const uint32_t* offsets, const int4* rect,
                              uint32_t n, int tiles_x, uint64_t* pairs)
{
    if (n == 0) return cudaSuccess;
    k_emit<<<(n + 255) / 256, 256, 0, s>>>(ids, offsets, rect, n, tiles_x, pairs); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tile_ranges(cudaStream_t s, const uint64_t* pairs, uint32_t P, uint32_t T, uint2* ranges)
{
    if (P == 0) return cudaSuccess;
    k_ranges<<<(P + 255) / 256, 256, 0, s>>>(pairs, P, T, ranges); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_finalize_bins(cudaStream_t s, const uint64_t* pairs, uint32_t P, uint32_t n, const float* depth,
                                 uint64_t* keys, uint32_t* vals)
{
    if (P == 0) return cudaSuccess;
    k_finalize<<<(P + 255) / 256, 256, 0, s>>>(pairs, P, n, depth, keys, vals); note_launch();
    return cudaGetLastError();
}

}  // namespace gs
