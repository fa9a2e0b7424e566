// Heaviest tiles first: the order in which the blend takes its tiles, from the
// durations its blocks recorded in the previous frame (a bucket sort in
// logarithmic buckets, four per octave).  Any permutation gives the same
// images; this one shortens the tail of the launch.  One block of any size.
#pragma once
#include <cstdint>

namespace gs {

constexpr int kOrderBuckets = 128;
static_assert(kOrderBuckets % 32 == 0, "buckets are scanned by one warp, a whole number per lane");

// order[0 .. T) receives base + the tile indices 0 .. T - 1, heaviest first
__device__ __forceinline__ void tile_order_block(const uint32_t* __restrict__ work, uint32_t T,
                                                 uint32_t* __restrict__ order, uint32_t base = 0)
{
    __shared__ uint32_t s_cnt[kOrderBuckets];
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    auto bucket = [](uint32_t w) {   // 4 per octave, heaviest = 0
        const int b = w ? (int)(4.f * log2f((float)w)) : 0;
        return kOrderBuckets - 1 - min(b, kOrderBuckets - 1);
    };
    for (uint32_t t = threadIdx.x; t < T; t += blockDim.x) atomicAdd(&s_cnt[bucket(work[t])], 1u);
    __syncthreads();
    if (threadIdx.x < 32) {   // exclusive scan of the buckets: 4 per lane, then across the warp
        constexpr int kPer = kOrderBuckets / 32;
        const int lane = threadIdx.x;
        uint32_t c[kPer], sum = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            c[k] = s_cnt[lane * kPer + k];
            sum += c[k];
        }
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        uint32_t run = x - sum;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            s_cnt[lane * kPer + k] = run;
            run += c[k];
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < T; t += blockDim.x) order[atomicAdd(&s_cnt[bucket(work[t])], 1u)] = base + t;
}

}  // namespace gs
