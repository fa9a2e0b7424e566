// Front-to-back order of the Gaussians (Sec. 4: Gaussians are blended sorted
// by depth) and the pair offsets in that order, in one persistent launch.
//
// For up to kDsMaxSlice Gaussians per SM the whole sort runs as a single
// cooperative kernel, one 1024-thread block per SM, each block owning a
// contiguous slice of the sequence:
//   4 stable LSD passes over the 8-bit digits of the FP32 depth bits (ids in
//   ascending order ride along): load the slice, rank it by digit with one
//   ballot per digit bit and per-warp running counters (stable), reorder it by
//   digit in shared memory, publish the block's digit counts (and add them to
//   the digit totals), grid barrier, derive the global offset of each of the
//   block's digit runs, write the runs out (coalesced), grid barrier;
//   then the exclusive scan of supers_touched[id] in the sorted order (block
//   sums, grid barrier, block prefixes), which gives each Gaussian's first
//   pair slot.
// This replaces a histogram kernel, four one-sweep passes and a scan kernel
// (seven launches whose time is dominated by latency at this size) with one.
//
// Grid barriers spin at most kGridSpinLimit times; on expiry the block records
// kDevTimeout in the error word and carries on (outputs undefined, no hang).
#include <cooperative_groups.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kDsThreads = 1024;
constexpr int kDsWarps = kDsThreads / 32;
constexpr int kDsRadix = 256;
constexpr int kDsPasses = 4;
constexpr long kGridSpinLimit = 1L << 22;
constexpr int kDsPer = kDsMaxSlice / kDsThreads;   // slice elements per thread
// The pair count of each Gaussian rides along with its id through the passes:
// id in the low kIdBits bits, min(count, kCntEsc) above; kCntEsc means "look
// the count up" (rare: a Gaussian over 2047 super-tiles).
constexpr int kIdBits = 21;
constexpr uint32_t kIdMask = (1u << kIdBits) - 1u;
static_assert(kDsMaxN == kIdMask, "the persistent sort's size limit is the id field");
constexpr uint32_t kCntEsc = (1u << (32 - kIdBits)) - 1u;
static_assert(kDsPer * kDsThreads == kDsMaxSlice, "the slice is a whole number of elements per thread");

struct DsArgs {
    const uint32_t* keys_in;     // [n] depth keys in id order
    uint32_t* keys[2];           // ping-pong
    uint32_t* ids[2];
    const uint32_t* counts;      // [n] pair count per Gaussian (by id)
    uint32_t* offsets;           // [n + 1] exclusive scan in depth order
    uint32_t* cnt;               // [grid][256] per-block digit counts
    uint32_t* tot;               // [4][256] digit totals per pass (zeroed)
    unsigned long long* bsum;    // [grid] per-block count sums
    unsigned int* bar;           // [2] barrier counter and generation (zeroed)
    int* err;
    uint32_t n;
};

// Grid-wide barrier for a cooperative launch (all blocks resident).
__device__ __forceinline__ void grid_barrier(unsigned int* bar, int* err)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = bar + 1;
        const unsigned int gen = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long spins = 0;
            while (*vgen == gen) {
                if (++spins > kGridSpinLimit) {
                    atomicExch(err, kDevTimeout);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kDsThreads, 1) k_depth_sort_scan(DsArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t n = a.n;
    const uint32_t G = gridDim.x;
    const uint32_t slice = (n + G - 1) / G;
    const uint32_t lo = blockIdx.x * slice;
    const uint32_t hi = min(n, lo + slice);
    const uint32_t m = hi > lo ? hi - lo : 0u;
    const uint32_t cw = (m + kDsWarps - 1) / kDsWarps;   // elements per warp chunk

    uint32_t* s_key = reinterpret_cast<uint32_t*>(smem);
    uint32_t* s_id = s_key + kDsMaxSlice;
    uint32_t* s_key2 = s_id + kDsMaxSlice;                            // slice reordered by digit
    uint32_t* s_id2 = s_key2 + kDsMaxSlice;
    uint16_t* s_rank = reinterpret_cast<uint16_t*>(s_id2 + kDsMaxSlice);
    uint16_t* s_wcnt = s_rank + kDsMaxSlice;                          // [kDsWarps][256]
    uint32_t* s_off = reinterpret_cast<uint32_t*>(s_wcnt + kDsWarps * kDsRadix);   // [256]
    uint32_t* s_boff = s_off + kDsRadix;                              // [256] block-local digit starts
    uint32_t* s_wtot = s_boff + kDsRadix;                             // [kDsWarps]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;

    for (int pass = 0; pass < kDsPasses; ++pass) {
        const int shift = pass * 8;
        // ping-pong buffers chosen by condition (a run-time index into the
        // parameter struct would copy it to local memory)
        const bool odd = pass & 1;
        const uint32_t* src_key = pass == 0 ? a.keys_in : (odd ? a.keys[0] : a.keys[1]);
        const uint32_t* src_id = pass == 0 ? nullptr : (odd ? a.ids[0] : a.ids[1]);
        uint32_t* dst_key = odd ? a.keys[1] : a.keys[0];
        uint32_t* dst_id = odd ? a.ids[1] : a.ids[0];
        for (int i = tid; i < kDsWarps * kDsRadix; i += kDsThreads) s_wcnt[i] = 0;
        // stage the slice in shared memory: coalesced loads (L2, the previous
        // pass's scatter by other blocks), all of a thread's loads in flight at once
        {
            uint32_t rk[kDsPer], ri[kDsPer];
#pragma unroll
            for (int k = 0; k < kDsPer; ++k) {
                const uint32_t j = tid + k * kDsThreads;
                if (j < m) {
                    rk[k] = __ldcg(src_key + lo + j);
                    if (pass == 0) {
                        const uint32_t c = a.counts[lo + j];
                        ri[k] = (lo + j) | ((c < kCntEsc ? c : kCntEsc) << kIdBits);
                    } else {
                        ri[k] = __ldcg(src_id + lo + j);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kDsPer; ++k) {
                const uint32_t j = tid + k * kDsThreads;
                if (j < m) {
                    s_key[j] = rk[k];
                    s_id[j] = ri[k];
                }
            }
        }
        __syncthreads();
        // stable ranking: warp w ranks its chunk [w cw, (w+1) cw) 32 elements at a time
        const uint32_t wlo = warp * cw, whi = min(m, wlo + cw);
        for (uint32_t base = wlo; base < whi; base += 32) {
            const uint32_t j = base + lane;
            const bool valid = j < whi;
            const uint32_t d = valid ? (s_key[j] >> shift) & 0xFFu : 0u;
            // lanes holding the same digit: one ballot per digit bit (a match
            // instruction's cost grows with the distinct digits in the warp)
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const bool bit = (d >> b) & 1u;
                const uint32_t bal = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bal : ~bal;
            }
            uint32_t prev = 0;
            if (valid) prev = s_wcnt[warp * kDsRadix + d];
            __syncwarp();
            if (valid) {
                s_rank[j] = (uint16_t)(prev + __popc(peers & lt));
                if (lane == 31 - __clz(peers)) s_wcnt[warp * kDsRadix + d] = (uint16_t)(prev + __popc(peers));
            }
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive prefix over warps, the block's count (published,
        // and added to the digit total), and the block-local start of the digit
        if (tid < kDsRadix) {
            uint32_t run = 0;
            for (int w = 0; w < kDsWarps; ++w) {
                const uint32_t c = s_wcnt[w * kDsRadix + tid];
                s_wcnt[w * kDsRadix + tid] = (uint16_t)run;
                run += c;
            }
            a.cnt[(size_t)blockIdx.x * kDsRadix + tid] = run;
            if (run) atomicAdd(&a.tot[pass * kDsRadix + tid], run);
            uint32_t x = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_wtot[warp] = x;
            s_boff[tid] = x - run;
        }
        __syncthreads();
        if (tid < kDsRadix) {
            uint32_t wb = 0;
            for (int w = 0; w < warp; ++w) wb += s_wtot[w];
            s_boff[tid] += wb;
        }
        __syncthreads();
        // reorder the slice by digit (stable) in shared memory
        for (uint32_t j = tid; j < m; j += kDsThreads) {
            const uint32_t key = s_key[j];
            const uint32_t d = (key >> shift) & 0xFFu;
            const uint32_t lp = s_boff[d] + s_wcnt[(j / cw) * kDsRadix + d] + s_rank[j];
            s_key2[lp] = key;
            s_id2[lp] = s_id[j];
        }
        grid_barrier(a.bar, a.err);
        // global start of this block's run of each digit:
        // exclusive digit total + this digit's count in earlier blocks, the
        // latter summed by 4 groups of 256 threads (every 4th earlier block each)
        {
            uint32_t* s_part = reinterpret_cast<uint32_t*>(s_wcnt);   // [4][256]; s_wcnt is free here
            const uint32_t d = tid & (kDsRadix - 1), g = tid / kDsRadix;
            uint32_t p0 = 0, p1 = 0;
            uint32_t b = g;
            for (; b + 4 < blockIdx.x; b += 8) {
                p0 += __ldcg(a.cnt + (size_t)b * kDsRadix + d);
                p1 += __ldcg(a.cnt + (size_t)(b + 4) * kDsRadix + d);
            }
            if (b < blockIdx.x) p0 += __ldcg(a.cnt + (size_t)b * kDsRadix + d);
            s_part[g * kDsRadix + d] = p0 + p1;
        }
        __syncthreads();
        if (tid < kDsRadix) {
            const uint32_t* s_part = reinterpret_cast<const uint32_t*>(s_wcnt);
            const uint32_t tot = __ldcg(a.tot + pass * kDsRadix + tid);
            const uint32_t pre = s_part[tid] + s_part[kDsRadix + tid] + s_part[2 * kDsRadix + tid] +
                                 s_part[3 * kDsRadix + tid];
            uint32_t x = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_wtot[warp] = x;
            s_off[tid] = pre + x - tot - s_boff[tid];   // completed below with earlier warps' totals
        }
        __syncthreads();
        if (tid < kDsRadix) {
            uint32_t wb = 0;
            for (int w = 0; w < warp; ++w) wb += s_wtot[w];
            s_off[tid] += wb;
        }
        __syncthreads();
        // write the digit runs out: consecutive threads, consecutive addresses
        for (uint32_t j = tid; j < m; j += kDsThreads) {
            const uint32_t key = s_key2[j];
            const uint32_t pos = s_off[(key >> shift) & 0xFFu] + j;
            if (pos < n) {
                const uint32_t v = s_id2[j];
                if (pass + 1 < kDsPasses) {
                    dst_key[pos] = key;
                    dst_id[pos] = v;
                } else {   // last pass: plain ids, and the counts in sorted order in the free key buffer
                    dst_id[pos] = v & kIdMask;
                    dst_key[pos] = v >> kIdBits;
                }
            }
        }
        grid_barrier(a.bar, a.err);
    }

    // exclusive scan of counts[id] over the sorted slice.  Stage the sorted ids
    // and their gathered counts in shared memory (independent loads), then
    // thread t scans a contiguous run of E = ceil(m / 1024) positions.
    const uint32_t* sorted = ((kDsPasses - 1) & 1) ? a.ids[1] : a.ids[0];
    const uint32_t* sorted_cnt = ((kDsPasses - 1) & 1) ? a.keys[1] : a.keys[0];
    uint32_t* s_cnt = s_key;   // reuse
    {
        uint32_t rc[kDsPer];
#pragma unroll
        for (int k = 0; k < kDsPer; ++k) {
            const uint32_t j = tid + k * kDsThreads;
            rc[k] = j < m ? __ldcg(sorted_cnt + lo + j) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kDsPer; ++k) {
            const uint32_t j = tid + k * kDsThreads;
            if (j < m) {
                uint32_t c = rc[k];
                if (c == kCntEsc) {   // escaped: look the count up
                    const uint32_t id = __ldcg(sorted + lo + j);
                    c = id < n ? a.counts[id] : 0u;
                }
                s_cnt[j] = c;
            }
        }
    }
    __syncthreads();
    const uint32_t E = (m + kDsThreads - 1) / kDsThreads;
    const uint32_t t0 = min(m, tid * E), t1 = min(m, t0 + E);
    unsigned long long sum = 0;
    for (uint32_t j = t0; j < t1; ++j) sum += s_cnt[j];
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __shared__ unsigned long long s_w64[kDsWarps];
    if (lane == 31) s_w64[warp] = x;
    __syncthreads();
    unsigned long long wb = 0, btot = 0;
    for (int w = 0; w < kDsWarps; ++w) {
        const unsigned long long t = s_w64[w];
        wb += w < warp ? t : 0ull;
        btot += t;
    }
    if (tid == 0) a.bsum[blockIdx.x] = btot;
    // block-local exclusive prefixes, in place (s_id is free again)
    uint32_t run = (uint32_t)(wb + x - sum);
    for (uint32_t j = t0; j < t1; ++j) {
        const uint32_t c = s_cnt[j];
        s_id[j] = run;
        run += c;
    }
    grid_barrier(a.bar, a.err);
    // one warp reads the block sums (lane-strided) and broadcasts the prefix:
    // every thread reading them would hammer the same few L2 lines
    if (warp == 0) {
        unsigned long long bpre = 0, all = 0;
        for (uint32_t b = lane; b < G; b += 32) {
            const unsigned long long v = __ldcg(a.bsum + b);
            bpre += b < blockIdx.x ? v : 0ull;
            all += v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bpre += __shfl_xor_sync(0xffffffffu, bpre, o);
            all += __shfl_xor_sync(0xffffffffu, all, o);
        }
        if (lane == 0) {
            s_w64[0] = bpre;
            s_w64[1] = all;
        }
    }
    __syncthreads();
    const uint32_t bp = (uint32_t)s_w64[0];
    const unsigned long long all = s_w64[1];
#pragma unroll 4
    for (uint32_t j = tid; j < m; j += kDsThreads) a.offsets[lo + j] = bp + s_id[j];
    if (blockIdx.x == G - 1 && tid == 0) a.offsets[n] = (uint32_t)all;
}

int ds_grid(int device)
{
    static int cached_dev = -1, cached = 0;
    if (cached_dev == device) return cached;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    const size_t smem = depth_sort_smem_bytes();
    if (cudaFuncSetAttribute(k_depth_sort_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_depth_sort_scan, kDsThreads, smem) != cudaSuccess)
        return 0;
    cached_dev = device;
    cached = per_sm >= 1 ? sms : 0;
    return cached;
}

}  // namespace

size_t depth_sort_smem_bytes()
{
    return (size_t)kDsMaxSlice * (4 * 4 + 2) + (size_t)kDsWarps * kDsRadix * 2 + 2 * kDsRadix * 4 + kDsWarps * 4;
}

uint32_t depth_sort_capacity(int device)
{
    return (uint32_t)ds_grid(device) * (uint32_t)kDsMaxSlice;
}

cudaError_t launch_depth_sort_scan(cudaStream_t s, int device, const uint32_t* keys_in, uint32_t* keys[2],
                                   uint32_t* ids[2], const uint32_t* counts, uint32_t n, uint32_t* offsets,
                                   uint32_t* cnt_scratch, unsigned long long* bsum_scratch, unsigned int* bar,
                                   uint32_t* tot_scratch, int* err, int* out_idx, bool pre_zeroed)
{
    const int G = ds_grid(device);
    if (G <= 0 || n == 0 || n > (uint32_t)G * (uint32_t)kDsMaxSlice || n > kDsMaxN) return cudaErrorInvalidValue;
    // fewer blocks for small inputs (at least 1024 elements per block)
    const uint64_t want = ((uint64_t)n + 1023) / 1024;
    const uint32_t grid = (uint32_t)(want < (uint64_t)G ? want : (uint64_t)G);
    cudaError_t e = cudaSuccess;
    if (!pre_zeroed) {
        if ((e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(tot_scratch, 0, sizeof(uint32_t) * kDsPasses * kDsRadix, s)) != cudaSuccess) return e;
    }
    DsArgs a;
    a.keys_in = keys_in;
    a.keys[0] = keys[0] == keys_in ? keys[1] : keys[0];
    a.keys[1] = keys[0] == keys_in ? keys[0] : keys[1];
    a.ids[0] = ids[0];
    a.ids[1] = ids[1];
    a.counts = counts;
    a.offsets = offsets;
    a.cnt = cnt_scratch;
    a.tot = tot_scratch;
    a.bsum = bsum_scratch;
    a.bar = bar;
    a.err = err;
    a.n = n;
    // a cooperative launch (all blocks co-resident, checked against the
    // occupancy above); launched through cudaLaunchKernelEx so that it can be
    // recorded in a CUDA graph
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kDsThreads);
    cfg.dynamicSmemBytes = depth_sort_smem_bytes();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_depth_sort_scan, a);
    note_launch();
    *out_idx = (kDsPasses - 1) & 1;
    return e;
}

}  // namespace gs
