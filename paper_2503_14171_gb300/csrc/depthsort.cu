// Front-to-back order of the Gaussians (Sec. 4: Gaussians are blended sorted
// by depth) and the pair offsets in that order, in one persistent launch.
//
// For up to kDsMaxSlice Gaussians per SM the whole sort runs as a single
// cooperative kernel, one 1024-thread block per SM, each block owning a
// contiguous slice of the sequence.
//
// Key range.  Every visible depth is a positive FP32 value, and the order of
// positive FP32 values is that of their bit patterns, so subtracting the
// smallest visible key keeps the order; the keys of the Gaussians that emit no
// pair (0xFFFFFFFF) go last.  Once the slice is loaded, each block publishes
// the range of its visible keys, and after one grid barrier every block knows
// the whole range: when it spans fewer than 2^27 - 1 values (16 binades, a
// depth ratio up to 65536) the biased keys fit 27 bits and three passes of 9
// bits sort them, otherwise four.
//
// Each pass is a stable LSD pass over a 9-bit digit (ids in ascending order
// ride along): stage the slice, rank it by digit with one ballot per digit bit
// and per-warp running counters (stable), reorder it by digit in shared
// memory, publish the block's digit counts (and add them to the digit
// totals), grid barrier, derive the global offset of each of the block's digit
// runs, write the runs out (coalesced), grid barrier.
// The exclusive scan of supers_touched[id] in the sorted order (each
// Gaussian's first pair slot) rides on the last pass: a Gaussian's slot is
// the pair count of every Gaussian before it in the final order, i.e. of the
// lower digits (all blocks), of the same digit in earlier blocks, and of its
// own digit run before it.  So the last pass also scans the pair counts of
// its reordered slice and publishes their per-digit sums beside the digit
// counts; after its one grid barrier each block derives its runs' pair-slot
// bases exactly as it derives their positions, and writes the offsets with
// the ids (no barrier after it).  The passes alternate between the two
// buffers so that the last one always writes ids[1].
// This replaces a histogram kernel, four one-sweep passes and a scan kernel
// (seven launches whose time is dominated by latency at this size) with one.
//
// Grid barriers spin at most kGridSpinLimit times; on expiry the block records
// kDevTimeout in the error word and carries on (outputs undefined, no hang).
#include <atomic>
#include <mutex>

#include <cooperative_groups.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kDsThreads = 1024;
constexpr int kDsWarps = kDsThreads / 32;
constexpr int kDsBits = 9;
constexpr int kDsRadix = 1 << kDsBits;
constexpr int kDsMaxPasses = 4;                    // 36 bits: any 32-bit key
constexpr uint32_t kCulled = 0xFFFFFFFFu;          // key of a Gaussian that emits no pair
constexpr uint32_t kCulled3 = (1u << (3 * kDsBits)) - 1u;   // its biased key when three passes suffice
constexpr long kGridSpinLimit = 1L << 22;
constexpr int kDsPer = kDsMaxSlice / kDsThreads;   // slice elements per thread
static_assert(kDsTotWords == (kDsMaxPasses + 1) * kDsRadix, "digit totals of every pass, then the pair-count totals");
static_assert(kDsRadix == kDsRadixWords, "the scratch layout's digit count");
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
    uint32_t* cnt;               // [grid][512] per-block digit counts
    uint32_t* csum;              // [grid][512] per-block digit sums of the pair counts (last pass);
                                 // words 0, 1 of a block's row first carry its key range
    uint32_t* tot;               // [5][512] digit totals per pass, then the pair-count totals (zeroed)
    unsigned int* bar;           // [2] barrier counter and generation (zeroed); bar[2] stays zero
    int* err;
    uint32_t n;
    uint32_t inject_spins;       // > 0: block 0 first polls bar[2], which nothing sets, this many times
};

// Grid-wide barrier for a cooperative launch (all blocks resident).  Thread 0
// of each block arrives with an acquire-release add at GPU scope (it releases
// the block's writes, ordered before it by the CTA barrier, and acquires those
// of the blocks that arrived earlier); the last to arrive resets the count and
// publishes the next generation with a release add; the others poll the
// generation with acquire loads.
// Poll word (acquire loads) until it differs from `unchanged`, at most limit
// times; on expiry record kDevTimeout in the error word and return false.
__device__ __forceinline__ bool bounded_poll(const unsigned int* word, unsigned int unchanged, long limit, int* err)
{
    long spins = 0;
    unsigned int g;
    do {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(word) : "memory");
        if (g != unchanged) return true;
        if (++spins > limit) {
            atomicExch(err, kDevTimeout);
            return false;
        }
        __nanosleep(32);
    } while (true);
}

__device__ __forceinline__ void grid_barrier(unsigned int* bar, int* err)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int gen, arrived;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(bar + 1) : "memory");
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
        if (arrived == gridDim.x - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(bar) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar + 1) : "memory");
        } else {
            bounded_poll(bar + 1, gen, kGridSpinLimit, err);
        }
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
    constexpr uint32_t R = kDsRadix;

    uint32_t* s_key = reinterpret_cast<uint32_t*>(smem);
    uint32_t* s_id = s_key + kDsMaxSlice;
    uint32_t* s_key2 = s_id + kDsMaxSlice;                            // slice reordered by digit
    uint32_t* s_id2 = s_key2 + kDsMaxSlice;
    uint16_t* s_rank = reinterpret_cast<uint16_t*>(s_id2 + kDsMaxSlice);
    uint16_t* s_wcnt = s_rank + kDsMaxSlice;                          // [kDsWarps][R]
    uint32_t* s_off = reinterpret_cast<uint32_t*>(s_wcnt + kDsWarps * R);   // [R]
    uint32_t* s_boff = s_off + R;                                     // [R] block-local digit starts
    uint32_t* s_wtot = s_boff + R;                                    // [kDsWarps]
    // last pass only (s_rank is free once the slice is reordered): pair-count
    // scan value at each digit run's start, and each run's first pair slot
    // minus that value
    uint32_t* s_cbase = reinterpret_cast<uint32_t*>(s_rank);          // [R]
    uint32_t* s_obase = s_cbase + R;                                  // [R]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;

    // fault injection for the tests of the expiry path: a bounded wait for a
    // word nothing sets runs out and records kDevTimeout; the sort itself is
    // unaffected
    if (a.inject_spins && blockIdx.x == 0 && tid == 0) bounded_poll(a.bar + 2, 0u, (long)a.inject_spins, a.err);

    // ---- the slice's keys and the range of the visible ones ----
    uint32_t rk[kDsPer];
    {
        uint32_t kmin = kCulled, kmax = 0u;
#pragma unroll
        for (int k = 0; k < kDsPer; ++k) {
            const uint32_t j = tid + k * kDsThreads;
            rk[k] = kCulled;
            if (j < m) rk[k] = __ldcg(a.keys_in + lo + j);
            if (rk[k] != kCulled) {
                kmin = min(kmin, rk[k]);
                kmax = max(kmax, rk[k]);
            }
        }
        kmin = __reduce_min_sync(0xffffffffu, kmin);
        kmax = __reduce_max_sync(0xffffffffu, kmax);
        if (lane == 0) {
            s_off[warp] = kmin;
            s_off[kDsWarps + warp] = kmax;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kDsWarps; ++w) {
                kmin = min(kmin, s_off[w]);
                kmax = max(kmax, s_off[kDsWarps + w]);
            }
            a.csum[(size_t)blockIdx.x * R] = kmin;
            a.csum[(size_t)blockIdx.x * R + 1] = kmax;
        }
    }
    grid_barrier(a.bar, a.err);
    if (warp == 0) {
        uint32_t kmin = kCulled, kmax = 0u;
        for (uint32_t b = lane; b < G; b += 32) {
            kmin = min(kmin, __ldcg(a.csum + (size_t)b * R));
            kmax = max(kmax, __ldcg(a.csum + (size_t)b * R + 1));
        }
        kmin = __reduce_min_sync(0xffffffffu, kmin);
        kmax = __reduce_max_sync(0xffffffffu, kmax);
        if (lane == 0) {
            s_wtot[0] = kmin;
            s_wtot[1] = kmax;
        }
    }
    __syncthreads();
    const bool any = s_wtot[0] <= s_wtot[1];
    const uint32_t bias = any ? s_wtot[0] : 0u;
    const int P = (any ? s_wtot[1] - s_wtot[0] : 0u) < kCulled3 ? 3 : 4;
    const uint32_t culled = P == 3 ? kCulled3 : kCulled - bias;   // above every biased visible key
    __syncthreads();   // s_wtot is reused below
#pragma unroll
    for (int k = 0; k < kDsPer; ++k) {
        const uint32_t j = tid + k * kDsThreads;
        if (j < m) {
            s_key[j] = rk[k] == kCulled ? culled : rk[k] - bias;
            const uint32_t c = a.counts[lo + j];
            s_id[j] = (lo + j) | ((c < kCntEsc ? c : kCntEsc) << kIdBits);
        }
    }

    for (int pass = 0; pass < P; ++pass) {
        const bool last = pass == P - 1;
        const int shift = pass * kDsBits;
        // ping-pong buffers chosen by condition (a run-time index into the
        // parameter struct would copy it to local memory); the last pass
        // writes buffer 1
        const bool to1 = ((pass + P) & 1) != 0;
        const uint32_t* src_key = to1 ? a.keys[0] : a.keys[1];
        const uint32_t* src_id = to1 ? a.ids[0] : a.ids[1];
        uint32_t* dst_key = to1 ? a.keys[1] : a.keys[0];
        uint32_t* dst_id = to1 ? a.ids[1] : a.ids[0];
        for (int i = tid; i < kDsWarps * (int)R; i += kDsThreads) s_wcnt[i] = 0;
        // stage the slice in shared memory (the first pass has it already):
        // coalesced loads (L2, the previous pass's scatter by other blocks),
        // all of a thread's loads in flight at once
        if (pass > 0) {
            uint32_t ri[kDsPer];
#pragma unroll
            for (int k = 0; k < kDsPer; ++k) {
                const uint32_t j = tid + k * kDsThreads;
                if (j < m) {
                    rk[k] = __ldcg(src_key + lo + j);
                    ri[k] = __ldcg(src_id + lo + j);
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
            const uint32_t d = valid ? (s_key[j] >> shift) & (R - 1) : 0u;
            // lanes holding the same digit: one ballot per digit bit (a match
            // instruction's cost grows with the distinct digits in the warp)
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int b = 0; b < kDsBits; ++b) {
                const bool bit = (d >> b) & 1u;
                const uint32_t bal = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bal : ~bal;
            }
            uint32_t prev = 0;
            if (valid) prev = s_wcnt[warp * R + d];
            __syncwarp();
            if (valid) {
                s_rank[j] = (uint16_t)(prev + __popc(peers & lt));
                if (lane == 31 - __clz(peers)) s_wcnt[warp * R + d] = (uint16_t)(prev + __popc(peers));
            }
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive prefix over warps, the block's count (published,
        // and added to the digit total), and the block-local start of the digit
        if (tid < (int)R) {
            uint32_t run = 0;
            for (int w = 0; w < kDsWarps; ++w) {
                const uint32_t c = s_wcnt[w * R + tid];
                s_wcnt[w * R + tid] = (uint16_t)run;
                run += c;
            }
            a.cnt[(size_t)blockIdx.x * R + tid] = run;
            if (run) atomicAdd(&a.tot[pass * R + tid], run);
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
        if (tid < (int)R) {
            uint32_t wb = 0;
            for (int w = 0; w < warp; ++w) wb += s_wtot[w];
            s_boff[tid] += wb;
        }
        __syncthreads();
        // reorder the slice by digit (stable) in shared memory
        for (uint32_t j = tid; j < m; j += kDsThreads) {
            const uint32_t key = s_key[j];
            const uint32_t d = (key >> shift) & (R - 1);
            const uint32_t lp = s_boff[d] + s_wcnt[(j / cw) * R + d] + s_rank[j];
            s_key2[lp] = key;
            s_id2[lp] = s_id[j];
        }
        if (last) {
            // pair counts of the reordered slice, their exclusive scan (in
            // s_key, free now): thread t takes a contiguous run of E positions
            __syncthreads();
            const uint32_t E = (m + kDsThreads - 1) / kDsThreads;
            const uint32_t t0 = min(m, tid * E), t1 = min(m, t0 + E);
            uint32_t sum = 0;
            for (uint32_t j = t0; j < t1; ++j) {
                const uint32_t v = s_id2[j];
                uint32_t c = v >> kIdBits;
                if (c == kCntEsc) {   // escaped: look the count up
                    const uint32_t id = v & kIdMask;
                    c = id < n ? a.counts[id] : 0u;
                }
                s_key[j] = c;
                sum += c;
            }
            uint32_t x = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_wtot[warp] = x;
            __syncthreads();
            uint32_t wb = 0, btot = 0;
            for (int w = 0; w < kDsWarps; ++w) {
                const uint32_t t = s_wtot[w];
                wb += w < warp ? t : 0u;
                btot += t;
            }
            uint32_t run = wb + x - sum;
            for (uint32_t j = t0; j < t1; ++j) {
                const uint32_t c = s_key[j];
                s_key[j] = run;
                run += c;
            }
            __syncthreads();
            // per digit: the pair counts of its run (published, and added to
            // the digit's total) and the scan value at the run's start
            if (tid < (int)R) {
                const uint32_t r0 = s_boff[tid], r1 = tid + 1 < (int)R ? s_boff[tid + 1] : m;
                const uint32_t v0 = r0 < m ? s_key[r0] : btot, v1 = r1 < m ? s_key[r1] : btot;
                a.csum[(size_t)blockIdx.x * R + tid] = v1 - v0;
                if (v1 != v0) atomicAdd(&a.tot[kDsMaxPasses * R + tid], v1 - v0);
                s_cbase[tid] = v0;
            }
        }
        grid_barrier(a.bar, a.err);
        // global start of this block's run of each digit:
        // exclusive digit total + this digit's count in earlier blocks, the
        // latter summed by 2 groups of 512 threads (every other earlier block each)
        {
            uint32_t* s_part = reinterpret_cast<uint32_t*>(s_wcnt);   // [2][2][R]; s_wcnt is free here
            const uint32_t d = tid & (R - 1), g = tid / R;
            uint32_t p0 = 0, p1 = 0, q0 = 0, q1 = 0;
            uint32_t b = g;
            if (last) {   // the digit counts and the pair-count sums
                for (; b + 2 < blockIdx.x; b += 4) {
                    p0 += __ldcg(a.cnt + (size_t)b * R + d);
                    p1 += __ldcg(a.cnt + (size_t)(b + 2) * R + d);
                    q0 += __ldcg(a.csum + (size_t)b * R + d);
                    q1 += __ldcg(a.csum + (size_t)(b + 2) * R + d);
                }
                if (b < blockIdx.x) {
                    p0 += __ldcg(a.cnt + (size_t)b * R + d);
                    q0 += __ldcg(a.csum + (size_t)b * R + d);
                }
                s_part[2 * R + g * R + d] = q0 + q1;
            } else {
                for (; b + 2 < blockIdx.x; b += 4) {
                    p0 += __ldcg(a.cnt + (size_t)b * R + d);
                    p1 += __ldcg(a.cnt + (size_t)(b + 2) * R + d);
                }
                if (b < blockIdx.x) p0 += __ldcg(a.cnt + (size_t)b * R + d);
            }
            s_part[g * R + d] = p0 + p1;
        }
        __syncthreads();
        if (tid < (int)R) {
            const uint32_t* s_part = reinterpret_cast<const uint32_t*>(s_wcnt);
            const uint32_t tot = __ldcg(a.tot + pass * R + tid);
            const uint32_t pre = s_part[tid] + s_part[R + tid];
            uint32_t x = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_wtot[warp] = x;
            s_off[tid] = pre + x - tot - s_boff[tid];   // completed below with earlier warps' totals
            if (last) {
                // first pair slot of this block's run of digit tid, minus the
                // run's start in the slice's pair-count scan
                const uint32_t cpre = s_part[2 * R + tid] + s_part[3 * R + tid];
                const uint32_t ctot = __ldcg(a.tot + kDsMaxPasses * R + tid);
                uint32_t xc = ctot;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, xc, o);
                    if (lane >= o) xc += y;
                }
                if (lane == 31) s_wtot[R / 32 + warp] = xc;
                s_obase[tid] = cpre + xc - ctot - s_cbase[tid];   // completed below likewise
            }
        }
        __syncthreads();
        if (tid < (int)R) {
            uint32_t wb = 0;
            for (int w = 0; w < warp; ++w) wb += s_wtot[w];
            s_off[tid] += wb;
            if (last) {
                uint32_t wc = 0, all = 0;
                for (int w = 0; w < (int)R / 32; ++w) {
                    const uint32_t t = s_wtot[R / 32 + w];
                    wc += w < warp ? t : 0u;
                    all += t;
                }
                s_obase[tid] += wc;
                if (blockIdx.x == 0 && tid == 0) a.offsets[n] = all;   // the pair total
            }
        }
        __syncthreads();
        // write the digit runs out: consecutive threads, consecutive addresses
        for (uint32_t j = tid; j < m; j += kDsThreads) {
            const uint32_t key = s_key2[j];
            const uint32_t d = (key >> shift) & (R - 1);
            const uint32_t pos = s_off[d] + j;
            if (pos < n) {
                const uint32_t v = s_id2[j];
                if (!last) {
                    dst_key[pos] = key;
                    dst_id[pos] = v;
                } else {   // last pass: plain ids and their first pair slots
                    dst_id[pos] = v & kIdMask;
                    a.offsets[pos] = s_obase[d] + s_key[j];
                }
            }
        }
        if (!last) grid_barrier(a.bar, a.err);
    }
}

// Grid of the persistent sort on each device (its SM count, or 0 when one
// block per SM does not fit), computed once per device.  The cache is one
// atomic word per device (-1 = not yet known): concurrent first calls from
// several host threads compute the same value, and a reader never sees a
// value that belongs to another device.
constexpr int kDsMaxDevices = 64;
std::atomic<int> g_ds_grid[kDsMaxDevices] = {};
std::atomic<bool> g_ds_grid_init{false};
std::mutex g_ds_grid_mutex;

int ds_grid(int device)
{
    if (device < 0 || device >= kDsMaxDevices) return 0;
    if (!g_ds_grid_init.load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lock(g_ds_grid_mutex);
        if (!g_ds_grid_init.load(std::memory_order_relaxed)) {
            for (auto& v : g_ds_grid) v.store(-1, std::memory_order_relaxed);
            g_ds_grid_init.store(true, std::memory_order_release);
        }
    }
    const int known = g_ds_grid[device].load(std::memory_order_acquire);
    if (known >= 0) return known;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    const size_t smem = depth_sort_smem_bytes();
    if (cudaFuncSetAttribute(k_depth_sort_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_depth_sort_scan, kDsThreads, smem) != cudaSuccess)
        return 0;
    const int grid = per_sm >= 1 ? sms : 0;
    g_ds_grid[device].store(grid, std::memory_order_release);
    return grid;
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
                                   uint32_t* cnt_scratch, uint32_t* csum_scratch, unsigned int* bar,
                                   uint32_t* tot_scratch, int* err, int* out_idx, bool pre_zeroed,
                                   uint32_t inject_spins)
{
    const int G = ds_grid(device);
    if (G <= 0 || n == 0 || n > (uint32_t)G * (uint32_t)kDsMaxSlice || n > kDsMaxN) return cudaErrorInvalidValue;
    // fewer blocks for small inputs (at least 1024 elements per block)
    const uint64_t want = ((uint64_t)n + 1023) / 1024;
    const uint32_t grid = (uint32_t)(want < (uint64_t)G ? want : (uint64_t)G);
    cudaError_t e = cudaSuccess;
    if (!pre_zeroed) {
        if ((e = cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned int), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(tot_scratch, 0, sizeof(uint32_t) * kDsTotWords, s)) != cudaSuccess) return e;
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
    a.csum = csum_scratch;
    a.bar = bar;
    a.err = err;
    a.n = n;
    a.inject_spins = inject_spins;
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
    *out_idx = 1;   // the last pass writes ids[1]
    return e;
}

}  // namespace gs
