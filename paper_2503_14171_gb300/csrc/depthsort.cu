// Front-to-back order of the Gaussians (Sec. 4: Gaussians are blended sorted
// by depth) and the pair offsets in that order, in one persistent launch.
//
// For up to kDsMaxSlice Gaussians per SM the whole sort runs as a single
// cooperative kernel, one 1024-thread block per SM, each block owning a
// contiguous slice of the sequence.
//
// Key range.  Every visible depth is a positive FP32 value, and the order of
// positive FP32 values is that of their bit patterns, so subtracting the
// smallest visible key keeps the order.  The Gaussians that emit no pair (key
// 0xFFFFFFFF) go last in id order: each takes the biased key span + 1 + id,
// above every visible one.  Once the slice is loaded, each block publishes
// the range of its visible keys, and after one grid barrier every block knows
// the whole range: when span + n fits 27 bits (up to 16 binades of depth,
// less the Gaussian count) three passes of 9 bits sort the biased keys,
// otherwise four.
//
// Each pass is a stable LSD pass over a 9-bit digit (ids in ascending order
// ride along): stage the slice, rank it by digit (stable: per-warp lane-mask
// tables built with shared-memory atomics, per-warp running counters),
// reorder it by digit in shared memory, publish the
// block's digit counts (and add them to the digit totals), grid barrier,
// derive the global offset of each of the block's digit runs, write the runs
// out (coalesced), grid barrier.
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
constexpr long kGridSpinLimit = 1L << 22;
constexpr int kDsPer = kDsMaxSlice / kDsThreads;   // slice elements per thread
static_assert(kDsWarps * kDsRadix <= 2 * kDsMaxSlice, "the rank's lane-mask tables fit in s_key2 / s_id2");
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
    unsigned int* bar;           // [0] arrival counter of the grid barrier (zeroed); bar[2] stays zero
    int* err;
    uint32_t n;
    uint32_t inject_spins;       // > 0: block 0 first polls bar[2], which nothing sets, this many times
};

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

// Grid-wide barrier for a cooperative launch (all blocks resident): an
// arrival counter that only grows during the launch (zeroed before it), so
// that the k-th barrier is passed once it reaches k * gridDim.x.  Thread 0 of
// each block arrives with a release add at GPU scope (releasing the block's
// writes, ordered before it by the CTA barrier) and polls the counter with
// acquire loads.  The adds form one chain of read-modify-writes, so the load
// that reads the last arrival's value acquires the writes released by every
// earlier arrival.  One round trip to L2 per barrier, where a reset counter
// and a separate generation word take two.
__device__ __forceinline__ void grid_barrier(unsigned int* bar, unsigned int& target, int* err)
{
    __syncthreads();
    target += gridDim.x;
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        long spins = 0;
        unsigned int c;
        do {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(bar) : "memory");
            if ((int)(c - target) >= 0) break;
            if (++spins > kGridSpinLimit) {
                atomicExch(err, kDevTimeout);
                break;
            }
            __nanosleep(32);
        } while (true);
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
    uint16_t* s_wcnt = reinterpret_cast<uint16_t*>(s_id2 + kDsMaxSlice);   // [kDsWarps][R]
    uint32_t* s_off = reinterpret_cast<uint32_t*>(s_wcnt + kDsWarps * R);   // [R]
    uint32_t* s_boff = s_off + R;                                     // [R] block-local digit starts
    // last pass only: pair-count scan value at each digit run's start, and
    // each run's first pair slot minus that value
    uint32_t* s_cbase = s_boff + R;                                   // [R]
    uint32_t* s_obase = s_cbase + R;                                  // [R]
    uint32_t* s_wtot = s_obase + R;                                   // [kDsWarps]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;

    // fault injection for the tests of the expiry path: a bounded wait for a
    // word nothing sets runs out and records kDevTimeout; the sort itself is
    // unaffected
    if (a.inject_spins && blockIdx.x == 0 && tid == 0) bounded_poll(a.bar + 2, 0u, (long)a.inject_spins, a.err);

    unsigned int bar_target = 0;   // the grid barrier's arrival count to wait for
    // ---- the slice's keys (and pair counts) and the range of the visible keys ----
    uint32_t rk[kDsPer], rc[kDsPer];
    {
        uint32_t kmin = kCulled, kmax = 0u;
#pragma unroll
        for (int k = 0; k < kDsPer; ++k) {
            const uint32_t j = tid + k * kDsThreads;
            rk[k] = kCulled;
            rc[k] = 0u;
            if (j < m) {
                rk[k] = __ldcg(a.keys_in + lo + j);
                rc[k] = __ldcg(a.counts + lo + j);
            }
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
    grid_barrier(a.bar, bar_target, a.err);
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
    // a Gaussian that emits no pair takes the key cbase + id: above every
    // biased visible key and in id order, as equal keys would sort, but
    // distinct (equal digits in a warp make the ranking's atomics collide)
    const uint32_t cbase = any ? s_wtot[1] - s_wtot[0] + 1u : 0u;
    const int P = (uint64_t)cbase + n - 1u < (1ull << (3 * kDsBits)) ? 3 : 4;
    __syncthreads();   // s_wtot is reused below
#pragma unroll
    for (int k = 0; k < kDsPer; ++k) {
        const uint32_t j = tid + k * kDsThreads;
        if (j < m) {
            s_key[j] = rk[k] == kCulled ? cbase + lo + j : rk[k] - bias;
            s_id[j] = (lo + j) | ((rc[k] < kCntEsc ? rc[k] : kCntEsc) << kIdBits);
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
        for (int i = tid; i < kDsWarps * (int)R / 8; i += kDsThreads) reinterpret_cast<uint4*>(s_wcnt)[i] = make_uint4(0, 0, 0, 0);
        for (int i = tid; i < kDsWarps * (int)R / 4; i += kDsThreads)   // the rank's lane-mask tables
            reinterpret_cast<uint4*>(s_key2)[i] = make_uint4(0, 0, 0, 0);
        if (last && tid < (int)R) s_off[tid] = 0u;   // the last pass's per-digit pair-count sums
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
        // stable ranking: warp w ranks its chunk [w cw, (w+1) cw), at most
        // kDsPer groups of 32 (cw <= kDsMaxSlice / 32), in order.  The lanes
        // of a group that hold the same digit are found through a per-warp
        // table of lane masks, one word per digit (in s_key2 / s_id2, free
        // until the reorder, zeroed above): each lane ORs its bit into its
        // digit's word and reads the word back.  (Warp votes cost one ballot
        // per digit bit and a match instruction's cost grows with the
        // distinct digits in the warp; both run far below the shared-memory
        // atomics' rate.)  The highest lane of each digit then reads the
        // warp's running count of the digit, passes it to its peers, writes
        // it back advanced and clears the digit's word.  Each lane keeps its
        // digit and rank in dr (digit | rank << 16) for the reorder below.
        const uint32_t wlo = warp * cw, whi = min(m, wlo + cw);
        uint32_t* s_mask = s_key2 + warp * R;
        uint32_t dr[kDsPer];
#pragma unroll
        for (int g = 0; g < kDsPer; ++g) {
            if (wlo + g * 32 < whi) {   // warp-uniform
                const uint32_t j = wlo + g * 32 + lane;
                const bool valid = j < whi;
                const uint32_t d = valid ? (s_key[j] >> shift) & (R - 1) : 0u;
                if (valid) atomicOr(s_mask + d, 1u << lane);
                __syncwarp();
                const uint32_t peers = valid ? s_mask[d] : (1u << lane);   // an idle lane leads itself
                __syncwarp();   // every lane has read its word before the leaders clear it
                const int leader = 31 - __clz(peers);
                uint32_t prev = 0;
                if (valid && lane == leader) {
                    prev = s_wcnt[warp * R + d];
                    s_wcnt[warp * R + d] = (uint16_t)(prev + __popc(peers));
                    s_mask[d] = 0u;
                }
                prev = __shfl_sync(0xffffffffu, prev, leader);
                dr[g] = d | ((prev + __popc(peers & lt)) << 16);
                __syncwarp();   // the next group's lanes see the cleared words and the new counts
            }
        }
        // the last pass: each digit's sum of the pair counts of the block's
        // keys (s_off holds them until the barrier; a sum needs no order)
        if (last) {
#pragma unroll
            for (int g = 0; g < kDsPer; ++g) {
                const uint32_t j = wlo + g * 32 + lane;
                if (j < whi) {
                    const uint32_t v = s_id[j];
                    uint32_t c = v >> kIdBits;
                    if (c == kCntEsc) {   // escaped: look the count up
                        const uint32_t id = v & kIdMask;
                        c = id < n ? a.counts[id] : 0u;
                    }
                    if (c) atomicAdd(&s_off[dr[g] & 0xFFFFu], c);
                }
            }
        }
        __syncthreads();
        // per digit: exclusive prefix over warps, the block's count (published,
        // and added to the digit total), the last pass's pair-count sum
        // (likewise), and the block-local start of the digit
        if (tid < (int)R) {
            uint32_t run = 0;
            for (int w = 0; w < kDsWarps; ++w) {
                const uint32_t c = s_wcnt[w * R + tid];
                s_wcnt[w * R + tid] = (uint16_t)run;
                run += c;
            }
            a.cnt[(size_t)blockIdx.x * R + tid] = run;
            if (run) atomicAdd(&a.tot[pass * R + tid], run);
            if (last) {
                const uint32_t cs = s_off[tid];
                a.csum[(size_t)blockIdx.x * R + tid] = cs;
                if (cs) atomicAdd(&a.tot[kDsMaxPasses * R + tid], cs);
            }
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
        // each element's position in the block's digit-ordered slice (stable),
        // kept in dr: the reorder itself waits until after the barrier, where
        // it overlaps the loads of the cross-block prefix
#pragma unroll
        for (int g = 0; g < kDsPer; ++g) {
            const uint32_t j = wlo + g * 32 + lane;
            if (j < whi) {
                const uint32_t d = dr[g] & 0xFFFFu;
                dr[g] = s_boff[d] + s_wcnt[warp * R + d] + (dr[g] >> 16);
            }
        }
        grid_barrier(a.bar, bar_target, a.err);
        // global start of this block's run of each digit:
        // exclusive digit total + this digit's count in earlier blocks.  The
        // latter is summed with 16-byte loads: thread t takes digits
        // 4 (t mod 128) .. 4 (t mod 128) + 3 of the earlier blocks b = t / 128
        // (mod 8), four rows' loads in flight, into s_part[8][R] (and the
        // pair-count sums of the last pass into s_part[8 + 8][R]: s_wcnt is
        // free here and holds exactly these 16 R words).  The digit totals and
        // the first four rows are requested before the reorder.
        uint32_t tot = 0, ctot = 0;
        if (tid < (int)R) {
            tot = __ldcg(a.tot + pass * R + tid);
            if (last) ctot = __ldcg(a.tot + kDsMaxPasses * R + tid);
        }
        {
            uint32_t* s_part = reinterpret_cast<uint32_t*>(s_wcnt);
            const uint32_t q = tid & 127, g = tid >> 7;
            const uint4* cnt4 = reinterpret_cast<const uint4*>(a.cnt) + q;
            const uint4* csum4 = reinterpret_cast<const uint4*>(a.csum) + q;
            constexpr uint32_t RQ = R / 4;   // 16-byte words per row
            uint4 p = make_uint4(0, 0, 0, 0);
            {
                uint4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t b = g + 8 * u;
                    v[u] = b < blockIdx.x ? __ldcg(cnt4 + (size_t)b * RQ) : make_uint4(0, 0, 0, 0);
                }
                // reorder the slice by digit in shared memory, each lane
                // moving the elements it ranked
#pragma unroll
                for (int k = 0; k < kDsPer; ++k) {
                    const uint32_t j = wlo + k * 32 + lane;
                    if (j < whi) {
                        s_key2[dr[k]] = s_key[j];
                        s_id2[dr[k]] = s_id[j];
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) { p.x += v[u].x; p.y += v[u].y; p.z += v[u].z; p.w += v[u].w; }
            }
            {
                uint32_t b = g + 32;
                for (; b + 24 < blockIdx.x; b += 32) {
                    uint4 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) v[u] = __ldcg(cnt4 + (size_t)(b + 8 * u) * RQ);
#pragma unroll
                    for (int u = 0; u < 4; ++u) { p.x += v[u].x; p.y += v[u].y; p.z += v[u].z; p.w += v[u].w; }
                }
                for (; b < blockIdx.x; b += 8) {
                    const uint4 v = __ldcg(cnt4 + (size_t)b * RQ);
                    p.x += v.x; p.y += v.y; p.z += v.z; p.w += v.w;
                }
            }
            reinterpret_cast<uint4*>(s_part + g * R)[q] = p;
            if (last) {
                uint4 c = make_uint4(0, 0, 0, 0);
                uint32_t b = g;
                for (; b + 24 < blockIdx.x; b += 32) {
                    uint4 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) v[u] = __ldcg(csum4 + (size_t)(b + 8 * u) * RQ);
#pragma unroll
                    for (int u = 0; u < 4; ++u) { c.x += v[u].x; c.y += v[u].y; c.z += v[u].z; c.w += v[u].w; }
                }
                for (; b < blockIdx.x; b += 8) {
                    const uint4 v = __ldcg(csum4 + (size_t)b * RQ);
                    c.x += v.x; c.y += v.y; c.z += v.z; c.w += v.w;
                }
                reinterpret_cast<uint4*>(s_part + (8 + g) * R)[q] = c;
            }
        }
        __syncthreads();
        if (last) {
            // pair counts of the reordered slice, their exclusive scan (in
            // s_key, free now): thread t takes a contiguous run of E positions
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
            // per digit: the scan value at the run's start
            if (tid < (int)R) {
                const uint32_t r0 = s_boff[tid];
                s_cbase[tid] = r0 < m ? s_key[r0] : btot;
            }
            __syncthreads();   // s_wtot is reused below
        }
        if (tid < (int)R) {
            const uint32_t* s_part = reinterpret_cast<const uint32_t*>(s_wcnt);
            uint32_t pre = 0;
#pragma unroll
            for (int g = 0; g < 8; ++g) pre += s_part[g * R + tid];
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
                uint32_t cpre = 0;
#pragma unroll
                for (int g = 8; g < 16; ++g) cpre += s_part[g * R + tid];
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
        // (unrolled over the thread's kDsPer elements, so that their shared
        // loads issue back to back)
#pragma unroll
        for (int k = 0; k < kDsPer; ++k) {
            const uint32_t j = tid + k * kDsThreads;
            if (j < m) {
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
        }
        if (!last) grid_barrier(a.bar, bar_target, a.err);
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
    return (size_t)kDsMaxSlice * 4 * 4 + (size_t)kDsWarps * kDsRadix * 2 + 4 * kDsRadix * 4 + kDsWarps * 4;
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
