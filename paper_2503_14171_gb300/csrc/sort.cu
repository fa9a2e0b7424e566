// Device-wide primitives for the binning stage: a stable LSD radix sort in the
// single-pass ("one sweep") form -- one global digit histogram for all passes,
// then one kernel per 8-bit digit that ranks its tile of keys with warp
// multi-split, resolves the tile's global digit offsets by decoupled look-back
// over its predecessors, stages the keys in digit order in shared memory and
// writes them out in coalesced runs -- and an exclusive scan.
//
// Every wait on another block is bounded: after kSpinLimit polls the block
// records kDevTimeout in the context's error word and proceeds (its output is
// then undefined, the GPU is never hung).
#include <atomic>

#include "gs_internal.cuh"
#include "tile_order.cuh"

namespace gs {
namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kThreads = 256;              // one thread per digit in the digit phases
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 12;                 // keys per thread (12: 3072-key tiles; 8 measured 1.5 and 5 µs slower per frame at 960x540 and 1920x1080)
constexpr int kTileKeys = kThreads * kItems;
constexpr int kMaxPasses = 8;              // the callers' histogram ([8][256]) and counter ([8]) buffers
constexpr uint32_t kFlagAgg = 1u << 30;    // status word: 2-bit flag | 30-bit count
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1;
constexpr long kSpinLimit = 1L << 22;
constexpr int kLookback = 8;               // predecessor tiles read per look-back round trip

static_assert(kThreads == kRadix, "digit phases use one thread per digit");

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift)
{
    return (uint32_t)(key >> shift) & (kRadix - 1);
}

// Stable rank of this lane's key among the keys of its digit that the warp has
// ranked so far (warp multi-split).  The lanes holding the same digit are
// found through the warp's table of lane masks (one word per digit, zero
// between calls): each lane ORs its bit into its digit's word and reads the
// word back.  (One warp ballot per digit bit, or a match instruction, costs
// far more issue time on this part than these shared-memory atomics.)  The
// highest lane of each digit reads the warp's running count of the digit,
// passes it to its peers, writes it back advanced and clears the word.
// valid = false (a slot past the end): returns 0 and touches nothing.
__device__ __forceinline__ uint32_t warp_rank(uint32_t* __restrict__ mask, uint32_t* __restrict__ count, uint32_t d,
                                              bool valid, int lane, uint32_t lt)
{
    if (valid) atomicOr(mask + d, 1u << lane);
    __syncwarp();
    const uint32_t peers = valid ? mask[d] : (1u << lane);   // an idle lane leads itself
    __syncwarp();   // every lane has read its word before the leaders clear it
    const int leader = 31 - __clz(peers);
    uint32_t prev = 0;
    if (valid && lane == leader) {
        prev = count[d];
        count[d] = prev + __popc(peers);
        mask[d] = 0u;
    }
    prev = __shfl_sync(0xffffffffu, prev, leader);
    __syncwarp();   // the next call's lanes see the cleared words and the new counts
    return prev + __popc(peers & lt);
}

// Histogram of every pass's digit over all keys, in per-warp shared-memory
// sub-histograms (a key shared by a whole warp, e.g. the exponent byte of a
// depth, costs one 32-way serialised atomic instead of block-wide contention).
constexpr int kHistPasses = 5;   // up to 40 bits (the (view, depth) keys of a batch of views)
template <typename K>
__global__ void __launch_bounds__(kThreads) k_radix_hist(const K* __restrict__ keys, uint32_t n, int bit_lo,
                                                         int passes, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t s_hist[kWarps][kHistPasses][kRadix];
    for (int i = threadIdx.x; i < kWarps * kHistPasses * kRadix; i += kThreads) (&s_hist[0][0][0])[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    const uint32_t stride = gridDim.x * kThreads;
    for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
        const K key = keys[i];
#pragma unroll
        for (int p = 0; p < kHistPasses; ++p)
            if (p < passes) atomicAdd(&s_hist[warp][p][digit_of(key, bit_lo + p * kRadixBits)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < min(passes, kHistPasses) * kRadix; i += kThreads) {
        uint32_t v = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) v += (&s_hist[w][0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// Exclusive prefix of each pass's 256 counts (one block per pass).
__global__ void __launch_bounds__(kThreads) k_radix_hist_scan(uint32_t* __restrict__ hist)
{
    __shared__ uint32_t s_warp[kWarps];
    uint32_t* h = hist + blockIdx.x * kRadix;
    const uint32_t v = h[threadIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t base = 0;
    for (int w = 0; w < warp; ++w) base += s_warp[w];
    h[threadIdx.x] = base + x - v;
}

template <typename K, bool HAS_VAL>
struct OnesweepSmem {
    uint32_t warp_hist[kWarps][kRadix];   // per-warp digit counts, then their exclusive prefix
    uint32_t local_start[kRadix];         // exclusive prefix of the tile's digit counts
    uint32_t global_base[kRadix];         // output index of the tile's first key of each digit, minus local_start
    uint32_t warp_tot[kWarps];
    uint32_t tile;
    union {
        K keys[kTileKeys];                // the tile in digit order
        uint32_t mask[kWarps][kRadix];    // before that, the ranking's per-warp lane-mask tables
    };
    uint32_t vals[HAS_VAL ? kTileKeys : 1];
};

// One tile of a one-sweep pass (the tile index taken from a counter in launch
// order, so every predecessor tile is running or done).
template <typename K, bool HAS_VAL>
__device__ __forceinline__ void onesweep_tile(OnesweepSmem<K, HAS_VAL>& S, const K* __restrict__ keys_in,
                                              K* __restrict__ keys_out, const uint32_t* __restrict__ vals_in,
                                              uint32_t* __restrict__ vals_out, uint32_t n, int shift,
                                              const uint32_t* __restrict__ digit_base,
                                              uint32_t* __restrict__ status, uint32_t* __restrict__ tile_counter,
                                              int* __restrict__ err)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kWarps * kRadix; i += kThreads) {
        (&S.warp_hist[0][0])[i] = 0;
        (&S.mask[0][0])[i] = 0;
    }
    if (tid == 0) S.tile = atomicAdd(tile_counter, 1u);   // tiles are taken in launch order
    __syncthreads();
    const uint32_t tile = S.tile;
    const uint32_t base = tile * (uint32_t)kTileKeys;
    if (base >= n) return;

    K key[kItems];
    uint32_t val[kItems];
    uint32_t dig[kItems];
    uint32_t rank[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t idx = base + warp * (kItems * 32) + i * 32 + lane;
        const bool valid = idx < n;
        key[i] = valid ? keys_in[idx] : K(0);
        if (HAS_VAL) val[i] = valid ? vals_in[idx] : 0u;
        dig[i] = valid ? digit_of(key[i], shift) : (uint32_t)kRadix;
    }
    // warp multi-split: rank among earlier keys of the same digit in this warp
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        rank[i] = warp_rank(S.mask[warp], S.warp_hist[warp], dig[i], dig[i] < (uint32_t)kRadix, lane, lt);
    __syncthreads();

    // thread d: per-warp exclusive prefix for digit d and the tile's count
    const uint32_t d = tid;
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = S.warp_hist[w][d];
        S.warp_hist[w][d] = total;
        total += c;
    }
    volatile uint32_t* st = status + (size_t)tile * kRadix + d;
    *st = (tile == 0 ? kFlagInc : kFlagAgg) | total;

    // exclusive scan of the tile's digit counts
    uint32_t x = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) S.warp_tot[warp] = x;
    __syncthreads();
    uint32_t wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += S.warp_tot[w];
    const uint32_t local_start = wbase + x - total;
    S.local_start[d] = local_start;

    // decoupled look-back over earlier tiles for digit d, kLookback tiles per
    // round trip (tiles before 0 read as an inclusive zero)
    uint32_t excl = 0;
    if (tile > 0) {
        long spins = 0;
        int j = (int)tile - 1;
        while (true) {
            uint32_t sw[kLookback];
#pragma unroll
            for (int w = 0; w < kLookback; ++w)
                sw[w] = j - w >= 0 ? *(volatile const uint32_t*)(status + (size_t)(j - w) * kRadix + d) : kFlagInc;
            int used = 0;
            bool inc = false, blocked = false;
#pragma unroll
            for (int w = 0; w < kLookback; ++w) {
                if (inc || blocked) continue;
                const uint32_t f = sw[w] & ~kValueMask;
                if (f == 0u) {
                    blocked = true;
                    continue;
                }
                excl += sw[w] & kValueMask;
                ++used;
                inc = f == kFlagInc;
            }
            if (inc) break;
            j -= used;
            if (blocked && ++spins > kSpinLimit) {
                atomicExch(err, kDevTimeout);
                break;
            }
        }
        *st = kFlagInc | ((excl + total) & kValueMask);
    }
    S.global_base[d] = digit_base[d] + excl - local_start;
    __syncthreads();

    // stage keys in digit order
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t dd = dig[i];
        if (dd < (uint32_t)kRadix) {
            const uint32_t lp = S.local_start[dd] + S.warp_hist[warp][dd] + rank[i];
            S.keys[lp] = key[i];
            if (HAS_VAL) S.vals[lp] = val[i];
        }
    }
    __syncthreads();
    const uint32_t count = min((uint32_t)kTileKeys, n - base);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t p = i * kThreads + tid;
        if (p < count) {
            const K k = S.keys[p];
            const uint32_t g = S.global_base[digit_of(k, shift)] + p;
            if (g < n) {
                keys_out[g] = k;
                if (HAS_VAL) vals_out[g] = S.vals[p];
            } else {   // inconsistent look-back state: report instead of writing out of bounds
                atomicExch(err, kDevCheck);
            }
        }
    }
}

// The single-array pass (the same steps as onesweep_tile, kept as one kernel
// body: its own code measured 4 us faster per 2.5M-pair pass than a call of
// the shared tile function).
template <typename K, bool HAS_VAL>
__global__ void __launch_bounds__(kThreads, 4) k_onesweep(const K* __restrict__ keys_in, K* __restrict__ keys_out,
                                                       const uint32_t* __restrict__ vals_in,
                                                       uint32_t* __restrict__ vals_out, uint32_t n, int shift,
                                                       const uint32_t* __restrict__ digit_base,
                                                       uint32_t* __restrict__ status,
                                                       uint32_t* __restrict__ tile_counter, int* __restrict__ err,
                                                       const uint32_t* __restrict__ n_dev)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& S = *reinterpret_cast<OnesweepSmem<K, HAS_VAL>*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (n_dev) n = min(n, *n_dev);   // key count known on the device only; surplus tiles exit

    for (int i = tid; i < kWarps * kRadix; i += kThreads) {
        (&S.warp_hist[0][0])[i] = 0;
        (&S.mask[0][0])[i] = 0;
    }
    if (tid == 0) S.tile = atomicAdd(tile_counter, 1u);   // tiles are taken in launch order
    __syncthreads();
    const uint32_t tile = S.tile;
    const uint32_t base = tile * (uint32_t)kTileKeys;
    if (base >= n) return;

    K key[kItems];
    uint32_t val[kItems];
    uint32_t dig[kItems];
    uint32_t rank[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t idx = base + warp * (kItems * 32) + i * 32 + lane;
        const bool valid = idx < n;
        key[i] = valid ? keys_in[idx] : K(0);
        if (HAS_VAL) val[i] = valid ? vals_in[idx] : 0u;
        dig[i] = valid ? digit_of(key[i], shift) : (uint32_t)kRadix;
    }
    // warp multi-split: rank among earlier keys of the same digit in this warp
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kItems; ++i)
        rank[i] = warp_rank(S.mask[warp], S.warp_hist[warp], dig[i], dig[i] < (uint32_t)kRadix, lane, lt);
    __syncthreads();

    // thread d: per-warp exclusive prefix for digit d and the tile's count
    const uint32_t d = tid;
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = S.warp_hist[w][d];
        S.warp_hist[w][d] = total;
        total += c;
    }
    volatile uint32_t* st = status + (size_t)tile * kRadix + d;
    *st = (tile == 0 ? kFlagInc : kFlagAgg) | total;

    // exclusive scan of the tile's digit counts
    uint32_t x = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) S.warp_tot[warp] = x;
    __syncthreads();
    uint32_t wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += S.warp_tot[w];
    const uint32_t local_start = wbase + x - total;
    S.local_start[d] = local_start;

    // decoupled look-back over earlier tiles for digit d, kLookback tiles per
    // round trip (tiles before 0 read as an inclusive zero)
    uint32_t excl = 0;
    if (tile > 0) {
        long spins = 0;
        int j = (int)tile - 1;
        while (true) {
            uint32_t sw[kLookback];
#pragma unroll
            for (int w = 0; w < kLookback; ++w)
                sw[w] = j - w >= 0 ? *(volatile const uint32_t*)(status + (size_t)(j - w) * kRadix + d) : kFlagInc;
            int used = 0;
            bool inc = false, blocked = false;
#pragma unroll
            for (int w = 0; w < kLookback; ++w) {
                if (inc || blocked) continue;
                const uint32_t f = sw[w] & ~kValueMask;
                if (f == 0u) {
                    blocked = true;
                    continue;
                }
                excl += sw[w] & kValueMask;
                ++used;
                inc = f == kFlagInc;
            }
            if (inc) break;
            j -= used;
            if (blocked && ++spins > kSpinLimit) {
                atomicExch(err, kDevTimeout);
                break;
            }
        }
        *st = kFlagInc | ((excl + total) & kValueMask);
    }
    S.global_base[d] = digit_base[d] + excl - local_start;
    __syncthreads();

    // stage keys in digit order
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t dd = dig[i];
        if (dd < (uint32_t)kRadix) {
            const uint32_t lp = S.local_start[dd] + S.warp_hist[warp][dd] + rank[i];
            S.keys[lp] = key[i];
            if (HAS_VAL) S.vals[lp] = val[i];
        }
    }
    __syncthreads();
    const uint32_t count = min((uint32_t)kTileKeys, n - base);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const uint32_t p = i * kThreads + tid;
        if (p < count) {
            const K k = S.keys[p];
            const uint32_t g = S.global_base[digit_of(k, shift)] + p;
            if (g < n) {
                keys_out[g] = k;
                if (HAS_VAL) vals_out[g] = S.vals[p];
            } else {   // inconsistent look-back state: report instead of writing out of bounds
                atomicExch(err, kDevCheck);
            }
        }
    }
}

// One pass over several independent key arrays (the pair lists of a batch of
// views) in one launch: blocks [first[s], first[s + 1]) serve segment s, which
// sorts its own keys with its own digit histogram, look-back states and tile
// counter exactly as k_onesweep sorts one array.  A segment with fewer passes
// than the launch's pass index has no blocks.
template <typename K, bool HAS_VAL>
__global__ void __launch_bounds__(kThreads, 4) k_onesweep_segs(const __grid_constant__ SortSegs g, int pass)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& S = *reinterpret_cast<OnesweepSmem<K, HAS_VAL>*>(smem_raw);
    int sg = 0;
    while (sg + 1 < g.count && (int)blockIdx.x >= g.seg[sg + 1].first_block) ++sg;
    const SortSeg& q = g.seg[sg];
    if (pass >= q.passes) return;
    uint32_t n = q.cap;
    if (q.n_dev) n = min(n, *q.n_dev);
    const int cur = pass & 1;
    onesweep_tile<K, HAS_VAL>(S, reinterpret_cast<const K*>(q.keys[cur]), reinterpret_cast<K*>(q.keys[cur ^ 1]),
                              HAS_VAL ? q.vals[cur] : nullptr, HAS_VAL ? q.vals[cur ^ 1] : nullptr, n,
                              q.bit_lo + pass * kRadixBits, q.hist + pass * kRadix,
                              q.status + (size_t)pass * q.tiles * kRadix, q.counters + pass, q.err);
}

// Digit histograms of every pass of each segment (blocks [first[s], first[s +
// 1]) count segment s's keys), accumulated into the segments' zeroed
// histograms; then one block per (segment, pass) turns them into exclusive
// prefixes.
constexpr int kSegHistItems = 16;   // keys per thread of the histogram blocks
__global__ void __launch_bounds__(kThreads) k_radix_hist_segs(const __grid_constant__ SortSegs g)
{
    __shared__ uint32_t s_hist[4][kRadix];
    int sg = 0;
    while (sg + 1 < g.count && (int)blockIdx.x >= g.seg[sg + 1].first_block) ++sg;
    const SortSeg& q = g.seg[sg];
    const int passes = min(q.passes, 4);
    for (int i = threadIdx.x; i < 4 * kRadix; i += kThreads) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t n = q.cap;
    const uint32_t base = (blockIdx.x - q.first_block) * (uint32_t)(kThreads * kSegHistItems);
    const uint32_t* keys = reinterpret_cast<const uint32_t*>(q.keys[0]);
#pragma unroll 4
    for (int k = 0; k < kSegHistItems; ++k) {
        const uint32_t i = base + k * kThreads + threadIdx.x;
        if (i < n) {
            const uint32_t key = keys[i];
            for (int p = 0; p < passes; ++p)
                atomicAdd(&s_hist[p][(key >> (q.bit_lo + p * kRadixBits)) & (kRadix - 1)], 1u);
        }
    }
    __syncthreads();
    uint32_t* h = const_cast<uint32_t*>(q.hist);
    for (int i = threadIdx.x; i < passes * kRadix; i += kThreads) {
        const uint32_t v = (&s_hist[0][0])[i];
        if (v) atomicAdd(&h[i], v);
    }
}

__global__ void __launch_bounds__(kThreads) k_radix_hist_scan_segs(const __grid_constant__ SortSegs g)
{
    const int sg = blockIdx.x / 4, p = blockIdx.x % 4;
    const SortSeg& q = g.seg[sg];
    if (p >= q.passes) return;
    __shared__ uint32_t s_warp[kWarps];
    uint32_t* h = const_cast<uint32_t*>(q.hist) + p * kRadix;
    const uint32_t v = h[threadIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t b = 0;
    for (int w = 0; w < warp; ++w) b += s_warp[w];
    h[threadIdx.x] = b + x - v;
}

// The one-sweep kernels' dynamic shared memory attribute, set once per device
// (an atomic bit per device: concurrent first calls set the same value).
template <typename K, bool HAS_VAL>
cudaError_t onesweep_attr()
{
    static std::atomic<uint64_t> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    const int smem = (int)sizeof(OnesweepSmem<K, HAS_VAL>);
    if ((e = cudaFuncSetAttribute(k_onesweep<K, HAS_VAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_onesweep_segs<K, HAS_VAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess)
        return e;
    done.fetch_or(bit, std::memory_order_acq_rel);
    return cudaSuccess;
}

template <typename K, bool HAS_VAL>
cudaError_t radix_sort_impl(cudaStream_t s, K* keys[2], uint32_t* vals[2], uint32_t n, int bit_lo, int bit_hi,
                            uint32_t* hist, uint32_t* status, uint32_t* counters, int* err, int* out_idx,
                            bool hist_ready, const uint32_t* n_dev = nullptr, bool pre_zeroed = false)
{
    *out_idx = 0;
    if (n <= 1 || bit_hi <= bit_lo) return cudaSuccess;
    const int passes = (bit_hi - bit_lo + kRadixBits - 1) / kRadixBits;
    if (passes > kMaxPasses) return cudaErrorInvalidValue;
    const uint32_t tiles = (n + kTileKeys - 1) / kTileKeys;
    cudaError_t e;
    if (!pre_zeroed) {
        if ((e = cudaMemsetAsync(status, 0, sizeof(uint32_t) * (size_t)passes * tiles * kRadix, s)) != cudaSuccess)
            return e;
        if ((e = cudaMemsetAsync(counters, 0, sizeof(uint32_t) * passes, s)) != cudaSuccess) return e;
    }
    if (!hist_ready) {
        if (passes > kHistPasses) return cudaErrorInvalidValue;   // the histogram kernel holds kHistPasses passes
        if ((e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * passes * kRadix, s)) != cudaSuccess) return e;
        const uint32_t hb = (n + kThreads * 8 - 1) / (kThreads * 8);
        const int hist_blocks = (int)(hb < 152u * 8u ? hb : 152u * 8u);
        k_radix_hist<K><<<hist_blocks, kThreads, 0, s>>>(keys[0], n, bit_lo, passes, hist); note_launch();
        k_radix_hist_scan<<<passes, kThreads, 0, s>>>(hist); note_launch();
    }
    const size_t smem = sizeof(OnesweepSmem<K, HAS_VAL>);
    if ((e = onesweep_attr<K, HAS_VAL>()) != cudaSuccess) return e;
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = bit_lo + p * kRadixBits;
        k_onesweep<K, HAS_VAL><<<tiles, kThreads, smem, s>>>(
            keys[cur], keys[cur ^ 1], HAS_VAL ? vals[cur] : nullptr, HAS_VAL ? vals[cur ^ 1] : nullptr, n, shift,
            hist + p * kRadix, status + (size_t)p * tiles * kRadix, counters + p, err, n_dev); note_launch();
        cur ^= 1;
    }
    *out_idx = cur;
    return cudaGetLastError();
}

// ---- exclusive scan of per-Gaussian counts gathered through the depth order ----
// Single pass with decoupled look-back: each block takes the next tile of 4096
// positions (in launch order), sums its gathered counts, publishes the sum,
// resolves its exclusive prefix from its predecessors (one warp reads 32
// predecessor tiles per round trip, bounded wait), and writes its offsets.
// Tile states are 64-bit (2-bit flag | 62-bit value), so the total is exact;
// per-position offsets are 32-bit and valid whenever the total is < 2^32.
// A second count array is reduced alongside (one 64-bit atomic per block).
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kScanRow = kScanItems + 4;   // a lane's row of offsets in shared memory, padded
constexpr unsigned long long kScanAgg = 1ull << 62;
constexpr unsigned long long kScanInc = 2ull << 62;
constexpr unsigned long long kScanMask = (1ull << 62) - 1;

template <bool PACKED>
__global__ void __launch_bounds__(kScanThreads) k_scan_onepass(const uint32_t* __restrict__ counts,
                                                               const uint32_t* __restrict__ side,
                                                               const uint32_t* __restrict__ ids, uint32_t n,
                                                               uint32_t* __restrict__ offsets,
                                                               unsigned long long* __restrict__ status,
                                                               uint32_t* __restrict__ tile_counter,
                                                               unsigned long long* __restrict__ totals,
                                                               int* __restrict__ err)
{
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    __shared__ __align__(16) uint32_t s_out[kScanThreads / 32][32 * kScanRow];
    __shared__ unsigned long long s_prefix;
    __shared__ uint32_t s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t ntiles = (n + kScanTile - 1) / kScanTile;
    // blocked arrangement: thread t owns positions [t*16, t*16 + 16) of the
    // tile, loaded as four 16-byte words where the pointer allows
    const uint32_t base = tile * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    unsigned long long sum = 0, sum2 = 0;
    uint32_t w[kScanItems];
    if (base + kScanItems <= n && (reinterpret_cast<uintptr_t>(ids) & 15u) == 0) {
        const uint4* p4 = reinterpret_cast<const uint4*>(ids + base);
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            const uint4 t = p4[q];
            w[4 * q] = t.x; w[4 * q + 1] = t.y; w[4 * q + 2] = t.z; w[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) w[i] = base + i < n ? ids[base + i] : (PACKED ? 0u : n);
    }
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint32_t k = base + i;
        if (PACKED) {   // the count rides with the entry (escaped ones looked up)
            const uint32_t id = w[i] & kPackedIdxMask;
            uint32_t c = w[i] >> kPackedIdxBits;
            if (c == kPackedCntEsc) c = id < n ? counts[id] : 0u;
            v[i] = k < n ? c : 0u;
        } else {
            const uint32_t id = w[i];
            v[i] = id < n ? counts[id] : 0u;
            if (side != nullptr && id < n) sum2 += side[id];
        }
        sum += v[i];
    }
    // block scan of the per-thread sums
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    // side total: warp reduce, one atomic per warp
    unsigned long long z = sum2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_down_sync(0xffffffffu, z, o);
    if (lane == 0 && z) atomicAdd(&totals[1], z);
    __syncthreads();
    unsigned long long wbase = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        const unsigned long long t = s_warp[w];
        wbase += w < warp ? t : 0ull;
        tot += t;
    }
    // publish, then look back (warp 0)
    if (warp == 0) {
        volatile unsigned long long* st = status + tile;
        if (lane == 0) *st = (tile == 0 ? kScanInc : kScanAgg) | tot;
        unsigned long long excl = 0;
        if (tile > 0) {
            long spins = 0;
            int j = (int)tile - 1;
            while (true) {
                const int jj = j - lane;
                const unsigned long long sv =
                    jj >= 0 ? *(volatile const unsigned long long*)(status + jj) : kScanInc;
                const unsigned long long f = sv & ~kScanMask;
                // lanes up to the first inclusive one count; a not-ready lane before it blocks
                const uint32_t inc_mask = __ballot_sync(0xffffffffu, f == kScanInc);
                const uint32_t zero_mask = __ballot_sync(0xffffffffu, f == 0ull);
                const int first_inc = inc_mask ? __ffs(inc_mask) - 1 : 32;
                const int first_zero = zero_mask ? __ffs(zero_mask) - 1 : 32;
                const int upto = min(first_inc, first_zero);            // lanes [0, upto) are aggregates
                unsigned long long add = (lane < upto || (lane == first_inc && first_inc < first_zero))
                                             ? (sv & kScanMask) : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) add += __shfl_down_sync(0xffffffffu, add, o);
                add = __shfl_sync(0xffffffffu, add, 0);
                excl += add;
                if (first_inc < first_zero) break;
                j -= upto;
                if (first_zero < 32 && ++spins > (1L << 22)) {
                    if (lane == 0) atomicExch(err, kDevTimeout);
                    break;
                }
            }
            if (lane == 0) *st = kScanInc | ((excl + tot) & kScanMask);
        }
        if (lane == 0) {
            s_prefix = excl;
            if (tile == ntiles - 1) totals[0] = excl + tot;
        }
    }
    __syncthreads();
    uint32_t run = (uint32_t)(s_prefix + wbase + x - sum);
    // a warp whose 512 positions all lie below n writes them through its
    // shared-memory rows (20-word stride: conflict-free 16-byte accesses) as
    // 512 contiguous bytes per instruction; the ragged tail writes in place
    const uint32_t wbase_k = tile * kScanTile + warp * 32 * kScanItems;
    if (wbase_k + 32 * kScanItems <= n && (reinterpret_cast<uintptr_t>(offsets) & 15u) == 0) {
        uint32_t* row = &s_out[warp][lane * kScanRow];
#pragma unroll
        for (int q = 0; q < kScanItems / 4; ++q) {
            uint4 t;
            t.x = run; run += v[4 * q];
            t.y = run; run += v[4 * q + 1];
            t.z = run; run += v[4 * q + 2];
            t.w = run; run += v[4 * q + 3];
            *reinterpret_cast<uint4*>(row + 4 * q) = t;
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kScanItems / 4; ++j) {
            const int e = j * 128 + lane * 4;
            const uint4 t = *reinterpret_cast<const uint4*>(&s_out[warp][(e / kScanItems) * kScanRow + e % kScanItems]);
            *reinterpret_cast<uint4*>(offsets + wbase_k + e) = t;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const uint32_t k = base + i;
            if (k < n) offsets[k] = run;
            run += v[i];
        }
    }
    if (tile == ntiles - 1 && threadIdx.x == kScanThreads - 1) offsets[n] = (uint32_t)(s_prefix + tot);
}

}  // namespace

int radix_passes(int bit_lo, int bit_hi)
{
    return bit_hi > bit_lo ? (bit_hi - bit_lo + kRadixBits - 1) / kRadixBits : 0;
}

size_t radix_status_words(uint32_t n, int bit_lo, int bit_hi)
{
    const size_t tiles = (n + kTileKeys - 1) / kTileKeys;
    return (size_t)radix_passes(bit_lo, bit_hi) * tiles * kRadix + kRadix;
}

cudaError_t radix_sort_u32_pairs(cudaStream_t s, uint32_t* keys[2], uint32_t* vals[2], uint32_t n, int bit_lo,
                                 int bit_hi, uint32_t* hist, uint32_t* status, uint32_t* counters, int* err,
                                 int* out_idx)
{
    return radix_sort_impl<uint32_t, true>(s, keys, vals, n, bit_lo, bit_hi, hist, status, counters, err, out_idx,
                                           false, nullptr);
}

cudaError_t radix_sort_u64_pairs(cudaStream_t s, uint64_t* keys[2], uint32_t* vals[2], uint32_t n, int bit_lo,
                                 int bit_hi, uint32_t* hist, uint32_t* status, uint32_t* counters, int* err,
                                 int* out_idx)
{
    return radix_sort_impl<uint64_t, true>(s, keys, vals, n, bit_lo, bit_hi, hist, status, counters, err, out_idx,
                                           false, nullptr);
}

cudaError_t radix_sort_u64_keys(cudaStream_t s, uint64_t* keys[2], uint32_t n, int bit_lo, int bit_hi,
                                uint32_t* hist, uint32_t* status, uint32_t* counters, int* err, int* out_idx,
                                bool hist_ready, const uint32_t* n_dev, bool pre_zeroed)
{
    uint32_t* no_vals[2] = {nullptr, nullptr};
    if (n_dev && !hist_ready) return cudaErrorInvalidValue;   // the histogram kernels need the count on the host
    if (pre_zeroed && !hist_ready) return cudaErrorInvalidValue;
    return radix_sort_impl<uint64_t, false>(s, keys, no_vals, n, bit_lo, bit_hi, hist, status, counters, err,
                                            out_idx, hist_ready, n_dev, pre_zeroed);
}

// Per-super-tile counts -> (a) the exclusive digit histograms of every radix
// pass over the super-tile bits (bits [32, 32 + 8 passes) of the pair keys) and
// (b) the [start, end) range of every super-tile's run in the sorted list.
// One block; Ts <= kMaxSupersForCounts.
//
// With a capacity check (out != nullptr): the pair totals stay on the device.
// If the frame's super-tile pairs exceed in.cap (the pair buffers) or its tile
// pairs (the sum of the odd entries of in.slots) exceed in.max_pairs, every
// range is left empty (the blend then sees no Gaussians), out->count = 0 so
// the sort does nothing, and the error word reports the overflow;
// out->needed / out->tile_pairs keep the frame's totals for the host.
__device__ __forceinline__ void supers_to_hist_block(uint32_t* __restrict__ counts, uint32_t Ts, int passes,
                                                     uint32_t* __restrict__ hist, uint2* __restrict__ ranges,
                                                     const PairCheckIn& in, PairCheckOut* out, int* __restrict__ err)
{
    __shared__ uint32_t s_hist[kHistPasses][kRadix];
    __shared__ uint32_t s_warp[kWarps];
    __shared__ unsigned long long s_sum[kWarps];
    __shared__ int s_ok;
    for (int i = threadIdx.x; i < kHistPasses * kRadix; i += kThreads) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    // the counts arrive as kCountCopies partial arrays; fold them into copy 0
    unsigned long long mine = 0;
    for (uint32_t t = threadIdx.x; t < Ts; t += kThreads) {
        uint32_t c = 0;
        for (int k = 0; k < kCountCopies; ++k) c += counts[(size_t)k * Ts + t];
        counts[t] = c;
        mine += c;
        for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][(t >> (p * kRadixBits)) & (kRadix - 1)], c);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the emitted pairs must fit the pair buffers (in.cap; 0: unchecked): a
    // frame beyond the reservation (out != NULL) is reported as a capacity
    // overflow, a count above the exactly sized buffers as a failed check
    // (only after an expired bounded wait upstream); either way the ranges are
    // left empty, so no later kernel reads beyond the buffers
    if (out || in.cap) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        if (lane == 0) s_sum[warp] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long ps = 0, p = 0;
            for (int w = 0; w < kWarps; ++w) ps += s_sum[w];
            bool ok = ps <= in.cap;
            if (out) {
                for (int k = 0; k < kTotalSlots; ++k) p += in.slots[2 * k + 1];
                ok = ok && p <= in.max_pairs;
                out->needed = ps;
                out->tile_pairs = p;
                out->count = ok ? (uint32_t)ps : 0u;
            }
            if (!ok && err) atomicExch(err, out ? kDevCapacity : kDevCheck);
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) {
            for (uint32_t t = threadIdx.x; t < Ts; t += kThreads) ranges[t] = make_uint2(0u, 0u);
            return;
        }
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        const uint32_t v = s_hist[p][threadIdx.x];
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t b = 0;
        for (int w = 0; w < warp; ++w) b += s_warp[w];
        hist[p * kRadix + threadIdx.x] = b + x - v;
        __syncthreads();
    }
    // ranges: exclusive scan of the counts in super-tile order
    uint32_t carry = 0;
    for (uint32_t t0 = 0; t0 < Ts; t0 += kThreads) {
        const uint32_t t = t0 + threadIdx.x;
        const uint32_t v = t < Ts ? counts[t] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t b = 0, tot = 0;
        for (int w = 0; w < kWarps; ++w) {
            b += w < warp ? s_warp[w] : 0u;
            tot += s_warp[w];
        }
        if (t < Ts) {
            const uint32_t st = carry + b + x - v;
            ranges[t] = v ? make_uint2(st, st + v) : make_uint2(0u, 0u);
        }
        carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) k_supers_to_hist(uint32_t* __restrict__ counts, uint32_t Ts,
                                                             int passes, uint32_t* __restrict__ hist,
                                                             uint2* __restrict__ ranges, PairCheckIn in,
                                                             PairCheckOut* out, int* __restrict__ err,
                                                             const uint32_t* __restrict__ order_work,
                                                             uint32_t order_T, uint32_t* __restrict__ order)
{
    if (blockIdx.x == 1) {   // beside it, independent of it: the next blend's tile order
        tile_order_block(order_work, order_T, order);
        return;
    }
    supers_to_hist_block(counts, Ts, passes, hist, ranges, in, out, err);
}

// The per-view counts of a batch of views: block v folds view v's counts into
// its histograms, ranges and pair check, as k_supers_to_hist does for a frame.
__global__ void __launch_bounds__(kThreads) k_supers_to_hist_views(const __grid_constant__ HistViews b,
                                                                   int* __restrict__ err)
{
    const HistView& h = b.v[blockIdx.x];
    supers_to_hist_block(h.counts, h.Ts, h.passes, h.hist, h.ranges, h.in, h.out, err);
}

cudaError_t launch_supers_to_hist_views(cudaStream_t s, const HistViews& b, int* err)
{
    if (b.V <= 0) return cudaSuccess;
    k_supers_to_hist_views<<<b.V, kThreads, 0, s>>>(b, err); note_launch();
    return cudaGetLastError();
}

template <typename K, bool HAS_VAL>
cudaError_t radix_sort_segs_impl(cudaStream_t s, SortSegs g)
{
    int max_passes = 0;
    for (int k = 0; k < g.count; ++k) {
        if (g.seg[k].passes > kMaxPasses) return cudaErrorInvalidValue;
        max_passes = max_passes > g.seg[k].passes ? max_passes : g.seg[k].passes;
    }
    const size_t smem = sizeof(OnesweepSmem<K, HAS_VAL>);
    cudaError_t ea = onesweep_attr<K, HAS_VAL>();
    if (ea != cudaSuccess) return ea;
    for (int p = 0; p < max_passes; ++p) {
        int blocks = 0;
        for (int k = 0; k < g.count; ++k) {
            g.seg[k].first_block = blocks;
            if (p < g.seg[k].passes) blocks += (int)g.seg[k].tiles;
        }
        if (blocks == 0) continue;
        k_onesweep_segs<K, HAS_VAL><<<blocks, kThreads, smem, s>>>(g, p); note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t radix_sort_u64_segs(cudaStream_t s, SortSegs g)
{
    return radix_sort_segs_impl<uint64_t, false>(s, g);
}

cudaError_t radix_sort_u32_pairs_segs(cudaStream_t s, SortSegs g)
{
    int blocks = 0;
    for (int k = 0; k < g.count; ++k) {
        if (g.seg[k].passes > 4 || g.seg[k].n_dev) return cudaErrorInvalidValue;   // host-known counts, <= 32 bits
        g.seg[k].first_block = blocks;
        blocks += (int)((g.seg[k].cap + kThreads * kSegHistItems - 1) / (kThreads * kSegHistItems));
    }
    if (blocks > 0) {
        k_radix_hist_segs<<<blocks, kThreads, 0, s>>>(g); note_launch();
        k_radix_hist_scan_segs<<<4 * g.count, kThreads, 0, s>>>(g); note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return radix_sort_segs_impl<uint32_t, true>(s, g);
}

uint32_t radix_tiles(uint32_t n)
{
    return (n + kTileKeys - 1) / kTileKeys;
}

cudaError_t launch_supers_to_hist(cudaStream_t s, uint32_t* counts, uint32_t Ts, int passes, uint32_t* hist,
                                  uint2* ranges, PairCheckIn in, PairCheckOut* out, int* err,
                                  const uint32_t* order_work, uint32_t order_T, uint32_t* order)
{
    const int blocks = order && order_work && order_T > 0 ? 2 : 1;
    k_supers_to_hist<<<blocks, kThreads, 0, s>>>(counts, Ts, passes, hist, ranges, in, out, err, order_work, order_T,
                                                 order); note_launch();
    return cudaGetLastError();
}

size_t scan_partials_count(uint32_t n)
{
    return (n + kScanTile - 1) / kScanTile + 1;
}

cudaError_t launch_scan_gathered(cudaStream_t s, const uint32_t* counts, const uint32_t* side, const uint32_t* ids,
                                 uint32_t n, uint32_t* offsets, unsigned long long* scratch, uint32_t* counter,
                                 unsigned long long* totals, int* err, bool packed)
{
    const uint32_t nt = (n + kScanTile - 1) / kScanTile;
    if (packed && (side != nullptr || n > kPackedIdxMask)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(totals, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaMemsetAsync(offsets, 0, sizeof(uint32_t), s);
    if ((e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * nt, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
    if (packed)
        k_scan_onepass<true><<<nt, kScanThreads, 0, s>>>(counts, side, ids, n, offsets, scratch, counter, totals, err);
    else
        k_scan_onepass<false><<<nt, kScanThreads, 0, s>>>(counts, side, ids, n, offsets, scratch, counter, totals, err);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gs
