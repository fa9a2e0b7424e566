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
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kThreads = 256;              // one thread per digit in the digit phases
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;                 // keys per thread
constexpr int kTileKeys = kThreads * kItems;
constexpr int kMaxPasses = 8;
constexpr uint32_t kFlagAgg = 1u << 30;    // status word: 2-bit flag | 30-bit count
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1;
constexpr long kSpinLimit = 1L << 22;

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

// Histogram of every pass's digit over all keys; warp-aggregated shared-memory
// counting (many keys share a digit, e.g. the exponent byte of depths).
template <typename K>
__global__ void __launch_bounds__(kThreads) k_radix_hist(const K* __restrict__ keys, uint32_t n, int bit_lo,
                                                         int passes, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t s_hist[kMaxPasses][kRadix];
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += kThreads) (&s_hist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t stride = gridDim.x * kThreads;
    // whole warps iterate together so __match_any_sync sees all lanes
    const uint32_t n_round = (n + 31u) & ~31u;
    for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < n_round; i += stride) {
        const bool valid = i < n;
        const K key = valid ? keys[i] : K(0);
        for (int p = 0; p < passes; ++p) {
            const uint32_t d = valid ? digit_of(key, bit_lo + p * kRadixBits) : kRadix;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const int leader = 31 - __clz(peers);
            if (valid && (int)(threadIdx.x & 31) == leader) atomicAdd(&s_hist[p][d], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kThreads) {
        const uint32_t v = (&s_hist[0][0])[i];
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
    K keys[kTileKeys];
    uint32_t vals[HAS_VAL ? kTileKeys : 1];
};

template <typename K, bool HAS_VAL>
__global__ void __launch_bounds__(kThreads) k_onesweep(const K* __restrict__ keys_in, K* __restrict__ keys_out,
                                                       const uint32_t* __restrict__ vals_in,
                                                       uint32_t* __restrict__ vals_out, uint32_t n, int shift,
                                                       const uint32_t* __restrict__ digit_base,
                                                       uint32_t* __restrict__ status,
                                                       uint32_t* __restrict__ tile_counter, int* __restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& S = *reinterpret_cast<OnesweepSmem<K, HAS_VAL>*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int i = tid; i < kWarps * kRadix; i += kThreads) (&S.warp_hist[0][0])[i] = 0;
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
    for (int i = 0; i < kItems; ++i) {
        const uint32_t d = dig[i];
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const int leader = 31 - __clz(peers);
        uint32_t prev = 0;
        if (d < (uint32_t)kRadix) prev = S.warp_hist[warp][d];
        rank[i] = prev + __popc(peers & lt);
        __syncwarp();
        if (lane == leader && d < (uint32_t)kRadix) S.warp_hist[warp][d] = prev + __popc(peers);
        __syncwarp();
    }
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

    // decoupled look-back over earlier tiles for digit d
    uint32_t excl = 0;
    if (tile > 0) {
        long spins = 0;
        int j = (int)tile - 1;
        while (j >= 0) {
            const uint32_t s = *(volatile const uint32_t*)(status + (size_t)j * kRadix + d);
            const uint32_t f = s & ~kValueMask;
            if (f == 0u) {
                if (++spins > kSpinLimit) {
                    atomicExch(err, kDevTimeout);
                    break;
                }
                continue;
            }
            excl += s & kValueMask;
            if (f == kFlagInc) break;
            --j;
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
            keys_out[g] = k;
            if (HAS_VAL) vals_out[g] = S.vals[p];
        }
    }
}

template <typename K, bool HAS_VAL>
cudaError_t radix_sort_impl(cudaStream_t s, K* keys[2], uint32_t* vals[2], uint32_t n, int bit_lo, int bit_hi,
                            uint32_t* hist, uint32_t* status, uint32_t* counters, int* err, int* out_idx)
{
    *out_idx = 0;
    if (n <= 1 || bit_hi <= bit_lo) return cudaSuccess;
    const int passes = (bit_hi - bit_lo + kRadixBits - 1) / kRadixBits;
    const uint32_t tiles = (n + kTileKeys - 1) / kTileKeys;
    cudaError_t e;
    if ((e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * passes * kRadix, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(status, 0, sizeof(uint32_t) * (size_t)passes * tiles * kRadix, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(counters, 0, sizeof(uint32_t) * passes, s)) != cudaSuccess) return e;
    const uint32_t hb = (n + kThreads * 8 - 1) / (kThreads * 8);
    const int hist_blocks = (int)(hb < 152u * 8u ? hb : 152u * 8u);
    k_radix_hist<K><<<hist_blocks, kThreads, 0, s>>>(keys[0], n, bit_lo, passes, hist); note_launch();
    k_radix_hist_scan<<<passes, kThreads, 0, s>>>(hist); note_launch();
    const size_t smem = sizeof(OnesweepSmem<K, HAS_VAL>);
    static bool attr_set = false;
    if (!attr_set) {
        e = cudaFuncSetAttribute(k_onesweep<K, HAS_VAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = bit_lo + p * kRadixBits;
        k_onesweep<K, HAS_VAL><<<tiles, kThreads, smem, s>>>(
            keys[cur], keys[cur ^ 1], HAS_VAL ? vals[cur] : nullptr, HAS_VAL ? vals[cur ^ 1] : nullptr, n, shift,
            hist + p * kRadix, status + (size_t)p * tiles * kRadix, counters + p, err); note_launch();
        cur ^= 1;
    }
    *out_idx = cur;
    return cudaGetLastError();
}

// ---- exclusive scan of tiles_touched gathered through the depth order ----
// Block totals are 64-bit so that the pair count P is exact even when it would
// not fit 32 bits (the caller then refuses the frame); per-item offsets are
// 32-bit and valid whenever P < 2^32.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename V>
__device__ __forceinline__ V block_exclusive_scan(V v, V* s_warp, V* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    V x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const V y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    V base = 0, tot = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        const V t = s_warp[w];
        if (w < warp) base += t;
        tot += t;
    }
    __syncthreads();
    *total = tot;
    return base + x - v;
}

// per block: sum of counts[ids[k]] -> partials[b], sum of side[ids[k]] -> partials2[b]
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ tt,
                                                              const uint32_t* __restrict__ side,
                                                              const uint32_t* __restrict__ ids, uint32_t n,
                                                              unsigned long long* __restrict__ partials,
                                                              unsigned long long* __restrict__ partials2)
{
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    const uint32_t base = blockIdx.x * kScanTile;
    unsigned long long sum = 0, sum2 = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint32_t idx = base + i * kScanThreads + threadIdx.x;
        if (idx < n) {
            const uint32_t id = ids[idx];
            if (id < n) {
                sum += tt[id];
                if (side) sum2 += side[id];
            }
        }
    }
    unsigned long long tot, tot2;
    block_exclusive_scan<unsigned long long>(sum, s_warp, &tot);
    block_exclusive_scan<unsigned long long>(sum2, s_warp, &tot2);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = tot;
        partials2[blockIdx.x] = tot2;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partials(unsigned long long* __restrict__ partials,
                                                                unsigned long long* __restrict__ partials2,
                                                                uint32_t nb)
{
    __shared__ unsigned long long s_warp[kScanThreads / 32];
    unsigned long long carry = 0, carry2 = 0;
    for (uint32_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        const uint32_t i = b0 + threadIdx.x;
        const unsigned long long v = i < nb ? partials[i] : 0ull;
        const unsigned long long v2 = i < nb ? partials2[i] : 0ull;
        unsigned long long tot, tot2;
        const unsigned long long ex = block_exclusive_scan<unsigned long long>(v, s_warp, &tot);
        block_exclusive_scan<unsigned long long>(v2, s_warp, &tot2);
        if (i < nb) partials[i] = carry + ex;
        carry += tot;
        carry2 += tot2;
    }
    if (threadIdx.x == 0) {
        partials[nb] = carry;
        partials2[nb] = carry2;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t* __restrict__ tt,
                                                             const uint32_t* __restrict__ ids, uint32_t n,
                                                             const unsigned long long* __restrict__ partials,
                                                             uint32_t* __restrict__ out)
{
    __shared__ uint32_t s_warp[kScanThreads / 32];
    const uint32_t base = blockIdx.x * kScanTile;
    // blocked arrangement: thread t owns items [t*kScanItems, (t+1)*kScanItems)
    uint32_t v[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint32_t idx = base + threadIdx.x * kScanItems + i;
        const uint32_t id = idx < n ? ids[idx] : n;
        v[i] = id < n ? tt[id] : 0u;
        sum += v[i];
    }
    uint32_t tot;
    uint32_t run = (uint32_t)partials[blockIdx.x] + block_exclusive_scan<uint32_t>(sum, s_warp, &tot);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint32_t idx = base + threadIdx.x * kScanItems + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (uint32_t)partials[gridDim.x];
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
    return radix_sort_impl<uint32_t, true>(s, keys, vals, n, bit_lo, bit_hi, hist, status, counters, err, out_idx);
}

cudaError_t radix_sort_u64_keys(cudaStream_t s, uint64_t* keys[2], uint32_t n, int bit_lo, int bit_hi,
                                uint32_t* hist, uint32_t* status, uint32_t* counters, int* err, int* out_idx)
{
    uint32_t* no_vals[2] = {nullptr, nullptr};
    return radix_sort_impl<uint64_t, false>(s, keys, no_vals, n, bit_lo, bit_hi, hist, status, counters, err,
                                            out_idx);
}

size_t scan_partials_count(uint32_t n)
{
    return (n + kScanTile - 1) / kScanTile + 1;
}

cudaError_t launch_scan_gathered(cudaStream_t s, const uint32_t* tt, const uint32_t* side, const uint32_t* ids,
                                 uint32_t n, uint32_t* offsets, unsigned long long* partials)
{
    const uint32_t nb = (n + kScanTile - 1) / kScanTile;
    unsigned long long* partials2 = partials + nb + 1;
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(offsets, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
        return cudaMemsetAsync(partials, 0, 2 * sizeof(unsigned long long), s);
    }
    k_scan_reduce<<<nb, kScanThreads, 0, s>>>(tt, side, ids, n, partials, partials2); note_launch();
    k_scan_partials<<<1, kScanThreads, 0, s>>>(partials, partials2, nb); note_launch();
    k_scan_apply<<<nb, kScanThreads, 0, s>>>(tt, ids, n, partials, offsets); note_launch();
    return cudaGetLastError();
}

}  // namespace gs
