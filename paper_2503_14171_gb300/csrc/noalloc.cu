// gs_render_with_grads_noalloc: the render with screen-space derivatives for
// callers that must not allocate device memory.
//
// Some hosts embed the renderer where cudaMalloc is not available or not
// allowed while frames are produced: a memory manager that owns every device
// byte (a game engine or a VR compositor with a fixed budget), a plugin that
// may only use the buffers its host hands it, or a real-time loop that must
// never hit an allocation stall.  This entry point runs the same kernels as
// gs_render_with_grads (projection, persistent depth sort and offset scan,
// super-tile emission and sort, blend with derivatives) but takes every
// scratch buffer from one file-scope device array of kNaScratchBytes, so it
// calls no cudaMalloc, cudaFree or other allocating routine.
//
// The array belongs to the library: every GPU that loads it holds the array
// until the process exits.  Host code cannot use the array's name as a device
// address, so the first call on each device (with that device current) asks
// the runtime for the address with cudaGetSymbolAddress and keeps it; make
// that first call before any stream capture.  All calls share the array and
// it keeps the last call's contents: what must start at zero is cleared on
// every call, and two calls whose work overlaps on the GPU (different streams,
// different host threads) race on it.  Host-side state is per call (the
// readbacks are locals) apart from the per-device address, which is an
// atomic word, so calls from several host threads on different devices are
// independent.
#include <algorithm>
#include <atomic>

#include "gs_internal.cuh"

namespace gs {
namespace {

// Limits of the scratch-free path.
constexpr uint32_t kNaMaxGaussians = 16384;
constexpr uint32_t kNaMaxPixels = 65536;        // W * H (e.g. 256 x 256)
constexpr uint32_t kNaMaxSide = 4096;
constexpr uint32_t kNaMaxSuperPairs = 262144;   // (super-tile, Gaussian) pairs
constexpr uint32_t kNaMaxBlocks = 512;          // SMs the persistent depth sort may use
constexpr uint32_t kNaMaxSupers = 1024;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of the buffers carved from the array.
constexpr size_t kOffRec0 = 0;
constexpr size_t kOffRec1 = kOffRec0 + align256(16ull * kNaMaxGaussians);
constexpr size_t kOffRec2 = kOffRec1 + align256(16ull * kNaMaxGaussians);
constexpr size_t kOffDepth = kOffRec2 + align256(16ull * kNaMaxGaussians);
constexpr size_t kOffRadius = kOffDepth + align256(4ull * kNaMaxGaussians);
constexpr size_t kOffRect = kOffRadius + align256(4ull * kNaMaxGaussians);
constexpr size_t kOffTiles = kOffRect + align256(8ull * kNaMaxGaussians);
constexpr size_t kOffSupers = kOffTiles + align256(4ull * kNaMaxGaussians);
constexpr size_t kOffKey0 = kOffSupers + align256(4ull * kNaMaxGaussians);
constexpr size_t kOffKey1 = kOffKey0 + align256(4ull * kNaMaxGaussians);
constexpr size_t kOffId0 = kOffKey1 + align256(4ull * kNaMaxGaussians);
constexpr size_t kOffId1 = kOffId0 + align256(4ull * kNaMaxGaussians);
constexpr size_t kOffOffsets = kOffId1 + align256(4ull * kNaMaxGaussians);
constexpr size_t kOffTotals = kOffOffsets + align256(4ull * (kNaMaxGaussians + 1));
constexpr size_t kOffDs = kOffTotals + align256(8ull * (2 * kTotalSlots + 4));   // the persistent depth sort's scratch
constexpr size_t kOffDsSum = kOffDs + align256(ds_scratch_bytes(kNaMaxBlocks));   // the fallback scan's partials
constexpr size_t kOffSCounts = kOffDsSum + align256(8ull * kNaMaxBlocks);
constexpr size_t kOffSRanges = kOffSCounts + align256(4ull * kCountCopies * kNaMaxSupers);
constexpr size_t kOffHist = kOffSRanges + align256(8ull * kNaMaxSupers);
constexpr size_t kOffStatus = kOffHist + align256(4ull * 8 * 256);
constexpr size_t kOffCounter = kOffStatus + align256(4ull * (256 * (kNaMaxSuperPairs / 2048 + 1) * 2 + 256));
constexpr size_t kOffErr = kOffCounter + 256;
constexpr size_t kOffPairs0 = kOffErr + 256;
constexpr size_t kOffPairs1 = kOffPairs0 + align256(8ull * kNaMaxSuperPairs);
constexpr size_t kNaScratchBytes = kOffPairs1 + align256(8ull * kNaMaxSuperPairs);   // about 6.6 MB

static_assert(kNaMaxSupers <= (uint32_t)kMaxSupersForCounts, "super-tile counts are accumulated in shared memory");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

constexpr int kNaMaxDevices = 64;
std::atomic<unsigned char*> g_na_base[kNaMaxDevices] = {};    // device address of the array, per device

template <typename T>
T* at(unsigned char* base, size_t off)
{
    return reinterpret_cast<T*>(base + off);
}

int bits_for_na(uint32_t v)
{
    int b = 0;
    while (b < 32 && (uint64_t(1) << b) < v) ++b;
    return b;
}

CameraParams na_camera(const gs_camera& cam, int W, int H)
{
    CameraParams p;
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) p.R[3 * r + k] = cam.viewmat[4 * r + k];
        p.t[r] = cam.viewmat[4 * r + 3];
    }
    for (int k = 0; k < 3; ++k)
        p.campos[k] = -(p.R[0 * 3 + k] * p.t[0] + p.R[1 * 3 + k] * p.t[1] + p.R[2 * 3 + k] * p.t[2]);
    p.fx = cam.fx;
    p.fy = cam.fy;
    p.cx = cam.cx;
    p.cy = cam.cy;
    p.znear = cam.znear;
    p.lim_x = 1.3f * ((float)W / (2.f * cam.fx));
    p.lim_y = 1.3f * ((float)H / (2.f * cam.fy));
    return p;
}

#define NA_CUDA(expr)                                 \
    do {                                              \
        if ((expr) != cudaSuccess) {                  \
            cudaGetLastError();                       \
            return GS_ERR_CUDA;                       \
        }                                             \
    } while (0)

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" gs_status gs_render_with_grads_noalloc(const gs_gaussians* g, const gs_camera* cam, int32_t W, int32_t H,
                                                  const gs_options* opt, void* stream, float* out_C,
                                                  float* out_grads)
{
    gs_options o{};
    o.tile = kTile;
    o.mode = GS_MODE_3DGS;
    if (opt) o = *opt;
    if (o.tile != kTile || (o.mode != GS_MODE_3DGS && o.mode != GS_MODE_EXACT)) return GS_ERR_INVALID_ARG;
    // every call waits for its pair count and its error word: no flag applies
    if (o.flags != 0 || o.max_pairs < 0) return GS_ERR_INVALID_ARG;
    if (!g || !cam || !out_C || !out_grads) return GS_ERR_INVALID_ARG;
    if (W < 1 || H < 1 || (uint32_t)W > kNaMaxSide || (uint32_t)H > kNaMaxSide) return GS_ERR_INVALID_ARG;
    if ((uint64_t)W * (uint64_t)H > kNaMaxPixels) return GS_ERR_CAPACITY;
    if (g->n < 0) return GS_ERR_INVALID_ARG;
    if ((uint64_t)g->n > kNaMaxGaussians) return GS_ERR_CAPACITY;
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || (!g->sh && !g->rgb)))
        return GS_ERR_INVALID_ARG;
    if (g->sh && (g->sh_degree < 0 || g->sh_degree > 3)) return GS_ERR_INVALID_ARG;
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;

    // per-device set-up: the device address of the scratch array
    int dev = 0;
    NA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) return GS_ERR_INVALID_ARG;
    unsigned char* base = g_na_base[dev].load(std::memory_order_acquire);
    if (!base) {   // concurrent first calls look up the same address
        void* ptr = nullptr;
        NA_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        base = static_cast<unsigned char*>(ptr);
        g_na_base[dev].store(base, std::memory_order_release);
    }

    const uint32_t n = (uint32_t)g->n;
    const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
    const int ks = super_side(tiles_x, tiles_y, o.mode);
    const int stiles_x = (tiles_x + ks - 1) / ks, stiles_y = (tiles_y + ks - 1) / ks;
    const uint32_t Ts = (uint32_t)(stiles_x * stiles_y);
    if (Ts > kNaMaxSupers) return GS_ERR_CAPACITY;

    Records rec{at<float4>(base, kOffRec0), at<float4>(base, kOffRec1), at<float4>(base, kOffRec2)};
    unsigned long long* totals = at<unsigned long long>(base, kOffTotals);
    unsigned long long* scan_tot = totals + 2 * kTotalSlots;
    int* err = at<int>(base, kOffErr);
    uint32_t* ids[2] = {at<uint32_t>(base, kOffId0), at<uint32_t>(base, kOffId1)};
    uint32_t* keys[2] = {at<uint32_t>(base, kOffKey0), at<uint32_t>(base, kOffKey1)};
    uint32_t* offsets = at<uint32_t>(base, kOffOffsets);
    uint2* sranges = at<uint2>(base, kOffSRanges);

    // cleared on every call: pair totals, the error word, the super-tile counts and ranges
    NA_CUDA(cudaMemsetAsync(totals, 0, 8ull * (2 * kTotalSlots + 4), s));
    NA_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    NA_CUDA(cudaMemsetAsync(sranges, 0, sizeof(uint2) * Ts, s));

    const CameraParams cp = na_camera(*cam, W, H);
    unsigned long long h_totals[2 * kTotalSlots] = {};   // pair totals (pageable; the copy completes before use)
    if (n > 0) {
        NA_CUDA(launch_project(s, *g, cp, W, H, tiles_x, tiles_y, ks, o.mode, rec, at<float>(base, kOffDepth),
                               at<int>(base, kOffRadius), at<ushort4>(base, kOffRect), at<uint32_t>(base, kOffTiles),
                               at<uint32_t>(base, kOffSupers), keys[0], ids[0], totals));
        // pair totals to pageable host memory (a synchronous copy; no pinned buffer)
        NA_CUDA(cudaMemcpyAsync(h_totals, totals, sizeof(h_totals), cudaMemcpyDeviceToHost, s));
        NA_CUDA(cudaStreamSynchronize(s));
    }
    unsigned long long Ps64 = 0, P64 = 0;
    for (int k = 0; k < kTotalSlots; ++k) {
        Ps64 += h_totals[2 * k];
        P64 += h_totals[2 * k + 1];
    }
    if (Ps64 > kNaMaxSuperPairs) return GS_ERR_CAPACITY;
    // the (tile, Gaussian) pair limit of the options, as gs_render_with_grads applies it
    const unsigned long long limit =
        o.max_pairs > 0 ? (unsigned long long)std::min<int64_t>(o.max_pairs, kMaxPairs) : (unsigned long long)kMaxPairs;
    if (P64 > limit) return GS_ERR_CAPACITY;
    const uint32_t Ps = (uint32_t)Ps64;

    int sorted = 0;
    const uint32_t ds_cap = n > 1 ? depth_sort_capacity(dev) : 0u;
    if (n > 1 && n <= ds_cap && n <= kDsMaxN && ds_cap / kDsMaxSlice <= kNaMaxBlocks) {
        const size_t G = ds_cap / kDsMaxSlice;
        NA_CUDA(launch_depth_sort_scan(s, dev, keys[0], keys, ids, at<uint32_t>(base, kOffSupers), n, offsets,
                                       at<uint32_t>(base, kOffDs + ds_cnt_offset(G)),
                                       at<uint32_t>(base, kOffDs + ds_csum_offset(G)),
                                       at<unsigned int>(base, kOffDs + ds_bar_offset(G)),
                                       at<uint32_t>(base, kOffDs + ds_tot_offset(G)), err, &sorted));
    } else {
        if (n > 1)
            NA_CUDA(radix_sort_u32_pairs(s, keys, ids, n, 0, 32, at<uint32_t>(base, kOffHist),
                                         at<uint32_t>(base, kOffStatus), at<uint32_t>(base, kOffCounter), err,
                                         &sorted));
        NA_CUDA(launch_scan_gathered(s, at<uint32_t>(base, kOffSupers), nullptr, ids[sorted], n, offsets,
                                     at<unsigned long long>(base, kOffDsSum), at<uint32_t>(base, kOffCounter),
                                     scan_tot, err));
    }

    uint64_t* pairs[2] = {at<uint64_t>(base, kOffPairs0), at<uint64_t>(base, kOffPairs1)};
    uint32_t* scounts = at<uint32_t>(base, kOffSCounts);
    uint32_t* hist = at<uint32_t>(base, kOffHist);
    const int sbits = bits_for_na(Ts);
    const int spasses = radix_passes(32, 32 + sbits);
    NA_CUDA(cudaMemsetAsync(scounts, 0, sizeof(uint32_t) * kCountCopies * Ts, s));
    NA_CUDA(launch_emit_pairs(s, ids[sorted], offsets, at<ushort4>(base, kOffRect), n, ks, stiles_x, pairs[0],
                              scounts, Ts, Ps));
    NA_CUDA(launch_supers_to_hist(s, scounts, Ts, spasses, hist, sranges, PairCheckIn{nullptr, Ps ? Ps : 1u, 0},
                                  nullptr, err));
    int psorted = 0;
    if (Ps > 1 && Ts > 1)
        NA_CUDA(radix_sort_u64_keys(s, pairs, Ps, 32, 32 + sbits, hist, at<uint32_t>(base, kOffStatus),
                                    at<uint32_t>(base, kOffCounter), err, &psorted, true));

    BlendArgs a;
    a.W = W;
    a.H = H;
    a.tiles_x = tiles_x;
    a.tiles_y = tiles_y;
    a.stiles_x = stiles_x;
    a.ks = ks;
    a.n = n;
    a.sranges = sranges;
    a.pair_words = reinterpret_cast<const uint32_t*>(pairs[psorted]);
    a.rect = at<ushort4>(base, kOffRect);
    a.rec = rec;
    a.bg = make_float3(o.bg[0], o.bg[1], o.bg[2]);
    a.out_C = out_C;
    a.out_G = out_grads;
    a.state = nullptr;
    a.count = nullptr;
    a.order = nullptr;
    a.work = nullptr;
    NA_CUDA(launch_blend(s, true, o.mode, a));

    // report a bounded device wait that expired (outputs are then undefined)
    int h_err = 0;
    NA_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (h_err == kDevTimeout) return GS_ERR_TIMEOUT;
    if (h_err != kDevOk) return GS_ERR_DEVICE_CHECK;
    return GS_OK;
}
