// C ABI of libgs (declared in include/gs.h): context, scratch management and the
// orchestration of the kernels of each call.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "gs_internal.cuh"

using namespace gs;

int64_t& gs::launch_counter()
{
    thread_local int64_t count = 0;
    return count;
}

namespace {

// Adds the kernels launched during one API call to the context's tally.
struct LaunchTally {
    gs_ctx* c;
    int64_t start;
    explicit LaunchTally(gs_ctx* ctx) : c(ctx), start(launch_counter()) {}
    ~LaunchTally()
    {
        if (c) c->launches += launch_counter() - start;
    }
};

gs_status fail(gs_ctx* c, gs_status st, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

gs_status cuda_fail(gs_ctx* c, cudaError_t e, const char* where)
{
    cudaGetLastError();   // clear a sticky-free error so the context stays usable
    return fail(c, e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA, "%s: %s", where,
                cudaGetErrorString(e));
}

#define GS_CUDA(ctx, expr)                                    \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr); \
    } while (0)

// Grow a scratch buffer to at least `bytes` (1.25x headroom).  Frees only after
// the stream has drained, so in-flight kernels never lose their memory.
gs_status ensure(gs_ctx* c, DevBuf& b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return GS_OK;
    if (c->reserved)   // after gs_reserve no call allocates
        return fail(c, GS_ERR_CAPACITY, "a buffer of %zu bytes exceeds the reserved capacity", bytes);
    size_t want = bytes + bytes / 4;
    if (c->inject_alloc_countdown >= 0 && c->inject_alloc_countdown-- == 0)   // gs_debug_inject
        return fail(c, GS_ERR_OOM, "cudaMalloc(%zu) failed: injected allocation failure", want);
    if (b.p) {
        GS_CUDA(c, cudaStreamSynchronize(c->stream));
        cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GS_ERR_OOM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    b.cap = want;
    return GS_OK;
}

void release(DevBuf& b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

template <typename T>
T* as(DevBuf& b)
{
    return reinterpret_cast<T*>(b.p);
}


// The next blend's tile order, computed beside the projection's histogram
// kernel (a 256-thread block) when the recorded durations belong to this tile
// layout and the tiles are few enough for that block (else the blend launches
// its own 1024-thread ordering: 8160 tiles of a 1920 x 1080 frame took the
// shared launch from 7.6 to 20.3 us).
struct OrderJob {
    const uint32_t* work = nullptr;
    uint32_t T = 0;
    uint32_t* order = nullptr;
};
OrderJob order_job(gs_ctx* c, uint32_t T)
{
    OrderJob j;
    constexpr uint32_t kMaxSharedOrderTiles = 4096;
    if (T > 0 && T <= kMaxSharedOrderTiles && c->work_tiles == (int64_t)T && c->tile_work.cap >= sizeof(uint32_t) * T &&
        c->tile_order.cap >= sizeof(uint32_t) * T) {
        j.work = as<uint32_t>(c->tile_work);
        j.T = T;
        j.order = as<uint32_t>(c->tile_order);
    }
    return j;
}

int bits_for(uint32_t v)   // number of bits to represent values < v (v >= 1)
{
    int b = 0;
    while (b < 32 && (uint64_t(1) << b) < v) ++b;
    return b;
}

gs_status check_options(gs_ctx* c, const gs_options* o)
{
    if (o->tile != kTile) return fail(c, GS_ERR_INVALID_ARG, "tile must be %d", kTile);
    if (o->mode != GS_MODE_3DGS && o->mode != GS_MODE_EXACT) return fail(c, GS_ERR_INVALID_ARG, "bad mode");
    if (o->max_pairs < 0) return fail(c, GS_ERR_INVALID_ARG, "max_pairs < 0");
    if (o->flags & ~(GS_FLAG_NO_HOST_WAIT | GS_FLAG_BWD_RECOMPUTE))
        return fail(c, GS_ERR_INVALID_ARG, "unknown flags 0x%x", o->flags);
    return GS_OK;
}

gs_status check_gaussians(gs_ctx* c, const gs_gaussians* g)
{
    if (!g) return fail(c, GS_ERR_INVALID_ARG, "gaussians == NULL");
    if (g->n < 0 || g->n > 0x7FFFFFFF) return fail(c, GS_ERR_INVALID_ARG, "n out of range");
    if (g->n == 0) return GS_OK;
    if (!g->means || !g->log_scales || !g->quats || !g->opacity_logits)
        return fail(c, GS_ERR_INVALID_ARG, "a required Gaussian array is NULL");
    if (!g->sh && !g->rgb) return fail(c, GS_ERR_INVALID_ARG, "both sh and rgb are NULL");
    if (g->sh && (g->sh_degree < 0 || g->sh_degree > 3)) return fail(c, GS_ERR_INVALID_ARG, "sh_degree not in 0..3");
    return GS_OK;
}

CameraParams make_camera(const gs_camera& cam, int W, int H)
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

gs_status read_device_error(gs_ctx* c)
{
    int h = 0;
    GS_CUDA(c, cudaMemcpyAsync(&h, c->errword.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    if (h != kDevOk) {
        GS_CUDA(c, cudaMemsetAsync(c->errword.p, 0, sizeof(int), c->stream));
        if (h == kDevTimeout) return fail(c, GS_ERR_TIMEOUT, "a bounded device wait expired");
        if (h == kDevCapacity) {
            PairCheckOut o{};
            if (c->pair_check.p) {
                GS_CUDA(c, cudaMemcpy(&o, c->pair_check.p, sizeof(o), cudaMemcpyDeviceToHost));
            }
            return fail(c, GS_ERR_CAPACITY,
                        "a frame needed %llu super-tile pairs (reserved %lld) and %llu tile pairs (limit %lld); "
                        "it was rendered without Gaussians", o.needed, (long long)c->res_pairs, o.tile_pairs,
                        (long long)(c->opt.max_pairs > 0 ? c->opt.max_pairs : kMaxPairs));
        }
        return fail(c, GS_ERR_DEVICE_CHECK, "a device-side check failed (code %d)", h);
    }
    return GS_OK;
}

gs_status do_project(gs_ctx* c, const gs_gaussians* g, const gs_camera* cam, int W, int H)
{
    if (!cam) return fail(c, GS_ERR_INVALID_ARG, "camera == NULL");
    if (W < 1 || H < 1 || W > (1 << 20) || H > (1 << 20)) return fail(c, GS_ERR_INVALID_ARG, "bad image size");
    gs_status st = check_gaussians(c, g);
    if (st != GS_OK) return st;
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return fail(c, GS_ERR_INVALID_ARG, "fx, fy must be > 0");
    c->have_proj = false;
    c->have_state = false;
    c->order_ready = false;
    c->batch_views = 0;
    const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
    const int ks = super_side(tiles_x, tiles_y, c->opt.mode);
    const int stiles_x = (tiles_x + ks - 1) / ks, stiles_y = (tiles_y + ks - 1) / ks;
    const int64_t T = (int64_t)tiles_x * tiles_y;
    const int64_t Ts = (int64_t)stiles_x * stiles_y;
    if (T > 0x7FFFFFFF) return fail(c, GS_ERR_INVALID_ARG, "too many tiles");
    if (Ts > 65536) return fail(c, GS_ERR_INVALID_ARG, "more than 65536 super-tiles (image over 16384 x 16384)");
    const uint32_t n = (uint32_t)g->n;
    const bool no_wait = (c->opt.flags & GS_FLAG_NO_HOST_WAIT) != 0;
    if (no_wait) {
        if (!c->reserved) return fail(c, GS_ERR_NOT_READY, "GS_FLAG_NO_HOST_WAIT needs gs_reserve first");
        if ((int64_t)n > c->res_n || T > c->res_tiles || Ts > c->res_supers || (int64_t)W * H > c->res_pixels)
            return fail(c, GS_ERR_CAPACITY, "frame (n %u, %d x %d) exceeds the reserved sizes", n, W, H);
    }

    // per-Gaussian scratch
    if ((st = ensure(c, c->rec0, sizeof(float4) * n)) || (st = ensure(c, c->rec1, sizeof(float4) * n)) ||
        (st = ensure(c, c->rec2, sizeof(float4) * n)) || (st = ensure(c, c->depth, sizeof(float) * n)) ||
        (st = ensure(c, c->radius, sizeof(int) * n)) || (st = ensure(c, c->rect, sizeof(ushort4) * n)) ||
        (st = ensure(c, c->tiles_touched, sizeof(uint32_t) * n)) ||
        (st = ensure(c, c->supers_touched, sizeof(uint32_t) * n)) ||
        (st = ensure(c, c->dkey[0], sizeof(uint32_t) * n)) || (st = ensure(c, c->dkey[1], sizeof(uint32_t) * n)) ||
        (st = ensure(c, c->did[0], sizeof(uint32_t) * n)) || (st = ensure(c, c->did[1], sizeof(uint32_t) * n)) ||
        (st = ensure(c, c->offsets, sizeof(uint32_t) * (n + 1))) ||
        (st = ensure(c, c->scan_partials, sizeof(unsigned long long) * scan_partials_count(n))) ||
        (st = ensure(c, c->scan_totals, (2 * kTotalSlots + 4) * sizeof(unsigned long long))) ||
        (st = ensure(c, c->super_counts, sizeof(uint32_t) * kCountCopies * Ts)) ||
        (st = ensure(c, c->sranges, sizeof(uint2) * Ts)) || (st = ensure(c, c->sort_hist, sizeof(uint32_t) * 8 * 256)) ||
        (st = ensure(c, c->sort_status, sizeof(uint32_t) * radix_status_words(n, 0, 32))) ||
        (st = ensure(c, c->sort_counter, sizeof(uint32_t) * 8)))
        return st;

    const Records rec{as<float4>(c->rec0), as<float4>(c->rec1), as<float4>(c->rec2)};
    const CameraParams cp = make_camera(*cam, W, H);
    c->last_g = *g;
    c->last_cam = cp;
    // scan_totals: [0, 2 kTotalSlots) slot pairs (super-tile pairs, tile pairs)
    // from the projection, then 2 scan totals and the scan tile counter
    unsigned long long* totals = as<unsigned long long>(c->scan_totals);
    unsigned long long* scan_tot = totals + 2 * kTotalSlots;
    // counters of the frame's later kernels, cleared by the projection kernel
    const uint32_t ds_cap = n > 1 ? depth_sort_capacity(c->device) : 0u;
    const bool persistent = n > 1 && n <= ds_cap && n <= kDsMaxN;
    const size_t G = ds_cap / kDsMaxSlice;
    const bool counted = Ts <= kMaxSupersForCounts;
    const int sbits = bits_for((uint32_t)Ts);
    const int spasses = radix_passes(32, 32 + sbits);
    ZeroList zl{};
    if (persistent) {
        if ((st = ensure(c, c->ds_scratch, ds_scratch_bytes(G)))) return st;
        unsigned char* base = as<unsigned char>(c->ds_scratch);
        zl.p[zl.count] = reinterpret_cast<uint32_t*>(base + ds_zero_offset(G));   // barrier and totals
        zl.words[zl.count++] = ds_zero_words();
    }
    if (counted) {
        zl.p[zl.count] = as<uint32_t>(c->super_counts);
        zl.words[zl.count++] = (uint32_t)(kCountCopies * Ts);
    }
    // the pair sort's look-back states and tile counters -- only when the depth
    // sort is the persistent kernel: the one-sweep depth sort uses the same
    // state buffer, so the pair sort then clears it itself
    const bool pairs_prezeroed = no_wait && Ts > 1 && persistent;
    if (pairs_prezeroed) {
        zl.p[zl.count] = as<uint32_t>(c->sort_status);
        zl.words[zl.count++] = (uint32_t)radix_status_words((uint32_t)c->res_pairs, 32, 32 + sbits);
        zl.p[zl.count] = as<uint32_t>(c->sort_counter);
        zl.words[zl.count++] = (uint32_t)spasses;
    }
    GS_CUDA(c, cudaMemsetAsync(totals, 0, 2 * kTotalSlots * sizeof(unsigned long long), c->stream));
    GS_CUDA(c, launch_project(c->stream, *g, cp, W, H, tiles_x, tiles_y, ks, c->opt.mode, rec, as<float>(c->depth),
                              as<int>(c->radius), as<ushort4>(c->rect), as<uint32_t>(c->tiles_touched),
                              as<uint32_t>(c->supers_touched), as<uint32_t>(c->dkey[0]), as<uint32_t>(c->did[0]),
                              totals, &zl));
    if (!no_wait) {
        // the pair totals travel to the host while the depth sort runs
        GS_CUDA(c, cudaMemcpyAsync(c->h_scalar, totals, 2 * kTotalSlots * sizeof(unsigned long long),
                                   cudaMemcpyDeviceToHost, c->stream));
        GS_CUDA(c, cudaEventRecord(c->totals_ready, c->stream));
    }

    // depth order (stable radix sort of the FP32 depth bits, ids ascending) and
    // the super-tile pair offsets in that order
    int sorted = 0;
    if (persistent) {
        unsigned char* base = as<unsigned char>(c->ds_scratch);
        uint32_t* keys[2] = {as<uint32_t>(c->dkey[0]), as<uint32_t>(c->dkey[1])};
        uint32_t* vals[2] = {as<uint32_t>(c->did[0]), as<uint32_t>(c->did[1])};
        GS_CUDA(c, launch_depth_sort_scan(c->stream, c->device, keys[0], keys, vals, as<uint32_t>(c->supers_touched), n,
                                          as<uint32_t>(c->offsets), reinterpret_cast<uint32_t*>(base + ds_cnt_offset(G)),
                                          reinterpret_cast<uint32_t*>(base + ds_csum_offset(G)),
                                          reinterpret_cast<unsigned int*>(base + ds_bar_offset(G)),
                                          reinterpret_cast<uint32_t*>(base + ds_tot_offset(G)),
                                          as<int>(c->errword), &sorted, true, c->inject_wait_spins));
        c->inject_wait_spins = 0;
    } else {
        if (n > 1) {
            uint32_t* keys[2] = {as<uint32_t>(c->dkey[0]), as<uint32_t>(c->dkey[1])};
            uint32_t* vals[2] = {as<uint32_t>(c->did[0]), as<uint32_t>(c->did[1])};
            GS_CUDA(c, radix_sort_u32_pairs(c->stream, keys, vals, n, 0, 32, as<uint32_t>(c->sort_hist),
                                            as<uint32_t>(c->sort_status), as<uint32_t>(c->sort_counter),
                                            as<int>(c->errword), &sorted));
        }
        GS_CUDA(c, launch_scan_gathered(c->stream, as<uint32_t>(c->supers_touched), nullptr,
                                        as<uint32_t>(c->did[sorted]), n, as<uint32_t>(c->offsets),
                                        as<unsigned long long>(c->scan_partials),
                                        reinterpret_cast<uint32_t*>(scan_tot + 2), scan_tot, as<int>(c->errword)));
    }
    c->sorted_ids_buf = sorted;
    const uint32_t* ids = as<uint32_t>(c->did[sorted]);
    const int64_t limit = c->opt.max_pairs > 0 ? std::min<int64_t>(c->opt.max_pairs, kMaxPairs) : kMaxPairs;

    if (no_wait) {
        // the pair totals stay on the device: emit into the reserved buffers and
        // let the histogram kernel check the frame against their capacity
        const uint32_t cap = (uint32_t)c->res_pairs;
        uint64_t* pairs[2] = {as<uint64_t>(c->pairs[0]), as<uint64_t>(c->pairs[1])};
        PairCheckOut* chk = as<PairCheckOut>(c->pair_check);
        GS_CUDA(c, launch_emit_pairs(c->stream, ids, as<uint32_t>(c->offsets), as<ushort4>(c->rect), n, ks, stiles_x,
                                     pairs[0], as<uint32_t>(c->super_counts), (uint32_t)Ts, cap));
        const OrderJob job = order_job(c, (uint32_t)(tiles_x * tiles_y));
        GS_CUDA(c, launch_supers_to_hist(c->stream, as<uint32_t>(c->super_counts), (uint32_t)Ts, spasses,
                                         as<uint32_t>(c->sort_hist), as<uint2>(c->sranges),
                                         PairCheckIn{totals, cap, (unsigned long long)limit}, chk,
                                         as<int>(c->errword), job.work, job.T, job.order));
        c->order_ready = job.order != nullptr;
        int psorted = 0;
        if (Ts > 1 && cap > 1)
            GS_CUDA(c, radix_sort_u64_keys(c->stream, pairs, cap, 32, 32 + sbits, as<uint32_t>(c->sort_hist),
                                           as<uint32_t>(c->sort_status), as<uint32_t>(c->sort_counter),
                                           as<int>(c->errword), &psorted, true, &chk->count, pairs_prezeroed));
        c->sorted_pairs_buf = psorted;
        c->n = n;
        c->W = W;
        c->H = H;
        c->ks = ks;
        c->tiles_x = tiles_x;
        c->tiles_y = tiles_y;
        c->stiles_x = stiles_x;
        c->stiles_y = stiles_y;
        c->P = -1;
        c->Ps = -1;
        c->totals_known = false;
        c->have_proj = true;
        return GS_OK;
    }

    GS_CUDA(c, cudaEventSynchronize(c->totals_ready));
    unsigned long long Ps64 = 0, P64 = 0;
    for (int k = 0; k < kTotalSlots; ++k) {
        Ps64 += c->h_scalar[2 * k];
        P64 += c->h_scalar[2 * k + 1];
    }
    if ((int64_t)P64 > limit)
        return fail(c, GS_ERR_CAPACITY, "pair count %llu exceeds the limit %lld", P64, (long long)limit);
    if ((int64_t)Ps64 > kMaxPairs)
        return fail(c, GS_ERR_CAPACITY, "super-tile pair count %llu exceeds %lld", Ps64, (long long)kMaxPairs);
    const uint32_t Ps = (uint32_t)Ps64;

    if ((st = ensure(c, c->pairs[0], sizeof(uint64_t) * Ps)) || (st = ensure(c, c->pairs[1], sizeof(uint64_t) * Ps)))
        return st;
    if ((st = ensure(c, c->sort_status, sizeof(uint32_t) * std::max(radix_status_words(Ps, 32, 32 + sbits),
                                                                    radix_status_words(n, 0, 32)))))
        return st;
    uint64_t* pairs[2] = {as<uint64_t>(c->pairs[0]), as<uint64_t>(c->pairs[1])};
    GS_CUDA(c, launch_emit_pairs(c->stream, ids, as<uint32_t>(c->offsets), as<ushort4>(c->rect), n, ks, stiles_x,
                                 pairs[0], counted ? as<uint32_t>(c->super_counts) : nullptr, (uint32_t)Ts, Ps));
    int psorted = 0;
    if (counted) {
        // digit histograms of the super-tile passes and the super-tile ranges,
        // both from the per-super-tile counts (checked against the buffers)
        const OrderJob job = order_job(c, (uint32_t)(tiles_x * tiles_y));
        GS_CUDA(c, launch_supers_to_hist(c->stream, as<uint32_t>(c->super_counts), (uint32_t)Ts, spasses,
                                         as<uint32_t>(c->sort_hist), as<uint2>(c->sranges),
                                         PairCheckIn{nullptr, Ps ? Ps : 1u, 0}, nullptr, as<int>(c->errword),
                                         job.work, job.T, job.order));
        c->order_ready = job.order != nullptr;
        if (Ps > 1 && Ts > 1)
            GS_CUDA(c, radix_sort_u64_keys(c->stream, pairs, Ps, 32, 32 + sbits, as<uint32_t>(c->sort_hist),
                                           as<uint32_t>(c->sort_status), as<uint32_t>(c->sort_counter),
                                           as<int>(c->errword), &psorted, true));
    } else {
        if (Ps > 1 && Ts > 1)
            GS_CUDA(c, radix_sort_u64_keys(c->stream, pairs, Ps, 32, 32 + sbits, as<uint32_t>(c->sort_hist),
                                           as<uint32_t>(c->sort_status), as<uint32_t>(c->sort_counter),
                                           as<int>(c->errword), &psorted, false));
        GS_CUDA(c, cudaMemsetAsync(c->sranges.p, 0, sizeof(uint2) * Ts, c->stream));
        GS_CUDA(c, launch_ranges(c->stream, pairs[psorted], Ps, (uint32_t)Ts, as<uint2>(c->sranges)));
    }
    c->sorted_pairs_buf = psorted;

    c->n = n;
    c->W = W;
    c->H = H;
    c->ks = ks;
    c->tiles_x = tiles_x;
    c->tiles_y = tiles_y;
    c->stiles_x = stiles_x;
    c->stiles_y = stiles_y;
    c->P = (int64_t)P64;
    c->Ps = Ps;
    c->totals_known = true;
    c->have_proj = true;
    return GS_OK;
}

BlendArgs blend_args(gs_ctx* c, float* out_C, float* out_grads)
{
    BlendArgs a;
    a.W = c->W;
    a.H = c->H;
    a.tiles_x = c->tiles_x;
    a.tiles_y = c->tiles_y;
    a.stiles_x = c->stiles_x;
    a.ks = c->ks;
    a.n = (uint32_t)c->n;
    a.sranges = as<uint2>(c->sranges);
    a.pair_words = reinterpret_cast<const uint32_t*>(c->pairs[c->sorted_pairs_buf].p);
    a.rect = as<ushort4>(c->rect);
    a.rec = Records{as<float4>(c->rec0), as<float4>(c->rec1), as<float4>(c->rec2)};
    a.bg = make_float3(c->opt.bg[0], c->opt.bg[1], c->opt.bg[2]);
    a.out_C = out_C;
    a.out_G = out_grads;
    a.state = as<float4>(c->state);
    a.count = as<int>(c->count);
    a.order = nullptr;
    a.work = nullptr;
    return a;
}

gs_status do_blend(gs_ctx* c, float* out_C, float* out_grads)
{
    if (!c->have_proj) return fail(c, GS_ERR_NOT_READY, "no projection: call gs_project first");
    if (!out_C) return fail(c, GS_ERR_INVALID_ARG, "out_C == NULL");
    const size_t npix = (size_t)c->W * c->H;
    gs_status st;
    if ((st = ensure(c, c->state, sizeof(float4) * npix)) || (st = ensure(c, c->count, sizeof(int) * npix))) return st;
    // tiles heaviest first, by the durations the previous frame's blocks recorded
    const uint32_t T = (uint32_t)(c->tiles_x * c->tiles_y);
    if ((st = ensure(c, c->tile_work, sizeof(uint32_t) * T)) || (st = ensure(c, c->tile_order, sizeof(uint32_t) * T)))
        return st;
    if (c->work_tiles != (int64_t)T) {   // a new tile layout: no history yet
        GS_CUDA(c, cudaMemsetAsync(c->tile_work.p, 0, sizeof(uint32_t) * T, c->stream));
        c->work_tiles = T;
    }
    if (!c->order_ready)   // else the projection's histogram launch computed it
        GS_CUDA(c, launch_tile_order(c->stream, as<uint32_t>(c->tile_work), T, as<uint32_t>(c->tile_order)));
    c->order_ready = false;
    BlendArgs a = blend_args(c, out_C, out_grads);
    a.order = as<uint32_t>(c->tile_order);
    a.work = as<uint32_t>(c->tile_work);
    GS_CUDA(c, launch_blend(c->stream, out_grads != nullptr, c->opt.mode, a));
    c->have_state = true;
    c->state_grads = out_grads != nullptr;
    return GS_OK;
}

}  // namespace

extern "C" {

const char* gs_status_string(gs_status s)
{
    switch (s) {
    case GS_OK: return "GS_OK";
    case GS_ERR_INVALID_ARG: return "GS_ERR_INVALID_ARG";
    case GS_ERR_CUDA: return "GS_ERR_CUDA";
    case GS_ERR_OOM: return "GS_ERR_OOM";
    case GS_ERR_CAPACITY: return "GS_ERR_CAPACITY";
    case GS_ERR_TIMEOUT: return "GS_ERR_TIMEOUT";
    case GS_ERR_DEVICE_CHECK: return "GS_ERR_DEVICE_CHECK";
    case GS_ERR_NOT_READY: return "GS_ERR_NOT_READY";
    }
    return "GS_ERR_UNKNOWN";
}

const char* gs_last_error(const gs_ctx* ctx)
{
    return ctx ? ctx->err : "";
}

gs_status gs_create(gs_ctx** out, void* stream, const gs_options* opt)
{
    if (!out) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    gs_options o{};
    o.tile = kTile;
    o.mode = GS_MODE_3DGS;
    if (opt) o = *opt;
    if (check_options(nullptr, &o) != GS_OK) return GS_ERR_INVALID_ARG;
    gs_ctx* c = new (std::nothrow) gs_ctx();
    if (!c) return GS_ERR_OOM;
    c->opt = o;
    c->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return GS_ERR_CUDA;
    }
    if (cudaMallocHost((void**)&c->h_scalar, 2 * kTotalSlots * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return GS_ERR_OOM;
    }
    if (cudaEventCreateWithFlags(&c->totals_ready, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(c->h_scalar);
        delete c;
        return GS_ERR_CUDA;
    }
    if (ensure(c, c->errword, sizeof(int)) != GS_OK) {
        cudaFreeHost(c->h_scalar);
        delete c;
        return GS_ERR_OOM;
    }
    if (cudaMemsetAsync(c->errword.p, 0, sizeof(int), c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
        cudaGetLastError();
        release(c->errword);
        cudaFreeHost(c->h_scalar);
        delete c;
        return GS_ERR_CUDA;
    }
    *out = c;
    return GS_OK;
}

gs_status gs_destroy(gs_ctx* c)
{
    if (!c) return GS_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->stream);
    DevBuf* bufs[] = {&c->rec0, &c->rec1, &c->rec2, &c->depth, &c->radius, &c->rect, &c->tiles_touched,
                      &c->supers_touched, &c->dkey[0], &c->dkey[1], &c->did[0], &c->did[1], &c->offsets,
                      &c->scan_partials, &c->scan_totals, &c->super_counts, &c->ds_scratch, &c->pairs[0],
                      &c->pairs[1],
                      &c->sort_hist, &c->sort_status,
                      &c->sort_counter, &c->sranges, &c->tile_count, &c->tile_start, &c->state, &c->count,
                      &c->errword, &c->grad2d, &c->pair_check, &c->tile_work, &c->tile_order,
                      &c->vrec0, &c->vrec1, &c->vrec2, &c->vrect, &c->vsupers, &c->vkey, &c->vtotals,
                      &c->views_dev, &c->vpairs0, &c->vpairs1, &c->vsranges, &c->vwork, &c->vorder, &c->vqueue,
                      &c->vsortv, &c->vcounts, &c->vhist, &c->vstatus, &c->vdhist, &c->vdstatus, &c->ckpt};
    for (DevBuf* b : bufs) release(*b);
    if (c->h_scalar) cudaFreeHost(c->h_scalar);
    if (c->totals_ready) cudaEventDestroy(c->totals_ready);
    cudaGetLastError();
    delete c;
    return GS_OK;
}

gs_status gs_set_stream(gs_ctx* c, void* stream)
{
    if (!c) return GS_ERR_INVALID_ARG;
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    c->stream = (cudaStream_t)stream;
    return GS_OK;
}

gs_status gs_set_options(gs_ctx* c, const gs_options* opt)
{
    if (!c || !opt) return GS_ERR_INVALID_ARG;
    gs_status st = check_options(c, opt);
    if (st != GS_OK) return st;
    c->opt = *opt;
    c->have_proj = false;
    c->have_state = false;
    c->order_ready = false;
    c->batch_views = 0;
    return GS_OK;
}

gs_status gs_project(gs_ctx* c, const gs_gaussians* g, const gs_camera* cam, int32_t W, int32_t H)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    return do_project(c, g, cam, W, H);
}

gs_status gs_render_binned(gs_ctx* c, float* out_C, float* out_grads)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    return do_blend(c, out_C, out_grads);
}

gs_status gs_render_with_grads(gs_ctx* c, const gs_gaussians* g, const gs_camera* cam, int32_t W, int32_t H,
                               float* out_C, float* out_grads)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (!out_C || !out_grads) return fail(c, GS_ERR_INVALID_ARG, "out_C and out_grads are required");
    gs_status st = do_project(c, g, cam, W, H);
    if (st != GS_OK) return st;
    return do_blend(c, out_C, out_grads);
}

gs_status gs_render(gs_ctx* c, const gs_gaussians* g, const gs_camera* cam, int32_t W, int32_t H, float* out_C)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (!out_C) return fail(c, GS_ERR_INVALID_ARG, "out_C is required");
    gs_status st = do_project(c, g, cam, W, H);
    if (st != GS_OK) return st;
    return do_blend(c, out_C, nullptr);
}

gs_status gs_upscale(gs_ctx* c, const float* C, const float* grads, int32_t W, int32_t H, int32_t factor,
                     float* out)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (!C || !grads || !out) return fail(c, GS_ERR_INVALID_ARG, "NULL image pointer");
    if (W < 2 || H < 2) return fail(c, GS_ERR_INVALID_ARG, "upscale needs W, H >= 2");
    if (factor < 1 || factor > 16) return fail(c, GS_ERR_INVALID_ARG, "factor must be in 1..16");
    if ((int64_t)W * factor > (1 << 24) || (int64_t)H * factor > (1 << 24))
        return fail(c, GS_ERR_INVALID_ARG, "output too large");
    GS_CUDA(c, launch_upscale(c->stream, C, grads, W, H, factor, out, as<int>(c->errword)));
    return GS_OK;
}

namespace {

gs_status check_sizes(gs_ctx* c, int32_t W, int32_t H, int32_t W2, int32_t H2, int32_t min_side)
{
    if (W < min_side || H < min_side) return fail(c, GS_ERR_INVALID_ARG, "input must be at least %d x %d", min_side, min_side);
    if (W2 < W || H2 < H || (int64_t)W2 > 16ll * W || (int64_t)H2 > 16ll * H)
        return fail(c, GS_ERR_INVALID_ARG, "output %d x %d must be 1 to 16 times the input %d x %d", W2, H2, W, H);
    if (W2 > (1 << 24) || H2 > (1 << 24)) return fail(c, GS_ERR_INVALID_ARG, "output too large");
    return GS_OK;
}

}  // namespace

gs_status gs_upscale_to(gs_ctx* c, const float* C, const float* grads, int32_t W, int32_t H, int32_t W2, int32_t H2,
                        float* out)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (!C || !grads || !out) return fail(c, GS_ERR_INVALID_ARG, "NULL image pointer");
    gs_status st = check_sizes(c, W, H, W2, H2, 2);
    if (st != GS_OK) return st;
    GS_CUDA(c, launch_upscale_to(c->stream, C, grads, W, H, W2, H2, out, as<int>(c->errword)));
    return GS_OK;
}

gs_status gs_upscale_mlp(gs_ctx* c, const float* C, const float* grads, int32_t W, int32_t H, int32_t W2, int32_t H2,
                         const float* params, float* out)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (!C || !grads || !out) return fail(c, GS_ERR_INVALID_ARG, "NULL image pointer");
    gs_status st = check_sizes(c, W, H, W2, H2, 2);
    if (st != GS_OK) return st;
    if (!params) {
        GS_CUDA(c, launch_upscale_to(c->stream, C, grads, W, H, W2, H2, out, as<int>(c->errword)));
        return GS_OK;
    }
    GS_CUDA(c, launch_mlp_upscale(c->stream, C, grads, W, H, W2, H2, params, out, as<int>(c->errword)));
    return GS_OK;
}

gs_status gs_mlp_samples(gs_ctx* c, const float* C, const float* grads, int32_t W, int32_t H, int32_t W2, int32_t H2,
                         const int32_t* pixels, int64_t M, const float* target_image, uint16_t* features, float* base,
                         float* target)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (M < 0) return fail(c, GS_ERR_INVALID_ARG, "M < 0");
    if (M == 0) return GS_OK;
    if (!C || !grads || !pixels || !features || !base) return fail(c, GS_ERR_INVALID_ARG, "NULL pointer");
    if ((target_image == nullptr) != (target == nullptr))
        return fail(c, GS_ERR_INVALID_ARG, "target_image and target go together");
    if (reinterpret_cast<uintptr_t>(features) % 16) return fail(c, GS_ERR_INVALID_ARG, "features not 16-byte aligned");
    gs_status st = check_sizes(c, W, H, W2, H2, 2);
    if (st != GS_OK) return st;
    GS_CUDA(c, launch_mlp_samples(c->stream, C, grads, W, H, W2, H2, pixels, M, target_image, features, base, target,
                                  as<int>(c->errword)));
    return GS_OK;
}

gs_status gs_mlp_gradient(gs_ctx* c, const float* params, const uint16_t* features, const float* base,
                          const float* target, int64_t M, float* grads, float* loss)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (M < 0) return fail(c, GS_ERR_INVALID_ARG, "M < 0");
    if (!params || !grads || (M > 0 && (!features || !base || !target)))
        return fail(c, GS_ERR_INVALID_ARG, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(features) % 16) return fail(c, GS_ERR_INVALID_ARG, "features not 16-byte aligned");
    GS_CUDA(c, launch_mlp_grad(c->stream, params, features, base, target, M, grads, loss, as<int>(c->errword)));
    return GS_OK;
}

gs_status gs_mlp_adam(gs_ctx* c, float* params, float* m, float* v, const float* grads, int32_t step, float lr,
                      float beta1, float beta2, float eps)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (!params || !m || !v || !grads) return fail(c, GS_ERR_INVALID_ARG, "NULL pointer");
    if (step < 1) return fail(c, GS_ERR_INVALID_ARG, "step must be >= 1");
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f && lr >= 0.f))
        return fail(c, GS_ERR_INVALID_ARG, "need 0 <= beta < 1, eps > 0, lr >= 0");
    GS_CUDA(c, launch_mlp_adam(c->stream, params, m, v, grads, step, lr, beta1, beta2, eps));
    return GS_OK;
}

gs_status gs_upscale_backward_to(gs_ctx* c, const float* dL_dout, int32_t W, int32_t H, int32_t W2, int32_t H2,
                                 float* dL_dC, float* dL_dgrads)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (!dL_dout || !dL_dC || !dL_dgrads) return fail(c, GS_ERR_INVALID_ARG, "NULL image pointer");
    gs_status st = check_sizes(c, W, H, W2, H2, 2);
    if (st != GS_OK) return st;
    GS_CUDA(c, launch_upscale_backward_to(c->stream, dL_dout, W, H, W2, H2, dL_dC, dL_dgrads));
    return GS_OK;
}

gs_status gs_upscale_bicubic(gs_ctx* c, const float* C, int32_t W, int32_t H, int32_t W2, int32_t H2, float a,
                             float* out)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (!C || !out) return fail(c, GS_ERR_INVALID_ARG, "NULL image pointer");
    if (!(a >= -2.f && a <= 0.f)) return fail(c, GS_ERR_INVALID_ARG, "a must be in [-2, 0]");
    gs_status st = check_sizes(c, W, H, W2, H2, 1);
    if (st != GS_OK) return st;
    GS_CUDA(c, launch_bicubic(c->stream, C, W, H, W2, H2, a, out));
    return GS_OK;
}

gs_status gs_upscale_backward(gs_ctx* c, const float* dL_dout, int32_t W, int32_t H, int32_t factor,
                              float* dL_dC, float* dL_dgrads)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (!dL_dout || !dL_dC || !dL_dgrads) return fail(c, GS_ERR_INVALID_ARG, "NULL image pointer");
    if (W < 2 || H < 2) return fail(c, GS_ERR_INVALID_ARG, "upscale needs W, H >= 2");
    if (factor < 1 || factor > 16) return fail(c, GS_ERR_INVALID_ARG, "factor must be in 1..16");
    if ((int64_t)W * factor > (1 << 24) || (int64_t)H * factor > (1 << 24))
        return fail(c, GS_ERR_INVALID_ARG, "output too large");
    GS_CUDA(c, launch_upscale_backward(c->stream, dL_dout, W, H, factor, dL_dC, dL_dgrads));
    return GS_OK;
}

namespace {

gs_status do_render_backward(gs_ctx* c, const float* dC, const float* dG, float* grad2d, const float* dout = nullptr,
                             int factor = 0)
{
    if ((!dC && !dout) || !grad2d) return fail(c, GS_ERR_INVALID_ARG, "dL_dC and grad2d are required");
    const bool recompute = (c->opt.flags & GS_FLAG_BWD_RECOMPUTE) != 0;
    if (!c->have_proj || (!recompute && (!c->have_state || !c->state_grads)))
        return fail(c, GS_ERR_NOT_READY, "no derivative blend since the last projection");
    gs_status st;
    if (recompute &&
        (st = ensure(c, c->ckpt, sizeof(float4) * kCkSlots * kTilePixels * (size_t)c->tiles_x * c->tiles_y)))
        return st;
    if (c->n > 0) GS_CUDA(c, cudaMemsetAsync(grad2d, 0, sizeof(float) * 9 * (size_t)c->n, c->stream));
    BlendBwdArgs a;
    a.W = c->W;
    a.H = c->H;
    a.tiles_x = c->tiles_x;
    a.stiles_x = c->stiles_x;
    a.ks = c->ks;
    a.n = (uint32_t)c->n;
    a.sranges = as<uint2>(c->sranges);
    a.pair_words = reinterpret_cast<const uint32_t*>(c->pairs[c->sorted_pairs_buf].p);
    a.rect = as<ushort4>(c->rect);
    a.rec = Records{as<float4>(c->rec0), as<float4>(c->rec1), as<float4>(c->rec2)};
    a.bg = make_float3(c->opt.bg[0], c->opt.bg[1], c->opt.bg[2]);
    a.state = as<float4>(c->state);
    a.count = as<int>(c->count);
    a.dC = dC;
    a.dG = dG;
    a.dout = dout;
    a.W2 = c->W * factor;
    a.H2 = c->H * factor;
    a.grad2d = grad2d;
    a.err = as<int>(c->errword);
    // the forward blend's tile order of this frame (heaviest first)
    a.order = c->work_tiles == (int64_t)c->tiles_x * c->tiles_y && c->tile_order.p ? as<uint32_t>(c->tile_order)
                                                                                   : nullptr;
    a.ckpt = recompute ? as<float4>(c->ckpt) : nullptr;
    GS_CUDA(c, launch_blend_backward(c->stream, c->opt.mode, a));
    return GS_OK;
}

gs_status do_project_backward(gs_ctx* c, const float* grad2d, const gs_gaussian_grads* out)
{
    if (!grad2d || !out) return fail(c, GS_ERR_INVALID_ARG, "grad2d and out are required");
    if (!c->have_proj) return fail(c, GS_ERR_NOT_READY, "no projection");
    if (c->n > 0 && (!out->means || !out->log_scales || !out->quats || !out->opacity_logits))
        return fail(c, GS_ERR_INVALID_ARG, "means, log_scales, quats and opacity_logits gradients are required");
    GS_CUDA(c, launch_project_backward(c->stream, c->last_g, c->last_cam, grad2d, *out));
    return GS_OK;
}

}  // namespace

gs_status gs_render_backward(gs_ctx* c, const float* dL_dC, const float* dL_dgrads, float* grad2d)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    return do_render_backward(c, dL_dC, dL_dgrads, grad2d);
}

gs_status gs_project_backward(gs_ctx* c, const float* grad2d, const gs_gaussian_grads* out)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    return do_project_backward(c, grad2d, out);
}

gs_status gs_backward(gs_ctx* c, const float* dL_dout, int32_t factor, const gs_gaussian_grads* out)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (!dL_dout || !out) return fail(c, GS_ERR_INVALID_ARG, "dL_dout and out are required");
    if (!c->have_proj ||
        (!(c->opt.flags & GS_FLAG_BWD_RECOMPUTE) && (!c->have_state || !c->state_grads)))
        return fail(c, GS_ERR_NOT_READY, "no derivative blend since the last projection");
    if (c->W < 2 || c->H < 2) return fail(c, GS_ERR_INVALID_ARG, "upscale needs W, H >= 2");
    if (factor < 1 || factor > 16) return fail(c, GS_ERR_INVALID_ARG, "factor must be in 1..16");
    gs_status st;
    if ((st = ensure(c, c->grad2d, sizeof(float) * 9 * (size_t)std::max<int64_t>(c->n, 1)))) return st;
    // the upscale's adjoint fused into the blend's: no low-res upstream planes
    if ((st = do_render_backward(c, nullptr, nullptr, as<float>(c->grad2d), dL_dout, factor)) != GS_OK) return st;
    return do_project_backward(c, as<float>(c->grad2d), out);
}

namespace {

// P and Ps of the last projection; after a frame without a host wait they are
// read from the device (waiting for the stream).
gs_status known_totals(gs_ctx* c)
{
    if (c->totals_known) return GS_OK;
    PairCheckOut o[kMaxViews] = {};
    const int k = c->batch_views > 0 ? c->batch_views : 1;   // after a batch: the sums over its views
    GS_CUDA(c, cudaMemcpyAsync(o, c->pair_check.p, sizeof(PairCheckOut) * k, cudaMemcpyDeviceToHost, c->stream));
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    c->P = c->Ps = 0;
    for (int v = 0; v < k; ++v) {
        c->P += (int64_t)o[v].tile_pairs;
        c->Ps += (int64_t)o[v].needed;
    }
    c->totals_known = true;
    return GS_OK;
}

}  // namespace

gs_status gs_pair_count(gs_ctx* c, int64_t* P)
{
    if (!c || !P) return GS_ERR_INVALID_ARG;
    if (!c->have_proj && c->batch_views == 0) return GS_ERR_NOT_READY;
    gs_status st = known_totals(c);
    if (st != GS_OK) return st;
    *P = c->P;
    return GS_OK;
}

gs_status gs_super_pair_count(gs_ctx* c, int64_t* Ps)
{
    if (!c || !Ps) return GS_ERR_INVALID_ARG;
    if (!c->have_proj && c->batch_views == 0) return GS_ERR_NOT_READY;
    gs_status st = known_totals(c);
    if (st != GS_OK) return st;
    *Ps = c->Ps;
    return GS_OK;
}

namespace {

gs_status reserve_impl(gs_ctx* c, int64_t n, int32_t V, int32_t W, int32_t H, int64_t super_pairs)
{
    if (n < 0 || n > 0x7FFFFFFF || W < 1 || H < 1 || super_pairs < 1 || super_pairs > kMaxPairs || V < 0 ||
        V > kMaxViews)
        return fail(c, GS_ERR_INVALID_ARG, "bad reserve sizes");
    const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
    const int stiles_x = (tiles_x + kSuperMax - 1) / kSuperMax, stiles_y = (tiles_y + kSuperMax - 1) / kSuperMax;
    const int64_t T = (int64_t)tiles_x * tiles_y;
    // every frame up to W x H: the largest super-tiles give at most Ts4 of them,
    // smaller ones (chosen only when they fit one sort pass) at most 256
    const int64_t Ts = std::max<int64_t>((int64_t)stiles_x * stiles_y, std::min<int64_t>(kSuperOnePass, T));
    if (Ts > kMaxSupersForCounts)
        return fail(c, GS_ERR_INVALID_ARG, "%lld super-tiles exceed %d", (long long)Ts, kMaxSupersForCounts);
    const size_t un = (size_t)std::max<int64_t>(n, 1), pix = (size_t)W * H;
    const uint32_t nn = (uint32_t)un;
    c->reserved = false;
    gs_status st;
    const int sbits = bits_for((uint32_t)Ts);
    const uint32_t ds_cap = depth_sort_capacity(c->device);
    const size_t G = ds_cap / kDsMaxSlice;
    if ((st = ensure(c, c->rec0, sizeof(float4) * un)) || (st = ensure(c, c->rec1, sizeof(float4) * un)) ||
        (st = ensure(c, c->rec2, sizeof(float4) * un)) || (st = ensure(c, c->depth, sizeof(float) * un)) ||
        (st = ensure(c, c->radius, sizeof(int) * un)) || (st = ensure(c, c->rect, sizeof(ushort4) * un)) ||
        (st = ensure(c, c->tiles_touched, sizeof(uint32_t) * un)) ||
        (st = ensure(c, c->supers_touched, sizeof(uint32_t) * un)) ||
        (st = ensure(c, c->dkey[0], sizeof(uint32_t) * un)) || (st = ensure(c, c->dkey[1], sizeof(uint32_t) * un)) ||
        (st = ensure(c, c->did[0], sizeof(uint32_t) * un)) || (st = ensure(c, c->did[1], sizeof(uint32_t) * un)) ||
        (st = ensure(c, c->offsets, sizeof(uint32_t) * (un + 1))) ||
        (st = ensure(c, c->scan_partials, sizeof(unsigned long long) * scan_partials_count(nn))) ||
        (st = ensure(c, c->scan_totals, (2 * kTotalSlots + 4) * sizeof(unsigned long long))) ||
        (st = ensure(c, c->super_counts, sizeof(uint32_t) * kCountCopies * Ts)) ||
        (st = ensure(c, c->sranges, sizeof(uint2) * Ts)) || (st = ensure(c, c->sort_hist, sizeof(uint32_t) * 8 * 256)) ||
        (st = ensure(c, c->sort_status,
                     sizeof(uint32_t) * std::max(radix_status_words((uint32_t)super_pairs, 32, 32 + sbits),
                                                 radix_status_words(nn, 0, 32)))) ||
        (st = ensure(c, c->sort_counter, sizeof(uint32_t) * 8)) ||
        (st = ensure(c, c->ds_scratch, ds_scratch_bytes(G))) ||
        (st = ensure(c, c->pairs[0], sizeof(uint64_t) * (size_t)super_pairs)) ||
        (st = ensure(c, c->pairs[1], sizeof(uint64_t) * (size_t)super_pairs)) ||
        (st = ensure(c, c->state, sizeof(float4) * pix)) || (st = ensure(c, c->count, sizeof(int) * pix)) ||
        (st = ensure(c, c->tile_count, sizeof(uint32_t) * T)) || (st = ensure(c, c->tile_start, sizeof(uint32_t) * T)) ||
        (st = ensure(c, c->tile_work, sizeof(uint32_t) * T)) || (st = ensure(c, c->tile_order, sizeof(uint32_t) * T)) ||
        (st = ensure(c, c->grad2d, sizeof(float) * 9 * un)) ||
        (st = ensure(c, c->pair_check, sizeof(PairCheckOut))) ||
        ((c->opt.flags & GS_FLAG_BWD_RECOMPUTE) &&
         (st = ensure(c, c->ckpt, sizeof(float4) * kCkSlots * kTilePixels * (size_t)T))))
        return st;
    if (V > 0) {
        const size_t vn = un * (size_t)V;
        if (vn >= 0xFFFFFFFFull)
            return fail(c, GS_ERR_CAPACITY, "%d views of %lld Gaussians exceed 2^32 entries", V, (long long)n);
        // the views' depth sorts: 32-bit keys, both ping-pong halves in the
        // first pair buffer (free until the views' pairs are emitted), values
        // in vkey and vsortv
        const size_t per_view = std::max<size_t>((size_t)super_pairs, un);
        if ((st = ensure(c, c->vsortv, sizeof(uint32_t) * vn)) ||
            (st = ensure(c, c->vdhist, sizeof(uint32_t) * 4 * 256 * (size_t)V)) ||
            (st = ensure(c, c->vdstatus, sizeof(uint32_t) * (radix_status_words(nn, 0, 32) + 8) * V)) ||
            (st = ensure(c, c->offsets, sizeof(uint32_t) * (vn + 1))) ||
            (st = ensure(c, c->scan_partials, sizeof(unsigned long long) * scan_partials_count((uint32_t)vn))) ||
            (st = ensure(c, c->sort_status, sizeof(uint32_t) * std::max(radix_status_words(nn, 0, 32),
                                                                         radix_status_words((uint32_t)super_pairs, 32,
                                                                                            32 + sbits)))))
            return st;
        if ((st = ensure(c, c->vrec0, sizeof(float4) * vn)) || (st = ensure(c, c->vrec1, sizeof(float4) * vn)) ||
            (st = ensure(c, c->vrec2, sizeof(float4) * vn)) || (st = ensure(c, c->vrect, sizeof(ushort4) * vn)) ||
            (st = ensure(c, c->vsupers, sizeof(uint32_t) * vn)) || (st = ensure(c, c->vkey, sizeof(uint32_t) * vn)) ||
            (st = ensure(c, c->vtotals, sizeof(unsigned long long) * 2 * kTotalSlots * (size_t)V)) ||
            (st = ensure(c, c->views_dev, sizeof(ViewDesc) * kMaxViews)) ||
            (st = ensure(c, c->vpairs0, sizeof(uint64_t) * per_view * V)) ||
            (st = ensure(c, c->vpairs1, sizeof(uint64_t) * per_view * V)) ||
            (st = ensure(c, c->vsranges, sizeof(uint2) * (size_t)Ts * V)) ||
            (st = ensure(c, c->vwork, sizeof(uint32_t) * (size_t)T * V)) ||
            (st = ensure(c, c->vorder, sizeof(uint32_t) * (size_t)T * V)) ||
            (st = ensure(c, c->vqueue, sizeof(uint32_t))) ||
            (st = ensure(c, c->vcounts, sizeof(uint32_t) * kCountCopies * (size_t)Ts * V)) ||
            (st = ensure(c, c->vhist, sizeof(uint32_t) * 8 * 256 * (size_t)V)) ||
            (st = ensure(c, c->vstatus, sizeof(uint32_t) *
                                            (radix_status_words((uint32_t)super_pairs, 32, 32 + sbits) + 8) * V)) ||
            (st = ensure(c, c->pair_check, sizeof(PairCheckOut) * (size_t)V)))
            return st;
        c->vstatus_stride = radix_status_words((uint32_t)super_pairs, 32, 32 + sbits) + 8;
        c->vdstatus_stride = radix_status_words(nn, 0, 32) + 8;
        GS_CUDA(c, cudaMemsetAsync(c->vwork.p, 0, sizeof(uint32_t) * (size_t)T * V, c->stream));
    }
    GS_CUDA(c, cudaStreamSynchronize(c->stream));
    c->res_views = V;
    c->res_n = n;
    c->res_pixels = (int64_t)pix;
    c->res_tiles = T;
    c->res_supers = Ts;
    c->res_pairs = super_pairs;
    c->reserved = true;
    return GS_OK;
}

}  // namespace

gs_status gs_reserve(gs_ctx* c, int64_t n, int32_t W, int32_t H, int64_t super_pairs)
{
    if (!c) return GS_ERR_INVALID_ARG;
    return reserve_impl(c, n, 0, W, H, super_pairs);
}

gs_status gs_reserve_views(gs_ctx* c, int64_t n, int32_t V, int32_t W, int32_t H, int64_t super_pairs)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (V < 1) return fail(c, GS_ERR_INVALID_ARG, "V must be >= 1");
    return reserve_impl(c, n, V, W, H, super_pairs);
}

namespace {

// A batch of views over one or several Gaussian sets (gs_render_views,
// gs_render_views_scenes).  Launches: per Gaussian set one projection of all
// its views; one stable sort of every (view, depth) key of the batch; one
// pair-offset scan; one emission; one histogram launch; one launch per pass
// of the pair sort over every view's pairs; one blend of every tile of every
// view; one upscale of every view.  No host wait.
gs_status render_views_impl(gs_ctx* c, const gs_gaussians* scenes, int32_t S, const int32_t* scene_of_view, int32_t V,
                            const gs_camera* cams, const int32_t* Ws, const int32_t* Hs, float* const* out_C,
                            float* const* out_grads, const int32_t* factors, float* const* out_up)
{
    if (!(c->opt.flags & GS_FLAG_NO_HOST_WAIT) || !c->reserved || c->res_views < 1)
        return fail(c, GS_ERR_NOT_READY, "batched views need GS_FLAG_NO_HOST_WAIT and gs_reserve_views");
    if (V < 1 || V > c->res_views) return fail(c, GS_ERR_CAPACITY, "%d views, %d reserved", V, c->res_views);
    if (!scenes || S < 1 || S > kMaxViews) return fail(c, GS_ERR_INVALID_ARG, "1 <= S <= %d Gaussian sets", kMaxViews);
    if (!cams || !Ws || !Hs || !out_C || !out_grads) return fail(c, GS_ERR_INVALID_ARG, "NULL argument");
    gs_status st;
    for (int k = 0; k < S; ++k) {
        if ((st = check_gaussians(c, &scenes[k])) != GS_OK) return st;
        if (scenes[k].n > c->res_n)
            return fail(c, GS_ERR_CAPACITY, "Gaussian set %d: n %lld exceeds the reserved %lld", k,
                        (long long)scenes[k].n, (long long)c->res_n);
    }
    // views grouped by Gaussian set (each set's views contiguous, in view order)
    ViewBatch batch{};
    int order[kMaxViews];
    int set_first[kMaxViews + 1];
    uint32_t nview[kMaxViews];
    uint64_t total64 = 0;
    {
        int q = 0;
        for (int k = 0; k < S; ++k) {
            set_first[k] = q;
            for (int v = 0; v < V; ++v)
                if ((scene_of_view ? scene_of_view[v] : 0) == k) order[q++] = v;
        }
        set_first[S] = q;
        if (q != V) return fail(c, GS_ERR_INVALID_ARG, "a view's Gaussian set index is outside 0..%d", S - 1);
    }
    for (int v = 0; v < V; ++v) {
        const int W = Ws[v], H = Hs[v];
        if (W < 1 || H < 1 || !(cams[v].fx > 0.f) || !(cams[v].fy > 0.f) || !out_C[v] || !out_grads[v])
            return fail(c, GS_ERR_INVALID_ARG, "bad view %d", v);
        const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
        const int64_t T = (int64_t)tiles_x * tiles_y;
        const int ks = c->views_ks ? c->views_ks : super_side(tiles_x, tiles_y, c->opt.mode);
        const int64_t Ts = (int64_t)((tiles_x + ks - 1) / ks) * ((tiles_y + ks - 1) / ks);
        if (T > c->res_tiles || Ts > c->res_supers || (int64_t)W * H > c->res_pixels)
            return fail(c, GS_ERR_CAPACITY, "view %d (%d x %d) exceeds the reserved sizes", v, W, H);
        if (out_up && out_up[v]) {
            const int f = factors ? factors[v] : 0;
            if (f < 1 || f > 16 || W < 2 || H < 2) return fail(c, GS_ERR_INVALID_ARG, "bad upscale of view %d", v);
        }
        nview[v] = (uint32_t)scenes[scene_of_view ? scene_of_view[v] : 0].n;
    }
    // the view's entries in the batch arrays, in view order
    uint32_t start[kMaxViews + 1];
    for (int v = 0; v < V; ++v) {
        start[v] = (uint32_t)total64;
        total64 += nview[v];
    }
    start[V] = (uint32_t)total64;
    if (total64 > (uint64_t)c->res_n * (uint64_t)c->res_views || total64 >= 0xFFFFFFFFull)
        return fail(c, GS_ERR_CAPACITY, "the batch's %llu (view, Gaussian) entries exceed the reservation",
                    (unsigned long long)total64);
    const uint32_t total = (uint32_t)total64;
    for (int q = 0; q < V; ++q) {   // descriptions grouped by Gaussian set
        const int v = order[q];
        ViewDesc& d = batch.v[q];
        d.cam = make_camera(cams[v], Ws[v], Hs[v]);
        d.W = Ws[v];
        d.H = Hs[v];
        d.tiles_x = (Ws[v] + kTile - 1) / kTile;
        d.tiles_y = (Hs[v] + kTile - 1) / kTile;
        d.ks = c->views_ks ? c->views_ks : super_side(d.tiles_x, d.tiles_y, c->opt.mode);
        d.off = start[v];
        d.vid = v;
    }
    c->have_proj = false;
    c->have_state = false;
    c->order_ready = false;
    cudaStream_t s = c->stream;
    unsigned long long* vtot = as<unsigned long long>(c->vtotals);
    GS_CUDA(c, cudaMemsetAsync(vtot, 0, sizeof(unsigned long long) * 2 * kTotalSlots * V, s));
    GS_CUDA(c, launch_set_views(s, batch, V, as<ViewDesc>(c->views_dev)));
    // the views' depth sorts: keys in the first pair buffer (free until the
    // views' pairs are emitted), values (batch entries) in vkey and vsortv
    const size_t vcap = (size_t)c->res_n * c->res_views;
    uint32_t* k32[2] = {as<uint32_t>(c->vpairs0), as<uint32_t>(c->vpairs0) + vcap};
    uint32_t* v32[2] = {as<uint32_t>(c->vkey), as<uint32_t>(c->vsortv)};
    ViewOutputs vo;
    vo.rec = Records{as<float4>(c->vrec0), as<float4>(c->vrec1), as<float4>(c->vrec2)};
    vo.rect = as<ushort4>(c->vrect);
    vo.supers = as<uint32_t>(c->vsupers);
    vo.depth_key = k32[0];
    vo.gidx = v32[0];
    vo.totals = vtot;
    vo.pack_counts = total <= kPackedIdxMask;   // entries in the low 24 bits, the pair count above
    for (int k = 0; k < S; ++k) {   // one projection launch per Gaussian set, over its views
        const int nv = set_first[k + 1] - set_first[k];
        if (nv > 0)
            GS_CUDA(c, launch_project_views(s, scenes[k], as<ViewDesc>(c->views_dev) + set_first[k], nv, c->opt.mode,
                                            vo));
    }
    // every view's Gaussians in its own depth order (each view's stretch of
    // the batch sorted as a segment of its own: a stable sort of the 32-bit
    // depth keys, which start in id order), then the super-tile pair offsets
    // over the whole order
    {
        SortSegs ds{};
        ds.count = V;
        const size_t dstride = c->vdstatus_stride;
        GS_CUDA(c, cudaMemsetAsync(c->vdhist.p, 0, sizeof(uint32_t) * 4 * 256 * V, s));
        GS_CUDA(c, cudaMemsetAsync(c->vdstatus.p, 0, sizeof(uint32_t) * dstride * V, s));
        for (int v = 0; v < V; ++v) {
            SortSeg& q = ds.seg[v];
            for (int b = 0; b < 2; ++b) {
                q.keys[b] = k32[b] + start[v];
                q.vals[b] = v32[b] + start[v];
            }
            q.n_dev = nullptr;
            q.cap = nview[v];
            q.tiles = radix_tiles(nview[v]);
            q.passes = 4;   // even: the sorted entries land in v32[0]
            q.bit_lo = 0;
            q.hist = as<uint32_t>(c->vdhist) + (size_t)v * 4 * 256;
            q.status = as<uint32_t>(c->vdstatus) + (size_t)v * dstride;
            q.counters = q.status + dstride - 8;
            q.err = as<int>(c->errword);
        }
        GS_CUDA(c, radix_sort_u32_pairs_segs(s, ds));
    }
    const uint32_t* vsorted = v32[0];
    unsigned long long* scan_tot = as<unsigned long long>(c->scan_totals) + 2 * kTotalSlots;
    GS_CUDA(c, launch_scan_gathered(s, as<uint32_t>(c->vsupers), nullptr, vsorted, total, as<uint32_t>(c->offsets),
                                    as<unsigned long long>(c->scan_partials), reinterpret_cast<uint32_t*>(scan_tot + 2),
                                    scan_tot, as<int>(c->errword), vo.pack_counts));

    // per view: its pair buffers, counts, histograms, sort state and ranges
    const int64_t limit = c->opt.max_pairs > 0 ? std::min<int64_t>(c->opt.max_pairs, kMaxPairs) : kMaxPairs;
    const uint32_t cap = (uint32_t)c->res_pairs;
    const size_t counts_stride = (size_t)kCountCopies * c->res_supers;
    const size_t status_stride = c->vstatus_stride;
    PairCheckOut* chk = as<PairCheckOut>(c->pair_check);
    EmitViews ev{};
    HistViews hv{};
    SortSegs sg{};
    BlendViews bv;
    bv.V = V;
    bv.start[0] = 0;
    UpscaleViews uv;
    uv.V = 0;
    uv.start[0] = 0;
    ev.V = hv.V = sg.count = V;
    GS_CUDA(c, cudaMemsetAsync(c->vcounts.p, 0, sizeof(uint32_t) * counts_stride * V, s));
    GS_CUDA(c, cudaMemsetAsync(c->vstatus.p, 0, sizeof(uint32_t) * status_stride * V, s));
    for (int v = 0; v < V; ++v) {
        const int q = [&] { for (int i = 0; i < V; ++i) if (order[i] == v) return i; return 0; }();
        const ViewDesc& d = batch.v[q];
        const int stiles_x = (d.tiles_x + d.ks - 1) / d.ks, stiles_y = (d.tiles_y + d.ks - 1) / d.ks;
        const uint32_t Ts = (uint32_t)(stiles_x * stiles_y);
        const int sbits = bits_for(Ts);
        const int spasses = Ts > 1 ? radix_passes(32, 32 + sbits) : 0;
        uint64_t* pairs[2] = {as<uint64_t>(c->vpairs0) + (size_t)v * cap, as<uint64_t>(c->vpairs1) + (size_t)v * cap};
        uint32_t* counts_v = as<uint32_t>(c->vcounts) + (size_t)v * counts_stride;
        uint32_t* hist_v = as<uint32_t>(c->vhist) + (size_t)v * 8 * 256;
        uint32_t* status_v = as<uint32_t>(c->vstatus) + (size_t)v * status_stride;
        uint2* sranges_v = as<uint2>(c->vsranges) + (size_t)v * c->res_supers;
        EmitView& e = ev.v[v];
        e.pairs = pairs[0];
        e.counts = counts_v;
        e.start = start[v];
        e.n = nview[v];
        e.cap = cap;
        e.Ts = Ts;
        e.ks = d.ks;
        e.stiles_x = stiles_x;
        HistView& h = hv.v[v];
        h.counts = counts_v;
        h.Ts = Ts;
        h.passes = spasses;
        h.hist = hist_v;
        h.ranges = sranges_v;
        h.in = PairCheckIn{vtot + (size_t)v * 2 * kTotalSlots, cap, (unsigned long long)limit};
        h.out = chk + v;
        SortSeg& g = sg.seg[v];
        g.keys[0] = pairs[0];
        g.keys[1] = pairs[1];
        g.n_dev = &chk[v].count;
        g.cap = cap;
        g.tiles = radix_tiles(cap);
        g.passes = spasses;
        g.bit_lo = 32;
        g.hist = hist_v;
        g.status = status_v;
        g.counters = status_v + status_stride - 8;   // the last 8 words of the view's (zeroed) state
        g.err = as<int>(c->errword);
        BlendArgs& a = bv.a[v];
        a.W = d.W;
        a.H = d.H;
        a.tiles_x = d.tiles_x;
        a.tiles_y = d.tiles_y;
        a.stiles_x = stiles_x;
        a.ks = d.ks;
        a.n = nview[v];
        a.sranges = sranges_v;
        a.pair_words = reinterpret_cast<const uint32_t*>(pairs[spasses & 1]);
        a.rect = as<ushort4>(c->vrect) + start[v];
        a.rec = Records{as<float4>(c->vrec0) + start[v], as<float4>(c->vrec1) + start[v],
                        as<float4>(c->vrec2) + start[v]};
        a.bg = make_float3(c->opt.bg[0], c->opt.bg[1], c->opt.bg[2]);
        a.out_C = out_C[v];
        a.out_G = out_grads[v];
        a.state = nullptr;
        a.count = nullptr;
        a.order = nullptr;
        a.work = nullptr;
        bv.start[v + 1] = bv.start[v] + d.tiles_x * d.tiles_y;
        if (out_up && out_up[v]) {
            UpscaleView& u = uv.v[uv.V];
            u.C = out_C[v];
            u.G = out_grads[v];
            u.W = d.W;
            u.H = d.H;
            u.W2 = d.W * factors[v];
            u.H2 = d.H * factors[v];
            u.out = out_up[v];
            uv.start[uv.V + 1] = uv.start[uv.V] + upscale_tiles(u.W2, u.H2);
            ++uv.V;
        }
    }
    GS_CUDA(c, launch_emit_views(s, ev, vsorted, as<uint32_t>(c->offsets), as<ushort4>(c->vrect), total,
                                 vo.pack_counts));
    GS_CUDA(c, launch_supers_to_hist_views(s, hv, as<int>(c->errword)));
    GS_CUDA(c, radix_sort_u64_segs(s, sg));
    const int tiles_total = bv.start[V];
    bv.work = as<uint32_t>(c->vwork);
    bv.queue = as<uint32_t>(c->vqueue);
    bv.order = nullptr;
    if (c->views_sched == 1) {   // heaviest tiles of the last batch first
        GS_CUDA(c, launch_tile_order(s, as<uint32_t>(c->vwork), (uint32_t)tiles_total, as<uint32_t>(c->vorder)));
        bv.order = as<uint32_t>(c->vorder);
    } else if (c->views_sched == 3) {   // the views in order, each view's heaviest tiles first
        GS_CUDA(c, launch_tile_order_views(s, as<uint32_t>(c->vwork), bv.start, V, as<uint32_t>(c->vorder)));
        bv.order = as<uint32_t>(c->vorder);
    }
    GS_CUDA(c, launch_blend_views(s, c->opt.mode, bv, c->views_map, c->views_sched == 2));
    if (uv.V > 0) GS_CUDA(c, launch_upscale_views(s, uv));
    c->totals_known = false;
    c->batch_views = V;
    return GS_OK;
}

}  // namespace

gs_status gs_render_views(gs_ctx* c, const gs_gaussians* g, int32_t V, const gs_camera* cams, const int32_t* Ws,
                          const int32_t* Hs, float* const* out_C, float* const* out_grads, const int32_t* factors,
                          float* const* out_up)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (!g) return fail(c, GS_ERR_INVALID_ARG, "gaussians == NULL");
    return render_views_impl(c, g, 1, nullptr, V, cams, Ws, Hs, out_C, out_grads, factors, out_up);
}

gs_status gs_render_views_scenes(gs_ctx* c, const gs_gaussians* scenes, int32_t S, const int32_t* scene_of_view,
                                 int32_t V, const gs_camera* cams, const int32_t* Ws, const int32_t* Hs,
                                 float* const* out_C, float* const* out_grads, const int32_t* factors,
                                 float* const* out_up)
{
    if (!c) return GS_ERR_INVALID_ARG;
    LaunchTally tally(c);
    if (!scene_of_view) return fail(c, GS_ERR_INVALID_ARG, "scene_of_view == NULL");
    return render_views_impl(c, scenes, S, scene_of_view, V, cams, Ws, Hs, out_C, out_grads, factors, out_up);
}

gs_status gs_views_config(gs_ctx* c, int32_t warp_map, int32_t schedule, int32_t super_side_tiles)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (warp_map < 0 || warp_map > 1 || schedule < 0 || schedule > 3)
        return fail(c, GS_ERR_INVALID_ARG, "warp_map in {0, 1}, schedule in {0, 1, 2, 3}");
    if (super_side_tiles != 0 && super_side_tiles != kSuperMax)
        return fail(c, GS_ERR_INVALID_ARG, "super-tile side 0 (per view) or %d", kSuperMax);
    c->views_map = warp_map;
    c->views_sched = schedule;
    c->views_ks = super_side_tiles;
    return GS_OK;
}

namespace {

gs_status autotune_impl(gs_ctx* c, const gs_gaussians* scenes, int32_t S, const int32_t* scene_of_view, int32_t V,
                        const gs_camera* cams, const int32_t* Ws, const int32_t* Hs, float* const* out_C,
                        float* const* out_grads, const int32_t* factors, float* const* out_up, int32_t reps,
                        float* ms, int32_t* best)
{
    if (reps < 1) return fail(c, GS_ERR_INVALID_ARG, "reps must be >= 1");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GS_CUDA(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, GS_ERR_CUDA, "cudaEventCreate failed");
    }
    float best_ms = 0.f;
    int best_k = -1;
    gs_status st = GS_OK;
    for (int k = 0; k < GS_VIEWS_CONFIGS && st == GS_OK; ++k) {
        c->views_map = k & 1;
        c->views_sched = (k >> 1) & 3;
        c->views_ks = (k >> 3) ? kSuperMax : 0;
        // one untimed batch: first use of the variant, and tile durations for schedules 1 and 3
        st = render_views_impl(c, scenes, S, scene_of_view, V, cams, Ws, Hs, out_C, out_grads, factors, out_up);
        if (st != GS_OK) break;
        if (cudaEventRecord(e0, c->stream) != cudaSuccess) { st = fail(c, GS_ERR_CUDA, "event"); break; }
        for (int r = 0; r < reps && st == GS_OK; ++r)
            st = render_views_impl(c, scenes, S, scene_of_view, V, cams, Ws, Hs, out_C, out_grads, factors, out_up);
        if (st != GS_OK) break;
        float t = 0.f;
        if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            st = fail(c, GS_ERR_CUDA, "event timing failed");
            break;
        }
        t /= (float)reps;
        if (ms) ms[k] = t;
        if (best_k < 0 || t < best_ms) {
            best_ms = t;
            best_k = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GS_OK) return st;
    c->views_map = best_k & 1;
    c->views_sched = (best_k >> 1) & 3;
    c->views_ks = (best_k >> 3) ? kSuperMax : 0;
    if (best) *best = best_k;
    return read_device_error(c);
}

}  // namespace

gs_status gs_autotune_views(gs_ctx* c, const gs_gaussians* g, int32_t V, const gs_camera* cams, const int32_t* Ws,
                            const int32_t* Hs, float* const* out_C, float* const* out_grads, const int32_t* factors,
                            float* const* out_up, int32_t reps, float* ms, int32_t* best)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!g) return fail(c, GS_ERR_INVALID_ARG, "gaussians == NULL");
    return autotune_impl(c, g, 1, nullptr, V, cams, Ws, Hs, out_C, out_grads, factors, out_up, reps, ms, best);
}

gs_status gs_autotune_views_scenes(gs_ctx* c, const gs_gaussians* scenes, int32_t S, const int32_t* scene_of_view,
                                   int32_t V, const gs_camera* cams, const int32_t* Ws, const int32_t* Hs,
                                   float* const* out_C, float* const* out_grads, const int32_t* factors,
                                   float* const* out_up, int32_t reps, float* ms, int32_t* best)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!scene_of_view) return fail(c, GS_ERR_INVALID_ARG, "scene_of_view == NULL");
    return autotune_impl(c, scenes, S, scene_of_view, V, cams, Ws, Hs, out_C, out_grads, factors, out_up, reps, ms,
                         best);
}

gs_status gs_read_projected(gs_ctx* c, float* mean2d, float* conic, float* rgb, float* opacity, float* depth,
                            int32_t* radius, int32_t* tiles_touched)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!c->have_proj) return fail(c, GS_ERR_NOT_READY, "no projection");
    const Records rec{as<float4>(c->rec0), as<float4>(c->rec1), as<float4>(c->rec2)};
    GS_CUDA(c, launch_unpack_projected(c->stream, rec, as<int>(c->radius), as<uint32_t>(c->tiles_touched),
                                       as<float>(c->depth), (uint32_t)c->n, mean2d, conic, rgb, opacity, depth,
                                       radius, tiles_touched));
    return GS_OK;
}

gs_status gs_read_bins(gs_ctx* c, uint64_t* keys, uint32_t* vals, uint32_t* ranges, int64_t capacity)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!c->have_proj) return fail(c, GS_ERR_NOT_READY, "no projection");
    gs_status st0 = known_totals(c);
    if (st0 != GS_OK) return st0;
    if ((keys || vals) && capacity < c->P) return fail(c, GS_ERR_CAPACITY, "capacity %lld < P %lld",
                                                       (long long)capacity, (long long)c->P);
    LaunchTally tally(c);
    const size_t T = (size_t)c->tiles_x * c->tiles_y;
    gs_status st;
    if ((st = ensure(c, c->tile_count, sizeof(uint32_t) * T)) || (st = ensure(c, c->tile_start, sizeof(uint32_t) * T)))
        return st;
    GS_CUDA(c, launch_tile_lists(c->stream, as<uint64_t>(c->pairs[c->sorted_pairs_buf]), as<uint2>(c->sranges),
                                 as<ushort4>(c->rect), as<float>(c->depth), (uint32_t)c->n, c->tiles_x, c->tiles_y,
                                 c->ks, c->stiles_x, as<uint32_t>(c->tile_count), as<uint32_t>(c->tile_start), keys, vals,
                                 reinterpret_cast<uint2*>(ranges)));
    return GS_OK;
}

gs_status gs_read_state(gs_ctx* c, float* state, int32_t* count)
{
    if (!c) return GS_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, GS_ERR_NOT_READY, "no blend state");
    const size_t npix = (size_t)c->W * c->H;
    if (state) {
        // float4 per pixel -> four planes
        GS_CUDA(c, cudaMemcpy2DAsync(state, sizeof(float), c->state.p, sizeof(float4), sizeof(float), npix,
                                     cudaMemcpyDeviceToDevice, c->stream));
        for (int k = 1; k < 4; ++k)
            GS_CUDA(c, cudaMemcpy2DAsync(state + k * npix, sizeof(float), as<float>(c->state) + k, sizeof(float4),
                                         sizeof(float), npix, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (count) GS_CUDA(c, cudaMemcpyAsync(count, c->count.p, sizeof(int) * npix, cudaMemcpyDeviceToDevice, c->stream));
    return GS_OK;
}

gs_status gs_read_tile_work(gs_ctx* c, uint32_t* work)
{
    if (!c || !work) return GS_ERR_INVALID_ARG;
    if (!c->have_state) return fail(c, GS_ERR_NOT_READY, "no blend state");
    const size_t T = (size_t)c->tiles_x * c->tiles_y;
    GS_CUDA(c, cudaMemcpyAsync(work, c->tile_work.p, sizeof(uint32_t) * T, cudaMemcpyDeviceToDevice, c->stream));
    return GS_OK;
}

gs_status gs_blend_stats(gs_ctx* c, int64_t* counts)
{
    if (!c || !counts) return GS_ERR_INVALID_ARG;
    if (!c->have_proj) return fail(c, GS_ERR_NOT_READY, "no projection");
    LaunchTally tally(c);
    DevBuf tmp;
    if (cudaMalloc(&tmp.p, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GS_ERR_OOM, "gs_blend_stats: cudaMalloc failed");
    }
    tmp.cap = 2 * sizeof(unsigned long long);
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(tmp.p, 0, 2 * sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) {
        const BlendArgs a = blend_args(c, nullptr, nullptr);
        e = launch_blend_stats(c->stream, c->opt.mode, a, as<unsigned long long>(tmp));
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, tmp.p, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    release(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "gs_blend_stats");
    counts[0] = (int64_t)h[0];
    counts[1] = (int64_t)h[1];
    return GS_OK;
}

gs_status gs_debug_inject(gs_ctx* c, int32_t what, int64_t value)
{
    if (!c) return GS_ERR_INVALID_ARG;
    switch (what) {
    case GS_INJECT_NONE:
        c->inject_wait_spins = 0;
        c->inject_alloc_countdown = -1;
        return GS_OK;
    case GS_INJECT_WAIT_EXPIRY:
        if (value < 1 || value > (1 << 24)) return fail(c, GS_ERR_INVALID_ARG, "polls must be in 1..2^24");
        c->inject_wait_spins = (uint32_t)value;
        return GS_OK;
    case GS_INJECT_ALLOC_FAILURE:
        if (value < 0) return fail(c, GS_ERR_INVALID_ARG, "countdown must be >= 0");
        c->inject_alloc_countdown = value;
        return GS_OK;
    }
    return fail(c, GS_ERR_INVALID_ARG, "unknown injection %d", what);
}

gs_status gs_launch_count(const gs_ctx* c, int64_t* count)
{
    if (!c || !count) return GS_ERR_INVALID_ARG;
    *count = c->launches;
    return GS_OK;
}

gs_status gs_synchronize(gs_ctx* c)
{
    if (!c) return GS_ERR_INVALID_ARG;
    return read_device_error(c);
}

}  // extern "C"
