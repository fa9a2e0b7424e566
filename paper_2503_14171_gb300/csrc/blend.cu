// Front-to-back blend of each tile's Gaussians with the analytic screen-space
// derivatives of the pixel colour (Sec. 4 blend equation; Sec. 5 "3DGS Image
// Gradients"; supplement "Forward pass").
//
// One 256-thread block per 16x16 tile, one pixel per thread (each warp an 8x4
// block of pixels).  Binning is done
// per super-tile of ks x ks tiles (ks = 1, 2 or 4 per frame): the block walks
// its super-tile's depth-ordered list 256 candidates at a time,
// keeps the Gaussians whose pair marks this tile (an order-preserving
// block compaction, so the kept sequence is exactly the tile's own
// front-to-back list) and stages their records in shared memory until at
// least 256 are staged (or the list ends), then blends them.  The next
// round's candidate ids and rects are fetched before the staged records are
// used, hiding their latency.  A pixel stops when its transmittance would fall
// below 1e-4; the block leaves once every pixel stopped.
//
// The exponent is kept in base 2: the record stores the conic scaled by
// log2(e), g2 = A2 dx^2 + B2 dx dy + C2 dy^2 = g log2(e), and alpha = sigma 2^g2.
//
// The state carried per pixel is the transmittance T = 1 - A and its
// derivatives (the paper's A-recurrences with the sign flipped): tracking T
// multiplicatively keeps it accurate in FP32 where A approaches 1.  With
// alpha_x = alpha g_x, alpha_y = alpha g_y, alpha_xy = alpha (g_x g_y + g_xy):
//   w   = T alpha                       (colour weight)
//   w_x = alpha (T g_x + T_x)           = T alpha_x + T_x alpha
//   w_y = alpha (T g_y + T_y)
//   w_xy = alpha (T (g_x g_y + g_xy) + T_x g_y + T_y g_x + T_xy)
//   C += c w, C_x += c w_x, C_y += c w_y, C_xy += c w_xy
//   T *= (1 - alpha), T_x -= w_x, T_y -= w_y, T_xy -= w_xy
// (identical to B_i, A_i and their derivatives in the supplement, T = 1 - A).
#include <algorithm>

#include "blend_common.cuh"

namespace gs {
namespace {

constexpr int kStage = 2 * kCand;        // staged records per batch (>= kCand before blending)

// Records the walk takes together, and the launch bound (blocks per SM) that
// leaves the registers for them: with derivatives 3 records at 4 blocks/SM
// (64 registers), without 2 at 5 (48); WIDE (frames of at most 4 tiles per
// SM, one wave of blocks): 4 records at 3 blocks/SM.  Measured per (records,
// blocks/SM), derivative blend at 960x540 / 640x360 / 480x270 / 320x180 and
// plain blend at 1920x1080, in µs: (1, 5) 176 / - / 121 / - / 340; (2, 4)
// 164-174 / - / 96-100 / - / 313-334; (3, 4) 164-170 / 106-109 / 96-100 / 86-90 /
// 320; (3, 3) 180 / 104 / 92 / 88 / 320; (4, 3) 180 / 104 / 92 / 86 / 320;
// (2, 5) 180 / - / 113 / - / 313.
template <bool GRADS, bool WIDE = false>
__host__ __device__ constexpr int blend_unroll() { return WIDE ? 4 : GRADS ? 3 : 2; }
template <bool GRADS, bool WIDE = false>
__host__ __device__ constexpr int blend_min_blocks() { return WIDE ? 3 : GRADS ? 4 : 5; }

struct PixelState {
    float T, Txy;
    float2 TxTy;
    float2 C01, X01, Y01, Z01, XY2, CZ2;   // channel pairs (0, 1); channel 2 as (X2, Y2) and (C2, Z2)
    int last;
    bool done;
};

__device__ __forceinline__ void init(PixelState& p, bool inside)
{
    const float2 z = make_float2(0.f, 0.f);
    p.T = 1.f;
    p.Txy = 0.f;
    p.TxTy = z;
    p.C01 = p.X01 = p.Y01 = p.Z01 = p.XY2 = p.CZ2 = z;
    p.last = 0;
    p.done = !inside;
}

// One (pixel, Gaussian) pair: g2 is the exponent in base 2, (dx, dy) the offset
// from the mean, r0 = (mu_x, mu_y, -a, -c), r1 = (A2, B2, C2, reject threshold),
// c = (r, g, b, sigma).  Returns true if the pair was blended.
template <bool GRADS, int MODE>
__device__ __forceinline__ bool blend_pair(PixelState& p, float g2, float dx, float dy, const float4& r0,
                                           const float4& r1, const float4& c, int idx)
{
    if (MODE == GS_MODE_3DGS && g2 < r1.w) return false;   // sigma e^g < 1/255 for sure
    float alpha = c.w * pow2(g2);
    bool clamped = false;
    if (MODE == GS_MODE_3DGS) {
        if (alpha < (1.f / 255.f)) return false;
        clamped = alpha > 0.99f;
        alpha = fminf(alpha, 0.99f);
    }
    // every multiply-add below is spelled out (fmaf, or an intrinsic that is
    // never fused): the walk's unrolled copies of this function then round
    // alike wherever the compiler places them
    const float2 tw = mul2(make_float2(p.T, p.T), make_float2(__fsub_rn(1.f, alpha), alpha));   // (T (1 - alpha), T alpha)
    const float Tn = tw.x;
    if (MODE == GS_MODE_3DGS && Tn < 1e-4f) {
        p.done = true;
        return false;
    }
    const float w = tw.y;
    const float2 c01 = make_float2(c.x, c.y);
    p.C01 = fma2(c01, make_float2(w, w), p.C01);
    if (!GRADS) p.CZ2.x = fmaf(c.z, w, p.CZ2.x);
    if (GRADS) {
        const float bn = r1.y * kLn2;                       // -b
        // (g_x, g_y) = (-(a dx + b dy), -(b dx + c dy))
        const float2 g = fma2(make_float2(r0.z, r0.w), make_float2(dx, dy), mul2(make_float2(bn, bn), make_float2(dy, dx)));
        float gx = g.x, gy = g.y;
        float gxy = fmaf(gx, gy, bn);                       // g_x g_y + g_xy
        if (clamped) { gx = 0.f; gy = 0.f; gxy = 0.f; }
        const float2 wxy2 = mul2(make_float2(alpha, alpha), fma2(make_float2(p.T, p.T), make_float2(gx, gy), p.TxTy));
        const float wxy = alpha * fmaf(p.T, gxy, fmaf(p.TxTy.x, gy, fmaf(p.TxTy.y, gx, p.Txy)));
        p.X01 = fma2(c01, make_float2(wxy2.x, wxy2.x), p.X01);
        p.Y01 = fma2(c01, make_float2(wxy2.y, wxy2.y), p.Y01);
        p.Z01 = fma2(c01, make_float2(wxy, wxy), p.Z01);
        const float2 cz = make_float2(c.z, c.z);
        p.XY2 = fma2(cz, wxy2, p.XY2);
        p.CZ2 = fma2(cz, make_float2(w, wxy), p.CZ2);
        p.TxTy = sub2(p.TxTy, wxy2);
        p.Txy = __fsub_rn(p.Txy, wxy);
    }
    p.T = Tn;
    p.last = idx + 1;
    return true;
}

template <bool GRADS>
__device__ __forceinline__ void store(const BlendArgs& a, const PixelState& p, int x, int y)
{
    const size_t plane = (size_t)a.W * a.H;
    const size_t pix = (size_t)y * a.W + x;
    a.out_C[pix] = fmaf(p.T, a.bg.x, p.C01.x);
    a.out_C[plane + pix] = fmaf(p.T, a.bg.y, p.C01.y);
    a.out_C[2 * plane + pix] = fmaf(p.T, a.bg.z, p.CZ2.x);
    if (GRADS) {
        float* G = a.out_G;
        G[pix] = fmaf(p.TxTy.x, a.bg.x, p.X01.x);
        G[plane + pix] = fmaf(p.TxTy.x, a.bg.y, p.X01.y);
        G[2 * plane + pix] = fmaf(p.TxTy.x, a.bg.z, p.XY2.x);
        G[3 * plane + pix] = fmaf(p.TxTy.y, a.bg.x, p.Y01.x);
        G[4 * plane + pix] = fmaf(p.TxTy.y, a.bg.y, p.Y01.y);
        G[5 * plane + pix] = fmaf(p.TxTy.y, a.bg.z, p.XY2.y);
        G[6 * plane + pix] = fmaf(p.Txy, a.bg.x, p.Z01.x);
        G[7 * plane + pix] = fmaf(p.Txy, a.bg.y, p.Z01.y);
        G[8 * plane + pix] = fmaf(p.Txy, a.bg.z, p.CZ2.y);
    }
    if (a.state) a.state[pix] = make_float4(p.T, p.TxTy.x, p.TxTy.y, p.Txy);
    if (a.count) a.count[pix] = p.last;
}

// One tile of a blend.  STATS: count the (pixel, Gaussian) pairs evaluated
// (every list entry a pixel passes before it stops, the oracle's count) and
// blended, instead of writing images (used once, outside timed regions, to
// size the FLOP count).  MAP: the pixels of each warp, 0 = an 8 x 4 block
// (two blocks across, four down: a compact block makes the lanes of a warp
// agree more often on whether a Gaussian reaches them), 1 = a 16 x 2 strip.
// work_slot, when given, receives the tile's duration (clock64 / 16).
template <bool GRADS, int MODE, bool STATS, int MAP, int U>
__device__ __forceinline__ void blend_tile(const BlendArgs& a, int tile, unsigned long long* __restrict__ stats,
                                           uint32_t* work_slot)
{
    // U records taken together by the walk below: their loads and exponents
    // are formed before any of them is applied (they do not depend on the
    // pixel's state), which leaves the walk's dependency chain the state
    // update alone
    __shared__ float4 s_r0[kStage];
    __shared__ float4 s_r1[kStage];
    __shared__ float4 s_r2[kStage];
    __shared__ int s_wcnt[kWarps];

    const long long t_start = clock64();
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lx = MAP == 0 ? ((warp & 1) << 3) | (lane & 7) : lane & 15;
    const int ly = MAP == 0 ? ((warp >> 1) << 2) | (lane >> 3) : (warp << 1) | (lane >> 4);
    const int x = tx * kTile + lx, y = ty * kTile + ly;
    const float px = (float)x, py = (float)y;
    const uint32_t lanemask_lt = (1u << lane) - 1u;

    const int ksh = __ffs(a.ks) - 1;   // ks = 1, 2 or 4
    const int S = (ty >> ksh) * a.stiles_x + (tx >> ksh);
    const uint2 sr = a.sranges[S];
    const int total = (int)(sr.y - sr.x);

    PixelState p;
    init(p, x < a.W && y < a.H);
    uint32_t n_eval = 0, n_acc = 0;
    int list_base = 0;   // position of the batch's first record in the tile's list

    // candidate of the first round
    const int tbit = (ty & (a.ks - 1)) * a.ks + (tx & (a.ks - 1));   // this tile in the pair masks
    uint32_t cid = 0xFFFFFFFFu;
    bool chit = false;
    if ((int)threadIdx.x < total) chit = pair_hit(a.pair_words, sr.x + threadIdx.x, a.n, tbit, cid);

    int c0 = 0;
    while (c0 < total) {
        if (__syncthreads_count(p.done) == kThreads) break;
        // stage rounds of kCand candidates until >= kCand records are staged
        int staged = 0;
        while (c0 < total && staged < kCand) {
            const bool hit = chit;
            const uint32_t ball = __ballot_sync(0xffffffffu, hit);
            if (lane == 0) s_wcnt[warp] = __popc(ball);
            __syncthreads();
            int wbase = 0, tot = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const int cw = s_wcnt[w];
                wbase += w < warp ? cw : 0;
                tot += cw;
            }
            if (hit) {
                const int pos = staged + wbase + __popc(ball & lanemask_lt);
                s_r0[pos] = a.rec.r0[cid];
                s_r1[pos] = a.rec.r1[cid];
                s_r2[pos] = a.rec.r2[cid];
            }
            staged += tot;
            c0 += kCand;
            // fetch the next round's candidate
            const int cn = c0 + (int)threadIdx.x;
            cid = 0xFFFFFFFFu;
            chit = false;
            if (cn < total) chit = pair_hit(a.pair_words, sr.x + cn, a.n, tbit, cid);
            __syncthreads();   // s_wcnt is reused by the next round; staged records are visible
        }
        int k = 0;
        for (; k + U - 1 < staged && !p.done; k += U) {
            float4 q0[U], q1[U];
            float qdx[U], qdy[U], qg2[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                q0[u] = s_r0[k + u];
                q1[u] = s_r1[k + u];
                const float2 d = sub2(make_float2(px, py), make_float2(q0[u].x, q0[u].y));
                qdx[u] = d.x;
                qdy[u] = d.y;
                qg2[u] = exponent2(q1[u], qdx[u], qdy[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (u > 0 && p.done) break;
                if (STATS) ++n_eval;
                if (MODE == GS_MODE_3DGS && qg2[u] < q1[u].w) continue;
                const float4 c = s_r2[k + u];
                if (blend_pair<GRADS, MODE>(p, qg2[u], qdx[u], qdy[u], q0[u], q1[u], c, list_base + k + u) && STATS)
                    ++n_acc;
            }
        }
        for (; k < staged && !p.done; ++k) {   // the batch's last records, one at a time
            const float4 r0 = s_r0[k];
            const float4 r1 = s_r1[k];
            const float dx = px - r0.x, dy = py - r0.y;
            if (STATS) ++n_eval;
            const float g2 = exponent2(r1, dx, dy);
            if (MODE == GS_MODE_3DGS && g2 < r1.w) continue;
            const float4 c = s_r2[k];
            if (blend_pair<GRADS, MODE>(p, g2, dx, dy, r0, r1, c, list_base + k) && STATS) ++n_acc;
        }
        list_base += staged;
    }
    if (STATS) {
        unsigned long long e = n_eval, acc = n_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_down_sync(0xffffffffu, e, o);
            acc += __shfl_down_sync(0xffffffffu, acc, o);
        }
        if (lane == 0) {
            atomicAdd(&stats[0], e);
            atomicAdd(&stats[1], acc);
        }
        return;
    }
    if (work_slot && threadIdx.x == 0) *work_slot = (uint32_t)min((clock64() - t_start) >> 4, 0xFFFFFFFFll);
    if (x < a.W && y < a.H) store<GRADS>(a, p, x, y);
}

template <bool GRADS, int MODE, bool STATS = false, bool WIDE = false>
__global__ void __launch_bounds__(kThreads, blend_min_blocks<GRADS, WIDE>())
    k_blend(BlendArgs a, unsigned long long* __restrict__ stats = nullptr)
{
    const int tile = a.order ? (int)a.order[blockIdx.x] : (int)blockIdx.x;
    blend_tile<GRADS, MODE, STATS, 0, blend_unroll<GRADS, WIDE>()>(a, tile, stats, a.work ? a.work + tile : nullptr);
}

// The tiles of every view of a batch in one launch: job j is global tile
// order[j] (or j), the tiles of view v being start[v] .. start[v + 1] - 1.
// PERSIST: a grid of resident blocks takes jobs from a counter in turn;
// otherwise one block per job.
template <bool GRADS, int MODE, int MAP, bool PERSIST>
__global__ void __launch_bounds__(kThreads, blend_min_blocks<GRADS>()) k_blend_views(const __grid_constant__ BlendViews b)
{
    __shared__ int s_job;
    const int total = b.start[b.V];
    for (int j = PERSIST ? -1 : (int)blockIdx.x;;) {
        if (PERSIST) {
            __syncthreads();          // the previous tile's shared state is no longer read
            if (threadIdx.x == 0) s_job = (int)atomicAdd(b.queue, 1u);
            __syncthreads();
            j = s_job;
            if (j >= total) break;
        }
        const int g = b.order ? (int)b.order[j] : j;
        int v = 0;
        while (v + 1 < b.V && g >= b.start[v + 1]) ++v;
        blend_tile<GRADS, MODE, false, MAP, blend_unroll<GRADS>()>(b.a[v], g - b.start[v], nullptr,
                                                                 b.work ? b.work + g : nullptr);
        if (!PERSIST) break;
    }
}

template <bool GRADS, int MODE>
cudaError_t launch_t(cudaStream_t s, const BlendArgs& a)
{
    const int T = a.tiles_x * a.tiles_y;
    bool wide = false;
    if (GRADS) {   // one wave of blocks at 4 per SM: the WIDE shape
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            wide = T <= 4 * sms;
    }
    if (wide)
        k_blend<GRADS, MODE, false, GRADS><<<T, kThreads, 0, s>>>(a);
    else
        k_blend<GRADS, MODE><<<T, kThreads, 0, s>>>(a);
    note_launch();
    return cudaGetLastError();
}

template <int MODE, int MAP, bool PERSIST>
cudaError_t launch_views_t(cudaStream_t s, const BlendViews& b, int grid)
{
    k_blend_views<true, MODE, MAP, PERSIST><<<grid, kThreads, 0, s>>>(b); note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend_stats(cudaStream_t s, int mode, const BlendArgs& a, unsigned long long* stats)
{
    const int tiles = a.tiles_x * a.tiles_y;
    if (mode == GS_MODE_EXACT)
        k_blend<true, GS_MODE_EXACT, true><<<tiles, kThreads, 0, s>>>(a, stats);
    else
        k_blend<true, GS_MODE_3DGS, true><<<tiles, kThreads, 0, s>>>(a, stats);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_blend_views(cudaStream_t s, int mode, const BlendViews& b, int map, bool persistent)
{
    const int total = b.start[b.V];
    if (total <= 0) return cudaSuccess;
    int grid = total;
    if (persistent) {
        // resident blocks: as many as fit (blocks per SM by the occupancy calculator)
        int dev = 0, sms = 1, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (mode == GS_MODE_EXACT)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, map ? k_blend_views<true, GS_MODE_EXACT, 1, true>
                                                                       : k_blend_views<true, GS_MODE_EXACT, 0, true>,
                                                          kThreads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, map ? k_blend_views<true, GS_MODE_3DGS, 1, true>
                                                                       : k_blend_views<true, GS_MODE_3DGS, 0, true>,
                                                          kThreads, 0);
        grid = std::min(total, std::max(1, sms * std::max(1, per_sm)));
        cudaError_t e = cudaMemsetAsync(b.queue, 0, sizeof(uint32_t), s);
        if (e != cudaSuccess) return e;
    }
    if (mode == GS_MODE_EXACT) {
        if (persistent) return map ? launch_views_t<GS_MODE_EXACT, 1, true>(s, b, grid)
                                   : launch_views_t<GS_MODE_EXACT, 0, true>(s, b, grid);
        return map ? launch_views_t<GS_MODE_EXACT, 1, false>(s, b, grid)
                   : launch_views_t<GS_MODE_EXACT, 0, false>(s, b, grid);
    }
    if (persistent) return map ? launch_views_t<GS_MODE_3DGS, 1, true>(s, b, grid)
                               : launch_views_t<GS_MODE_3DGS, 0, true>(s, b, grid);
    return map ? launch_views_t<GS_MODE_3DGS, 1, false>(s, b, grid) : launch_views_t<GS_MODE_3DGS, 0, false>(s, b, grid);
}

cudaError_t launch_blend(cudaStream_t s, bool grads, int mode, const BlendArgs& a)
{
    if (grads)
        return mode == GS_MODE_EXACT ? launch_t<true, GS_MODE_EXACT>(s, a) : launch_t<true, GS_MODE_3DGS>(s, a);
    return mode == GS_MODE_EXACT ? launch_t<false, GS_MODE_EXACT>(s, a) : launch_t<false, GS_MODE_3DGS>(s, a);
}

}  // namespace gs
