// Front-to-back blend of each tile's Gaussians with the analytic screen-space
// derivatives of the pixel colour (Sec. 4 blend equation; Sec. 5 "3DGS Image
// Gradients"; supplement "Forward pass").
//
// One 256-thread block per 16x16 tile, one pixel per thread.  Binning is done
// per 64x64 super-tile (4x4 tiles): the block walks its super-tile's
// depth-ordered list 256 candidates at a time, keeps the Gaussians whose tile
// rect covers this tile (an order-preserving block compaction, so the kept
// sequence is exactly the tile's own front-to-back list), stages their records
// in shared memory and blends them.  The next round's candidate ids and rects
// are fetched before the current batch is blended, hiding their latency.  A
// pixel stops when its transmittance would fall below 1e-4; a warp whose
// pixels have all stopped skips the rest of each batch, and the block leaves
// once every pixel stopped.
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
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kBlock = kTilePixels;   // 256
constexpr int kWarps = kBlock / 32;

__device__ __forceinline__ bool covers(ushort4 r, int tx, int ty)
{
    return (int)r.x <= tx && tx <= (int)r.z && (int)r.y <= ty && ty <= (int)r.w;
}

// STATS: count the (pixel, Gaussian) pairs evaluated and blended instead of
// writing images (used once, outside timed regions, to size the FLOP count).
template <bool GRADS, int MODE, bool STATS = false>
__global__ void __launch_bounds__(kBlock) k_blend(BlendArgs a, unsigned long long* __restrict__ stats = nullptr)
{
    __shared__ float4 s_r0[kBlock];
    __shared__ float4 s_r1[kBlock];
    __shared__ float4 s_r2[kBlock];
    __shared__ int s_wcnt[kWarps];

    const int tile = blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
    const int x = tx * kTile + lx, y = ty * kTile + ly;
    const bool inside = x < a.W && y < a.H;
    const float px = (float)x, py = (float)y;
    // centre of this warp's 16 x 2 pixel strip (rows 2 warp, 2 warp + 1 of the tile)
    const float wcx = (float)(tx * kTile) + 7.5f, wcy = (float)(ty * kTile + 2 * warp) + 0.5f;
    const uint32_t lanemask_lt = (1u << lane) - 1u;

    const int S = (ty / kSuper) * a.stiles_x + (tx / kSuper);
    const uint2 sr = a.sranges[S];
    const int total = (int)(sr.y - sr.x);

    float T = 1.f, Tx = 0.f, Ty = 0.f, Txy = 0.f;
    float C0 = 0.f, C1 = 0.f, C2 = 0.f;
    float X0 = 0.f, X1 = 0.f, X2 = 0.f;
    float Y0 = 0.f, Y1 = 0.f, Y2 = 0.f;
    float Z0 = 0.f, Z1 = 0.f, Z2 = 0.f;
    int last = 0;
    int list_base = 0;    // position of this round's first kept Gaussian in the tile's list
    bool done = !inside;
    uint32_t n_eval = 0, n_acc = 0;

    // candidate of the first round
    uint32_t cid = 0xFFFFFFFFu;
    ushort4 crect = make_ushort4(1, 1, 0, 0);
    if ((int)threadIdx.x < total) {
        cid = a.pair_words[2 * (size_t)(sr.x + threadIdx.x)];
        if (cid < a.n) crect = a.rect[cid];
    }

    for (int c0 = 0; c0 < total; c0 += kBlock) {
        if (__syncthreads_count(done) == kBlock) break;
        // order-preserving compaction of the candidates that cover this tile
        const bool hit = cid < a.n && covers(crect, tx, ty);
        const uint32_t ball = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) s_wcnt[warp] = __popc(ball);
        __syncthreads();
        int wbase = 0, batch = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const int cw = s_wcnt[w];
            wbase += w < warp ? cw : 0;
            batch += cw;
        }
        if (hit) {
            const int pos = wbase + __popc(ball & lanemask_lt);
            s_r0[pos] = a.rec.r0[cid];
            s_r1[pos] = a.rec.r1[cid];
            s_r2[pos] = a.rec.r2[cid];
        }
        // fetch the next round's candidate while this batch is blended
        const int cn = c0 + kBlock + (int)threadIdx.x;
        cid = 0xFFFFFFFFu;
        if (cn < total) {
            cid = a.pair_words[2 * (size_t)(sr.x + cn)];
            if (cid < a.n) crect = a.rect[cid];
        }
        __syncthreads();
        for (int k = 0; !done && k < batch; ++k) {
            const float4 r0 = s_r0[k];
            if (STATS) ++n_eval;   // every list entry a pixel passes before it stops (the oracle's count)
            // warp-uniform skip: the Gaussian's alpha >= 1/255 box misses this warp's 16 x 2 strip
            if (fabsf(r0.x - wcx) > r0.z + 7.5f || fabsf(r0.y - wcy) > r0.w + 0.5f) continue;
            const float4 r1 = s_r1[k];
            const float dx = px - r0.x, dy = py - r0.y;
            // g = -1/2 (a dx^2 + 2 b dx dy + c dy^2)
            const float g = -0.5f * (r1.x * dx * dx + r1.z * dy * dy) - r1.y * dx * dy;
            if (MODE == GS_MODE_3DGS && g < r1.w) continue;     // sigma e^g < 1/255 for sure
            const float4 c = s_r2[k];
            float alpha = c.w * __expf(g);
            bool clamped = false;
            if (MODE == GS_MODE_3DGS) {
                if (alpha < (1.f / 255.f)) continue;
                clamped = alpha > 0.99f;
                alpha = fminf(alpha, 0.99f);
            }
            const float Tn = T * (1.f - alpha);
            if (MODE == GS_MODE_3DGS && Tn < 1e-4f) {
                done = true;
                break;
            }
            const float w = alpha * T;
            C0 = fmaf(c.x, w, C0);
            C1 = fmaf(c.y, w, C1);
            C2 = fmaf(c.z, w, C2);
            if (GRADS) {
                float gx = -(r1.x * dx + r1.y * dy);
                float gy = -(r1.y * dx + r1.z * dy);
                float gxy = fmaf(gx, gy, -r1.y);
                if (clamped) { gx = 0.f; gy = 0.f; gxy = 0.f; }
                const float wx = alpha * fmaf(T, gx, Tx);
                const float wy = alpha * fmaf(T, gy, Ty);
                const float wxy = alpha * (T * gxy + Tx * gy + Ty * gx + Txy);
                X0 = fmaf(c.x, wx, X0); X1 = fmaf(c.y, wx, X1); X2 = fmaf(c.z, wx, X2);
                Y0 = fmaf(c.x, wy, Y0); Y1 = fmaf(c.y, wy, Y1); Y2 = fmaf(c.z, wy, Y2);
                Z0 = fmaf(c.x, wxy, Z0); Z1 = fmaf(c.y, wxy, Z1); Z2 = fmaf(c.z, wxy, Z2);
                Tx -= wx;
                Ty -= wy;
                Txy -= wxy;
            }
            T = Tn;
            last = list_base + k + 1;
            if (STATS) ++n_acc;
        }
        list_base += batch;
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
    if (!inside) return;
    const size_t plane = (size_t)a.W * a.H;
    const size_t pix = (size_t)y * a.W + x;
    a.out_C[pix] = fmaf(T, a.bg.x, C0);
    a.out_C[plane + pix] = fmaf(T, a.bg.y, C1);
    a.out_C[2 * plane + pix] = fmaf(T, a.bg.z, C2);
    if (GRADS) {
        float* G = a.out_G;
        G[pix] = fmaf(Tx, a.bg.x, X0);
        G[plane + pix] = fmaf(Tx, a.bg.y, X1);
        G[2 * plane + pix] = fmaf(Tx, a.bg.z, X2);
        G[3 * plane + pix] = fmaf(Ty, a.bg.x, Y0);
        G[4 * plane + pix] = fmaf(Ty, a.bg.y, Y1);
        G[5 * plane + pix] = fmaf(Ty, a.bg.z, Y2);
        G[6 * plane + pix] = fmaf(Txy, a.bg.x, Z0);
        G[7 * plane + pix] = fmaf(Txy, a.bg.y, Z1);
        G[8 * plane + pix] = fmaf(Txy, a.bg.z, Z2);
    }
    if (a.state) a.state[pix] = make_float4(T, Tx, Ty, Txy);
    if (a.count) a.count[pix] = last;
}

template <bool GRADS, int MODE>
cudaError_t launch_t(cudaStream_t s, const BlendArgs& a)
{
    k_blend<GRADS, MODE><<<a.tiles_x * a.tiles_y, kBlock, 0, s>>>(a); note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend_stats(cudaStream_t s, int mode, const BlendArgs& a, unsigned long long* stats)
{
    const int tiles = a.tiles_x * a.tiles_y;
    if (mode == GS_MODE_EXACT)
        k_blend<true, GS_MODE_EXACT, true><<<tiles, kBlock, 0, s>>>(a, stats);
    else
        k_blend<true, GS_MODE_3DGS, true><<<tiles, kBlock, 0, s>>>(a, stats);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_blend(cudaStream_t s, bool grads, int mode, const BlendArgs& a)
{
    if (grads)
        return mode == GS_MODE_EXACT ? launch_t<true, GS_MODE_EXACT>(s, a) : launch_t<true, GS_MODE_3DGS>(s, a);
    return mode == GS_MODE_EXACT ? launch_t<false, GS_MODE_EXACT>(s, a) : launch_t<false, GS_MODE_3DGS>(s, a);
}

}  // namespace gs
