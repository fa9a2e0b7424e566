// Front-to-back blend of each tile's Gaussians with the analytic screen-space
// derivatives of the pixel colour (Sec. 4 blend equation; Sec. 5 "3DGS Image
// Gradients"; supplement "Forward pass").
//
// One 256-thread block per 16x16 tile, one pixel per thread.  The tile's list
// is walked in batches of 256 records staged in shared memory (one global load
// per record per block, broadcast reads per pixel).  A pixel stops when its
// transmittance would fall below 1e-4; a warp whose pixels have all stopped
// skips the rest of each batch, and the block leaves once every pixel stopped.
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

// STATS: count the (pixel, Gaussian) pairs evaluated and blended instead of
// writing images (used once, outside timed regions, to size the FLOP count).
template <bool GRADS, int MODE, bool STATS = false>
__global__ void __launch_bounds__(kBlock) k_blend(int W, int H, int tiles_x, uint32_t n, const uint2* __restrict__ ranges,
                                                  const uint32_t* __restrict__ pair_words, Records rec, float3 bg,
                                                  float* __restrict__ out_C, float* __restrict__ out_G,
                                                  float4* __restrict__ state, int* __restrict__ count_out,
                                                  unsigned long long* __restrict__ stats = nullptr)
{
    __shared__ float4 s_r0[kBlock];
    __shared__ float4 s_r1[kBlock];
    __shared__ float4 s_r2[kBlock];

    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int lx = threadIdx.x & (kTile - 1), ly = threadIdx.x / kTile;
    const int x = tx * kTile + lx, y = ty * kTile + ly;
    const bool inside = x < W && y < H;
    const float px = (float)x, py = (float)y;

    const uint2 rg = ranges[tile];
    const int total = (int)(rg.y - rg.x);

    float T = 1.f, Tx = 0.f, Ty = 0.f, Txy = 0.f;
    float C0 = 0.f, C1 = 0.f, C2 = 0.f;
    float X0 = 0.f, X1 = 0.f, X2 = 0.f;
    float Y0 = 0.f, Y1 = 0.f, Y2 = 0.f;
    float Z0 = 0.f, Z1 = 0.f, Z2 = 0.f;
    int last = 0;
    bool done = !inside;
    uint32_t n_eval = 0, n_acc = 0;

    for (int b0 = 0; b0 < total; b0 += kBlock) {
        if (__syncthreads_count(done) == kBlock) break;
        const int j = b0 + threadIdx.x;
        if (j < total) {
            // low word of the (tile << 32 | id) pair
            const uint32_t id = pair_words[2 * (size_t)(rg.x + j)];
            if (id < n) {
                s_r0[threadIdx.x] = rec.r0[id];
                s_r1[threadIdx.x] = rec.r1[id];
                s_r2[threadIdx.x] = rec.r2[id];
            } else {   // only after an expired bounded wait in the sort: a record that never blends
                s_r0[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                s_r1[threadIdx.x] = make_float4(0.f, 0.f, INFINITY, 0.f);
                s_r2[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        const int cnt = min(kBlock, total - b0);
        for (int k = 0; !done && k < cnt; ++k) {
            const float4 a = s_r0[k];
            const float4 b = s_r1[k];
            const float dx = px - a.x, dy = py - a.y;
            if (STATS) ++n_eval;
            // g = -1/2 (a dx^2 + 2 b dx dy + c dy^2)
            const float g = -0.5f * (a.z * dx * dx + b.x * dy * dy) - a.w * dx * dy;
            if (MODE == GS_MODE_3DGS && g < b.z) continue;     // sigma e^g < 1/255 for sure
            float alpha = b.y * __expf(g);
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
            const float4 c = s_r2[k];
            const float w = alpha * T;
            C0 = fmaf(c.x, w, C0);
            C1 = fmaf(c.y, w, C1);
            C2 = fmaf(c.z, w, C2);
            if (GRADS) {
                float gx = -(a.z * dx + a.w * dy);
                float gy = -(a.w * dx + b.x * dy);
                float gxy = fmaf(gx, gy, -a.w);
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
            last = b0 + k + 1;
            if (STATS) ++n_acc;
        }
    }
    if (STATS) {
        unsigned long long e = n_eval, a = n_acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_down_sync(0xffffffffu, e, o);
            a += __shfl_down_sync(0xffffffffu, a, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&stats[0], e);
            atomicAdd(&stats[1], a);
        }
        return;
    }
    if (!inside) return;
    const size_t plane = (size_t)W * H;
    const size_t pix = (size_t)y * W + x;
    out_C[pix] = fmaf(T, bg.x, C0);
    out_C[plane + pix] = fmaf(T, bg.y, C1);
    out_C[2 * plane + pix] = fmaf(T, bg.z, C2);
    if (GRADS) {
        out_G[pix] = fmaf(Tx, bg.x, X0);
        out_G[plane + pix] = fmaf(Tx, bg.y, X1);
        out_G[2 * plane + pix] = fmaf(Tx, bg.z, X2);
        out_G[3 * plane + pix] = fmaf(Ty, bg.x, Y0);
        out_G[4 * plane + pix] = fmaf(Ty, bg.y, Y1);
        out_G[5 * plane + pix] = fmaf(Ty, bg.z, Y2);
        out_G[6 * plane + pix] = fmaf(Txy, bg.x, Z0);
        out_G[7 * plane + pix] = fmaf(Txy, bg.y, Z1);
        out_G[8 * plane + pix] = fmaf(Txy, bg.z, Z2);
    }
    if (state) state[pix] = make_float4(T, Tx, Ty, Txy);
    if (count_out) count_out[pix] = last;
}

template <bool GRADS, int MODE>
cudaError_t launch_t(cudaStream_t s, int W, int H, int tiles_x, int tiles_y, uint32_t n, const uint2* ranges,
                     const uint64_t* pairs, Records rec, float3 bg, float* out_C, float* out_G, float4* state,
                     int* count)
{
    const int tiles = tiles_x * tiles_y;
    k_blend<GRADS, MODE><<<tiles, kBlock, 0, s>>>(W, H, tiles_x, n, ranges, reinterpret_cast<const uint32_t*>(pairs),
                                                 rec, bg, out_C, out_G, state, count); note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_blend_stats(cudaStream_t s, int mode, int W, int H, int tiles_x, int tiles_y, uint32_t n,
                               const uint2* ranges, const uint64_t* pairs, Records rec,
                               unsigned long long* stats)
{
    const int tiles = tiles_x * tiles_y;
    const float3 bg = make_float3(0.f, 0.f, 0.f);
    const uint32_t* pw = reinterpret_cast<const uint32_t*>(pairs);
    if (mode == GS_MODE_EXACT)
        k_blend<true, GS_MODE_EXACT, true><<<tiles, kBlock, 0, s>>>(W, H, tiles_x, n, ranges, pw, rec, bg, nullptr,
                                                                  nullptr, nullptr, nullptr, stats);
    else
        k_blend<true, GS_MODE_3DGS, true><<<tiles, kBlock, 0, s>>>(W, H, tiles_x, n, ranges, pw, rec, bg, nullptr,
                                                                 nullptr, nullptr, nullptr, stats);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_blend(cudaStream_t s, bool grads, int mode, int W, int H, int tiles_x, int tiles_y, uint32_t n,
                         const uint2* ranges, const uint64_t* pairs, Records rec, float bg0, float bg1, float bg2,
                         float* out_C, float* out_grads, float4* state, int* count)
{
    const float3 bg = make_float3(bg0, bg1, bg2);
    if (grads) {
        if (mode == GS_MODE_EXACT)
            return launch_t<true, GS_MODE_EXACT>(s, W, H, tiles_x, tiles_y, n, ranges, pairs, rec, bg, out_C,
                                                 out_grads, state, count);
        return launch_t<true, GS_MODE_3DGS>(s, W, H, tiles_x, tiles_y, n, ranges, pairs, rec, bg, out_C, out_grads,
                                            state, count);
    }
    if (mode == GS_MODE_EXACT)
        return launch_t<false, GS_MODE_EXACT>(s, W, H, tiles_x, tiles_y, n, ranges, pairs, rec, bg, out_C, nullptr,
                                              state, count);
    return launch_t<false, GS_MODE_3DGS>(s, W, H, tiles_x, tiles_y, n, ranges, pairs, rec, bg, out_C, nullptr, state,
                                         count);
}

}  // namespace gs
