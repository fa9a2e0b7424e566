// Adjoint of the derivative blend (supplement "Backward Pass").
//
// Reverse mode on the forward's own recurrences.  Per blended pair, with the
// state (T, T_x, T_y, T_xy) before the step and the weights
//   w = alpha T, w_x = alpha (T g_x + T_x), w_y = alpha (T g_y + T_y),
//   w_xy = alpha (T g_xy' + T_x g_y + T_y g_x + T_xy)   (g_xy' = g_x g_y + g_xy),
// the step adds c w (and c w_x, ...) to the outputs and subtracts w (w_x, ...)
// from the state.  Walking back to front with the adjoint lambda of the state
// (initialised from the background term, output += bg T):
//   G_w = u . c - lambda_T  (likewise G_wx, G_wy, G_wxy with u_x, u_y, u_xy)
//   dL/dc = u w + u_x w_x + u_y w_y + u_xy w_xy
//   lambda_T  += G_w alpha + G_wx alpha_x + G_wy alpha_y + G_wxy alpha_xy
//   lambda_Tx += G_wx alpha + G_wxy alpha_y,  lambda_Ty += G_wy alpha + G_wxy alpha_x,
//   lambda_Txy += G_wxy alpha
//   G_alpha = G_w T + G_wx T_x + G_wy T_y + G_wxy T_xy,  G_alpha_x = G_wx T + G_wxy T_y,
//   G_alpha_y = G_wy T + G_wxy T_x,  G_alpha_xy = G_wxy T
// and, through alpha = sigma e^g (alpha_x = alpha g_x, ...):
//   dL/dg = alpha (G_alpha + G_alpha_x g_x + G_alpha_y g_y + G_alpha_xy g_xy'),
//   dL/dg_x = alpha (G_alpha_x + G_alpha_xy g_y), dL/dg_y = alpha (G_alpha_y + G_alpha_xy g_x),
//   dL/dg_xy = alpha G_alpha_xy,  dL/dsigma = dL/dg / sigma,
// then to the mean and the conic by differentiating g, g_x, g_y, g_xy = -b.
// A clamped alpha (0.99) is a constant: no gradient to sigma or the geometry.
//
// The state before each step is recovered from the state after it by
// inverting the update: T = T'/(1 - alpha), T_x = (T_x' + alpha T g_x)/(1 -
// alpha), ... (the supplement's inversion trick written for T = 1 - A).  Two
// variants anchor that walk:
//  * inversion: from the final state the forward blend stored, through the
//    whole list (each alpha = 0.99 step scales the rounding of the recovered
//    state by up to 100, and such factors compound along the list);
//  * recompute: the block first re-runs the forward walk of its tile (the
//    transmittance state alone, every decision on the same FP32 values as the
//    forward) and checkpoints the exact state at the start of each round of
//    candidates; walking back, each round starts from the exact state at its
//    end, so the inversion spans one round's entries (about 60 at the 960 x
//    540 workload) instead of the whole list.  The forward's stored state and
//    counts are not used (the recomputed ones are).  Checkpoints go to global
//    scratch, kCkSlots per tile; a tile with more rounds keeps every second
//    one, then every fourth, ...
//
// Algorithmic work (FP32 operations, FMA = 2) per blended pair: g_x, g_y, g_xy'
// 9; the state before the step 19; the weights w.. 14; dL/dc 21; G_w.. 24;
// alpha_x.. 3; the adjoint update 18; G_alpha.. 14; dL/dg.. 14; the six
// geometric and opacity terms 28; the sum over the tile's pixels 9: 173.
// Re-evaluating a pair (d, g2, alpha) is 10, as in the forward.
//
// List walk.  A tile's front-to-back list is its super-tile's list filtered by
// the tile rects (as in the forward).  The block first streams the super-tile
// list in rounds of 256 candidates, recording the tile's list position at the
// start of each round, until the largest stored count of its pixels is
// covered.  It then replays the rounds last to first: each round's hits are
// compacted in order into shared memory and walked back to front; a pixel takes
// part in the entries below its own count, and every decision (reject, cut-off,
// clamp) is re-taken on the same FP32 values as the forward.  Round starts are
// kept for 1024 rounds at a time; longer lists are replayed in segments of 1024
// rounds, each recounted from a stored segment start.  Per list entry the block
// reduces the pixels' 9 gradients (a transposed warp sum, then shared-memory
// atomics) and adds one set per tile and Gaussian to global memory.
//
// The upstream gradient is either given per low-res pixel (dL/dC and dL/d of
// the derivative planes) or, fused, as the gradient of the upscaled image: each
// pixel then gathers its own upstream values through the upscale's adjoint
// before the walk, and the low-res planes never exist in memory.
#include "blend_common.cuh"
#include "spline_common.cuh"

namespace gs {
namespace {

constexpr int kMaxRounds = 1024;   // round starts kept in shared memory
constexpr int kMaxSegs = 256;      // segments of kMaxRounds rounds (lists up to 2^26 candidates)

struct BwdPixel {
    float px, py;
    int last;
    float T, Tx, Ty, Txy;          // state after the entries not yet walked back
    float lT, lTx, lTy, lTxy;      // its adjoint
    float uC[3], uX[3], uY[3], uZ[3];
};

// The part of one list entry's step that does not depend on the pixel's
// state: the pair's offset, exponent, decisions, alpha and its slopes, and the
// upstream gradients dotted with the colour.  The walk forms it for a group of
// entries before applying them (bwd_apply) one after the other.
struct BwdPrep {
    float dx, dy, alpha, gx, gy, gxy, bn, iom, ax, ay, axy;
    float dC, dX, dY, dZ;   // u . c of the four upstream gradient groups
    float sigma, ca, cc;
    bool keep, clamped;
};

template <int MODE>
__device__ __forceinline__ void bwd_prep(const BwdPixel& p, const float4& r0, const float4& r1, const float4& c,
                                         bool listed, BwdPrep& q)
{
    q.dx = p.px - r0.x;
    q.dy = p.py - r0.y;
    const float g2 = exponent2(r1, q.dx, q.dy);
    q.keep = listed && !(MODE == GS_MODE_3DGS && g2 < r1.w);
    q.clamped = false;
    q.alpha = 0.f;
    if (q.keep) {
        float alpha = c.w * pow2(g2);
        if (MODE == GS_MODE_3DGS) {
            if (alpha < (1.f / 255.f)) q.keep = false;
            q.clamped = alpha > 0.99f;
            alpha = fminf(alpha, 0.99f);
        }
        q.alpha = alpha;
    }
    q.bn = r1.y * kLn2;   // -b
    q.gx = fmaf(r0.z, q.dx, q.bn * q.dy);
    q.gy = fmaf(r0.w, q.dy, q.bn * q.dx);
    q.gxy = fmaf(q.gx, q.gy, q.bn);
    if (q.clamped) { q.gx = 0.f; q.gy = 0.f; q.gxy = 0.f; }
    q.iom = __fdividef(1.f, __fsub_rn(1.f, q.alpha));
    q.ax = q.alpha * q.gx;
    q.ay = q.alpha * q.gy;
    q.axy = q.alpha * q.gxy;
    q.dC = fmaf(p.uC[2], c.z, fmaf(p.uC[1], c.y, p.uC[0] * c.x));
    q.dX = fmaf(p.uX[2], c.z, fmaf(p.uX[1], c.y, p.uX[0] * c.x));
    q.dY = fmaf(p.uY[2], c.z, fmaf(p.uY[1], c.y, p.uY[0] * c.x));
    q.dZ = fmaf(p.uZ[2], c.z, fmaf(p.uZ[1], c.y, p.uZ[0] * c.x));
    q.sigma = c.w;
    q.ca = -r0.z;
    q.cc = -r0.w;
}

// The state-dependent rest of one list entry's step for one pixel: the
// pixel's 9 gradient terms in v and the state and its adjoint stepped back;
// false (v untouched) for an entry the forward did not blend.
__device__ __forceinline__ bool bwd_apply(BwdPixel& p, const BwdPrep& q, float v[9])
{
    if (!q.keep) return false;
    const float alpha = q.alpha, gx = q.gx, gy = q.gy, gxy = q.gxy, iom = q.iom;
    const float T0 = p.T * iom;
    const float Tx0 = fmaf(alpha * T0, gx, p.Tx) * iom;
    const float Ty0 = fmaf(alpha * T0, gy, p.Ty) * iom;
    const float Txy0 = fmaf(alpha, fmaf(T0, gxy, fmaf(Tx0, gy, Ty0 * gx)), p.Txy) * iom;
    const float w = alpha * T0;
    const float wx = alpha * fmaf(T0, gx, Tx0);
    const float wy = alpha * fmaf(T0, gy, Ty0);
    const float wxy = alpha * fmaf(T0, gxy, fmaf(Tx0, gy, fmaf(Ty0, gx, Txy0)));
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
        v[6 + ch] = fmaf(p.uZ[ch], wxy, fmaf(p.uY[ch], wy, fmaf(p.uX[ch], wx, p.uC[ch] * w)));
    const float Gw = __fsub_rn(q.dC, p.lT);
    const float Gwx = __fsub_rn(q.dX, p.lTx);
    const float Gwy = __fsub_rn(q.dY, p.lTy);
    const float Gwxy = __fsub_rn(q.dZ, p.lTxy);
    p.lT = __fadd_rn(p.lT, fmaf(Gwxy, q.axy, fmaf(Gwy, q.ay, fmaf(Gwx, q.ax, Gw * alpha))));
    p.lTx = __fadd_rn(p.lTx, fmaf(Gwxy, q.ay, Gwx * alpha));
    p.lTy = __fadd_rn(p.lTy, fmaf(Gwxy, q.ax, Gwy * alpha));
    p.lTxy = fmaf(Gwxy, alpha, p.lTxy);
    if (!q.clamped) {
        const float Ga = fmaf(Gwxy, Txy0, fmaf(Gwy, Ty0, fmaf(Gwx, Tx0, Gw * T0)));
        const float Gax = fmaf(Gwxy, Ty0, Gwx * T0);
        const float Gay = fmaf(Gwxy, Tx0, Gwy * T0);
        const float Gaxy = Gwxy * T0;
        const float dg = alpha * fmaf(Gaxy, gxy, fmaf(Gay, gy, fmaf(Gax, gx, Ga)));
        const float dgx = alpha * fmaf(Gaxy, gy, Gax);
        const float dgy = alpha * fmaf(Gaxy, gx, Gay);
        const float dgxy = alpha * Gaxy;
        const float cb = -q.bn;
        const float dx = q.dx, dy = q.dy;
        v[0] = fmaf(cb, dgy, fmaf(q.ca, dgx, -dg * gx));
        v[1] = fmaf(q.cc, dgy, fmaf(cb, dgx, -dg * gy));
        v[2] = fmaf(-0.5f * dx * dx, dg, -dx * dgx);
        v[3] = __fsub_rn(fmaf(-dx * dy, dg, fmaf(-dy, dgx, -dx * dgy)), dgxy);
        v[4] = fmaf(-0.5f * dy * dy, dg, -dy * dgy);
        v[5] = __fdividef(dg, q.sigma);
    }
    p.T = T0; p.Tx = Tx0; p.Ty = Ty0; p.Txy = Txy0;
    return true;
}

// Sum of v[0..8] over the warp into acc[0..8] (shared memory): a transposed
// exchange halves the values a lane carries at each of the first three steps,
// so lane L ends with the sum of value (L >> 2) & 7 (14 shuffles for the 9
// values instead of 45), then 2 atomic instructions.
__device__ __forceinline__ void warp_sum9_to_shared(float v[9], int lane, float* acc)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float r = __shfl_xor_sync(0xffffffffu, b4 ? v[j] : v[j + 4], 16);
        v[j] = (b4 ? v[j + 4] : v[j]) + r;
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float r = __shfl_xor_sync(0xffffffffu, b3 ? v[j] : v[j + 2], 8);
        v[j] = (b3 ? v[j + 2] : v[j]) + r;
    }
    {
        const float r = __shfl_xor_sync(0xffffffffu, b2 ? v[0] : v[1], 4);
        v[0] = (b2 ? v[1] : v[0]) + r;
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    float t8 = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t8 += __shfl_xor_sync(0xffffffffu, t8, o);
    if ((lane & 3) == 0) atomicAdd(&acc[lane >> 2], v[0]);
    if (lane == 0) atomicAdd(&acc[8], t8);
}

// The forward blend's step of the transmittance state alone (same expressions
// and decisions as the forward), given the pair's offset (dx, dy) and
// exponent g2.  Returns true if the pair was blended; sets done when the
// pixel stops before it.
template <int MODE>
__device__ __forceinline__ bool fwd_state_step(BwdPixel& p, bool& done, float dx, float dy, float g2,
                                               const float4& r0, const float4& r1, float sigma)
{
    if (MODE == GS_MODE_3DGS && g2 < r1.w) return false;
    float alpha = sigma * pow2(g2);
    bool clamped = false;
    if (MODE == GS_MODE_3DGS) {
        if (alpha < (1.f / 255.f)) return false;
        clamped = alpha > 0.99f;
        alpha = fminf(alpha, 0.99f);
    }
    const float Tn = p.T * __fsub_rn(1.f, alpha);   // as the forward's blend_pair
    if (MODE == GS_MODE_3DGS && Tn < 1e-4f) {
        done = true;
        return false;
    }
    const float bn = r1.y * kLn2;
    float gx = fmaf(r0.z, dx, bn * dy);
    float gy = fmaf(r0.w, dy, bn * dx);
    float gxy = fmaf(gx, gy, bn);
    if (clamped) { gx = 0.f; gy = 0.f; gxy = 0.f; }
    const float wx = alpha * fmaf(p.T, gx, p.Tx);
    const float wy = alpha * fmaf(p.T, gy, p.Ty);
    const float wxy = alpha * fmaf(p.T, gxy, fmaf(p.Tx, gy, fmaf(p.Ty, gx, p.Txy)));
    p.Tx = __fsub_rn(p.Tx, wx);
    p.Ty = __fsub_rn(p.Ty, wy);
    p.Txy = __fsub_rn(p.Txy, wxy);
    p.T = Tn;
    return true;
}

// Four blocks per SM: the register cap of 64 costs the 3DGS instantiation 20 B
// of spills, and the fourth block's warps hide more of the gather and
// barrier latency than the spills add.
template <int MODE, bool RECOMPUTE>
__global__ void __launch_bounds__(kThreads, 4) k_blend_bwd(BlendBwdArgs a)
{
    __shared__ float4 s_r0[kCand];
    __shared__ float4 s_r1[kCand];
    __shared__ float4 s_r2[kCand];
    __shared__ uint32_t s_id[kCand];
    __shared__ float s_acc[kCand][9];
    __shared__ int s_round[kMaxRounds];
    __shared__ int s_seg[kMaxSegs];
    __shared__ int s_wcnt[kWarps];
    __shared__ int s_max[kWarps];

    const int tile = a.order ? (int)a.order[blockIdx.x] : (int)blockIdx.x;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lanemask_lt = (1u << lane) - 1u;
    // each warp an 8 x 4 block of pixels, as in the forward blend
    const int x = tx * kTile + (((warp & 1) << 3) | (lane & 7));
    const int y = ty * kTile + (((warp >> 1) << 2) | (lane >> 3));
    const bool inside = x < a.W && y < a.H;
    const size_t plane = (size_t)a.W * a.H;
    const size_t pix = inside ? (size_t)y * a.W + x : 0;

    BwdPixel p;
    p.px = (float)x;
    p.py = (float)y;
    p.last = 0;
    p.T = 1.f; p.Tx = 0.f; p.Ty = 0.f; p.Txy = 0.f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) { p.uC[ch] = 0.f; p.uX[ch] = 0.f; p.uY[ch] = 0.f; p.uZ[ch] = 0.f; }
    if (inside) {
        if (!RECOMPUTE) {
            p.last = a.count[pix];
            const float4 st = a.state[pix];
            p.T = st.x; p.Tx = st.y; p.Ty = st.z; p.Txy = st.w;
        }
        if (a.dout) {   // the upscale's adjoint at this pixel, fused
            float acc[3][4];
            upscale_adjoint_at(a.dout, a.W, a.H, a.W2, a.H2, x, y, acc);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                p.uC[ch] = acc[ch][0];
                p.uX[ch] = acc[ch][1];
                p.uY[ch] = acc[ch][2];
                p.uZ[ch] = acc[ch][3];
            }
        } else {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                p.uC[ch] = a.dC[ch * plane + pix];
                if (a.dG) {
                    p.uX[ch] = a.dG[(0 * 3 + ch) * plane + pix];
                    p.uY[ch] = a.dG[(1 * 3 + ch) * plane + pix];
                    p.uZ[ch] = a.dG[(2 * 3 + ch) * plane + pix];
                }
            }
        }
    }
    // adjoint of the state after the last step: output += bg (T, T_x, T_y, T_xy)
    p.lT = p.uC[0] * a.bg.x + p.uC[1] * a.bg.y + p.uC[2] * a.bg.z;
    p.lTx = p.uX[0] * a.bg.x + p.uX[1] * a.bg.y + p.uX[2] * a.bg.z;
    p.lTy = p.uY[0] * a.bg.x + p.uY[1] * a.bg.y + p.uY[2] * a.bg.z;
    p.lTxy = p.uZ[0] * a.bg.x + p.uZ[1] * a.bg.y + p.uZ[2] * a.bg.z;

#pragma unroll
    for (int q = 0; q < 9; ++q) s_acc[threadIdx.x][q] = 0.f;

    const int ksh = __ffs(a.ks) - 1;   // ks = 1, 2 or 4
    const int S = (ty >> ksh) * a.stiles_x + (tx >> ksh);
    const uint2 sr = a.sranges[S];
    const int total = (int)(sr.y - sr.x);
    const int tbit = (ty & (a.ks - 1)) * a.ks + (tx & (a.ks - 1));   // this tile in the pair masks

    int filt = 0, R = 0;
    int ck_stride = 1, ck_used = 0;   // recompute: checkpoint of round r in slot r / ck_stride
    float4* ck = RECOMPUTE ? a.ckpt + (size_t)tile * kCkSlots * kThreads + threadIdx.x : nullptr;
    if (RECOMPUTE) {
        // pass 1: the forward walk of the tile (transmittance state and counts),
        // round by round, with the exact state checkpointed at round starts
        bool done = !inside;
        for (int c0 = 0; c0 < total; c0 += kCand, ++R) {
            if (__syncthreads_count(done) == kThreads) break;
            if (R % kMaxRounds == 0) {
                if (R / kMaxRounds >= kMaxSegs) {
                    if (threadIdx.x == 0) atomicExch(a.err, kDevCheck);
                    break;
                }
                if (threadIdx.x == 0) s_seg[R / kMaxRounds] = filt;
            }
            if (threadIdx.x == 0) s_round[R % kMaxRounds] = filt;
            if (R % ck_stride == 0) {
                if (R / ck_stride == kCkSlots) {   // full: keep every second checkpoint
#pragma unroll 1
                    for (int j = 1; j < kCkSlots / 2; ++j) ck[(size_t)j * kThreads] = ck[(size_t)(2 * j) * kThreads];
                    ck_stride *= 2;
                }
                if (R % ck_stride == 0) {
                    ck[(size_t)(R / ck_stride) * kThreads] = make_float4(p.T, p.Tx, p.Ty, p.Txy);
                    ck_used = R / ck_stride + 1;
                }
            }
            const int c = c0 + (int)threadIdx.x;
            uint32_t id = 0xFFFFFFFFu;
            bool hit = false;
            if (c < total) hit = pair_hit(a.pair_words, sr.x + c, a.n, tbit, id);
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
                const int k = wbase + __popc(ball & lanemask_lt);
                s_r0[k] = a.rec.r0[id];
                s_r1[k] = a.rec.r1[id];
                s_r2[k].w = a.rec.r2[id].w;
            }
            __syncthreads();
            // in groups of 3, as the forward walks: the records' offsets and
            // exponents first, then the state steps in order
            int k = 0;
            for (; k + 2 < tot && !done; k += 3) {
                float4 q0[3], q1[3];
                float qdx[3], qdy[3], qg2[3], qs[3];
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    q0[u] = s_r0[k + u];
                    q1[u] = s_r1[k + u];
                    qs[u] = s_r2[k + u].w;
                    qdx[u] = p.px - q0[u].x;
                    qdy[u] = p.py - q0[u].y;
                    qg2[u] = exponent2(q1[u], qdx[u], qdy[u]);
                }
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    if (u > 0 && done) break;
                    if (fwd_state_step<MODE>(p, done, qdx[u], qdy[u], qg2[u], q0[u], q1[u], qs[u]))
                        p.last = filt + k + u + 1;
                }
            }
            for (; k < tot && !done; ++k) {
                const float4 r0 = s_r0[k], r1 = s_r1[k];
                const float dx = p.px - r0.x, dy = p.py - r0.y;
                if (fwd_state_step<MODE>(p, done, dx, dy, exponent2(r1, dx, dy), r0, r1, s_r2[k].w)) p.last = filt + k + 1;
            }
            filt += tot;
        }
        __syncthreads();
    }
    // the block's longest prefix of the tile list
    int m = p.last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_max[warp] = m;
    __syncthreads();
    int M = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) M = max(M, s_max[w]);

    // pass 1 (inversion): the tile's list position at the start of each round of candidates
    for (int c0 = 0; !RECOMPUTE && c0 < total && filt < M; c0 += kCand, ++R) {
        if (R % kMaxRounds == 0) {
            if (R / kMaxRounds >= kMaxSegs) break;
            if (threadIdx.x == 0) s_seg[R / kMaxRounds] = filt;
        }
        if (threadIdx.x == 0) s_round[R % kMaxRounds] = filt;
        const int c = c0 + (int)threadIdx.x;
        bool hit = false;
        if (c < total) {
            uint32_t id;
            hit = pair_hit(a.pair_words, sr.x + c, a.n, tbit, id);
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) s_wcnt[warp] = __popc(ball);
        __syncthreads();
        int tot = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) tot += s_wcnt[w];
        __syncthreads();
        filt += tot;
    }
    if (filt < M) {   // the list ended (or is too long) before the stored counts: report, walk what exists
        if (threadIdx.x == 0) atomicExch(a.err, kDevCheck);
        M = filt;
    }

    // pass 2: replay the rounds last to first
    const int nseg = (R + kMaxRounds - 1) / kMaxRounds;
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int rb = seg * kMaxRounds, re = min(R, rb + kMaxRounds);
        if (seg != nseg - 1) {   // pass 1 kept the round starts of the last segment only
            __syncthreads();
            int f = s_seg[seg];
            for (int r = rb; r < re; ++r) {
                if (threadIdx.x == 0) s_round[r - rb] = f;
                const int c = r * kCand + (int)threadIdx.x;
                bool hit = false;
                if (c < total) {
                    uint32_t id;
                    hit = pair_hit(a.pair_words, sr.x + c, a.n, tbit, id);
                }
                const uint32_t ball = __ballot_sync(0xffffffffu, hit);
                if (lane == 0) s_wcnt[warp] = __popc(ball);
                __syncthreads();
                int tot = 0;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) tot += s_wcnt[w];
                __syncthreads();
                f += tot;
            }
        }
        __syncthreads();
        for (int r = re - 1; r >= rb; --r) {
            const int fb = s_round[r - rb];
            if (RECOMPUTE && r + 1 < R && (r + 1) % ck_stride == 0 && (r + 1) / ck_stride < ck_used) {
                // the exact state at the end of this round (the next round's start)
                const float4 st = ck[(size_t)((r + 1) / ck_stride) * kThreads];
                p.T = st.x; p.Tx = st.y; p.Ty = st.z; p.Txy = st.w;
            }
            const int c = r * kCand + (int)threadIdx.x;
            uint32_t id = 0xFFFFFFFFu;
            bool hit = false;
            if (c < total) hit = pair_hit(a.pair_words, sr.x + c, a.n, tbit, id);
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
            const int cnt = min(tot, M - fb);   // entries at list positions >= M are not needed
            if (hit) {
                const int k = wbase + __popc(ball & lanemask_lt);
                if (k < cnt) {
                    s_id[k] = id;
                    s_r0[k] = a.rec.r0[id];
                    s_r1[k] = a.rec.r1[id];
                    s_r2[k] = a.rec.r2[id];
                }
            }
            __syncthreads();
            // entries in groups of two: both prepared (state-independent part)
            // before either is applied, which leaves the state's step the
            // loop-carried chain
            int k = cnt - 1;
            for (; k >= 1; k -= 2) {
                BwdPrep qa, qb;
                bwd_prep<MODE>(p, s_r0[k], s_r1[k], s_r2[k], fb + k < p.last, qa);
                bwd_prep<MODE>(p, s_r0[k - 1], s_r1[k - 1], s_r2[k - 1], fb + k - 1 < p.last, qb);
                {
                    float v[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) v[q] = 0.f;
                    const bool contrib = bwd_apply(p, qa, v);
                    if (__any_sync(0xffffffffu, contrib)) warp_sum9_to_shared(v, lane, s_acc[k]);
                }
                {
                    float v[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) v[q] = 0.f;
                    const bool contrib = bwd_apply(p, qb, v);
                    if (__any_sync(0xffffffffu, contrib)) warp_sum9_to_shared(v, lane, s_acc[k - 1]);
                }
            }
            if (k == 0) {
                BwdPrep q0;
                bwd_prep<MODE>(p, s_r0[0], s_r1[0], s_r2[0], fb < p.last, q0);
                float v[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) v[q] = 0.f;
                const bool contrib = bwd_apply(p, q0, v);
                if (__any_sync(0xffffffffu, contrib)) warp_sum9_to_shared(v, lane, s_acc[0]);
            }
            __syncthreads();
            if ((int)threadIdx.x < cnt) {
                float* g = a.grad2d + (size_t)s_id[threadIdx.x] * 9;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const float val = s_acc[threadIdx.x][q];
                    if (val != 0.f) atomicAdd(g + q, val);
                    s_acc[threadIdx.x][q] = 0.f;
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_blend_backward(cudaStream_t s, int mode, const BlendBwdArgs& a)
{
    const int tiles = a.tiles_x * ((a.H + kTile - 1) / kTile);
    if (tiles == 0) return cudaSuccess;
    if (a.ckpt) {
        if (mode == GS_MODE_EXACT)
            k_blend_bwd<GS_MODE_EXACT, true><<<tiles, kThreads, 0, s>>>(a);
        else
            k_blend_bwd<GS_MODE_3DGS, true><<<tiles, kThreads, 0, s>>>(a);
    } else {
        if (mode == GS_MODE_EXACT)
            k_blend_bwd<GS_MODE_EXACT, false><<<tiles, kThreads, 0, s>>>(a);
        else
            k_blend_bwd<GS_MODE_3DGS, false><<<tiles, kThreads, 0, s>>>(a);
    }
    note_launch();
    return cudaGetLastError();
}

}  // namespace gs
