// Learned residual on top of the spline upscale: a per-output-pixel MLP
// 50 -> 64 -> 64 -> 3 (ReLU) that reads the 48 values the spline reads (C,
// dC/dx, dC/dy, d2C/dxdy of the three channels at the four corners of the
// pixel's cell) and the local coordinates (t, u), and adds its output to the
// spline value.  The paper's method is the spline alone (Sec. 5); this is an
// optional extension on the same inputs, with the spline as the fallback.
//
// Feature order: f[12 k + 3 q + c] = quantity q (C, C_x, C_y, C_xy) of channel
// c at corner k ((i, j), (i+1, j), (i, j+1), (i+1, j+1)); f[48] = t, f[49] = u.
// Parameters: one FP32 vector W1 [64][50], b1 [64], W2 [64][64], b2 [64],
// W3 [3][64], b3 [3] (7619 values).  The matrices enter the tensor core as
// BF16 (round to nearest even), the biases stay FP32; accumulation is FP32.
// Activations enter each product as BF16: the features, h1 and h2 (and, in the
// reverse mode, d2 and d1).
//
// Kernels (tcgen05, one CTA of 128 threads per 128 samples at a time, a
// persistent grid; see umma.cuh for the operand layout):
//   k_mlp_upscale   inference fused into the upscale: per 128 output pixels
//                   gather the 48 corner values (once, for both the spline and
//                   the features), evaluate the spline, stage the BF16
//                   features as the A operand, two MMAs (M 128, N 64, K 64)
//                   and a third (N 16, the 64 -> 3 output layer) with ReLU
//                   epilogues from tensor memory, write spline + residual.
//   k_mlp_samples   training samples: features (BF16 rows of 64), spline value
//                   and target at given output pixels.
//   k_mlp_grad      forward and reverse mode of the MSE loss over M samples:
//                   h1 = relu(W1 f + b1) and h2 = relu(W2 h1 + b2) as in
//                   inference (h2 narrowed to BF16 for the output layer, which
//                   runs on the FP32 cores here); d3 = 2 e / (3 M);
//                   d2 = (W3^T d3) [z2 > 0] on the
//                   FP32 cores; d1 = (W2^T d2) [z1 > 0] as an MMA against W2^T;
//                   the weight gradients of both hidden layers in one MMA per
//                   tile, P Q^T with P = [d2^T ; d1^T] (128 units x 128
//                   samples) and Q = [h1^T ; f^T] (128 x 128, the feature rows
//                   carrying a constant 1 in slot 50 for the bias gradients),
//                   accumulated in tensor memory over the CTA's tiles; dW3 and
//                   db3 on the FP32 cores.
//   k_mlp_adam      Adam with bias correction (Kingma and Ba, 2015).
#include <algorithm>
#include <cmath>

#include "gs_internal.cuh"
#include "spline_common.cuh"
#include "umma.cuh"

namespace gs {
namespace {

using namespace umma;

constexpr int kIn = 50, kHid = 64, kOut = 3;
constexpr int kRows = 128;                 // samples per tile = MMA M
constexpr int kThreads = 128;              // one sample (accumulator lane) per thread
constexpr uint32_t kLbo = 128;             // core matrices adjacent in K
constexpr uint32_t kSbo64 = 1024;          // 8-row groups of a K = 64 operand
constexpr uint32_t kSbo128 = 2048;         // 8-row groups of a K = 128 operand
constexpr uint32_t kWaitLimit = 1u << 22;  // mbarrier polls before giving up

constexpr int oW1 = 0, oB1 = oW1 + kHid * kIn, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kOut * kHid, kParams = oB3 + kOut;
static_assert(kParams == GS_MLP_PARAMS, "parameter layout");

// byte offset of element (r, k) of a K-major no-swizzle operand
__device__ __forceinline__ uint32_t kmaj(int r, int k, uint32_t sbo)
{
    return (uint32_t)(r >> 3) * sbo + (uint32_t)(k >> 3) * kLbo + (uint32_t)(r & 7) * 16 + (uint32_t)(k & 7) * 2;
}

__device__ __forceinline__ void st_bf16(uint8_t* base, uint32_t off, float v)
{
    *reinterpret_cast<uint16_t*>(base + off) = (uint16_t)(pack_bf16x2(v, 0.f) & 0xFFFFu);
}

// The weights of the first two layers as BF16 B operands (N = 64 rows, K = 64):
// w1 (n = unit, k = feature; features 50..63 zero), w2 (n = out, k = in) and,
// when w2t != nullptr, its transpose (n = in, k = out).  W3 rounded to BF16
// values in FP32; biases in FP32.
__device__ void stage_weights(const float* __restrict__ P, uint8_t* w1, uint8_t* w2, uint8_t* w2t, float* w3,
                              float* b1, float* b2, float* b3)
{
    for (int e = threadIdx.x; e < kHid * 64; e += blockDim.x) {
        const int n = e >> 6, k = e & 63;
        st_bf16(w1, kmaj(n, k, kSbo64), k < kIn ? P[oW1 + n * kIn + k] : 0.f);
        const float v = P[oW2 + n * kHid + k];
        st_bf16(w2, kmaj(n, k, kSbo64), v);
        if (w2t) st_bf16(w2t, kmaj(k, n, kSbo64), v);
    }
    for (int e = threadIdx.x; e < kOut * kHid; e += blockDim.x) w3[e] = bf16_round(P[oW3 + e]);
    for (int e = threadIdx.x; e < kHid; e += blockDim.x) {
        b1[e] = P[oB1 + e];
        b2[e] = P[oB2 + e];
    }
    if (threadIdx.x < kOut) b3[threadIdx.x] = P[oB3 + threadIdx.x];
}

// The 48 corner values of output pixel (X, Y) in feature order, its local
// coordinates, and the spline value (the Hermite patch of the cell).
__device__ __forceinline__ void pixel_inputs(const float* __restrict__ C, const float* __restrict__ G, int W, int H,
                                             int W2, int H2, int X, int Y, float (&f)[48], float& t, float& u,
                                             float (&sp)[3])
{
    int i, j;
    cell_of(X, W, W2, i, t);
    cell_of(Y, H, H2, j, u);
    const size_t plane = (size_t)W * H;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const size_t o = (size_t)(j + (k >> 1)) * W + i + (k & 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            f[12 * k + c] = __ldg(C + c * plane + o);
            f[12 * k + 3 + c] = __ldg(G + c * plane + o);
            f[12 * k + 6 + c] = __ldg(G + (3 + c) * plane + o);
            f[12 * k + 9 + c] = __ldg(G + (6 + c) * plane + o);
        }
    }
    const float4 hx = hermite(t), hy = hermite(u);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float Hx = (k & 1) ? hx.y : hx.x, Gx = (k & 1) ? hx.w : hx.z;
            const float Hy = (k >> 1) ? hy.y : hy.x, Gy = (k >> 1) ? hy.w : hy.z;
            acc = fmaf(Hx * Hy, f[12 * k + c], acc);
            acc = fmaf(Gx * Hy, f[12 * k + 3 + c], acc);
            acc = fmaf(Hx * Gy, f[12 * k + 6 + c], acc);
            acc = fmaf(Gx * Gy, f[12 * k + 9 + c], acc);
        }
        sp[c] = acc;
    }
}

// 64 BF16 feature values of one sample as 8 chunks of 8 (16 bytes each);
// slots 50..63 are zero
__device__ __forceinline__ void feature_chunks(const float (&f)[48], float t, float u, uint4 (&q)[8])
{
#pragma unroll
    for (int c = 0; c < 6; ++c)
        q[c] = make_uint4(pack_bf16x2(f[8 * c], f[8 * c + 1]), pack_bf16x2(f[8 * c + 2], f[8 * c + 3]),
                          pack_bf16x2(f[8 * c + 4], f[8 * c + 5]), pack_bf16x2(f[8 * c + 6], f[8 * c + 7]));
    q[6] = make_uint4(pack_bf16x2(t, u), 0u, 0u, 0u);
    q[7] = make_uint4(0u, 0u, 0u, 0u);
}

// row r of a K = 64 operand from 8 chunks
__device__ __forceinline__ void store_row(uint8_t* op, int r, const uint4 (&q)[8])
{
#pragma unroll
    for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4*>(op + kmaj(r, 8 * c, kSbo64)) = q[c];
}

// the four K = 16 steps of D = A B^T with A, B K = 64 operands
__device__ __forceinline__ void mma_k64(uint32_t d, uint32_t a, uint32_t b, uint32_t idesc)
{
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
        mma_bf16(d, smem_desc(a + kk * 2 * kLbo, kLbo, kSbo64), smem_desc(b + kk * 2 * kLbo, kLbo, kSbo64), idesc,
                 kk > 0);
}

// ------------------------------------------------------------------ inference

// A tile is 32 x 4 output pixels: thread tid takes pixel (tid % 32, tid / 32),
// so warp w owns output row w of the tile and accumulator lanes 32 w .. 32 w +
// 31.  The tile's low-res footprint (at most 33 x 5 pixels for W2 >= W,
// H2 >= H: the cells of 32 consecutive columns span at most 31 cells) is staged
// in shared memory with coalesced loads, each low-res pixel as three float4
// holding its 12 values (C, C_x, C_y, C_xy) x (r, g, b) -- the feature order
// of one corner.  Cell indices and Hermite weights of the tile's 32 columns
// and 4 rows are computed once per tile.
constexpr int kTileW = 32, kTileH = 4;
constexpr int kFootW = kTileW + 1, kFootH = kTileH + 1;
static_assert(kTileW * kTileH == kRows, "one tile per MMA");

struct InferSmem {
    uint8_t a[kRows * 128];          // A operand: features, then h1
    uint8_t w1[kHid * 128];
    uint8_t w2[kHid * 128];
    uint8_t w3[16 * 128];            // W3 as a B operand: N = 16 rows (3 used), K = 64
    float4 b1[kHid / 4], b2[kHid / 4];
    float tx[kTileW], ty[kTileH];    // local coordinates t, u
    int cx[kTileW], cy[kTileH];      // absolute cell indices
    float b3[4];
    uint64_t bar;
    uint32_t tmem;
};
// followed in dynamic shared memory by the footprint: fpw x fph low-res pixels
// (fpw = ceil(31 W / W2) + 2 <= 33, fph = ceil(3 H / H2) + 2 <= 5), three float4 each

constexpr uint32_t kInferCols = 64;   // D1, D2 and D3 share columns 0..63

// element e (0..11) of a corner's three float4
__device__ __forceinline__ float corner_value(const float4 (&v)[3], int e)
{
    const float4 q = v[e >> 2];
    switch (e & 3) {
    case 0: return q.x;
    case 1: return q.y;
    case 2: return q.z;
    default: return q.w;
    }
}

__global__ void __launch_bounds__(kThreads, 6) k_mlp_upscale(const float* __restrict__ C, const float* __restrict__ G,
                                                             int W, int H, int W2, int H2, int fpw,
                                                             const float* __restrict__ P, float* __restrict__ out,
                                                             int* __restrict__ err)
{
    extern __shared__ __align__(128) uint8_t smem_raw[];
    InferSmem& s = *reinterpret_cast<InferSmem*>(smem_raw);
    float4* const foot = reinterpret_cast<float4*>(smem_raw + sizeof(InferSmem));
    const int tid = threadIdx.x, warp = tid >> 5, lx = tid & 31, ly = tid >> 5;
    for (int e = tid; e < kHid * 64; e += kThreads) {
        const int n = e >> 6, k = e & 63;
        st_bf16(s.w1, kmaj(n, k, kSbo64), k < kIn ? P[oW1 + n * kIn + k] : 0.f);
        st_bf16(s.w2, kmaj(n, k, kSbo64), P[oW2 + n * kHid + k]);
    }
    for (int e = tid; e < 16 * 64; e += kThreads) {
        const int n = e >> 6, k = e & 63;
        st_bf16(s.w3, kmaj(n, k, kSbo64), n < kOut ? P[oW3 + n * kHid + k] : 0.f);
    }
    if (tid < kHid) {
        reinterpret_cast<float*>(s.b1)[tid] = P[oB1 + tid];
        reinterpret_cast<float*>(s.b2)[tid] = P[oB2 + tid];
    }
    if (tid < kOut) s.b3[tid] = P[oB3 + tid];
    if (tid == 0) {
        mbar_init(&s.bar, 1);
        mbar_init_fence();
    }
    if (warp == 0) {
        tmem_alloc(&s.tmem, kInferCols);
        tmem_relinquish();
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s.tmem;
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    const uint32_t sa = smem_u32(s.a), w1 = smem_u32(s.w1), w2 = smem_u32(s.w2), w3 = smem_u32(s.w3);
    constexpr uint32_t idesc = idesc_bf16(kRows, kHid);
    constexpr uint32_t idesc3 = idesc_bf16(kRows, 16);
    const int tiles_x = (W2 + kTileW - 1) / kTileW;
    const long long ntiles = (long long)tiles_x * ((H2 + kTileH - 1) / kTileH);
    const size_t plane = (size_t)W * H, plane2 = (size_t)W2 * H2;
    uint32_t phase = 0;
    bool ok = true;
    bool late = false;   // this thread's wait for an MMA ran out (the block leaves at its next barrier)
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tyi = (int)(tile / tiles_x);
        const int X0 = (int)(tile - (long long)tyi * tiles_x) * kTileW, Y0 = tyi * kTileH;
        // cells of the tile's columns and rows (clamped to the last pixel)
        if (tid < kTileW) {
            int ci;
            float t;
            cell_of(min(X0 + tid, W2 - 1), W, W2, ci, t);
            s.cx[tid] = ci;
            s.tx[tid] = t;
        } else if (tid < kTileW + kTileH) {
            const int r = tid - kTileW;
            int cj;
            float u;
            cell_of(min(Y0 + r, H2 - 1), H, H2, cj, u);
            s.cy[r] = cj;
            s.ty[r] = u;
        }
        if (__syncthreads_or(late)) {
            ok = false;
            break;
        }
        const int i0 = s.cx[0], j0 = s.cy[0];
        const int fw = s.cx[kTileW - 1] + 2 - i0, fh = s.cy[kTileH - 1] + 2 - j0;   // <= fpw x fph
        for (int e = tid; e < fw * fh; e += kThreads) {
            const int fy = e / fw, fx = e - fy * fw;
            const size_t o = (size_t)(j0 + fy) * W + i0 + fx;
            float4* d = foot + 3 * (fy * fpw + fx);
            d[0] = make_float4(__ldg(C + o), __ldg(C + plane + o), __ldg(C + 2 * plane + o), __ldg(G + o));
            d[1] = make_float4(__ldg(G + plane + o), __ldg(G + 2 * plane + o), __ldg(G + 3 * plane + o),
                               __ldg(G + 4 * plane + o));
            d[2] = make_float4(__ldg(G + 5 * plane + o), __ldg(G + 6 * plane + o), __ldg(G + 7 * plane + o),
                               __ldg(G + 8 * plane + o));
        }
        __syncthreads();
        // this pixel: spline value and BF16 features (row tid of A)
        const int X = X0 + lx, Y = Y0 + ly;
        float sp0 = 0.f, sp1 = 0.f, sp2 = 0.f;
        {
            const int li = s.cx[lx] - i0, lj = s.cy[ly] - j0;
            const float4 hx = hermite(s.tx[lx]), hy = hermite(s.ty[ly]);
            float4 v[4][3];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4* src = foot + 3 * ((lj + (k >> 1)) * fpw + li + (k & 1));
                v[k][0] = src[0];
                v[k][1] = src[1];
                v[k][2] = src[2];
                const float Hx = (k & 1) ? hx.y : hx.x, Gx = (k & 1) ? hx.w : hx.z;
                const float Hy = (k >> 1) ? hy.y : hy.x, Gy = (k >> 1) ? hy.w : hy.z;
                const float wv = Hx * Hy, wdx = Gx * Hy, wdy = Hx * Gy, wdxy = Gx * Gy;
                sp0 = fmaf(wv, v[k][0].x, sp0);
                sp1 = fmaf(wv, v[k][0].y, sp1);
                sp2 = fmaf(wv, v[k][0].z, sp2);
                sp0 = fmaf(wdx, v[k][0].w, sp0);
                sp1 = fmaf(wdx, v[k][1].x, sp1);
                sp2 = fmaf(wdx, v[k][1].y, sp2);
                sp0 = fmaf(wdy, v[k][1].z, sp0);
                sp1 = fmaf(wdy, v[k][1].w, sp1);
                sp2 = fmaf(wdy, v[k][2].x, sp2);
                sp0 = fmaf(wdxy, v[k][2].y, sp0);
                sp1 = fmaf(wdxy, v[k][2].z, sp1);
                sp2 = fmaf(wdxy, v[k][2].w, sp2);
            }
            // feature f = 12 k + e is element e of corner k; chunk c holds f = 8c .. 8c + 7
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                uint32_t w4[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int f = 8 * c + 2 * j;
                    w4[j] = pack_bf16x2(corner_value(v[f / 12], f % 12), corner_value(v[(f + 1) / 12], (f + 1) % 12));
                }
                *reinterpret_cast<uint4*>(s.a + kmaj(tid, 8 * c, kSbo64)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
            *reinterpret_cast<uint4*>(s.a + kmaj(tid, 48, kSbo64)) =
                make_uint4(pack_bf16x2(s.tx[lx], s.ty[ly]), 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(s.a + kmaj(tid, 56, kSbo64)) = make_uint4(0u, 0u, 0u, 0u);
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
            mma_k64(tmem, sa, w1, idesc);
            mma_commit(&s.bar);
        }
        late |= !mbar_wait(&s.bar, phase, kWaitLimit);   // each thread reads only its own accumulator lane
        phase ^= 1u;
        fence_after_sync();
        // layer 1 epilogue: h1 = relu(z1 + b1) as the BF16 row of A (the MMA
        // that read the features is complete)
#pragma unroll
        for (int g = 0; g < 4; g += 2) {      // two loads in flight per wait
            float z[2][16];
            tmem_ld16(tmem + lane + 16 * g, z[0]);
            tmem_ld16(tmem + lane + 16 * g + 16, z[1]);
            tmem_wait_ld();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t w[8];
                bias_relu_bf16(z[h], s.b1 + 4 * (g + h), w);
                *reinterpret_cast<uint4*>(s.a + kmaj(tid, 16 * (g + h), kSbo64)) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4*>(s.a + kmaj(tid, 16 * (g + h) + 8, kSbo64)) =
                    make_uint4(w[4], w[5], w[6], w[7]);
            }
        }
        fence_async_smem();
        fence_before_sync();
        if (__syncthreads_or(late)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            fence_after_sync();
            mma_k64(tmem, sa, w2, idesc);      // every thread has read D1
            mma_commit(&s.bar);
        }
        late |= !mbar_wait(&s.bar, phase, kWaitLimit);   // each thread reads only its own accumulator lane
        phase ^= 1u;
        fence_after_sync();
        // layer 2 epilogue: h2 = relu(z2 + b2) as the BF16 row of A (the MMA
        // that read h1 is complete)
#pragma unroll
        for (int g = 0; g < 4; g += 2) {      // two loads in flight per wait
            float z[2][16];
            tmem_ld16(tmem + lane + 16 * g, z[0]);
            tmem_ld16(tmem + lane + 16 * g + 16, z[1]);
            tmem_wait_ld();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t w[8];
                bias_relu_bf16(z[h], s.b2 + 4 * (g + h), w);
                *reinterpret_cast<uint4*>(s.a + kmaj(tid, 16 * (g + h), kSbo64)) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4*>(s.a + kmaj(tid, 16 * (g + h) + 8, kSbo64)) =
                    make_uint4(w[4], w[5], w[6], w[7]);
            }
        }
        fence_async_smem();
        fence_before_sync();
        if (__syncthreads_or(late)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            fence_after_sync();
            mma_k64(tmem, sa, w3, idesc3);     // the output layer, N = 16 (3 used)
            mma_commit(&s.bar);
        }
        late |= !mbar_wait(&s.bar, phase, kWaitLimit);   // each thread reads only its own accumulator lane
        phase ^= 1u;
        fence_after_sync();
        float r0, r1, r2;
        {
            float z[16];
            tmem_ld16(tmem + lane, z);
            tmem_wait_ld();
            r0 = z[0] + s.b3[0];
            r1 = z[1] + s.b3[1];
            r2 = z[2] + s.b3[2];
        }
        if (X < W2 && Y < H2) {
            const size_t o = (size_t)Y * W2 + X;
            out[o] = sp0 + r0;
            out[plane2 + o] = sp1 + r1;
            out[2 * plane2 + o] = sp2 + r2;
        }
        fence_before_sync();
    }
    ok = !__syncthreads_or(late || !ok);   // a wait in the last tile may have run out
    if (!ok && tid == 0) atomicExch(err, kDevTimeout);
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, kInferCols);
}

// ------------------------------------------------------------------ training samples

__global__ void k_mlp_samples(const float* __restrict__ C, const float* __restrict__ G, int W, int H, int W2, int H2,
                              const int* __restrict__ pix, long long M, const float* __restrict__ target_img,
                              uint16_t* __restrict__ feat, float* __restrict__ base, float* __restrict__ target,
                              int* __restrict__ err)
{
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int X = pix[2 * m], Y = pix[2 * m + 1];
    uint4 q[8];
    float sp[3] = {0.f, 0.f, 0.f};
    if (X < 0 || X >= W2 || Y < 0 || Y >= H2) {
        atomicExch(err, kDevCheck);
#pragma unroll
        for (int c = 0; c < 8; ++c) q[c] = make_uint4(0u, 0u, 0u, 0u);
    } else {
        float f[48], t, u;
        pixel_inputs(C, G, W, H, W2, H2, X, Y, f, t, u, sp);
        feature_chunks(f, t, u, q);
    }
    uint4* dst = reinterpret_cast<uint4*>(feat + m * 64);
#pragma unroll
    for (int c = 0; c < 8; ++c) dst[c] = q[c];
#pragma unroll
    for (int c = 0; c < 3; ++c) base[3 * m + c] = sp[c];
    if (target && target_img) {
        const bool in = X >= 0 && X < W2 && Y >= 0 && Y < H2;
        const size_t plane2 = (size_t)W2 * H2, o = in ? (size_t)Y * W2 + X : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) target[3 * m + c] = in ? target_img[c * plane2 + o] : 0.f;
    }
}

// ------------------------------------------------------------------ training: forward + reverse mode

struct TrainSmem {
    uint8_t a[kRows * 128];     // A operand rows: features, then h1, then d2
    uint8_t pm[kRows * 256];    // P = [d2^T ; d1^T]: 128 units x 128 samples (K = samples)
    uint8_t qm[kRows * 256];    // Q = [h1^T ; f^T]:  128 x 128
    uint8_t w1[kHid * 128];
    uint8_t w2[kHid * 128];
    uint8_t w2t[kHid * 128];
    float h2[kRows][kHid + 1];
    float d3[kRows][4];
    float w3[kOut * kHid];
    float b1[kHid], b2[kHid], b3[4];
    float red[kThreads / 32];
    uint64_t bar;
    uint32_t tmem;
};

// D1 / D3: columns 0..63, D2: 64..127, weight gradients 128..255
constexpr uint32_t kTrainCols = 256;
constexpr uint16_t kBf16One = 0x3F80;

__device__ __forceinline__ void st_u16(uint8_t* base, uint32_t off, uint32_t bits)
{
    *reinterpret_cast<uint16_t*>(base + off) = (uint16_t)(bits & 0xFFFFu);
}

__global__ void __launch_bounds__(kThreads) k_mlp_grad(const float* __restrict__ P, const uint16_t* __restrict__ feat,
                                                       const float* __restrict__ base,
                                                       const float* __restrict__ target, long long M, float scale,
                                                       float inv, float* __restrict__ grads,
                                                       float* __restrict__ loss, int* __restrict__ err)
{
    extern __shared__ __align__(128) uint8_t smem_raw[];
    TrainSmem& s = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    stage_weights(P, s.w1, s.w2, s.w2t, s.w3, s.b1, s.b2, s.b3);
    if (tid == 0) {
        mbar_init(&s.bar, 1);
        mbar_init_fence();
    }
    if (warp == 0) {
        tmem_alloc(&s.tmem, kTrainCols);
        tmem_relinquish();
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s.tmem;
    const uint32_t lane = (uint32_t)(warp * 32) << 16;
    const uint32_t sa = smem_u32(s.a), sp = smem_u32(s.pm), sq = smem_u32(s.qm);
    const uint32_t w1 = smem_u32(s.w1), w2 = smem_u32(s.w2), w2t = smem_u32(s.w2t);
    constexpr uint32_t idesc64 = idesc_bf16(kRows, kHid);
    constexpr uint32_t idesc128 = idesc_bf16(kRows, 128);
    const long long ntiles = (M + kRows - 1) / kRows;
    const int ku = tid & 63, half = tid >> 6;
    float acc3[3] = {0.f, 0.f, 0.f}, accb3 = 0.f, lsum = 0.f;
    uint32_t phase = 0;
    bool ok = true, first = true;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long m = tile * kRows + tid;
        const bool active = m < M;
        // features: row tid of A (slots 50..63 zero) and column tid of Q rows
        // 64.. (slot 50 = 1, the bias input)
        {
            uint4 q[8];
            if (active) {
                const uint4* src = reinterpret_cast<const uint4*>(feat + m * 64);
#pragma unroll
                for (int c = 0; c < 8; ++c) q[c] = src[c];
                q[6] = make_uint4(q[6].x, 0u, 0u, 0u);
                q[7] = make_uint4(0u, 0u, 0u, 0u);
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) q[c] = make_uint4(0u, 0u, 0u, 0u);
            }
            store_row(s.a, tid, q);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const uint32_t w[4] = {q[c].x, q[c].y, q[c].z, q[c].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    st_u16(s.qm, kmaj(kHid + 8 * c + 2 * e, tid, kSbo128), w[e]);
                    st_u16(s.qm, kmaj(kHid + 8 * c + 2 * e + 1, tid, kSbo128), w[e] >> 16);
                }
            }
            st_u16(s.qm, kmaj(kHid + kIn, tid, kSbo128), active ? kBf16One : 0u);
        }
        float bs[3] = {0.f, 0.f, 0.f}, tg[3] = {0.f, 0.f, 0.f};
        if (active) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                bs[c] = base[3 * m + c];
                tg[c] = target[3 * m + c];
            }
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
            mma_k64(tmem, sa, w1, idesc64);
            mma_commit(&s.bar);
        }
        ok = __syncthreads_and(mbar_wait(&s.bar, phase, kWaitLimit));
        phase ^= 1u;
        if (!ok) break;
        fence_after_sync();
        // layer 1: mask of z1 > 0; h1 as row tid of A and column tid of Q rows 0..63
        uint32_t mask1[2] = {0u, 0u};
        {
            uint4 q[8];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                float z[16];
                tmem_ld16(tmem + lane + 16 * g, z);
                tmem_wait_ld();
                uint32_t bits[8];
#pragma unroll
                for (int k = 0; k < 16; k += 2) {
                    const int n = 16 * g + k;
                    const float z0 = z[k] + s.b1[n], z1 = z[k + 1] + s.b1[n + 1];
                    if (z0 > 0.f) mask1[n >> 5] |= 1u << (n & 31);
                    if (z1 > 0.f) mask1[(n + 1) >> 5] |= 1u << ((n + 1) & 31);
                    bits[k >> 1] = pack_bf16x2(fmaxf(z0, 0.f), fmaxf(z1, 0.f));
                    st_u16(s.qm, kmaj(n, tid, kSbo128), bits[k >> 1]);
                    st_u16(s.qm, kmaj(n + 1, tid, kSbo128), bits[k >> 1] >> 16);
                }
                q[2 * g] = make_uint4(bits[0], bits[1], bits[2], bits[3]);
                q[2 * g + 1] = make_uint4(bits[4], bits[5], bits[6], bits[7]);
            }
            store_row(s.a, tid, q);
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
            mma_k64(tmem + kHid, sa, w2, idesc64);
            mma_commit(&s.bar);
        }
        ok = __syncthreads_and(mbar_wait(&s.bar, phase, kWaitLimit));
        phase ^= 1u;
        if (!ok) break;
        fence_after_sync();
        // layer 2 and the output: h2, r = W3 h2 + b3, e = base + r - target,
        // d3 = 2 e / (3 M); then d2 = (W3^T d3) [z2 > 0] as row tid of A and
        // column tid of P rows 0..63
        uint32_t mask2[2] = {0u, 0u};
        {
            float r0 = s.b3[0], r1 = s.b3[1], r2 = s.b3[2];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                float z[16];
                tmem_ld16(tmem + lane + kHid + 16 * g, z);
                tmem_wait_ld();
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int n = 16 * g + k;
                    const float zz = z[k] + s.b2[n];
                    if (zz > 0.f) mask2[n >> 5] |= 1u << (n & 31);
                    const float h = bf16_round(fmaxf(zz, 0.f));   // as the output layer reads it
                    s.h2[tid][n] = h;
                    r0 = fmaf(s.w3[n], h, r0);
                    r1 = fmaf(s.w3[kHid + n], h, r1);
                    r2 = fmaf(s.w3[2 * kHid + n], h, r2);
                }
            }
            const float e0 = active ? bs[0] + r0 - tg[0] : 0.f;
            const float e1 = active ? bs[1] + r1 - tg[1] : 0.f;
            const float e2 = active ? bs[2] + r2 - tg[2] : 0.f;
            lsum = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, lsum)));
            const float d0 = e0 * scale, d1 = e1 * scale, d2 = e2 * scale;
            s.d3[tid][0] = d0;
            s.d3[tid][1] = d1;
            s.d3[tid][2] = d2;
            uint4 q[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                uint32_t bits[4];
#pragma unroll
                for (int k = 0; k < 8; k += 2) {
                    const int n = 8 * g + k;
                    float v0 = fmaf(s.w3[n], d0, fmaf(s.w3[kHid + n], d1, s.w3[2 * kHid + n] * d2));
                    float v1 = fmaf(s.w3[n + 1], d0, fmaf(s.w3[kHid + n + 1], d1, s.w3[2 * kHid + n + 1] * d2));
                    v0 = (mask2[n >> 5] >> (n & 31)) & 1u ? v0 : 0.f;
                    v1 = (mask2[(n + 1) >> 5] >> ((n + 1) & 31)) & 1u ? v1 : 0.f;
                    bits[k >> 1] = pack_bf16x2(v0, v1);
                    st_u16(s.pm, kmaj(n, tid, kSbo128), bits[k >> 1]);
                    st_u16(s.pm, kmaj(n + 1, tid, kSbo128), bits[k >> 1] >> 16);
                }
                q[g] = make_uint4(bits[0], bits[1], bits[2], bits[3]);
            }
            store_row(s.a, tid, q);
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
            mma_k64(tmem, sa, w2t, idesc64);     // D3[p][i] = sum_o d2[p][o] W2[o][i]
            mma_commit(&s.bar);
        }
        // while it runs: dW3 += d3^T h2, db3 += sum d3 (FP32, in registers)
#pragma unroll 4
        for (int r = 64 * half; r < 64 * half + 64; ++r) {
            const float h = s.h2[r][ku];
            acc3[0] = fmaf(s.d3[r][0], h, acc3[0]);
            acc3[1] = fmaf(s.d3[r][1], h, acc3[1]);
            acc3[2] = fmaf(s.d3[r][2], h, acc3[2]);
        }
        if (tid < kOut)
            for (int r = 0; r < kRows; ++r) accb3 += s.d3[r][tid];
        ok = __syncthreads_and(mbar_wait(&s.bar, phase, kWaitLimit));
        phase ^= 1u;
        if (!ok) break;
        fence_after_sync();
        // d1 = D3 [z1 > 0] as column tid of P rows 64..127
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            float z[16];
            tmem_ld16(tmem + lane + 16 * g, z);
            tmem_wait_ld();
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                const int n = 16 * g + k;
                const float v0 = (mask1[n >> 5] >> (n & 31)) & 1u ? z[k] : 0.f;
                const float v1 = (mask1[(n + 1) >> 5] >> ((n + 1) & 31)) & 1u ? z[k + 1] : 0.f;
                const uint32_t b = pack_bf16x2(v0, v1);
                st_u16(s.pm, kmaj(kHid + n, tid, kSbo128), b);
                st_u16(s.pm, kmaj(kHid + n + 1, tid, kSbo128), b >> 16);
            }
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < kRows / 16; ++kk)
                mma_bf16(tmem + 2 * kHid, smem_desc(sp + kk * 2 * kLbo, kLbo, kSbo128),
                         smem_desc(sq + kk * 2 * kLbo, kLbo, kSbo128), idesc128, !(first && kk == 0));
            mma_commit(&s.bar);
        }
        ok = __syncthreads_and(mbar_wait(&s.bar, phase, kWaitLimit));
        phase ^= 1u;
        if (!ok) break;
        first = false;
        fence_before_sync();
    }
    if (ok && !first) {
        fence_after_sync();
        // weight gradients of the hidden layers from tensor memory: lane tid is
        // unit tid of [d2 ; d1]; columns 0..63 pair with h1, 64..113 with the
        // features, 114 with the constant 1
#pragma unroll 1
        for (int g = 0; g < 8; ++g) {
            float z[16];
            tmem_ld16(tmem + lane + 2 * kHid + 16 * g, z);
            tmem_wait_ld();
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int n = 16 * g + k;
                if (tid < kHid) {
                    if (n < kHid) atomicAdd(grads + oW2 + tid * kHid + n, z[k]);
                    else if (n == kHid + kIn) atomicAdd(grads + oB2 + tid, z[k]);
                } else {
                    const int o = tid - kHid;
                    if (n >= kHid && n < kHid + kIn) atomicAdd(grads + oW1 + o * kIn + (n - kHid), z[k]);
                    else if (n == kHid + kIn) atomicAdd(grads + oB1 + o, z[k]);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) atomicAdd(grads + oW3 + c * kHid + ku, acc3[c]);
        if (tid < kOut) atomicAdd(grads + oB3 + tid, accb3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if ((tid & 31) == 0) s.red[warp] = lsum;
        __syncthreads();
        if (tid == 0) atomicAdd(loss, (s.red[0] + s.red[1] + s.red[2] + s.red[3]) * inv);
    }
    if (!ok && tid == 0) atomicExch(err, kDevTimeout);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0) tmem_dealloc(tmem, kTrainCols);
}

__global__ void k_mlp_adam(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, int n, float lr, float beta1, float beta2, float eps, float c1,
                           float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace

// CTAs of a tensor-memory kernel resident per SM: the limits of its registers,
// shared memory (with the largest carveout), threads and blocks per SM, and of
// the 512 tensor-memory columns.  (The runtime's occupancy calculator reports
// one CTA per SM for any kernel that allocates tensor memory.)
template <typename Kernel>
cudaError_t resident_ctas(Kernel k, int threads, size_t smem, uint32_t tmem_cols, int& per_sm)
{
    int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0, threads_sm = 0, blocks_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&blocks_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    // shared memory is allocated in 128-byte units; registers per warp in units
    // of 8 per thread, and a warp's registers come from one of the 4 sub-partitions
    const size_t per_cta_smem = (smem + fa.sharedSizeBytes + (size_t)reserved + 127) / 128 * 128;
    const int warps = (threads + 31) / 32;
    const int regs_warp = (fa.numRegs + 7) / 8 * 8 * 32;
    const int warps_by_regs = regs_warp > 0 ? 4 * ((regs_sm / 4) / regs_warp) : 64;
    int n = (int)std::min<size_t>((size_t)smem_sm / per_cta_smem, 64);
    n = std::min(n, warps_by_regs / warps);
    n = std::min(n, threads_sm / (warps * 32));
    n = std::min(n, blocks_sm);
    n = std::min(n, (int)(512 / tmem_cols));
    per_sm = std::max(1, n);
    return cudaSuccess;
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_mlp_upscale(cudaStream_t s, const float* C, const float* G, int W, int H, int W2, int H2,
                               const float* params, float* out, int* err)
{
    // footprint bound of a 32 x 4 tile: ceil(31 W / W2) + 2 columns, ceil(3 H / H2) + 2 rows
    const int fpw = std::min(kFootW, (int)((31ll * W + W2 - 1) / W2) + 2);
    const int fph = std::min(kFootH, (int)((3ll * H + H2 - 1) / H2) + 2);
    const size_t smem = sizeof(InferSmem) + 3 * sizeof(float4) * (size_t)fpw * fph;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_upscale, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long ntiles = (long long)((W2 + kTileW - 1) / kTileW) * ((H2 + kTileH - 1) / kTileH);
    if (ntiles == 0) return cudaSuccess;
    // persistent: as many CTAs as fit on an SM (six at 4x with 37 KB of shared
    // memory each, five at 2x and below); the largest shared-memory carveout
    // makes that many resident
    e = cudaFuncSetAttribute(k_mlp_upscale, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = resident_ctas(k_mlp_upscale, kThreads, smem, kInferCols, per_sm);
    if (e != cudaSuccess) return e;
    const long long grid = std::min<long long>(ntiles, (long long)per_sm * sm_count());
    k_mlp_upscale<<<(unsigned)grid, kThreads, smem, s>>>(C, G, W, H, W2, H2, fpw, params, out, err);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_mlp_samples(cudaStream_t s, const float* C, const float* G, int W, int H, int W2, int H2,
                               const int* pixels, long long M, const float* target_img, uint16_t* feat, float* base,
                               float* target, int* err)
{
    if (M == 0) return cudaSuccess;
    const long long blocks = (M + 127) / 128;
    k_mlp_samples<<<(unsigned)blocks, 128, 0, s>>>(C, G, W, H, W2, H2, pixels, M, target_img, feat, base, target,
                                                  err);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(cudaStream_t s, const float* params, const uint16_t* feat, const float* base,
                            const float* target, long long M, float* grads, float* loss, int* err)
{
    cudaError_t e = cudaMemsetAsync(grads, 0, sizeof(float) * kParams, s);
    if (e == cudaSuccess && loss) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    if (M == 0) return cudaSuccess;
    const size_t smem = sizeof(TrainSmem);
    e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long ntiles = (M + kRows - 1) / kRows;
    // one CTA per SM (~140 KB shared memory, 256 tensor-memory columns)
    const long long grid = std::min<long long>(ntiles, sm_count());
    const double inv = 1.0 / (3.0 * (double)M);
    k_mlp_grad<<<(unsigned)grid, kThreads, smem, s>>>(params, feat, base, target, M, (float)(2.0 * inv), (float)inv,
                                                      grads, loss, err);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(cudaStream_t s, float* params, float* m, float* v, const float* g, int step, float lr,
                            float beta1, float beta2, float eps)
{
    const double c1 = 1.0 / (1.0 - std::pow((double)beta1, step));
    const double c2 = 1.0 / (1.0 - std::pow((double)beta2, step));
    k_mlp_adam<<<(kParams + 255) / 256, 256, 0, s>>>(params, m, v, g, kParams, lr, beta1, beta2, eps, (float)c1,
                                                     (float)c2);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gs
