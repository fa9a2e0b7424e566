// Gradient-aware bicubic Hermite upscale (Sec. 5 "Spline Interpolation";
// supplement "Spline Image Interpolation").
//
// The patch of low-res cell (i, j) solves F = C A C^T, so
// p(t, u) = [1 t t^2 t^3] C^-1 F C^-T [1 u u^2 u^3]^T, and the rows of
// [1 t t^2 t^3] C^-1 are the cubic Hermite basis
//   h00 = (1 + 2t)(1 - t)^2, h01 = t^2 (3 - 2t), h10 = t (1 - t)^2, h11 = t^2 (t - 1),
// weighting f(0), f(1), f'(0), f'(1).  Hence
//   p = sum_{a,b in {0,1}} H_a(t) H_b(u) f(a,b) + G_a(t) H_b(u) f_x(a,b)
//                        + H_a(t) G_b(u) f_y(a,b) + G_a(t) G_b(u) f_xy(a,b)
// with H = (h00, h01), G = (h10, h11).
//
// Output pixel X samples the low-res point x = (X + 0.5)/s - 0.5; its cell is
// i = clamp(floor(x), 0, W - 2) and t = x - i (outside [0, 1] only in the border
// half-cells, where the edge patch is extrapolated).  Both come from integer
// arithmetic: x = (2X + 1 - s) / (2s).
//
// Launch: one 256-thread block per 64 x 16 tile of output pixels, 2 x 2 outputs
// per thread.  The block computes the cell index and the four basis weights of
// its 64 columns and 16 rows once (shared tables), stages the low-res footprint
// of the tile -- each pixel's 12 values (C, C_x, C_y, C_xy for three channels)
// packed as three float4 -- in shared memory with coalesced loads, and then
// evaluates each output with 12 vector shared loads and 48 FMAs.  HBM-bound:
// 48 B per low-res pixel in, 12 B per output pixel out.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreadsX = 32, kThreadsY = 8;
constexpr int kOutW = 2 * kThreadsX;    // 64
constexpr int kOutH = 2 * kThreadsY;    // 16
constexpr int kMaxFactor = 16;
// footprint of a 64 x 16 output tile: at most 64 + 1 x 16 + 1 cells (s = 1)
constexpr int kFootW = kOutW + 2;
constexpr int kFootH = kOutH + 2;

__device__ __forceinline__ void cell_of(int X, int s, int W, int& i, float& t)
{
    // x = (X + 0.5)/s - 0.5 = num/den with num = 2X + 1 - s, den = 2s: the cell is
    // an exact integer floor division and t = (num - den i)/den has one rounding
    const int num = 2 * X + 1 - s, den = 2 * s;
    int q = num >= 0 ? num / den : -((den - 1 - num) / den);
    q = q < 0 ? 0 : (q > W - 2 ? W - 2 : q);
    i = q;
    t = (float)(num - den * q) / (float)den;
}

__device__ __forceinline__ float4 hermite(float t)
{
    const float t2 = t * t;
    const float omt = 1.f - t;
    return make_float4((1.f + 2.f * t) * omt * omt, t2 * (3.f - 2.f * t), t * omt * omt, t2 * (t - 1.f));
}

// footprint pitch (in low-res pixels) for factor s: ceil(64 / s) + 2 columns
__host__ __device__ inline int foot_w(int s) { return min(kFootW, (kOutW + s - 1) / s + 2); }
__host__ __device__ inline int foot_h(int s) { return min(kFootH, (kOutH + s - 1) / s + 2); }

__global__ void __launch_bounds__(kThreadsX * kThreadsY) k_upscale(const float* __restrict__ Cimg,
                                                                   const float* __restrict__ G, int W, int H,
                                                                   int s, float* __restrict__ out)
{
    // per low-res pixel of the footprint, its 12 values packed in 3 float4: [fy][fx][3]
    extern __shared__ float4 sm[];
    __shared__ float4 s_wx[kOutW];             // basis weights (h00, h01, h10, h11) per output column
    __shared__ float4 s_wy[kOutH];
    __shared__ int s_cx[kOutW], s_cy[kOutH];   // cell index relative to the footprint origin
    const int W2 = W * s, H2 = H * s;
    const int X0 = blockIdx.x * kOutW, Y0 = blockIdx.y * kOutH;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kThreadsX + tx;

    int i0, j0, itmp, jtmp;
    float ttmp;
    cell_of(X0, s, W, i0, ttmp);
    cell_of(Y0, s, H, j0, ttmp);
    cell_of(min(X0 + kOutW - 1, W2 - 1), s, W, itmp, ttmp);
    cell_of(min(Y0 + kOutH - 1, H2 - 1), s, H, jtmp, ttmp);
    const int fw = itmp + 2 - i0, fh = jtmp + 2 - j0;   // <= foot_w(s) x foot_h(s)
    const int pitch = foot_w(s);

    if (tid < kOutW) {
        int ci;
        float t;
        cell_of(min(X0 + tid, W2 - 1), s, W, ci, t);
        s_cx[tid] = ci - i0;
        s_wx[tid] = hermite(t);
    } else if (tid < kOutW + kOutH) {
        const int r = tid - kOutW;
        int cj;
        float u;
        cell_of(min(Y0 + r, H2 - 1), s, H, cj, u);
        s_cy[r] = cj - j0;
        s_wy[r] = hermite(u);
    }
    // footprint: 12 planes, each a coalesced row-major fh x fw window
    const size_t plane = (size_t)W * H;
    for (int fy = ty; fy < fh; fy += kThreadsY) {
        const size_t row = (size_t)(j0 + fy) * W + i0;
        for (int fx = tx; fx < fw; fx += kThreadsX) {
            const float* c = Cimg + row + fx;
            const float* g = G + row + fx;
            float4* d = sm + 3 * (fy * pitch + fx);
            d[0] = make_float4(c[0], c[plane], c[2 * plane], g[0]);
            d[1] = make_float4(g[plane], g[2 * plane], g[3 * plane], g[4 * plane]);
            d[2] = make_float4(g[5 * plane], g[6 * plane], g[7 * plane], g[8 * plane]);
        }
    }
    __syncthreads();

    const size_t oplane = (size_t)W2 * H2;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int oy = ty + b * kThreadsY;
        const int Y = Y0 + oy;
        if (Y >= H2) continue;
        const float4 wy = s_wy[oy];
        const int lj = s_cy[oy];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int ox = tx + a * kThreadsX;
            const int X = X0 + ox;
            if (X >= W2) continue;
            const float4 wx = s_wx[ox];
            const int li = s_cx[ox];
            // corner (p, q), p, q in {0, 1}: value weight Hx_p Hy_q, d/dx weight Gx_p Hy_q,
            // d/dy weight Hx_p Gy_q, d2/dxdy weight Gx_p Gy_q
            float r = 0.f, gch = 0.f, bch = 0.f;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    const float hx = p ? wx.y : wx.x, gx = p ? wx.w : wx.z;
                    const float hy = q ? wy.y : wy.x, gy = q ? wy.w : wy.z;
                    const float wv = hx * hy, wdx = gx * hy, wdy = hx * gy, wdxy = gx * gy;
                    const float4* v = sm + 3 * ((lj + q) * pitch + li + p);
                    const float4 v0 = v[0];   // C r, C g, C b, Cx r
                    const float4 v1 = v[1];   // Cx g, Cx b, Cy r, Cy g
                    const float4 v2 = v[2];   // Cy b, Cxy r, Cxy g, Cxy b
                    r = fmaf(wv, v0.x, r);
                    gch = fmaf(wv, v0.y, gch);
                    bch = fmaf(wv, v0.z, bch);
                    r = fmaf(wdx, v0.w, r);
                    gch = fmaf(wdx, v1.x, gch);
                    bch = fmaf(wdx, v1.y, bch);
                    r = fmaf(wdy, v1.z, r);
                    gch = fmaf(wdy, v1.w, gch);
                    bch = fmaf(wdy, v2.x, bch);
                    r = fmaf(wdxy, v2.y, r);
                    gch = fmaf(wdxy, v2.z, gch);
                    bch = fmaf(wdxy, v2.w, bch);
                }
            }
            const size_t o = (size_t)Y * W2 + X;
            out[o] = r;
            out[oplane + o] = gch;
            out[2 * oplane + o] = bch;
        }
    }
}

// Adjoint of k_upscale.  The output is linear in the low-res values, so
// dL/d(value of low-res pixel (i, j)) = sum over the output pixels whose cell
// has (i, j) as a corner of (that corner's weight) * dL/dout.  Output pixel X
// has (i, .) as its left corner when its cell is i (weights h00, h10 of t) and
// as its right corner when its cell is i - 1 (weights h01, h11).  Cells are
// monotone in X, so the pixels of cell c are [first(c), first(c + 1)) with
// first(c) the smallest X whose clamped floor((2X + 1 - s) / (2s)) is >= c:
// 0 for c <= 0, W s for c > W - 2, else ceil((2 s c + s - 1) / 2).  One thread
// per low-res pixel gathers exactly its (2s)^2 output pixels with the
// separable weights: no atomics, each low-res value written once.
constexpr int kBwdX = 32, kBwdY = 8;

__device__ __forceinline__ int first_of_cell(int c, int s, int W)
{
    if (c <= 0) return 0;
    if (c > W - 2) return W * s;
    return (2 * s * c + s) / 2;   // ceil((2 s c + s - 1) / 2)
}

__global__ void __launch_bounds__(kBwdX * kBwdY) k_upscale_bwd(const float* __restrict__ dout, int W, int H, int s,
                                                               float* __restrict__ dC, float* __restrict__ dG)
{
    const int i = blockIdx.x * kBwdX + threadIdx.x;
    const int j = blockIdx.y * kBwdY + threadIdx.y;
    if (i >= W || j >= H) return;
    const int W2 = W * s, H2 = H * s;
    const size_t oplane = (size_t)W2 * H2;
    const float inv2s = 1.f / (float)(2 * s);
    const int xa = first_of_cell(i - 1, s, W), xm = first_of_cell(i, s, W), xb = first_of_cell(i + 1, s, W);
    const int ya = first_of_cell(j - 1, s, H), ym = first_of_cell(j, s, H), yb = first_of_cell(j + 1, s, H);
    // acc[ch][q], q: value (H H), d/dx (G H), d/dy (H G), d2/dxdy (G G)
    float acc[3][4];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[ch][q] = 0.f;
    for (int Y = ya; Y < yb; ++Y) {
        const bool right_y = Y < ym;            // cell j - 1: (., j) is its lower corner
        const int cj = right_y ? j - 1 : j;
        const float4 hy = hermite((float)(2 * Y + 1 - s - 2 * s * cj) * inv2s);
        const float wyH = right_y ? hy.y : hy.x, wyG = right_y ? hy.w : hy.z;
        const float* row = dout + (size_t)Y * W2;
        for (int X = xa; X < xb; ++X) {
            const bool right_x = X < xm;
            const int ci = right_x ? i - 1 : i;
            const float4 hx = hermite((float)(2 * X + 1 - s - 2 * s * ci) * inv2s);
            const float wxH = right_x ? hx.y : hx.x, wxG = right_x ? hx.w : hx.z;
            const float wHH = wxH * wyH, wGH = wxG * wyH, wHG = wxH * wyG, wGG = wxG * wyG;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float d = __ldg(row + ch * oplane + X);
                acc[ch][0] = fmaf(wHH, d, acc[ch][0]);
                acc[ch][1] = fmaf(wGH, d, acc[ch][1]);
                acc[ch][2] = fmaf(wHG, d, acc[ch][2]);
                acc[ch][3] = fmaf(wGG, d, acc[ch][3]);
            }
        }
    }
    const size_t plane = (size_t)W * H, pix = (size_t)j * W + i;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        dC[ch * plane + pix] = acc[ch][0];
        dG[(0 * 3 + ch) * plane + pix] = acc[ch][1];
        dG[(1 * 3 + ch) * plane + pix] = acc[ch][2];
        dG[(2 * 3 + ch) * plane + pix] = acc[ch][3];
    }
}

}  // namespace

cudaError_t launch_upscale_backward(cudaStream_t s, const float* dout, int W, int H, int factor, float* dC,
                                    float* dG)
{
    if (factor < 1 || factor > kMaxFactor || W < 2 || H < 2) return cudaErrorInvalidValue;
    dim3 grid((W + kBwdX - 1) / kBwdX, (H + kBwdY - 1) / kBwdY);
    k_upscale_bwd<<<grid, dim3(kBwdX, kBwdY), 0, s>>>(dout, W, H, factor, dC, dG); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_upscale(cudaStream_t s, const float* C, const float* grads, int W, int H, int factor, float* out)
{
    if (factor < 1 || factor > kMaxFactor) return cudaErrorInvalidValue;
    const int W2 = W * factor, H2 = H * factor;
    dim3 grid((W2 + kOutW - 1) / kOutW, (H2 + kOutH - 1) / kOutH);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_upscale, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(3 * sizeof(float4) * kFootW * kFootH));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const size_t smem = 3 * sizeof(float4) * foot_w(factor) * foot_h(factor);
    k_upscale<<<grid, dim3(kThreadsX, kThreadsY), smem, s>>>(C, grads, W, H, factor, out); note_launch();
    return cudaGetLastError();
}

}  // namespace gs
