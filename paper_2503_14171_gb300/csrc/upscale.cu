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
// half-cells, where the edge patch is extrapolated).
//
// Launch: one block per 32 x 8 tile of output pixels.  The block first stages
// the low-res footprint of its tile (all 12 planes) in shared memory with
// coalesced loads, then each thread writes its outputs; every low-res value is
// read from HBM once per block.  HBM-bound: 48 B per low-res pixel in,
// 12 B per output pixel out.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kOutW = 32;
constexpr int kOutH = 8;
constexpr int kMaxFactor = 16;
// footprint of a 32 x 8 output tile is at most ceil(32/s)+2 x ceil(8/s)+2 low-res pixels
constexpr int kFootW = kOutW + 2;
constexpr int kFootH = kOutH + 2;

__device__ __forceinline__ void hermite(float t, float& h0, float& h1, float& g0, float& g1)
{
    const float t2 = t * t;
    const float omt = 1.f - t;
    h0 = (1.f + 2.f * t) * omt * omt;
    h1 = t2 * (3.f - 2.f * t);
    g0 = t * omt * omt;
    g1 = t2 * (t - 1.f);
}

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

__global__ void __launch_bounds__(kOutW * kOutH) k_upscale(const float* __restrict__ Cimg,
                                                           const float* __restrict__ G, int W, int H, int s,
                                                           float* __restrict__ out)
{
    __shared__ float sm[12][kFootH][kFootW];
    const int W2 = W * s, H2 = H * s;
    const int X0 = blockIdx.x * kOutW, Y0 = blockIdx.y * kOutH;
    int i0, j0, itmp, jtmp;
    float ttmp;
    cell_of(X0, s, W, i0, ttmp);
    cell_of(Y0, s, H, j0, ttmp);
    cell_of(min(X0 + kOutW - 1, W2 - 1), s, W, itmp, ttmp);
    cell_of(min(Y0 + kOutH - 1, H2 - 1), s, H, jtmp, ttmp);
    const int fw = itmp + 2 - i0, fh = jtmp + 2 - j0;   // footprint size (<= kFootW x kFootH)
    const size_t plane = (size_t)W * H;
    const int nf = fw * fh;
    for (int q = threadIdx.x; q < 12 * nf; q += blockDim.x) {
        const int pl = q / nf, r = q - pl * nf;
        const int fy = r / fw, fx = r - fy * fw;
        const float* src = pl < 3 ? Cimg + pl * plane : G + (pl - 3) * plane;
        sm[pl][fy][fx] = src[(size_t)(j0 + fy) * W + (i0 + fx)];
    }
    __syncthreads();

    const int X = X0 + (threadIdx.x % kOutW), Y = Y0 + (threadIdx.x / kOutW);
    if (X >= W2 || Y >= H2) return;
    int i, j;
    float t, u;
    cell_of(X, s, W, i, t);
    cell_of(Y, s, H, j, u);
    const int li = i - i0, lj = j - j0;
    float hx0, hx1, gx0, gx1, hy0, hy1, gy0, gy1;
    hermite(t, hx0, hx1, gx0, gx1);
    hermite(u, hy0, hy1, gy0, gy1);
    const float w00 = hx0 * hy0, w10 = hx1 * hy0, w01 = hx0 * hy1, w11 = hx1 * hy1;
    const float x00 = gx0 * hy0, x10 = gx1 * hy0, x01 = gx0 * hy1, x11 = gx1 * hy1;
    const float y00 = hx0 * gy0, y10 = hx1 * gy0, y01 = hx0 * gy1, y11 = hx1 * gy1;
    const float z00 = gx0 * gy0, z10 = gx1 * gy0, z01 = gx0 * gy1, z11 = gx1 * gy1;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const int pv = ch, px = 3 + ch, py = 6 + ch, pxy = 9 + ch;
        float acc = w00 * sm[pv][lj][li];
        acc = fmaf(w10, sm[pv][lj][li + 1], acc);
        acc = fmaf(w01, sm[pv][lj + 1][li], acc);
        acc = fmaf(w11, sm[pv][lj + 1][li + 1], acc);
        acc = fmaf(x00, sm[px][lj][li], acc);
        acc = fmaf(x10, sm[px][lj][li + 1], acc);
        acc = fmaf(x01, sm[px][lj + 1][li], acc);
        acc = fmaf(x11, sm[px][lj + 1][li + 1], acc);
        acc = fmaf(y00, sm[py][lj][li], acc);
        acc = fmaf(y10, sm[py][lj][li + 1], acc);
        acc = fmaf(y01, sm[py][lj + 1][li], acc);
        acc = fmaf(y11, sm[py][lj + 1][li + 1], acc);
        acc = fmaf(z00, sm[pxy][lj][li], acc);
        acc = fmaf(z10, sm[pxy][lj][li + 1], acc);
        acc = fmaf(z01, sm[pxy][lj + 1][li], acc);
        acc = fmaf(z11, sm[pxy][lj + 1][li + 1], acc);
        out[(size_t)ch * W2 * H2 + (size_t)Y * W2 + X] = acc;
    }
}

}  // namespace

cudaError_t launch_upscale(cudaStream_t s, const float* C, const float* grads, int W, int H, int factor, float* out)
{
    if (factor < 1 || factor > kMaxFactor) return cudaErrorInvalidValue;
    const int W2 = W * factor, H2 = H * factor;
    dim3 grid((W2 + kOutW - 1) / kOutW, (H2 + kOutH - 1) / kOutH);
    k_upscale<<<grid, kOutW * kOutH, 0, s>>>(C, grads, W, H, factor, out); note_launch();
    return cudaGetLastError();
}

}  // namespace gs
