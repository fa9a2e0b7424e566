// The spline's sample-point map and Hermite basis (Sec. 5 "Spline
// Interpolation"), shared by the upscale kernels and the learned residual.
//
// Output pixel X of a W2-wide output samples the low-res point
// x = (X + 0.5) W / W2 - 0.5 = ((2X + 1) W - W2) / (2 W2); its cell is
// i = clamp(floor(x), 0, W - 2) (an exact integer division) and t = x - i (one
// rounding; outside [0, 1] only in the border half-cells).
#pragma once

namespace gs {

// floor(num / den) for den > 0
__device__ __forceinline__ long long floor_div(long long num, long long den)
{
    return num >= 0 ? num / den : -((den - 1 - num) / den);
}

// cell and local coordinate of output pixel X (clamped to [0, W - 2]); a
// negative numerator clamps to cell 0, and a quotient of 31-bit operands takes
// the 32-bit division (the same exact floor)
__device__ __forceinline__ void cell_of(int X, int W, int W2, int& i, float& t)
{
    const long long num = (2ll * X + 1) * W - W2, den = 2ll * W2;
    long long q;
    if (num < 0)
        q = 0;
    else if (num <= 0x7FFFFFFFll && den <= 0x7FFFFFFFll)
        q = (long long)((unsigned)num / (unsigned)den);
    else
        q = floor_div(num, den);
    q = q > W - 2 ? W - 2 : q;
    i = (int)q;
    t = (float)(num - den * q) / (float)den;
}

// cubic Hermite basis (h00, h01, h10, h11) at t: weights of f(0), f(1), f'(0), f'(1)
__device__ __forceinline__ float4 hermite(float t)
{
    const float t2 = t * t;
    const float omt = 1.f - t;
    return make_float4((1.f + 2.f * t) * omt * omt, t2 * (3.f - 2.f * t), t * omt * omt, t2 * (t - 1.f));
}

// Adjoint of the upscale at one low-res pixel.  The output is linear in the
// low-res values, so dL/d(value of low-res pixel (i, j)) = sum over the output
// pixels whose cell has (i, j) as a corner of (that corner's weight) * dL/dout.
// Output pixel X has (i, .) as its left corner when its cell is i (weights h00,
// h10 of t) and as its right corner when its cell is i - 1 (weights h01, h11).
// Cells are monotone in X, so the pixels of cell c are [first(c), first(c + 1))
// with first(c) the smallest X whose clamped cell is >= c: 0 for c <= 0, W2 for
// c > W - 2, else ceil((2 W2 c + W2 - W) / (2 W)).
__device__ __forceinline__ int first_of_cell(int c, int W, int W2)
{
    if (c <= 0) return 0;
    if (c > W - 2) return W2;
    const long long num = 2ll * W2 * c + W2 - W, den = 2ll * W;   // num > 0 for W2 >= W
    return (int)((num + den - 1) / den);
}

// acc[ch][q] = dL/d(quantity q of channel ch at (i, j)), q: value (weights
// H H), d/dx (G H), d/dy (H G), d2/dxdy (G G); dout [3][H2][W2]
__device__ __forceinline__ void upscale_adjoint_at(const float* __restrict__ dout, int W, int H, int W2, int H2,
                                                   int i, int j, float (&acc)[3][4])
{
    const size_t oplane = (size_t)W2 * H2;
    const float inv_x = 1.f / (float)(2 * W2), inv_y = 1.f / (float)(2 * H2);
    const int xa = first_of_cell(i - 1, W, W2), xm = first_of_cell(i, W, W2), xb = first_of_cell(i + 1, W, W2);
    const int ya = first_of_cell(j - 1, H, H2), ym = first_of_cell(j, H, H2), yb = first_of_cell(j + 1, H, H2);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[ch][q] = 0.f;
    // numerators of t = ((2X + 1) W - W2 - 2 W2 c) / (2 W2), stepped by 2W per
    // output pixel (|num| <= 3 W2 inside the footprint: 32-bit)
    const int nx0 = (int)((2ll * xa + 1) * W - W2 - 2ll * W2 * (i - 1));
    int ny = (int)((2ll * ya + 1) * H - H2 - 2ll * H2 * (j - 1));
    for (int Y = ya; Y < yb; ++Y, ny += 2 * H) {
        const bool right_y = Y < ym;            // cell j - 1: (., j) is its lower corner
        if (Y == ym) ny -= 2 * H2;              // now in cell j
        const float4 hy = hermite((float)ny * inv_y);
        const float wyH = right_y ? hy.y : hy.x, wyG = right_y ? hy.w : hy.z;
        const float* row = dout + (size_t)Y * W2;
        int nx = nx0;
        for (int X = xa; X < xb; ++X, nx += 2 * W) {
            const bool right_x = X < xm;
            if (X == xm) nx -= 2 * W2;
            const float4 hx = hermite((float)nx * inv_x);
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
}

}  // namespace gs
