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

}  // namespace gs
