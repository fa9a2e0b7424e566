// Definitions shared by the blend (blend.cu) and its adjoint (blend_bwd.cu):
// both evaluate every (pixel, Gaussian) pair with the same expressions, so the
// adjoint re-takes each of the forward's decisions on the same FP32 values.
#pragma once

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = kTilePixels;    // one pixel per thread
constexpr int kWarps = kThreads / 32;
constexpr int kCand = kThreads;          // super-tile list candidates examined per round
constexpr float kLn2 = 0.69314718055994531f;

__device__ __forceinline__ bool covers(ushort4 r, int tx, int ty)
{
    return (int)r.x <= tx && tx <= (int)r.z && (int)r.y <= ty && ty <= (int)r.w;
}

// A (super-tile, Gaussian) pair is mask << 48 | super-tile << 32 | id, with
// bit ks ly + lx of the mask set when the Gaussian's tile rect covers tile
// (lx, ly) of the super-tile's ks x ks tiles (ks = 1, 2 or 4).  pair_hit reads pair k (one
// coalesced 8-byte load) and tests the calling tile's bit.
__device__ __forceinline__ bool pair_hit(const uint32_t* __restrict__ pair_words, size_t k, uint32_t n, int bit,
                                         uint32_t& id)
{
    const uint2 w = reinterpret_cast<const uint2*>(pair_words)[k];
    id = w.x;
    return id < n && ((w.y >> (16 + bit)) & 1u);
}

// 2^x by the hardware's base-2 exponential (PTX ex2.approx.ftz.f32: about
// 2^-22 relative error; results below 2^-126 flush to zero -- in 3DGS mode no
// blended pair comes near that (alpha >= 1/255), in exact mode such a pair
// adds less than 1e-38).  The blend and its adjoint both take it, so the
// adjoint re-takes the forward's decisions on the same values.
__device__ __forceinline__ float pow2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed FP32 pairs (PTX fma/mul/sub .rn.f32x2): two lanes per instruction,
// each rounded exactly as the scalar fmaf / __fmul_rn / __fsub_rn, so a packed
// step gives the bits of the two scalar steps it replaces (the forward blend
// keeps the quantities it updates together in adjacent pairs; its images are
// bit-identical to the scalar form's).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// Exponent of a (pixel, Gaussian) pair in base 2: r1 = (A2, B2, C2, threshold)
// with g2 = A2 dx^2 + B2 dx dy + C2 dy^2 = g log2(e).
__device__ __forceinline__ float exponent2(const float4& r1, float dx, float dy)
{
    return fmaf(dx, fmaf(r1.x, dx, r1.y * dy), r1.z * dy * dy);
}

}  // namespace
}  // namespace gs
