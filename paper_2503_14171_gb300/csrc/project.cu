// Projection of 3D Gaussians to screen-space records (Sec. 4: Sigma = R S S^T R^T,
// EWA splatting Sigma' = J W Sigma W^T J^T), view-dependent SH colour, and the
// tile rect of each Gaussian.  One thread per Gaussian; HBM-bound (reads 60 B
// (RGB) to 236 B (SH degree 3) per Gaussian, writes 92 B).
#include <math.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

// Real spherical harmonics in Cartesian form on the unit sphere (d = x, y, z),
// index k = l^2 + l + m, Condon-Shortley phase, normalisation
// K_l^m = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0):
//   l=0: 1/(2 sqrt(pi))
//   l=1: sqrt(3/(4 pi)) * (-y, z, -x)
//   l=2: (1/2)sqrt(15/pi) xy, -(1/2)sqrt(15/pi) yz, (1/4)sqrt(5/pi)(3z^2-1),
//        -(1/2)sqrt(15/pi) xz, (1/4)sqrt(15/pi)(x^2-y^2)
//   l=3: -(1/4)sqrt(35/(2pi)) y(3x^2-y^2), (1/2)sqrt(105/pi) xyz,
//        -(1/4)sqrt(21/(2pi)) y(5z^2-1), (1/4)sqrt(7/pi) z(5z^2-3),
//        -(1/4)sqrt(21/(2pi)) x(5z^2-1), (1/4)sqrt(105/pi) z(x^2-y^2),
//        -(1/4)sqrt(35/(2pi)) x(x^2-3y^2)
constexpr float kY00 = 0.28209479177387814f;
constexpr float kY1 = 0.48860251190291992f;
constexpr float kY2a = 1.0925484305920792f;
constexpr float kY2b = 0.31539156525252005f;
constexpr float kY2c = 0.54627421529603959f;
constexpr float kY3a = 0.59004358992664352f;
constexpr float kY3b = 2.8906114426405538f;
constexpr float kY3c = 0.45704579946446572f;
constexpr float kY3d = 0.37317633259011540f;
constexpr float kY3e = 1.4453057213202769f;

__device__ __forceinline__ void sh_colour(const float* __restrict__ sh, int deg, float x, float y, float z,
                                          float out[3])
{
    float Y[16];
    Y[0] = kY00;
    int K = 1;
    if (deg >= 1) {
        Y[1] = -kY1 * y;
        Y[2] = kY1 * z;
        Y[3] = -kY1 * x;
        K = 4;
    }
    if (deg >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;
        Y[5] = -kY2a * y * z;
        Y[6] = kY2b * (3.f * zz - 1.f);
        Y[7] = -kY2a * x * z;
        Y[8] = kY2c * (xx - yy);
        K = 9;
        if (deg >= 3) {
            Y[9] = -kY3a * y * (3.f * xx - yy);
            Y[10] = kY3b * x * y * z;
            Y[11] = -kY3c * y * (5.f * zz - 1.f);
            Y[12] = kY3d * z * (5.f * zz - 3.f);
            Y[13] = -kY3c * x * (5.f * zz - 1.f);
            Y[14] = kY3e * z * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.f * yy);
            K = 16;
        }
    }
    float r = 0.f, g = 0.f, b = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (k < K) {
            r = fmaf(sh[3 * k + 0], Y[k], r);
            g = fmaf(sh[3 * k + 1], Y[k], g);
            b = fmaf(sh[3 * k + 2], Y[k], b);
        }
    }
    out[0] = fmaxf(0.f, r + 0.5f);
    out[1] = fmaxf(0.f, g + 0.5f);
    out[2] = fmaxf(0.f, b + 0.5f);
}

// 3D covariance Sigma = M M^T with M = R diag(s), R from the unit quaternion:
// S = (S00, S01, S02, S11, S12, S22); ok = false for a zero quaternion.
__device__ __forceinline__ void cov3d(const float* __restrict__ quats, const float* __restrict__ log_scales, int ii,
                                      float S[6], bool& ok)
{
    float qw = quats[4 * ii], qx = quats[4 * ii + 1], qy = quats[4 * ii + 2], qz = quats[4 * ii + 3];
    const float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
    ok = qn2 > 0.f;
    const float qinv = rsqrtf(qn2);
    qw *= qinv; qx *= qinv; qy *= qinv; qz *= qinv;
    const float s0 = expf(log_scales[3 * ii]), s1 = expf(log_scales[3 * ii + 1]), s2 = expf(log_scales[3 * ii + 2]);
    const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qw * qz), R02 = 2.f * (qx * qz + qw * qy);
    const float R10 = 2.f * (qx * qy + qw * qz), R11 = 1.f - 2.f * (qx * qx + qz * qz), R12 = 2.f * (qy * qz - qw * qx);
    const float R20 = 2.f * (qx * qz - qw * qy), R21 = 2.f * (qy * qz + qw * qx), R22 = 1.f - 2.f * (qx * qx + qy * qy);
    const float M00 = R00 * s0, M01 = R01 * s1, M02 = R02 * s2;
    const float M10 = R10 * s0, M11 = R11 * s1, M12 = R12 * s2;
    const float M20 = R20 * s0, M21 = R21 * s1, M22 = R22 * s2;
    S[0] = M00 * M00 + M01 * M01 + M02 * M02;
    S[1] = M00 * M10 + M01 * M11 + M02 * M12;
    S[2] = M00 * M20 + M01 * M21 + M02 * M22;
    S[3] = M10 * M10 + M11 * M11 + M12 * M12;
    S[4] = M10 * M20 + M11 * M21 + M12 * M22;
    S[5] = M20 * M20 + M21 * M21 + M22 * M22;
}

// One Gaussian in one view: EWA projection, conic, radius, mean and tile rect.
struct ViewProj {
    float pz, m2x, m2y, ca, cb, cc, rad;
    int4 rc;
    uint32_t ntiles, nsup;
    bool vis;
};

__device__ __forceinline__ ViewProj project_view(float mx3, float my3, float mz3, const float S[6], bool ok, float L,
                                                 const CameraParams& cam, int W, int H, int tiles_x, int tiles_y,
                                                 int ks, int mode)
{
    ViewProj o;
    const float S00 = S[0], S01 = S[1], S02 = S[2], S11 = S[3], S12 = S[4], S22 = S[5];
    const float px = fmaf(cam.R[0], mx3, fmaf(cam.R[1], my3, fmaf(cam.R[2], mz3, cam.t[0])));
    const float py = fmaf(cam.R[3], mx3, fmaf(cam.R[4], my3, fmaf(cam.R[5], mz3, cam.t[1])));
    const float pz = fmaf(cam.R[6], mx3, fmaf(cam.R[7], my3, fmaf(cam.R[8], mz3, cam.t[2])));
    bool vis = ok && pz > cam.znear;

    // Jacobian of the perspective map at the frustum-clamped mean, times W
    const float iz = 1.f / pz;
    const float txz = fminf(cam.lim_x, fmaxf(-cam.lim_x, px * iz));
    const float tyz = fminf(cam.lim_y, fmaxf(-cam.lim_y, py * iz));
    const float j00 = cam.fx * iz, j02 = -cam.fx * txz * iz;
    const float j11 = cam.fy * iz, j12 = -cam.fy * tyz * iz;
    // T = J W (2x3)
    const float T00 = j00 * cam.R[0] + j02 * cam.R[6];
    const float T01 = j00 * cam.R[1] + j02 * cam.R[7];
    const float T02 = j00 * cam.R[2] + j02 * cam.R[8];
    const float T10 = j11 * cam.R[3] + j12 * cam.R[6];
    const float T11 = j11 * cam.R[4] + j12 * cam.R[7];
    const float T12 = j11 * cam.R[5] + j12 * cam.R[8];
    // U = T Sigma
    const float U00 = T00 * S00 + T01 * S01 + T02 * S02;
    const float U01 = T00 * S01 + T01 * S11 + T02 * S12;
    const float U02 = T00 * S02 + T01 * S12 + T02 * S22;
    const float U10 = T10 * S00 + T11 * S01 + T12 * S02;
    const float U11 = T10 * S01 + T11 * S11 + T12 * S12;
    const float U12 = T10 * S02 + T11 * S12 + T12 * S22;
    const float c00 = U00 * T00 + U01 * T01 + U02 * T02 + 0.3f;
    const float c01 = U00 * T10 + U01 * T11 + U02 * T12;
    const float c11 = U10 * T10 + U11 * T11 + U12 * T12 + 0.3f;
    const float det = c00 * c11 - c01 * c01;
    vis = vis && det > 0.f;

    const float idet = 1.f / det;
    o.ca = c11 * idet;
    o.cb = -c01 * idet;
    o.cc = c00 * idet;
    const float mid = 0.5f * (c00 + c11);
    const float hd = 0.5f * (c00 - c11);
    const float lam = mid + sqrtf(hd * hd + c01 * c01);   // cancellation-free largest eigenvalue
    const float rad = ceilf(3.f * sqrtf(lam));
    const float m2x = fmaf(cam.fx, px * iz, cam.cx);
    const float m2y = fmaf(cam.fy, py * iz, cam.cy);

    vis = vis && isfinite(m2x) && isfinite(m2y) && isfinite(rad);
    // alpha = sigma e^g >= 1/255 only inside d^T Sigma'^-1 d <= 2L, L = ln(255 sigma)
    int4 rc = make_int4(0, 0, -1, -1);
    uint32_t ntiles = 0;
    if (vis) {
        if (mode == GS_MODE_EXACT) {
            rc = make_int4(0, 0, tiles_x - 1, tiles_y - 1);
            ntiles = (uint32_t)(tiles_x * tiles_y);
        } else if (L > 0.f) {
            // tiles holding a pixel centre (i, j) with |i - mx| <= hx, |j - my| <= hy:
            // the 3-sigma square cut to the bounding box of the alpha >= 1/255 ellipse
            const float hx = fminf(rad, sqrtf(2.f * L * c00));
            const float hy = fminf(rad, sqrtf(2.f * L * c11));
            const float lox = ceilf(m2x - hx), hix = floorf(m2x + hx);
            const float loy = ceilf(m2y - hy), hiy = floorf(m2y + hy);
            if (!(hix < 0.f || lox > (float)(W - 1) || hiy < 0.f || loy > (float)(H - 1) || lox > hix ||
                  loy > hiy)) {
                const int x0 = lox < 0.f ? 0 : (int)lox;
                const int y0 = loy < 0.f ? 0 : (int)loy;
                const int x1 = hix > (float)(W - 1) ? W - 1 : (int)hix;
                const int y1 = hiy > (float)(H - 1) ? H - 1 : (int)hiy;
                rc = make_int4(x0 / kTile, y0 / kTile, x1 / kTile, y1 / kTile);
                ntiles = (uint32_t)((rc.z - rc.x + 1) * (rc.w - rc.y + 1));
            }
        }
    }
    o.pz = pz;
    o.m2x = m2x;
    o.m2y = m2y;
    o.rad = rad;
    o.rc = rc;
    o.ntiles = ntiles;
    const int ksh = __ffs(ks) - 1;   // ks = 1, 2 or 4
    o.nsup = ntiles ? (uint32_t)(((rc.z >> ksh) - (rc.x >> ksh) + 1) * ((rc.w >> ksh) - (rc.y >> ksh) + 1)) : 0u;
    o.vis = vis;
    return o;
}

// The three records of a visible Gaussian in one view (colour from the SH
// coefficients shv, or rgb).  The blend evaluates the exponent in base 2:
// g2 = g log2(e) with g = -1/2 (a dx^2 + 2 b dx dy + c dy^2).  Reject
// threshold: g < ln(1/(255 sigma)) - 1e-4 guarantees sigma e^g < 1/255 in FP32,
// so the blend may skip the exponential there.
template <int DEG>
__device__ __forceinline__ void view_records(const ViewProj& v, float mx3, float my3, float mz3, const float* shv,
                                             const float* rgb, float op, float L, const CameraParams& cam, int mode,
                                             float4& r0, float4& r1, float4& r2)
{
    float col[3];
    if (DEG >= 0) {
        float dx = mx3 - cam.campos[0], dy = my3 - cam.campos[1], dz = mz3 - cam.campos[2];
        const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= dn; dy *= dn; dz *= dn;
        sh_colour(shv, DEG, dx, dy, dz, col);
    } else {
        col[0] = rgb[0];
        col[1] = rgb[1];
        col[2] = rgb[2];
    }
    constexpr float kLog2e = 1.4426950408889634f;
    const float thr = (mode == GS_MODE_EXACT) ? -INFINITY : (-L - 1e-4f) * kLog2e;
    r0 = make_float4(v.m2x, v.m2y, -v.ca, -v.cc);
    r1 = make_float4(-0.5f * kLog2e * v.ca, -kLog2e * v.cb, -0.5f * kLog2e * v.cc, thr);
    r2 = make_float4(col[0], col[1], col[2], op);
}

constexpr int kProjThreads = 128;

// Copy the SH coefficients of a warp's cnt Gaussians (contiguous, KF floats
// each) into s[gi][k].  From a 16-byte aligned source every lane first issues
// all of its 16-byte loads, then scatters them into the padded rows; otherwise
// (or for the last few floats) scalar coalesced loads.
// The reverse: write s[gi][k] of a warp's cnt Gaussians to dst (contiguous,
// KF floats each), 16-byte stores where dst is 16-byte aligned.
template <int KF, int PITCH>
__device__ __forceinline__ void unstage_sh(float* __restrict__ dst, const float (*s)[PITCH], int cnt, int lane)
{
    const int tot = cnt * KF;
    int done = 0;
    if ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        const int tot4 = tot >> 2;
        float4* dst4 = reinterpret_cast<float4*>(dst);
        for (int q = lane; q < tot4; q += 32) {
            float e[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int f = 4 * q + c, gi = f / KF;
                e[c] = s[gi][f - gi * KF];
            }
            dst4[q] = make_float4(e[0], e[1], e[2], e[3]);
        }
        done = 4 * tot4;
    }
    for (int f = done + lane; f < tot; f += 32) {
        const int gi = f / KF;
        dst[f] = s[gi][f - gi * KF];
    }
}

template <int KF, int PITCH>
__device__ __forceinline__ void stage_sh(float (*s)[PITCH], const float* __restrict__ src, int cnt, int lane)
{
    const int tot = cnt * KF;
    int done = 0;
    if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
        constexpr int kPer = (32 * KF / 4 + 31) / 32;   // float4 per lane for a full warp
        const int tot4 = tot >> 2;
        const float4* src4 = reinterpret_cast<const float4*>(src);
        float4 v[kPer];
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int q = lane + 32 * r;
            if (q < tot4) v[r] = __ldcs(src4 + q);
        }
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const int q = lane + 32 * r;
            if (q < tot4) {
                const float e[4] = {v[r].x, v[r].y, v[r].z, v[r].w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int f = 4 * q + c, gi = f / KF;
                    s[gi][f - gi * KF] = e[c];
                }
            }
        }
        done = 4 * tot4;
    }
    for (int f = done + lane; f < tot; f += 32) {
        const int gi = f / KF;
        s[gi][f - gi * KF] = src[f];
    }
}

// DEG: SH degree 0..3, or -1 for direct RGB colours.  Each warp first copies the
// SH coefficients of its 32 Gaussians (contiguous, (DEG+1)^2 * 3 floats each)
// into shared memory with coalesced loads; the row pitch is padded to an odd
// number of words so the per-thread reads are free of bank conflicts.
template <int DEG>
__global__ void __launch_bounds__(kProjThreads) k_project(
    int n, const float* __restrict__ means, const float* __restrict__ log_scales,
    const float* __restrict__ quats, const float* __restrict__ op_logits, const float* __restrict__ sh,
    const float* __restrict__ rgb_in, CameraParams cam, int W, int H, int tiles_x, int tiles_y, int ks,
    int mode, Records rec, float* __restrict__ depth_out, int* __restrict__ radius_out,
    ushort4* __restrict__ rect_out, uint32_t* __restrict__ tiles_out, uint32_t* __restrict__ supers_out,
    uint32_t* __restrict__ depth_key, uint32_t* __restrict__ ids, unsigned long long* __restrict__ totals,
    ZeroList zero)
{
    constexpr int KF = DEG >= 0 ? (DEG + 1) * (DEG + 1) * 3 : 1;   // floats per Gaussian
    {
        // clear the later kernels' counters (grid-stride over the whole grid)
        const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
#pragma unroll
        for (int z = 0; z < ZeroList::kMax; ++z)   // unrolled: constant indices keep the list in registers
            if (z < zero.count)
                for (uint32_t w = t; w < zero.words[z]; w += stride) zero.p[z][w] = 0u;
    }
    constexpr int PITCH = KF | 1;
    __shared__ float s_sh[kProjThreads / 32][32][PITCH];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (DEG >= 0) {
        const int wbase = blockIdx.x * blockDim.x + warp * 32;
        const int cnt = min(32, n - wbase);
        if (cnt > 0) stage_sh<KF, PITCH>(s_sh[warp], sh + (size_t)wbase * KF, cnt, lane);
        __syncwarp();
    }
    // every lane runs to the warp reduction below; the tail of the last warp
    // reads a valid Gaussian and writes nothing
    const bool inrange = i < n;
    const int ii = inrange ? i : n - 1;
    const float mx3 = means[3 * ii], my3 = means[3 * ii + 1], mz3 = means[3 * ii + 2];
    float S[6];
    bool qok;
    cov3d(quats, log_scales, ii, S, qok);
    const float op = 1.f / (1.f + expf(-op_logits[ii]));
    const float L = logf(255.f * op);
    const ViewProj v = project_view(mx3, my3, mz3, S, qok && inrange, L, cam, W, H, tiles_x, tiles_y, ks, mode);
    // frame totals of (super-tile, Gaussian) and (tile, Gaussian) pairs: they do
    // not depend on the depth order, so they are summed here -- per block, then
    // into one of kTotalSlots slot pairs (spreading the atomics), summed on the host
    __shared__ unsigned long long s_tot[2][kProjThreads / 32];
    unsigned long long wsum = v.nsup, wt = v.ntiles;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
        wt += __shfl_xor_sync(0xffffffffu, wt, o);
    }
    if (lane == 0) {
        s_tot[0][warp] = wsum;
        s_tot[1][warp] = wt;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        unsigned long long b = 0;
#pragma unroll
        for (int w = 0; w < kProjThreads / 32; ++w) b += s_tot[threadIdx.x][w];
        if (b) atomicAdd(&totals[2 * (blockIdx.x % kTotalSlots) + threadIdx.x], b);
    }
    if (!inrange) return;
    const int4 rc = v.rc;
    ids[i] = (uint32_t)i;
    tiles_out[i] = v.ntiles;
    supers_out[i] = v.nsup;
    rect_out[i] = v.ntiles ? make_ushort4((unsigned short)rc.x, (unsigned short)rc.y, (unsigned short)rc.z,
                                          (unsigned short)rc.w)
                           : make_ushort4(1, 1, 0, 0);
    radius_out[i] = v.vis ? (int)v.rad : 0;
    depth_out[i] = v.vis ? v.pz : 0.f;
    depth_key[i] = v.ntiles > 0 ? __float_as_uint(v.pz) : 0xFFFFFFFFu;
    if (!v.vis) {
        rec.r0[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        rec.r1[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        rec.r2[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    float4 r0, r1, r2;
    view_records<DEG>(v, mx3, my3, mz3, &s_sh[warp][lane][0], rgb_in + 3 * (DEG >= 0 ? 0 : i), op, L, cam, mode,
                      r0, r1, r2);
    rec.r0[i] = r0;
    rec.r1[i] = r1;
    rec.r2[i] = r2;
}

// Several views of one Gaussian set in one launch (a batch of cameras, e.g.
// stereo pairs): each thread reads its Gaussian once -- mean, scales,
// quaternion, opacity and the SH coefficients (staged through shared memory
// as in k_project) -- computes the view-independent 3D covariance and opacity
// once, then runs the per-view projection of k_project for every view (same
// expressions, so a view here equals a single-view k_project bit for bit).
// Per view it writes the records, tile rect, super-tile count and the batched
// depth sort's key and index at entry off + i of the outputs, and the view's
// pair totals into slot set vid.  A batch over several Gaussian sets runs one
// launch per set, each over the views that use it.
template <int DEG>
__global__ void __launch_bounds__(kProjThreads) k_project_views(
    int n, const float* __restrict__ means, const float* __restrict__ log_scales,
    const float* __restrict__ quats, const float* __restrict__ op_logits, const float* __restrict__ sh,
    const float* __restrict__ rgb_in, const ViewDesc* __restrict__ views, int V, int mode, ViewOutputs out)
{
    constexpr int KF = DEG >= 0 ? (DEG + 1) * (DEG + 1) * 3 : 1;
    constexpr int PITCH = KF | 1;
    __shared__ float s_sh[kProjThreads / 32][32][PITCH];
    __shared__ unsigned long long s_tot[2][kProjThreads / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (DEG >= 0) {
        const int wbase = blockIdx.x * blockDim.x + warp * 32;
        const int cnt = min(32, n - wbase);
        if (cnt > 0) stage_sh<KF, PITCH>(s_sh[warp], sh + (size_t)wbase * KF, cnt, lane);
        __syncwarp();
    }
    const bool inrange = i < n;
    const int ii = inrange ? i : n - 1;
    const float mx3 = means[3 * ii], my3 = means[3 * ii + 1], mz3 = means[3 * ii + 2];
    float S[6];
    bool qok;
    cov3d(quats, log_scales, ii, S, qok);
    const float op = 1.f / (1.f + expf(-op_logits[ii]));
    const float L = logf(255.f * op);
    for (int vi = 0; vi < V; ++vi) {
        const ViewDesc d = views[vi];
        const ViewProj v = project_view(mx3, my3, mz3, S, qok && inrange, L, d.cam, d.W, d.H, d.tiles_x, d.tiles_y,
                                        d.ks, mode);
        unsigned long long wsum = v.nsup, wt = v.ntiles;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
            wt += __shfl_xor_sync(0xffffffffu, wt, o);
        }
        if (lane == 0) {
            s_tot[0][warp] = wsum;
            s_tot[1][warp] = wt;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            unsigned long long b = 0;
#pragma unroll
            for (int w = 0; w < kProjThreads / 32; ++w) b += s_tot[threadIdx.x][w];
            if (b)
                atomicAdd(&out.totals[(size_t)d.vid * 2 * kTotalSlots + 2 * (blockIdx.x % kTotalSlots) + threadIdx.x],
                          b);
        }
        __syncthreads();   // s_tot is reused by the next view
        if (!inrange) continue;
        const size_t o = (size_t)d.off + i;
        const int4 rc = v.rc;
        out.supers[o] = v.nsup;
        out.rect[o] = v.ntiles ? make_ushort4((unsigned short)rc.x, (unsigned short)rc.y, (unsigned short)rc.z,
                                              (unsigned short)rc.w)
                               : make_ushort4(1, 1, 0, 0);
        out.depth_key[o] = v.ntiles > 0 ? __float_as_uint(v.pz) : 0xFFFFFFFFu;
        out.gidx[o] = out.pack_counts ? (uint32_t)o | (min(v.nsup, kPackedCntEsc) << kPackedIdxBits) : (uint32_t)o;
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
        if (v.vis)
            view_records<DEG>(v, mx3, my3, mz3, &s_sh[warp][lane][0], rgb_in + 3 * (DEG >= 0 ? 0 : i), op, L,
                              d.cam, mode, r0, r1, r2);
        out.rec.r0[o] = r0;
        out.rec.r1[o] = r1;
        out.rec.r2[o] = r2;
    }
}

// d Y_k / d(x, y, z) of the Cartesian SH polynomials above (deg <= 3); the
// caller projects the gradient onto the sphere's tangent plane.
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float Y[16], float dYx[16],
                                              float dYy[16], float dYz[16])
{
#pragma unroll
    for (int k = 0; k < 16; ++k) { Y[k] = 0.f; dYx[k] = 0.f; dYy[k] = 0.f; dYz[k] = 0.f; }
    Y[0] = kY00;
    if (deg >= 1) {
        Y[1] = -kY1 * y; dYy[1] = -kY1;
        Y[2] = kY1 * z;  dYz[2] = kY1;
        Y[3] = -kY1 * x; dYx[3] = -kY1;
    }
    if (deg >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kY2a * x * y;            dYx[4] = kY2a * y;  dYy[4] = kY2a * x;
        Y[5] = -kY2a * y * z;           dYy[5] = -kY2a * z; dYz[5] = -kY2a * y;
        Y[6] = kY2b * (3.f * zz - 1.f); dYz[6] = 6.f * kY2b * z;
        Y[7] = -kY2a * x * z;           dYx[7] = -kY2a * z; dYz[7] = -kY2a * x;
        Y[8] = kY2c * (xx - yy);        dYx[8] = 2.f * kY2c * x; dYy[8] = -2.f * kY2c * y;
        if (deg >= 3) {
            Y[9] = -kY3a * y * (3.f * xx - yy);
            dYx[9] = -6.f * kY3a * x * y;
            dYy[9] = -3.f * kY3a * (xx - yy);
            Y[10] = kY3b * x * y * z;
            dYx[10] = kY3b * y * z; dYy[10] = kY3b * x * z; dYz[10] = kY3b * x * y;
            Y[11] = -kY3c * y * (5.f * zz - 1.f);
            dYy[11] = -kY3c * (5.f * zz - 1.f); dYz[11] = -10.f * kY3c * y * z;
            Y[12] = kY3d * z * (5.f * zz - 3.f);
            dYz[12] = kY3d * (15.f * zz - 3.f);
            Y[13] = -kY3c * x * (5.f * zz - 1.f);
            dYx[13] = -kY3c * (5.f * zz - 1.f); dYz[13] = -10.f * kY3c * x * z;
            Y[14] = kY3e * z * (xx - yy);
            dYx[14] = 2.f * kY3e * x * z; dYy[14] = -2.f * kY3e * y * z; dYz[14] = kY3e * (xx - yy);
            Y[15] = -kY3a * x * (xx - 3.f * yy);
            dYx[15] = -3.f * kY3a * (xx - yy); dYy[15] = 6.f * kY3a * x * y;
        }
    }
}

// Adjoint of k_project (reverse mode, hand-derived), one thread per Gaussian.
// Upstream g2d [n][9] = dL/d(mean_x, mean_y, conic a, b, c, opacity, r, g, b).
// The forward quantities are recomputed, then:
//   conic Q = Sigma'^-1:   dL/dSigma' = -Q G Q, G = [[g_a, g_b/2], [g_b/2, g_c]]
//   Sigma' = T Sigma T^T (T = J W):  dL/dSigma = T^T G' T, dL/dT = 2 G' T Sigma
//   J at the clamped x/z, y/z:  through T = J W to the camera-space mean p
//   mean2D = (fx x/z + cx, fy y/z + cy);  p = W mu + t
//   Sigma = M M^T, M = R diag(s):  dL/dM = 2 dL/dSigma M -> R and s = exp(log s)
//   R(q / |q|): the quaternion derivatives of R, projected through the
//   normalisation;  opacity = sigmoid(logit)
//   colour = max(0, sum_k sh_k Y_k(d/|d|) + 1/2), d = mu - campos: dL/dsh and,
//   through the basis' gradient on the sphere, dL/dmu.
template <int DEG>
__global__ void __launch_bounds__(kProjThreads) k_project_bwd(
    int n, const float* __restrict__ means, const float* __restrict__ log_scales,
    const float* __restrict__ quats, const float* __restrict__ op_logits, const float* __restrict__ sh,
    CameraParams cam, const float* __restrict__ g2d, float* __restrict__ g_means, float* __restrict__ g_ls,
    float* __restrict__ g_quats, float* __restrict__ g_ol, float* __restrict__ g_sh, float* __restrict__ g_rgb)
{
    constexpr int KF = DEG >= 0 ? (DEG + 1) * (DEG + 1) * 3 : 1;
    constexpr int PITCH = KF | 1;
    __shared__ float s_sh[kProjThreads / 32][32][PITCH];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wbase = blockIdx.x * blockDim.x + warp * 32;
    const int wcnt = min(32, n - wbase);
    if (DEG >= 0 && wcnt > 0) stage_sh<KF, PITCH>(s_sh[warp], sh + (size_t)wbase * KF, wcnt, lane);
    __syncwarp();
    const bool inrange = i < n;
    float gshv[DEG >= 0 ? KF : 1];
#pragma unroll
    for (int k = 0; k < (DEG >= 0 ? KF : 1); ++k) gshv[k] = 0.f;
    float gm[3] = {0.f, 0.f, 0.f}, gl[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, go = 0.f;
    float gcol[3] = {0.f, 0.f, 0.f};
    if (inrange) {
        float g[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) g[q] = g2d[(size_t)i * 9 + q];
        gcol[0] = g[6]; gcol[1] = g[7]; gcol[2] = g[8];
        const float mx3 = means[3 * i], my3 = means[3 * i + 1], mz3 = means[3 * i + 2];
        const float px = fmaf(cam.R[0], mx3, fmaf(cam.R[1], my3, fmaf(cam.R[2], mz3, cam.t[0])));
        const float py = fmaf(cam.R[3], mx3, fmaf(cam.R[4], my3, fmaf(cam.R[5], mz3, cam.t[1])));
        const float pz = fmaf(cam.R[6], mx3, fmaf(cam.R[7], my3, fmaf(cam.R[8], mz3, cam.t[2])));
        float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
        const float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
        bool vis = pz > cam.znear && qn2 > 0.f;
        const float qinv = rsqrtf(qn2);
        qw *= qinv; qx *= qinv; qy *= qinv; qz *= qinv;
        const float sc[3] = {expf(log_scales[3 * i]), expf(log_scales[3 * i + 1]), expf(log_scales[3 * i + 2])};
        float R[3][3] = {{1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
                         {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
                         {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
        float M[3][3], S[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k) M[r][k] = R[r][k] * sc[k];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) S[r][c] = M[r][0] * M[c][0] + M[r][1] * M[c][1] + M[r][2] * M[c][2];
        const float iz = 1.f / pz;
        const float rx = px * iz, ry = py * iz;
        const bool inx = rx >= -cam.lim_x && rx <= cam.lim_x;
        const bool iny = ry >= -cam.lim_y && ry <= cam.lim_y;
        const float txz = fminf(cam.lim_x, fmaxf(-cam.lim_x, rx));
        const float tyz = fminf(cam.lim_y, fmaxf(-cam.lim_y, ry));
        const float J[2][3] = {{cam.fx * iz, 0.f, -cam.fx * txz * iz}, {0.f, cam.fy * iz, -cam.fy * tyz * iz}};
        float Tm[2][3];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Tm[r][c] = J[r][0] * cam.R[c] + J[r][1] * cam.R[3 + c] + J[r][2] * cam.R[6 + c];
        float TS[2][3];   // T Sigma
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) TS[r][c] = Tm[r][0] * S[0][c] + Tm[r][1] * S[1][c] + Tm[r][2] * S[2][c];
        const float c00 = TS[0][0] * Tm[0][0] + TS[0][1] * Tm[0][1] + TS[0][2] * Tm[0][2] + 0.3f;
        const float c01 = TS[0][0] * Tm[1][0] + TS[0][1] * Tm[1][1] + TS[0][2] * Tm[1][2];
        const float c11 = TS[1][0] * Tm[1][0] + TS[1][1] * Tm[1][1] + TS[1][2] * Tm[1][2] + 0.3f;
        const float det = c00 * c11 - c01 * c01;
        vis = vis && det > 0.f;
        if (vis) {
            const float idet = 1.f / det;
            const float Qa = c11 * idet, Qb = -c01 * idet, Qc = c00 * idet;
            // dL/dSigma' = -Q G Q
            const float G00 = g[2], G01 = 0.5f * g[3], G11 = g[4];
            const float QG00 = Qa * G00 + Qb * G01, QG01 = Qa * G01 + Qb * G11;
            const float QG10 = Qb * G00 + Qc * G01, QG11 = Qb * G01 + Qc * G11;
            const float gS00 = -(QG00 * Qa + QG01 * Qb);
            const float gS01 = -(QG00 * Qb + QG01 * Qc);
            const float gS11 = -(QG10 * Qb + QG11 * Qc);
            const float gS[2][2] = {{gS00, gS01}, {gS01, gS11}};
            // dL/dT = 2 gS T Sigma; dL/dSigma = T^T gS T
            float gT[2][3];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) gT[r][c] = 2.f * (gS[r][0] * TS[0][c] + gS[r][1] * TS[1][c]);
            float gSig[3][3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float t0 = gS[0][0] * Tm[0][c] + gS[0][1] * Tm[1][c];
                    const float t1 = gS[1][0] * Tm[0][c] + gS[1][1] * Tm[1][c];
                    gSig[r][c] = Tm[0][r] * t0 + Tm[1][r] * t1;
                }
            // T = J W: dL/dJ = dL/dT W^T (only the non-zero entries of J)
            float gJ[2][3];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    gJ[r][c] = gT[r][0] * cam.R[3 * c] + gT[r][1] * cam.R[3 * c + 1] + gT[r][2] * cam.R[3 * c + 2];
            // J entries as functions of p (the clamp passes no derivative)
            float gpx = 0.f, gpy = 0.f, gpz = 0.f;
            gpz += gJ[0][0] * (-cam.fx * iz * iz) + gJ[1][1] * (-cam.fy * iz * iz);
            // j02 = -fx txz / z
            gpz += gJ[0][2] * (cam.fx * txz * iz * iz);
            if (inx) { gpx += gJ[0][2] * (-cam.fx * iz * iz); gpz += gJ[0][2] * (cam.fx * px * iz * iz * iz); }
            gpz += gJ[1][2] * (cam.fy * tyz * iz * iz);
            if (iny) { gpy += gJ[1][2] * (-cam.fy * iz * iz); gpz += gJ[1][2] * (cam.fy * py * iz * iz * iz); }
            // mean2D
            gpx += g[0] * cam.fx * iz;
            gpy += g[1] * cam.fy * iz;
            gpz += -(g[0] * cam.fx * px + g[1] * cam.fy * py) * iz * iz;
            // p = W mu + t
#pragma unroll
            for (int c = 0; c < 3; ++c) gm[c] = cam.R[c] * gpx + cam.R[3 + c] * gpy + cam.R[6 + c] * gpz;
            // Sigma = M M^T
            float gR[3][3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float gM = 2.f * (gSig[r][0] * M[0][k] + gSig[r][1] * M[1][k] + gSig[r][2] * M[2][k]);
                    gR[r][k] = gM * sc[k];
                    gl[k] += gM * R[r][k] * sc[k];
                }
            // R(q^) and the normalisation q^ = q / |q|
            const float gw = 2.f * (-qz * gR[0][1] + qy * gR[0][2] + qz * gR[1][0] - qx * gR[1][2] - qy * gR[2][0] +
                                    qx * gR[2][1]);
            const float gx = 2.f * (qy * gR[0][1] + qz * gR[0][2] + qy * gR[1][0] - 2.f * qx * gR[1][1] -
                                    qw * gR[1][2] + qz * gR[2][0] + qw * gR[2][1] - 2.f * qx * gR[2][2]);
            const float gy = 2.f * (-2.f * qy * gR[0][0] + qx * gR[0][1] + qw * gR[0][2] + qx * gR[1][0] +
                                    qz * gR[1][2] - qw * gR[2][0] + qz * gR[2][1] - 2.f * qy * gR[2][2]);
            const float gz = 2.f * (-2.f * qz * gR[0][0] - qw * gR[0][1] + qx * gR[0][2] + qw * gR[1][0] -
                                    2.f * qz * gR[1][1] + qy * gR[1][2] + qx * gR[2][0] + qy * gR[2][1]);
            const float dotq = qw * gw + qx * gx + qy * gy + qz * gz;
            gq[0] = (gw - qw * dotq) * qinv;
            gq[1] = (gx - qx * dotq) * qinv;
            gq[2] = (gy - qy * dotq) * qinv;
            gq[3] = (gz - qz * dotq) * qinv;
            // opacity
            const float op = 1.f / (1.f + expf(-op_logits[i]));
            go = g[5] * op * (1.f - op);
            // colour
            if (DEG >= 0) {
                float dx = mx3 - cam.campos[0], dy = my3 - cam.campos[1], dz = mz3 - cam.campos[2];
                const float dn = rsqrtf(dx * dx + dy * dy + dz * dz);
                dx *= dn; dy *= dn; dz *= dn;
                float Y[16], Yx[16], Yy[16], Yz[16];
                sh_basis_grad(DEG, dx, dy, dz, Y, Yx, Yy, Yz);
                const float* shv = &s_sh[warp][lane][0];
                constexpr int K = DEG >= 0 ? (DEG + 1) * (DEG + 1) : 1;
                float gn[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float acc = 0.f;
#pragma unroll
                    for (int k = 0; k < K; ++k) acc = fmaf(shv[3 * k + ch], Y[k], acc);
                    const float gc = acc + 0.5f > 0.f ? gcol[ch] : 0.f;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        gshv[3 * k + ch] = gc * Y[k];
                        gn[0] = fmaf(gc * shv[3 * k + ch], Yx[k], gn[0]);
                        gn[1] = fmaf(gc * shv[3 * k + ch], Yy[k], gn[1]);
                        gn[2] = fmaf(gc * shv[3 * k + ch], Yz[k], gn[2]);
                    }
                }
                const float dotn = gn[0] * dx + gn[1] * dy + gn[2] * dz;
                gm[0] += (gn[0] - dx * dotn) * dn;
                gm[1] += (gn[1] - dy * dotn) * dn;
                gm[2] += (gn[2] - dz * dotn) * dn;
            }
        } else {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) gcol[ch] = 0.f;
        }
        g_means[3 * i] = gm[0]; g_means[3 * i + 1] = gm[1]; g_means[3 * i + 2] = gm[2];
        g_ls[3 * i] = gl[0]; g_ls[3 * i + 1] = gl[1]; g_ls[3 * i + 2] = gl[2];
        g_quats[4 * i] = gq[0]; g_quats[4 * i + 1] = gq[1]; g_quats[4 * i + 2] = gq[2]; g_quats[4 * i + 3] = gq[3];
        g_ol[i] = go;
        if (DEG < 0 && g_rgb) { g_rgb[3 * i] = gcol[0]; g_rgb[3 * i + 1] = gcol[1]; g_rgb[3 * i + 2] = gcol[2]; }
    }
    if (DEG >= 0 && g_sh) {
        // stage the SH gradients in shared memory and write them coalesced
        __syncwarp();
        if (inrange) {
#pragma unroll
            for (int k = 0; k < (DEG >= 0 ? KF : 1); ++k) s_sh[warp][lane][k] = gshv[k];
        }
        __syncwarp();
        if (wcnt > 0) unstage_sh<KF, PITCH>(g_sh + (size_t)wbase * KF, s_sh[warp], wcnt, lane);
    }
}

__global__ void k_unpack(Records rec, const int* __restrict__ radius, const uint32_t* __restrict__ tiles,
                         const float* __restrict__ depth_in, uint32_t n, float* mean2d, float* conic, float* rgb,
                         float* opacity, float* depth, int32_t* radius_out, int32_t* tiles_out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = rec.r0[i], b = rec.r1[i], c = rec.r2[i];
    if (mean2d) { mean2d[2 * i] = a.x; mean2d[2 * i + 1] = a.y; }
    // r0 = (mu, -a, -c), r1.y = -b log2(e)
    if (conic) { conic[3 * i] = -a.z; conic[3 * i + 1] = -b.y * 0.69314718055994531f; conic[3 * i + 2] = -a.w; }
    if (rgb) { rgb[3 * i] = c.x; rgb[3 * i + 1] = c.y; rgb[3 * i + 2] = c.z; }
    if (opacity) opacity[i] = c.w;
    if (depth) depth[i] = depth_in[i];
    if (radius_out) radius_out[i] = radius[i];
    if (tiles_out) tiles_out[i] = (int32_t)tiles[i];
}

}  // namespace

cudaError_t launch_project(cudaStream_t s, const gs_gaussians& g, const CameraParams& cam, int W, int H,
                           int tiles_x, int tiles_y, int ks, int mode, Records rec, float* depth, int* radius, ushort4* rect,
                           uint32_t* tiles_touched, uint32_t* supers_touched, uint32_t* depth_key, uint32_t* ids,
                           unsigned long long* totals,
                           const ZeroList* zero)
{
    const int n = (int)g.n;
    if (n == 0) {   // no kernel to clear the later kernels' counters
        for (int z = 0; zero && z < zero->count; ++z) {
            cudaError_t e = cudaMemsetAsync(zero->p[z], 0, sizeof(uint32_t) * zero->words[z], s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const int blocks = (n + kProjThreads - 1) / kProjThreads;
    const int deg = g.sh ? g.sh_degree : -1;
    ZeroList zl{};
    if (zero) zl = *zero;
#define GS_PROJECT(D)                                                                                              \
    k_project<D><<<blocks, kProjThreads, 0, s>>>(n, g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, g.rgb, \
                                                 cam, W, H, tiles_x, tiles_y, ks, mode, rec, depth, radius, rect,  \
                                                 tiles_touched, supers_touched, depth_key, ids, totals, zl)
    switch (deg) {
    case 0: GS_PROJECT(0); break;
    case 1: GS_PROJECT(1); break;
    case 2: GS_PROJECT(2); break;
    case 3: GS_PROJECT(3); break;
    default: GS_PROJECT(-1); break;
    }
#undef GS_PROJECT
    note_launch();
    return cudaGetLastError();
}

__global__ void k_set_views(ViewBatch b, int V, ViewDesc* __restrict__ dst)
{
    if ((int)threadIdx.x < V) dst[threadIdx.x] = b.v[threadIdx.x];
}

cudaError_t launch_set_views(cudaStream_t s, const ViewBatch& b, int V, ViewDesc* dst)
{
    if (V < 1 || V > kMaxViews) return cudaErrorInvalidValue;
    k_set_views<<<1, kMaxViews, 0, s>>>(b, V, dst); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_project_views(cudaStream_t s, const gs_gaussians& g, const ViewDesc* views, int V, int mode,
                                 const ViewOutputs& out)
{
    const int n = (int)g.n;
    if (n == 0 || V == 0) return cudaSuccess;
    const int blocks = (n + kProjThreads - 1) / kProjThreads;
    const int deg = g.sh ? g.sh_degree : -1;
#define GS_PROJECT_VIEWS(D)                                                                                        \
    k_project_views<D><<<blocks, kProjThreads, 0, s>>>(n, g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, \
                                                       g.rgb, views, V, mode, out)
    switch (deg) {
    case 0: GS_PROJECT_VIEWS(0); break;
    case 1: GS_PROJECT_VIEWS(1); break;
    case 2: GS_PROJECT_VIEWS(2); break;
    case 3: GS_PROJECT_VIEWS(3); break;
    default: GS_PROJECT_VIEWS(-1); break;
    }
#undef GS_PROJECT_VIEWS
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_project_backward(cudaStream_t s, const gs_gaussians& g, const CameraParams& cam,
                                    const float* grad2d, const gs_gaussian_grads& out)
{
    const int n = (int)g.n;
    if (n == 0) return cudaSuccess;
    const int blocks = (n + kProjThreads - 1) / kProjThreads;
    const int deg = g.sh ? g.sh_degree : -1;
#define GS_PROJECT_BWD(D)                                                                                        \
    k_project_bwd<D><<<blocks, kProjThreads, 0, s>>>(n, g.means, g.log_scales, g.quats, g.opacity_logits, g.sh, \
                                                     cam, grad2d, out.means, out.log_scales, out.quats,          \
                                                     out.opacity_logits, out.sh, out.rgb)
    switch (deg) {
    case 0: GS_PROJECT_BWD(0); break;
    case 1: GS_PROJECT_BWD(1); break;
    case 2: GS_PROJECT_BWD(2); break;
    case 3: GS_PROJECT_BWD(3); break;
    default: GS_PROJECT_BWD(-1); break;
    }
#undef GS_PROJECT_BWD
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_unpack_projected(cudaStream_t s, Records rec, const int* radius, const uint32_t* tiles_touched,
                                    const float* depth_in, uint32_t n, float* mean2d, float* conic, float* rgb,
                                    float* opacity, float* depth, int32_t* radius_out, int32_t* tiles_out)
{
    if (n == 0) return cudaSuccess;
    k_unpack<<<(n + 255) / 256, 256, 0, s>>>(rec, radius, tiles_touched, depth_in, n, mean2d, conic, rgb, opacity,
                                             depth, radius_out, tiles_out); note_launch();
    return cudaGetLastError();
}

}  // namespace gs
