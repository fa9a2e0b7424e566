// Gradient-aware bicubic Hermite upscale (Sec. 5 "Spline Interpolation";
// supplement "Spline Image Interpolation"), at any output size (integer or
// fractional factors, supplement "Qualitative Results for Different Upsampling
// Rates"), its adjoint, and the classical bicubic comparator.
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
// Output pixel X of a W2-wide output samples the low-res point
// x = (X + 0.5) W / W2 - 0.5 = ((2X + 1) W - W2) / (2 W2); its cell is
// i = clamp(floor(x), 0, W - 2) (an exact integer division) and t = x - i (one
// rounding; outside [0, 1] only in the border half-cells, where the edge patch
// is extrapolated).
//
// Separable evaluation.  Grouping the sum by the patch row b,
//   p = sum_b H_b(u) A_b + G_b(u) B_b,
//   A_b = sum_a H_a(t) f(a,b) + G_a(t) f_x(a,b),  B_b = sum_a H_a(t) f_y(a,b) + G_a(t) f_xy(a,b),
// where A_b and B_b depend only on the output column (through i and t) and the
// low-res row.  A thread owns one output column and a run of consecutive output
// rows; for factors >= 1 their cell rows step by 0 or 1, so each low-res row's
// (A, B) is formed once (8 FMAs per channel) and every output then costs 4 FMAs
// per channel.
//
// Launch: one 256-thread block per 64 x 32 tile of output pixels: 64 columns x
// 4 runs of 8 rows, a warp = 32 columns of one run (coalesced stores).  The
// block computes the cell index and the basis weights of its 64 columns and 32
// rows once (shared tables) and stages the low-res footprint of the tile -- each
// pixel's 12 values (C, C_x, C_y, C_xy for three channels) packed as three
// float4 -- in shared memory with coalesced loads.  48 B per low-res pixel in,
// 12 B per output pixel out.
#include <cuda.h>           // CUtensorMap (the type only; no driver library is linked)
#include <cudaTypedefs.h>   // the encoder's signature, fetched through the runtime

#include <atomic>
#include <mutex>

#include "gs_internal.cuh"
#include "spline_common.cuh"
#include "umma.cuh"

namespace gs {
namespace {

constexpr int kMaxFactor = 16;
// spline tiles
constexpr int kSplCols = 64, kSplRuns = 4, kSplRun = 8;
constexpr int kSplThreads = kSplCols * kSplRuns;   // 256
constexpr int kSplW = kSplCols;                    // 64
constexpr int kSplH = kSplRuns * kSplRun;          // 32
// footprint of a 64 x 32 output tile for W2 >= W: at most 63 + 2 x 31 + 2 cells
constexpr int kFootW = kSplW + 1;
constexpr int kFootH = kSplH + 1;

// footprint bound of a 64 x 32 output tile: ceil(63 W / W2) + 2 columns,
// ceil(31 H / H2) + 2 rows
__host__ __device__ int foot_w(int W, int W2) { return min(kFootW, (int)((63ll * W + W2 - 1) / W2) + 2); }
__host__ __device__ int foot_h(int H, int H2) { return min(kFootH, (int)((31ll * H + H2 - 1) / H2) + 2); }

// (A, B) of the three channels at footprint row r for the column with cell li
// and x weights w = (h00, h01, h10, h11)
__device__ __forceinline__ void spline_row(const float4* __restrict__ foot, int pitch, int r, int li, float4 w,
                                           float (&A)[3], float (&B)[3])
{
    const float4* v = foot + 3 * (r * pitch + li);
    const float4 a0 = v[0], a1 = v[1], a2 = v[2];   // corner a = 0: (C rgb, Cx r) (Cx gb, Cy rg) (Cy b, Cxy rgb)
    const float4 b0 = v[3], b1 = v[4], b2 = v[5];   // corner a = 1
    A[0] = fmaf(w.x, a0.x, fmaf(w.y, b0.x, fmaf(w.z, a0.w, w.w * b0.w)));
    A[1] = fmaf(w.x, a0.y, fmaf(w.y, b0.y, fmaf(w.z, a1.x, w.w * b1.x)));
    A[2] = fmaf(w.x, a0.z, fmaf(w.y, b0.z, fmaf(w.z, a1.y, w.w * b1.y)));
    B[0] = fmaf(w.x, a1.z, fmaf(w.y, b1.z, fmaf(w.z, a2.y, w.w * b2.y)));
    B[1] = fmaf(w.x, a1.w, fmaf(w.y, b1.w, fmaf(w.z, a2.z, w.w * b2.z)));
    B[2] = fmaf(w.x, a2.x, fmaf(w.y, b2.x, fmaf(w.z, a2.w, w.w * b2.w)));
}

// The 64 x (4 RUN) output tile at (X0, Y0) (one block of kSplThreads; RUN
// rows per thread: 8, or 16 for factors of 3 and more, whose footprints are small)
template <int RUN = kSplRun>
__device__ __forceinline__ void upscale_tile(const float* __restrict__ Cimg, const float* __restrict__ G, int W,
                                             int H, int W2, int H2, int pitch, float* __restrict__ out, int X0,
                                             int Y0)
{
    constexpr int kTH = kSplRuns * RUN;   // tile rows
    // per low-res pixel of the footprint, its 12 values packed in 3 float4: [fy][fx][3]
    extern __shared__ float4 sm[];
    __shared__ float4 s_wx[kSplW];   // basis weights (h00, h01, h10, h11) per output column
    __shared__ float4 s_wy[kTH];
    __shared__ int s_cx[kSplW], s_cy[kTH];   // cell index (absolute until the footprint origin is known)
    const int tid = threadIdx.x;
    const int col = tid & (kSplCols - 1), run = tid / kSplCols;

    if (tid < kSplW) {
        int ci;
        float t;
        cell_of(min(X0 + tid, W2 - 1), W, W2, ci, t);
        s_cx[tid] = ci;
        s_wx[tid] = hermite(t);
    } else if (tid < kSplW + kTH) {
        const int r = tid - kSplW;
        int cj;
        float u;
        cell_of(min(Y0 + r, H2 - 1), H, H2, cj, u);
        s_cy[r] = cj;
        s_wy[r] = hermite(u);
    }
    __syncthreads();
    const int i0 = s_cx[0], j0 = s_cy[0];
    const int fw = s_cx[kSplW - 1] + 2 - i0, fh = s_cy[kTH - 1] + 2 - j0;   // <= pitch x foot_h(H, H2)

    // footprint: pixel p of the row-major fh x fw window is loaded by thread
    // p mod 256 (coalesced in each of the 12 planes); two rounds of loads in
    // flight before the first store
    const size_t plane = (size_t)W * H;
    const int np = fw * fh;
    for (int p0 = 0; p0 < np; p0 += 2 * kSplThreads) {
        float v[2][12];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int p = p0 + r * kSplThreads + tid;
            if (p < np) {
                const int fy = p / fw, fx = p - fy * fw;
                const size_t o = (size_t)(j0 + fy) * W + i0 + fx;
#pragma unroll
                for (int k = 0; k < 3; ++k) v[r][k] = __ldg(Cimg + k * plane + o);
#pragma unroll
                for (int k = 0; k < 9; ++k) v[r][3 + k] = __ldg(G + k * plane + o);
            }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int p = p0 + r * kSplThreads + tid;
            if (p < np) {
                const int fy = p / fw, fx = p - fy * fw;
                float4* d = sm + 3 * (fy * pitch + fx);
                d[0] = make_float4(v[r][0], v[r][1], v[r][2], v[r][3]);
                d[1] = make_float4(v[r][4], v[r][5], v[r][6], v[r][7]);
                d[2] = make_float4(v[r][8], v[r][9], v[r][10], v[r][11]);
            }
        }
    }
    __syncthreads();

    const int X = X0 + col;
    const int y0 = run * RUN;
    if (X >= W2 || Y0 + y0 >= H2) return;   // no barrier follows
    const float4 wx = s_wx[col];
    const int li = s_cx[col] - i0;
    // rows cur and cur + 1 of the run's current cell (relative to the footprint)
    int cur = s_cy[y0] - j0;
    float A0[3], B0[3], A1[3], B1[3];
    spline_row(sm, pitch, cur, li, wx, A0, B0);
    spline_row(sm, pitch, cur + 1, li, wx, A1, B1);
    const size_t oplane = (size_t)W2 * H2;
    float* o = out + (size_t)(Y0 + y0) * W2 + X;
#pragma unroll
    for (int k = 0; k < RUN; ++k) {
        if (Y0 + y0 + k >= H2) break;
        const int lj = s_cy[y0 + k] - j0;
        if (lj != cur) {   // the next cell row (cells of consecutive rows step by at most one)
            cur = lj;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                A0[c] = A1[c];
                B0[c] = B1[c];
            }
            spline_row(sm, pitch, cur + 1, li, wx, A1, B1);
        }
        const float4 wy = s_wy[y0 + k];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            o[c * oplane] = fmaf(wy.x, A0[c], fmaf(wy.y, A1[c], fmaf(wy.z, B0[c], wy.w * B1[c])));
        o += W2;
    }
}

template <int RUN = kSplRun>
__global__ void __launch_bounds__(kSplThreads) k_upscale(const float* __restrict__ Cimg, const float* __restrict__ G,
                                                         int W, int H, int W2, int H2, int pitch,
                                                         float* __restrict__ out)
{
    upscale_tile<RUN>(Cimg, G, W, H, W2, H2, pitch, out, blockIdx.x * kSplW, blockIdx.y * (kSplRuns * RUN));
}

// The upscales of a batch of views in one launch: block b takes tile b - start[v]
// of view v (row-major over its tiles_x tiles per row).
__global__ void __launch_bounds__(kSplThreads) k_upscale_views(const __grid_constant__ UpscaleViews b)
{
    const int g = blockIdx.x;
    int v = 0;
    while (v + 1 < b.V && g >= b.start[v + 1]) ++v;
    const UpscaleView& u = b.v[v];
    const int t = g - b.start[v];
    const int tiles_x = (u.W2 + kSplW - 1) / kSplW;
    const int by = t / tiles_x, bx = t - by * tiles_x;
    upscale_tile(u.C, u.G, u.W, u.H, u.W2, u.H2, foot_w(u.W, u.W2), u.out, bx * kSplW, by * kSplH);
}

// ---------------------------------------------------------------- TMA-fed persistent form
//
// For low-res frames whose rows are a multiple of 16 bytes (W % 4 == 0) with
// 16-byte aligned planes, each block loops over output tiles (tile, tile +
// grid, ...) and evaluates exactly as upscale_tile, but its footprints arrive
// by the tensor memory accelerator: two shared-memory stages, each holding one
// 3-D box of the C planes and one of the G planes ([plane][row][column], the
// box's first column rounded down to a multiple of 4 as the copy requires),
// their completion counted on the stage's mbarrier.  The footprint of the
// tile after next is in flight while the block evaluates the current one, so
// the staging no longer stalls the block between its load and its
// evaluation.  Same products and sums as upscale_tile, hence the same bits.
constexpr int kUpStages = 2;
constexpr uint32_t kUpWaitLimit = 1u << 22;   // mbarrier polls before giving up

struct UpTma {
    int bw, bh;       // box: columns (a multiple of 4) and rows of a footprint
    int plane;        // bw * bh floats
    int gofs;         // offset (floats) of the G box in a stage, 128-byte aligned
    int stage;        // floats per stage, 128-byte aligned
};

__host__ __device__ inline UpTma up_tma_layout(int W, int H, int W2, int H2)
{
    UpTma l;
    // + 3: the first column rounded down to a multiple of 4; no wider or
    // taller than the frame (W is a multiple of 4 here)
    l.bw = min((foot_w(W, W2) + 3 + 3) & ~3, W);
    l.bh = min(foot_h(H, H2), H);
    l.plane = l.bw * l.bh;
    l.gofs = (3 * l.plane + 31) & ~31;
    l.stage = (l.gofs + 9 * l.plane + 31) & ~31;
    return l;
}

// (A, B) as spline_row, from the planar stage: value k of column x in row r at
// st[k * plane + r * bw + x] (k < 3: C; else G at gofs + (k - 3) * plane)
__device__ __forceinline__ void spline_row_planar(const float* __restrict__ st, const UpTma& l, int r, int li,
                                                  float4 w, float (&A)[3], float (&B)[3])
{
    const float* c = st + r * l.bw + li;
    const float* g = c + l.gofs;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float* cc = c + ch * l.plane;
        const float* gx = g + ch * l.plane;
        const float* gy = g + (3 + ch) * l.plane;
        const float* gxy = g + (6 + ch) * l.plane;
        A[ch] = fmaf(w.x, cc[0], fmaf(w.y, cc[1], fmaf(w.z, gx[0], w.w * gx[1])));
        B[ch] = fmaf(w.x, gy[0], fmaf(w.y, gy[1], fmaf(w.z, gxy[0], w.w * gxy[1])));
    }
}

__global__ void __launch_bounds__(kSplThreads) k_upscale_tma(const __grid_constant__ CUtensorMap tmC,
                                                             const __grid_constant__ CUtensorMap tmG, int W, int H,
                                                             int W2, int H2, const UpTma l, float* __restrict__ out,
                                                             int* __restrict__ err)
{
    extern __shared__ __align__(128) float st_raw[];   // kUpStages stages of l.stage floats, from a 128-byte boundary
    __shared__ __align__(8) uint64_t s_full[kUpStages];
    __shared__ float4 s_wx[kSplW];
    __shared__ float4 s_wy[kSplH];
    __shared__ int s_cx[kSplW], s_cy[kSplH];
    __shared__ int s_abort;
    const int tid = threadIdx.x;
    const int col = tid & (kSplCols - 1), run = tid / kSplCols;
    const int tiles_x = (W2 + kSplW - 1) / kSplW;
    const int ntiles = tiles_x * ((H2 + kSplH - 1) / kSplH);
    const uint32_t tx_bytes = 12u * (uint32_t)l.plane * 4u;
    const size_t oplane = (size_t)W2 * H2;
    float* const st_all = st_raw + ((128u - (umma::smem_u32(st_raw) & 127u)) & 127u) / 4u;

    // thread 0: the copies of tile t's footprint into stage s
    auto issue = [&](int t, int s) {
        const int X0 = (t % tiles_x) * kSplW, Y0 = (t / tiles_x) * kSplH;
        int i0, j0;
        float u;
        cell_of(X0, W, W2, i0, u);
        cell_of(Y0, H, H2, j0, u);
        float* dst = st_all + (size_t)s * l.stage;
        umma::mbar_arrive_expect_tx(&s_full[s], tx_bytes);
        umma::tma_load_3d(dst, &tmC, i0 & ~3, j0, 0, &s_full[s]);
        umma::tma_load_3d(dst + l.gofs, &tmG, i0 & ~3, j0, 0, &s_full[s]);
    };
    uint32_t issued0 = 0, issued1 = 0;   // thread 0: copies issued per stage
    if (tid == 0) {
        umma::mbar_init(&s_full[0], 1);
        umma::mbar_init(&s_full[1], 1);
        umma::mbar_init_fence();
        s_abort = 0;
    }
    __syncthreads();
    if (tid == 0) {
        if ((int)blockIdx.x < ntiles) { issue(blockIdx.x, 0); ++issued0; }
        if ((int)(blockIdx.x + gridDim.x) < ntiles) { issue(blockIdx.x + gridDim.x, 1); ++issued1; }
    }

    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int s = it & 1;
        const int X0 = (t % tiles_x) * kSplW, Y0 = (t / tiles_x) * kSplH;
        if (tid < kSplW) {
            int ci;
            float u;
            cell_of(min(X0 + tid, W2 - 1), W, W2, ci, u);
            s_cx[tid] = ci;
            s_wx[tid] = hermite(u);
        } else if (tid < kSplW + kSplH) {
            const int r = tid - kSplW;
            int cj;
            float u;
            cell_of(min(Y0 + r, H2 - 1), H, H2, cj, u);
            s_cy[r] = cj;
            s_wy[r] = hermite(u);
        }
        __syncthreads();   // tables of tile t
        if (!umma::mbar_wait(&s_full[s], (uint32_t)(it >> 1) & 1u, kUpWaitLimit)) {
            s_abort = 1;
            atomicExch(err, kDevTimeout);
        } else {
            const float* st = st_all + (size_t)s * l.stage;
            const int X = X0 + col;
            const int y0 = run * kSplRun;
            if (X < W2 && Y0 + y0 < H2) {
                const int i0 = s_cx[0], j0 = s_cy[0];
                const float4 wx = s_wx[col];
                const int li = s_cx[col] - (i0 & ~3);
                int cur = s_cy[y0] - j0;
                float A0[3], B0[3], A1[3], B1[3];
                spline_row_planar(st, l, cur, li, wx, A0, B0);
                spline_row_planar(st, l, cur + 1, li, wx, A1, B1);
                float* o = out + (size_t)(Y0 + y0) * W2 + X;
#pragma unroll
                for (int k = 0; k < kSplRun; ++k) {
                    if (Y0 + y0 + k >= H2) break;
                    const int lj = s_cy[y0 + k] - j0;
                    if (lj != cur) {
                        cur = lj;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            A0[c] = A1[c];
                            B0[c] = B1[c];
                        }
                        spline_row_planar(st, l, cur + 1, li, wx, A1, B1);
                    }
                    const float4 wy = s_wy[y0 + k];
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        o[c * oplane] = fmaf(wy.x, A0[c], fmaf(wy.y, A1[c], fmaf(wy.z, B0[c], wy.w * B1[c])));
                    o += W2;
                }
            }
        }
        __syncthreads();   // stage s and the tables read by every thread
        if (s_abort) break;
        if (tid == 0) {
            const int t2 = t + kUpStages * (int)gridDim.x;
            if (t2 < ntiles) {
                umma::fence_async_smem();   // the stage's reads ordered before the copy that overwrites it
                issue(t2, s);
                if (s) ++issued1; else ++issued0;
            }
        }
    }
    // after an expired wait: let this block's copies in flight land (bounded) before it exits
    if (s_abort && tid == 0) {
        if (issued0) umma::mbar_wait(&s_full[0], (issued0 - 1) & 1u, kUpWaitLimit);
        if (issued1) umma::mbar_wait(&s_full[1], (issued1 - 1) & 1u, kUpWaitLimit);
    }
}

// Adjoint of k_upscale (upscale_adjoint_at in spline_common.cuh): one thread
// per low-res pixel gathers exactly its output footprint with the separable
// weights; no atomics, each low-res value written once.
constexpr int kBwdX = 32, kBwdY = 8;

__global__ void __launch_bounds__(kBwdX * kBwdY) k_upscale_bwd(const float* __restrict__ dout, int W, int H, int W2,
                                                               int H2, float* __restrict__ dC, float* __restrict__ dG)
{
    const int i = blockIdx.x * kBwdX + threadIdx.x;
    const int j = blockIdx.y * kBwdY + threadIdx.y;
    if (i >= W || j >= H) return;
    float acc[3][4];
    upscale_adjoint_at(dout, W, H, W2, H2, i, j, acc);
    const size_t plane = (size_t)W * H, pix = (size_t)j * W + i;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        dC[ch * plane + pix] = acc[ch][0];
        dG[(0 * 3 + ch) * plane + pix] = acc[ch][1];
        dG[(1 * 3 + ch) * plane + pix] = acc[ch][2];
        dG[(2 * 3 + ch) * plane + pix] = acc[ch][3];
    }
}

// Classical bicubic comparator (Sec. 5: slopes from finite differences; Sec.
// 6: PyTorch's bicubic): cubic convolution of the colour samples with Keys'
// kernel of parameter a, sample indices clamped to the image,
//   W(d) = (a + 2)|d|^3 - (a + 3)|d|^2 + 1 (|d| <= 1), a|d|^3 - 5a|d|^2 + 8a|d| - 4a (1 < |d| < 2).
// Same tiling as k_upscale: per 64 x 16 output tile, per-column and per-row
// tap weights in shared tables and the clamped colour footprint staged as
// float4; 16 vector shared loads per output.  HBM-bound: 12 B per low-res
// pixel in, 12 B per output pixel out.
__device__ __forceinline__ float keys(float d, float a)   // d >= 0
{
    if (d <= 1.f) return ((a + 2.f) * d - (a + 3.f)) * d * d + 1.f;
    if (d < 2.f) return ((a * d - 5.f * a) * d + 8.f * a) * d - 4.f * a;
    return 0.f;
}

// first tap index floor(x) - 1 and the four tap weights of output pixel X
__device__ __forceinline__ void taps_of(int X, int W, int W2, float a, int& first, float4& w)
{
    const long long num = (2ll * X + 1) * W - W2, den = 2ll * W2;
    const long long fl = floor_div(num, den);
    const float t = (float)(num - den * fl) / (float)den;
    first = (int)fl - 1;
    w = make_float4(keys(1.f + t, a), keys(t, a), keys(1.f - t, a), keys(2.f - t, a));
}

// bicubic tiles: one 32 x 8-thread block per 64 x 16 outputs, 2 x 2 per thread
constexpr int kThreadsX = 32, kThreadsY = 8;
constexpr int kOutW = 2 * kThreadsX;   // 64
constexpr int kOutH = 2 * kThreadsY;   // 16
constexpr int kBicFootW = kOutW + 3;   // 63 + 4 taps for W2 >= W
constexpr int kBicFootH = kOutH + 3;

int bic_foot_w(int W, int W2) { return std::min(kBicFootW, (int)((63ll * W + W2 - 1) / W2) + 4); }
int bic_foot_h(int H, int H2) { return std::min(kBicFootH, (int)((15ll * H + H2 - 1) / H2) + 4); }

__global__ void __launch_bounds__(kThreadsX * kThreadsY) k_bicubic(const float* __restrict__ Cimg, int W, int H,
                                                                   int W2, int H2, float a, int pitch,
                                                                   float* __restrict__ out)
{
    extern __shared__ float4 sb[];             // [fh][pitch] clamped colour (r, g, b, 0)
    __shared__ float4 s_wx[kOutW];
    __shared__ float4 s_wy[kOutH];
    __shared__ int s_cx[kOutW], s_cy[kOutH];   // first tap relative to the footprint origin
    const int X0 = blockIdx.x * kOutW, Y0 = blockIdx.y * kOutH;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kThreadsX + tx;
    int i0, j0, i1, j1;
    float4 wtmp;
    taps_of(X0, W, W2, a, i0, wtmp);
    taps_of(Y0, H, H2, a, j0, wtmp);
    taps_of(min(X0 + kOutW - 1, W2 - 1), W, W2, a, i1, wtmp);
    taps_of(min(Y0 + kOutH - 1, H2 - 1), H, H2, a, j1, wtmp);
    const int fw = i1 + 4 - i0, fh = j1 + 4 - j0;   // <= pitch x bic_foot_h(H, H2)
    if (tid < kOutW) {
        int f;
        float4 w;
        taps_of(min(X0 + tid, W2 - 1), W, W2, a, f, w);
        s_cx[tid] = f - i0;
        s_wx[tid] = w;
    } else if (tid < kOutW + kOutH) {
        const int r = tid - kOutW;
        int f;
        float4 w;
        taps_of(min(Y0 + r, H2 - 1), H, H2, a, f, w);
        s_cy[r] = f - j0;
        s_wy[r] = w;
    }
    const size_t plane = (size_t)W * H;
    for (int fy = ty; fy < fh; fy += kThreadsY) {
        const int jj = min(max(j0 + fy, 0), H - 1);
        for (int fx = tx; fx < fw; fx += kThreadsX) {
            const int ii = min(max(i0 + fx, 0), W - 1);
            const float* c = Cimg + (size_t)jj * W + ii;
            sb[fy * pitch + fx] = make_float4(c[0], c[plane], c[2 * plane], 0.f);
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
        for (int q = 0; q < 2; ++q) {
            const int ox = tx + q * kThreadsX;
            const int X = X0 + ox;
            if (X >= W2) continue;
            const float4 wx = s_wx[ox];
            const int li = s_cx[ox];
            float r = 0.f, g = 0.f, bl = 0.f;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const float wl = l == 0 ? wy.x : (l == 1 ? wy.y : (l == 2 ? wy.z : wy.w));
                const float4* row = sb + (lj + l) * pitch + li;
                float hr = 0.f, hg = 0.f, hb = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float wk = k == 0 ? wx.x : (k == 1 ? wx.y : (k == 2 ? wx.z : wx.w));
                    const float4 v = row[k];
                    hr = fmaf(wk, v.x, hr);
                    hg = fmaf(wk, v.y, hg);
                    hb = fmaf(wk, v.z, hb);
                }
                r = fmaf(wl, hr, r);
                g = fmaf(wl, hg, g);
                bl = fmaf(wl, hb, bl);
            }
            const size_t o = (size_t)Y * W2 + X;
            out[o] = r;
            out[oplane + o] = g;
            out[2 * oplane + o] = bl;
        }
    }
}

bool sizes_ok(int W, int H, int W2, int H2, int min_side)
{
    return W >= min_side && H >= min_side && W2 >= W && H2 >= H && (long long)W2 <= (long long)kMaxFactor * W &&
           (long long)H2 <= (long long)kMaxFactor * H;
}

// The upscale kernels' dynamic shared memory limit (the largest footprint, at
// factor 1), set once per device: an atomic bit per device, so concurrent
// first calls from several host threads set the same value.
template <typename F>
cudaError_t upscale_attr(F kernel, std::atomic<uint64_t>& done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(3 * sizeof(float4) * kFootW * kFootH))) != cudaSuccess)
        return e;
    done.fetch_or(bit, std::memory_order_acq_rel);
    return cudaSuccess;
}
std::atomic<uint64_t> g_upscale_attr{0};
std::atomic<uint64_t> g_upscale_views_attr{0};

}  // namespace

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library), looked up once per process
PFN_cuTensorMapEncodeTiled_v12000 tma_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            (void)cudaGetLastError();
    });
    return fn;
}

// the 3-D map of `planes` W x H FP32 planes, boxes of bw x bh x planes
bool planes_map(CUtensorMap* m, const float* base, int W, int H, int planes, int bw, int bh)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)W * 4u, (cuuint64_t)W * H * 4u};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

std::atomic<uint64_t> g_upscale_tma_attr{0};
constexpr size_t kUpTmaMaxSmem = 227 * 1024 - 4096;   // dynamic share beside the static tables

// The TMA-fed form when the frame allows it: rows of 16-byte multiples,
// 16-byte aligned planes, both stages within one block's shared memory.
// Returns cudaErrorNotSupported (nothing launched) otherwise.
cudaError_t launch_upscale_tma(cudaStream_t s, const float* C, const float* grads, int W, int H, int W2, int H2,
                               float* out, int* err)
{
    if (!err || W % 4 != 0 || (reinterpret_cast<uintptr_t>(C) & 15u) || (reinterpret_cast<uintptr_t>(grads) & 15u))
        return cudaErrorNotSupported;
    // only where the staged form waits on more than one round of loads per
    // block (footprints of more than 2 x 256 pixels: factors below ~2.2);
    // with smaller footprints the staged form's single round costs less than
    // the persistent loop's waits (4x: 12.0 vs 14.2 us at 1920x1080; 2x: 16.4 vs 14.3 us)
    if (foot_w(W, W2) * foot_h(H, H2) <= 2 * kSplThreads) return cudaErrorNotSupported;
    const UpTma l = up_tma_layout(W, H, W2, H2);
    const size_t smem = (size_t)kUpStages * l.stage * sizeof(float) + 128;   // + the rounding to 128 bytes
    if (l.bw > 256 || l.bh > 256 || smem > kUpTmaMaxSmem) return cudaErrorNotSupported;
    CUtensorMap mC, mG;
    if (!planes_map(&mC, C, W, H, 3, l.bw, l.bh) || !planes_map(&mG, grads, W, H, 9, l.bw, l.bh))
        return cudaErrorNotSupported;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
    if (!bit || !(g_upscale_tma_attr.load(std::memory_order_acquire) & bit)) {
        if ((e = cudaFuncSetAttribute(k_upscale_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kUpTmaMaxSmem)) != cudaSuccess)
            return e;
        g_upscale_tma_attr.fetch_or(bit, std::memory_order_acq_rel);
    }
    int per_sm = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_upscale_tma, kSplThreads, smem)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int ntiles = upscale_tiles(W2, H2);
    const int grid = std::max(1, std::min(ntiles, std::max(1, per_sm) * sms));
    k_upscale_tma<<<grid, kSplThreads, smem, s>>>(mC, mG, W, H, W2, H2, l, out, err); note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_upscale_to(cudaStream_t s, const float* C, const float* grads, int W, int H, int W2, int H2,
                              float* out, int* err)
{
    if (!sizes_ok(W, H, W2, H2, 2)) return cudaErrorInvalidValue;
    {
        const cudaError_t e = launch_upscale_tma(s, C, grads, W, H, W2, H2, out, err);
        if (e != cudaErrorNotSupported) return e;
    }
    const int pitch = foot_w(W, W2);
    if (W2 >= 3 * W && H2 >= 3 * H) {   // 64 x 64 tiles: footprints of at most 23 x 23 pixels
        constexpr int kTH = kSplRuns * 16;
        const int fh = std::min(kTH + 1, (int)((63ll * H + H2 - 1) / H2) + 2);
        dim3 grid((W2 + kSplW - 1) / kSplW, (H2 + kTH - 1) / kTH);
        k_upscale<16><<<grid, kSplThreads, 3 * sizeof(float4) * pitch * fh, s>>>(C, grads, W, H, W2, H2, pitch, out);
        note_launch();
        return cudaGetLastError();
    }
    dim3 grid((W2 + kSplW - 1) / kSplW, (H2 + kSplH - 1) / kSplH);
    cudaError_t e = upscale_attr(k_upscale<>, g_upscale_attr);
    if (e != cudaSuccess) return e;
    const size_t smem = 3 * sizeof(float4) * pitch * foot_h(H, H2);
    k_upscale<><<<grid, kSplThreads, smem, s>>>(C, grads, W, H, W2, H2, pitch, out); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_upscale_views(cudaStream_t s, const UpscaleViews& b)
{
    const int total = b.start[b.V];
    if (total <= 0) return cudaSuccess;
    size_t smem = 0;
    for (int v = 0; v < b.V; ++v) {
        const UpscaleView& u = b.v[v];
        if (!sizes_ok(u.W, u.H, u.W2, u.H2, 2)) return cudaErrorInvalidValue;
        smem = std::max(smem, 3 * sizeof(float4) * foot_w(u.W, u.W2) * foot_h(u.H, u.H2));
    }
    cudaError_t e = upscale_attr(k_upscale_views, g_upscale_views_attr);
    if (e != cudaSuccess) return e;
    k_upscale_views<<<total, kSplThreads, smem, s>>>(b); note_launch();
    return cudaGetLastError();
}

int upscale_tiles(int W2, int H2)
{
    return ((W2 + kSplW - 1) / kSplW) * ((H2 + kSplH - 1) / kSplH);
}

cudaError_t launch_upscale(cudaStream_t s, const float* C, const float* grads, int W, int H, int factor, float* out,
                           int* err)
{
    if (factor < 1 || factor > kMaxFactor) return cudaErrorInvalidValue;
    return launch_upscale_to(s, C, grads, W, H, W * factor, H * factor, out, err);
}

cudaError_t launch_upscale_backward_to(cudaStream_t s, const float* dout, int W, int H, int W2, int H2, float* dC,
                                       float* dG)
{
    if (!sizes_ok(W, H, W2, H2, 2)) return cudaErrorInvalidValue;
    dim3 grid((W + kBwdX - 1) / kBwdX, (H + kBwdY - 1) / kBwdY);
    k_upscale_bwd<<<grid, dim3(kBwdX, kBwdY), 0, s>>>(dout, W, H, W2, H2, dC, dG); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_upscale_backward(cudaStream_t s, const float* dout, int W, int H, int factor, float* dC,
                                    float* dG)
{
    if (factor < 1 || factor > kMaxFactor) return cudaErrorInvalidValue;
    return launch_upscale_backward_to(s, dout, W, H, W * factor, H * factor, dC, dG);
}

cudaError_t launch_bicubic(cudaStream_t s, const float* C, int W, int H, int W2, int H2, float a, float* out)
{
    if (!sizes_ok(W, H, W2, H2, 1)) return cudaErrorInvalidValue;
    dim3 grid((W2 + kOutW - 1) / kOutW, (H2 + kOutH - 1) / kOutH);
    const int pitch = bic_foot_w(W, W2);
    const size_t smem = sizeof(float4) * pitch * bic_foot_h(H, H2);
    k_bicubic<<<grid, dim3(kThreadsX, kThreadsY), smem, s>>>(C, W, H, W2, H2, a, pitch, out); note_launch();
    return cudaGetLastError();
}

}  // namespace gs
