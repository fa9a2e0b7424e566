// Internal declarations shared by the libgs translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gs {

constexpr int kTile = 16;                 // tile side in pixels (16 x 16 = 256 pixels)
constexpr int kTilePixels = kTile * kTile;
// Tile binning works per super-tile of ks x ks tiles (ks = 1, 2 or 4: a pair
// carries a ks^2-bit mask of the tiles it covers).  super_side picks ks per
// frame: the smallest side whose super-tile count fits one 8-bit pass of the
// pair sort, else the largest.  Small super-tiles keep the blend's filtered
// walk short (a block scans its super-tile's whole list); at larger images the
// extra pairs and sort passes of small super-tiles cost more than they save.
// In exact mode every Gaussian is in every tile, so smaller super-tiles would
// only multiply the pairs: the largest side is used.
constexpr int kSuperMax = 4;
constexpr int kSuperOnePass = 256;        // super-tiles one 8-bit radix pass orders
inline int super_side(int tiles_x, int tiles_y, int mode)
{
    if (mode == GS_MODE_EXACT) return kSuperMax;
    for (int ks = 1; ks < kSuperMax; ks *= 2)
        if ((int64_t)((tiles_x + ks - 1) / ks) * ((tiles_y + ks - 1) / ks) <= kSuperOnePass) return ks;
    return kSuperMax;
}

// Device error word values (written by bounded waits / device checks).
constexpr int kDevOk = 0;
constexpr int kDevTimeout = 1;
constexpr int kDevCheck = 2;
constexpr int kDevCapacity = 3;   // a frame's pairs exceeded the reserved pair buffers

// The projection sums the frame's pair totals into kTotalSlots slot pairs
// (super-tile pairs, tile pairs) to spread its atomics; the host adds the slots.
constexpr int kTotalSlots = 32;
// Copies of the per-super-tile count array the emission kernel spreads its
// atomics over (summed by launch_supers_to_hist).
constexpr int kCountCopies = 32;

// Largest pair count the 30-bit look-back counters of the radix sort can hold.
constexpr int64_t kMaxPairs = (int64_t(1) << 30) - 1;

// Per-Gaussian record staged by the blend kernel (3 x 16 B):
//   r0 = (mean_x, mean_y, -conic_a, -conic_c)
//   r1 = (A2, B2, C2, thr2): the exponent in base 2, g2 = A2 dx^2 + B2 dx dy + C2 dy^2
//        = log2(e) * (-1/2)(a dx^2 + 2 b dx dy + c dy^2), and its reject threshold
//   r2 = (red, green, blue, opacity)
struct Records {
    float4* r0;
    float4* r1;
    float4* r2;
};

struct CameraParams {
    float R[9];        // world->camera rotation, row-major
    float t[3];        // world->camera translation
    float campos[3];   // camera centre in world coordinates, -R^T t
    float fx, fy, cx, cy, znear;
    float lim_x, lim_y;   // 1.3 tan(fov/2) clamp of the Jacobian's x/z, y/z
};

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

// Arguments of the blend kernel.
struct BlendArgs {
    int W, H, tiles_x, tiles_y, stiles_x;
    int ks;                        // super-tile side in tiles
    uint32_t n;
    const uint2* sranges;          // [super-tiles] list ranges
    const uint32_t* pair_words;    // sorted (super << 32 | id) pairs viewed as 32-bit words
    const ushort4* rect;           // [n] tile rect (x0, y0, x1, y1) inclusive
    Records rec;
    float3 bg;
    float* out_C;
    float* out_G;
    float4* state;
    int* count;
    // tile scheduling (optional): blocks take tiles in the order order[] (the
    // heaviest of the previous frame first) and record their duration in work[]
    const uint32_t* order;
    uint32_t* work;
};

// Order tiles by the recorded work of the previous frame, heaviest first
// (coarse: 4 buckets per octave of the recorded duration).
// The tiles of a batch of views (view v: start[v] .. start[v + 1] - 1), each
// view's heaviest first, the views in order.
cudaError_t launch_tile_order_views(cudaStream_t s, const uint32_t* work, const int* start, int V, uint32_t* order);
cudaError_t launch_tile_order(cudaStream_t s, const uint32_t* work, uint32_t T, uint32_t* order);

// Adjoint of the blend: the forward's binning (super-tile lists filtered per
// tile by the rects), its final per-pixel state and count, the upstream
// planes, and the 2D gradients [n][9] = (mean_x, mean_y, conic a, b, c,
// opacity, r, g, b), accumulated.
struct BlendBwdArgs {
    int W, H, tiles_x, stiles_x;
    int ks;                        // super-tile side in tiles
    uint32_t n;
    const uint2* sranges;          // [super-tiles] list ranges
    const uint32_t* pair_words;    // sorted (super << 32 | id) pairs viewed as 32-bit words
    const ushort4* rect;           // [n] tile rect
    Records rec;
    float3 bg;
    const float4* state;           // [W*H] final (T, T_x, T_y, T_xy)
    const int* count;              // [W*H] list position after the last blended Gaussian
    const float* dC;               // [3][H][W]
    const float* dG;               // [3 (x, y, xy)][3][H][W]
    // instead of dC / dG (when not null): the upstream gradient of the upscaled
    // image [3][H2][W2], taken through the upscale's adjoint per pixel
    const float* dout;
    int W2, H2;
    float* grad2d;                 // [n][9]
    int* err;
    const uint32_t* order;         // optional: tiles in this order (the forward's, heaviest first)
    // recompute variant (when not null): per tile kCkSlots x 256 checkpointed
    // states; state and count above are then not read
    float4* ckpt;
};
constexpr int kCkSlots = 8;   // checkpoints per tile of the recompute variant of the blend adjoint

}  // namespace gs

struct gs_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    gs_options opt{};
    char err[512] = {0};

    // last projection
    bool have_proj = false;
    bool have_state = false;
    int64_t n = 0;
    int W = 0, H = 0, tiles_x = 0, tiles_y = 0, stiles_x = 0, stiles_y = 0;
    int ks = gs::kSuperMax;             // super-tile side of the last projection
    int64_t P = 0;                      // (tile, Gaussian) pairs
    int64_t Ps = 0;                     // (super-tile, Gaussian) pairs

    // per Gaussian
    gs::DevBuf rec0, rec1, rec2;        // float4[n]
    gs::DevBuf depth;                   // float[n]
    gs::DevBuf radius;                  // int32[n]
    gs::DevBuf rect;                    // ushort4[n] inclusive tile rect
    gs::DevBuf tiles_touched;           // uint32[n] tiles of the rect
    gs::DevBuf supers_touched;          // uint32[n] super-tiles of the rect
    gs::DevBuf dkey[2], did[2];         // depth sort keys / ids, ping-pong
    gs::DevBuf offsets;                 // uint32[n + 1]
    gs::DevBuf scan_partials;           // uint64[tiles + 1] scan tile states
    gs::DevBuf scan_totals;             // uint64[2] + uint32 tile counter
    // per super-tile pair
    gs::DevBuf pairs[2];                // uint64[Ps] (super-tile << 32 | id), ping-pong
    // radix sort scratch
    gs::DevBuf sort_hist;               // uint32[passes][256]
    gs::DevBuf sort_status;             // uint32[passes][tiles][256]
    gs::DevBuf sort_counter;            // uint32[passes]
    gs::DevBuf super_counts;            // uint32[super-tiles]
    gs::DevBuf ds_scratch;              // persistent depth sort: per-block counts, sums, barrier
    cudaEvent_t totals_ready = nullptr; // recorded after the pair totals are copied to the host
    // per tile / pixel
    gs::DevBuf sranges;                 // uint2[super-tiles]
    gs::DevBuf tile_count, tile_start;  // uint32[tiles] (per-tile list materialisation)
    gs::DevBuf tile_work, tile_order;   // uint32[tiles]: last frame's block durations, this frame's order
    int64_t work_tiles = -1;            // tile count the recorded durations belong to
    bool order_ready = false;           // the projection computed the next blend's tile order
    gs::DevBuf state;                   // float4[W*H]
    gs::DevBuf count;                   // int32[W*H]
    gs::DevBuf errword;                 // int32
    // reverse mode
    bool state_grads = false;           // the last blend carried derivatives (its state is usable)
    gs_gaussians last_g{};              // inputs and camera of the last projection
    gs::CameraParams last_cam{};
    gs::DevBuf grad2d;                  // float[n][9]
    gs::DevBuf ckpt;                    // float4[tiles][kCkSlots][256]: the recompute adjoint's checkpoints
    // frames without a host wait (GS_FLAG_NO_HOST_WAIT): buffers reserved up front
    bool reserved = false;
    int64_t res_n = 0, res_pixels = 0, res_tiles = 0, res_supers = 0, res_pairs = 0;
    gs::DevBuf pair_check;              // gs::PairCheckOut, device side
    // batched views (gs_render_views): per-view projection outputs, view v at v * n
    int res_views = 0;
    gs::DevBuf vrec0, vrec1, vrec2;     // float4[V][n]
    gs::DevBuf vrect;                   // ushort4[V][n]
    gs::DevBuf vsupers, vkey;           // uint32[V][n]
    gs::DevBuf vsortv;                  // uint32[V][n]: the batched depth sort's second value buffer
    gs::DevBuf vtotals;                 // uint64[V][2 kTotalSlots]
    gs::DevBuf views_dev;               // gs::ViewDesc[kMaxViews]
    gs::DevBuf vpairs0, vpairs1;        // uint64[V][res_pairs]: each view's pairs (sort ping-pong)
    gs::DevBuf vsranges;                // uint2[V][res_supers]
    gs::DevBuf vwork, vorder;           // uint32[V * res_tiles]: tile durations / order of the batch
    gs::DevBuf vqueue;                  // uint32 job counter of the persistent batched blend
    gs::DevBuf vcounts;                 // uint32[V][kCountCopies][res_supers]: each view's super-tile counts
    gs::DevBuf vhist;                   // uint32[V][8][256]: each view's pair-sort digit histograms
    gs::DevBuf vstatus;                 // uint32[V][vstatus_stride]: each view's look-back states and counters
    size_t vstatus_stride = 0;
    gs::DevBuf vdhist;                  // uint32[V][4][256]: each view's depth-sort digit histograms
    gs::DevBuf vdstatus;                // uint32[V][vdstatus_stride]: each view's depth-sort states and counters
    size_t vdstatus_stride = 0;
    int batch_views = 0;                // views of the last batch (0: the last frame was a single view)
    int views_ks = 0;                   // batched views: super-tile side, 0 = per-view rule, or kSuperMax
    int views_map = 0;                  // batched blend: 0 = 8 x 4 warp blocks, 1 = 16 x 2
    int views_sched = 1;                // 0 = tile order, 1 = heaviest first (last batch), 2 = persistent
    bool totals_known = true;           // P, Ps valid on the host
    unsigned long long* h_scalar = nullptr;   // pinned host scalar for the pair count
    int sorted_ids_buf = 0;             // which did[] holds the depth-sorted ids
    int sorted_pairs_buf = 0;           // which pairs[] holds the sorted pairs
    int64_t launches = 0;               // kernels launched on behalf of this context
    // fault injection (gs_debug_inject): one-shot, consumed by the next use
    uint32_t inject_wait_spins = 0;     // the next persistent depth sort's extra wait runs out after this many polls
    int64_t inject_alloc_countdown = -1;   // the allocation after this many more fails (-1: none)
};

namespace gs {

// Kernel launches issued by this thread since the library was loaded (every
// launch site calls note_launch(); the API adds the delta of each call to the
// context's counter, exposed by gs_launch_count).
int64_t& launch_counter();
inline void note_launch() { ++launch_counter(); }

// ---- launchers (each returns the cudaError_t of its launch) ----
// One view of a batch: camera and image size.
struct ViewDesc {
    CameraParams cam;
    int W, H, tiles_x, tiles_y;
    int ks;         // super-tile side in tiles
    uint32_t off;   // the view's Gaussian i is entry off + i of the batch's per-(view, Gaussian) arrays
    int vid;        // the view's index in the batch
};
// Per-view outputs of the batched projection, view v's Gaussian i at entry
// g = off_v + i (totals: 2 kTotalSlots per view, at vid): records, rect,
// super-tiles touched, and the input of the views' depth sorts,
// depth_key[g] = FP32 depth bits (0xFFFFFFFF for a Gaussian without tiles)
// and gidx[g] = g, or with pack_counts (batches of fewer than 2^24 entries)
// g | min(supers[g], 255) << 24: the pair count then travels with the entry
// through the depth sorts (255: look it up).
constexpr uint32_t kPackedIdxBits = 24;
constexpr uint32_t kPackedIdxMask = (1u << kPackedIdxBits) - 1u;
constexpr uint32_t kPackedCntEsc = 255u;
struct ViewOutputs {
    Records rec;
    ushort4* rect;
    uint32_t* supers;
    uint32_t* depth_key;
    uint32_t* gidx;
    unsigned long long* totals;
    bool pack_counts = false;
};
cudaError_t launch_project_views(cudaStream_t s, const gs_gaussians& g, const ViewDesc* views, int V, int mode,
                                 const ViewOutputs& out);
// Copy a batch of view descriptions to device memory through kernel
// parameters (recorded by value in a CUDA graph; no host buffer involved).
constexpr int kMaxViews = 32;
struct ViewBatch {
    ViewDesc v[kMaxViews];
};
cudaError_t launch_set_views(cudaStream_t s, const ViewBatch& b, int V, ViewDesc* dst);
// ids[i] = i for i < n
cudaError_t launch_iota(cudaStream_t s, uint32_t* ids, uint32_t n);

// Buffers of later kernels in the frame that must start at zero; the
// projection kernel clears them (grid-stride) so the frame needs no memsets.
struct ZeroList {
    static constexpr int kMax = 6;
    uint32_t* p[kMax];
    uint32_t words[kMax];
    int count;
};

cudaError_t launch_project(cudaStream_t s, const gs_gaussians& g, const CameraParams& cam, int W, int H,
                           int tiles_x, int tiles_y, int ks, int mode, Records rec, float* depth, int* radius,
                           ushort4* rect, uint32_t* tiles_touched, uint32_t* supers_touched, uint32_t* depth_key,
                           uint32_t* ids, unsigned long long* totals,
                           const ZeroList* zero = nullptr);

// LSD radix sort of n keys (uint32 keys with uint32 values, or uint64 keys
// alone) on bits [bit_lo, bit_hi).  Ping-pong buffers: the result lands in
// buffer index *out_idx (0 or 1).  n is a host count.
cudaError_t radix_sort_u32_pairs(cudaStream_t s, uint32_t* keys[2], uint32_t* vals[2], uint32_t n,
                                 int bit_lo, int bit_hi, uint32_t* hist, uint32_t* status,
                                 uint32_t* counters, int* err, int* out_idx);
// (uint64 key, uint32 value) pairs likewise (at most 40 bits)
cudaError_t radix_sort_u64_pairs(cudaStream_t s, uint64_t* keys[2], uint32_t* vals[2], uint32_t n, int bit_lo,
                                 int bit_hi, uint32_t* hist, uint32_t* status, uint32_t* counters, int* err,
                                 int* out_idx);
// uint64 keys alone.  hist_ready: hist already holds the exclusive digit
// histograms of every pass (from launch_supers_to_hist), so the sort skips its
// histogram kernels.  n_dev (optional, needs hist_ready): the key count is
// min(n, *n_dev), read on the device; n is then the capacity the launch is
// sized for.
cudaError_t radix_sort_u64_keys(cudaStream_t s, uint64_t* keys[2], uint32_t n, int bit_lo, int bit_hi,
                                uint32_t* hist, uint32_t* status, uint32_t* counters, int* err,
                                int* out_idx, bool hist_ready, const uint32_t* n_dev = nullptr,
                                bool pre_zeroed = false);
// Largest super-tile count whose per-super-tile counts the emission kernel
// accumulates in shared memory (and turns into histograms + ranges).
constexpr int kMaxSupersForCounts = 4096;
// Device-side pair-count check of a frame whose totals the host does not read
// (see k_supers_to_hist): inputs slots (the projection's 2 x kTotalSlots pair
// totals), cap, max_pairs; outputs count (pairs to sort, 0 on overflow),
// needed and tile_pairs (the frame's totals).
struct PairCheckIn {
    const unsigned long long* slots;
    unsigned long long cap, max_pairs;
};
struct PairCheckOut {
    unsigned long long needed, tile_pairs;
    uint32_t count;
};
// order_work / order_T / order (optional): in a second block of the same
// launch, the next blend's tile order from the recorded durations (as
// launch_tile_order).
cudaError_t launch_supers_to_hist(cudaStream_t s, uint32_t* counts, uint32_t Ts, int passes, uint32_t* hist,
                                  uint2* ranges, PairCheckIn in = PairCheckIn{nullptr, 0, 0},
                                  PairCheckOut* out = nullptr, int* err = nullptr,
                                  const uint32_t* order_work = nullptr, uint32_t order_T = 0,
                                  uint32_t* order = nullptr);
size_t radix_status_words(uint32_t n, int bit_lo, int bit_hi);
int radix_passes(int bit_lo, int bit_hi);
uint32_t radix_tiles(uint32_t n);   // one-sweep tiles of n keys

// Several independent key arrays sorted in the same launches (the pair lists
// of a batch of views; each view's depth keys): segment s sorts keys[0] (and
// vals[0]) of min(cap, *n_dev) keys on bits [bit_lo, bit_lo + 8 passes) into
// keys[passes % 2] (vals[passes % 2]), with its own exclusive digit
// histograms hist [passes][256], look-back states status [passes][tiles][256]
// and tile counters [passes] (both zeroed beforehand).
constexpr int kMaxSortSegs = 32;
struct SortSeg {
    void* keys[2];
    uint32_t* vals[2];
    const uint32_t* n_dev;
    uint32_t cap, tiles;   // tiles = radix_tiles(cap)
    int passes, bit_lo;
    const uint32_t* hist;
    uint32_t* status;
    uint32_t* counters;
    int* err;
    int first_block;       // set by the launcher
};
struct SortSegs {
    SortSeg seg[kMaxSortSegs];
    int count;
};
cudaError_t radix_sort_u64_segs(cudaStream_t s, SortSegs g);   // uint64 keys alone, hist given
// uint32 keys with uint32 values, at most 4 passes, cap = the segment's count
// (n_dev null); the digit histograms are computed here (hist zeroed beforehand)
cudaError_t radix_sort_u32_pairs_segs(cudaStream_t s, SortSegs g);

// k_supers_to_hist for each view of a batch in one launch (block v: view v).
struct HistView {
    uint32_t* counts;
    uint32_t Ts;
    int passes;
    uint32_t* hist;
    uint2* ranges;
    PairCheckIn in;
    PairCheckOut* out;
};
struct HistViews {
    HistView v[kMaxSortSegs];
    int V;
};
cudaError_t launch_supers_to_hist_views(cudaStream_t s, const HistViews& b, int* err);

// exclusive scan of counts[ids[k]] over k -> offsets[k] (offsets[n] = total);
// totals[0] = exact 64-bit total, totals[1] = 64-bit total of side[ids[k]].
// scratch: scan_partials_count(n) 64-bit tile states; counter: one uint32.
// packed: ids[k] carry their count in the top 8 bits (ViewOutputs), the entry
// in the low 24; counts[] is read only for the escaped ones
cudaError_t launch_scan_gathered(cudaStream_t s, const uint32_t* counts, const uint32_t* side, const uint32_t* ids,
                                 uint32_t n, uint32_t* offsets, unsigned long long* scratch, uint32_t* counter,
                                 unsigned long long* totals, int* err, bool packed = false);
size_t scan_partials_count(uint32_t n);

// counts (may be NULL): kCountCopies x Ts per-super-tile pair counts accumulated
// while emitting (zeroed by the caller; Ts <= kMaxSupersForCounts)
// Depth sort + pair-offset scan in one cooperative launch (depthsort.cu), for
// up to depth_sort_capacity(device) Gaussians (kDsMaxSlice per SM).  keys[0]
// holds the depth keys on entry; the sorted ids land in ids[*out_idx].
constexpr uint32_t kDsMaxSlice = 10240;
constexpr uint32_t kDsMaxN = (1u << 21) - 1u;   // ids share a 32-bit word with the pair counts
size_t depth_sort_smem_bytes();
uint32_t depth_sort_capacity(int device);
// Scratch of a grid of up to G blocks, carved from one buffer of
// ds_scratch_bytes(G): per-block digit counts and pair-count sums ([G][512]
// words each), the grid barrier (64 bytes) and the totals (kDsTotWords words);
// the barrier and the totals (ds_zero_words() words from ds_zero_offset(G),
// contiguous) must be zero at launch unless the launcher clears them.
constexpr uint32_t kDsRadixWords = 512;
constexpr uint32_t kDsTotWords = 5 * kDsRadixWords;
constexpr size_t ds_cnt_offset(size_t) { return 0; }
constexpr size_t ds_csum_offset(size_t G) { return G * kDsRadixWords * 4; }
constexpr size_t ds_bar_offset(size_t G) { return 2 * G * kDsRadixWords * 4; }
constexpr size_t ds_tot_offset(size_t G) { return ds_bar_offset(G) + 64; }
constexpr size_t ds_scratch_bytes(size_t G) { return ds_tot_offset(G) + 4 * (size_t)kDsTotWords; }
constexpr size_t ds_zero_offset(size_t G) { return ds_bar_offset(G); }
constexpr uint32_t ds_zero_words() { return 16 + kDsTotWords; }
cudaError_t launch_depth_sort_scan(cudaStream_t s, int device, const uint32_t* keys_in, uint32_t* keys[2],
                                   uint32_t* ids[2], const uint32_t* counts, uint32_t n, uint32_t* offsets,
                                   uint32_t* cnt_scratch, uint32_t* csum_scratch, unsigned int* bar,
                                   uint32_t* tot_scratch, int* err, int* out_idx, bool pre_zeroed = false,
                                   uint32_t inject_spins = 0);

// pairs at offsets >= cap are counted but not written (the capacity check of
// launch_supers_to_hist then rejects the frame)
// id_base, rebase: the ids and offsets of one view within a batch sorted
// together (ids[k] - id_base is the view's own id; its pairs start at slot
// offsets[k] - offsets[0] of its pair buffer)
cudaError_t launch_emit_pairs(cudaStream_t s, const uint32_t* ids, const uint32_t* offsets, const ushort4* rect,
                              uint32_t n, int ks, int stiles_x, uint64_t* pairs, uint32_t* counts, uint32_t Ts,
                              uint32_t cap = 0xFFFFFFFFu, uint32_t id_base = 0, bool rebase = false);
// The emission of every view of a batch in one launch: view v owns positions
// [start, start + n) of the batched (view, depth, id) order sorted (global
// indices, view v's Gaussian i at start + i) and its own pair buffer (cap
// pairs), super-tile side ks, stiles_x and counts [kCountCopies][Ts] (zeroed).
struct EmitView {
    uint64_t* pairs;
    uint32_t* counts;
    uint32_t start, n, cap, Ts;
    int ks, stiles_x;
};
struct EmitViews {
    EmitView v[kMaxSortSegs];
    int V;
};
cudaError_t launch_emit_views(cudaStream_t s, const EmitViews& b, const uint32_t* sorted, const uint32_t* offsets,
                              const ushort4* rect, uint32_t total, bool packed = false);
cudaError_t launch_ranges(cudaStream_t s, const uint64_t* pairs, uint32_t P, uint32_t T, uint2* ranges);
// per-tile lists from the super-tile lists: counts, starts, ranges and (optionally) keys/vals
cudaError_t launch_tile_lists(cudaStream_t s, const uint64_t* spairs, const uint2* sranges, const ushort4* rect,
                              const float* depth, uint32_t n, int tiles_x, int tiles_y, int ks, int stiles_x,
                              uint32_t* count, uint32_t* start, uint64_t* keys, uint32_t* vals, uint2* ranges);
cudaError_t launch_unpack_projected(cudaStream_t s, Records rec, const int* radius, const uint32_t* tiles_touched,
                                    const float* depth_in, uint32_t n, float* mean2d, float* conic, float* rgb,
                                    float* opacity, float* depth, int32_t* radius_out, int32_t* tiles_out);

cudaError_t launch_blend(cudaStream_t s, bool grads, int mode, const BlendArgs& a);

// The derivative blends of a batch of views in one launch: view v's tiles are
// global tiles start[v] .. start[v + 1] - 1 (its args' order/work unused); jobs
// in the order `order` (optional), durations into `work` (optional).
constexpr int kMaxBatchViews = 32;
struct BlendViews {
    BlendArgs a[kMaxBatchViews];
    int start[kMaxBatchViews + 1];
    int V;
    const uint32_t* order;
    uint32_t* work;
    uint32_t* queue;   // job counter of the persistent variant
};
// map: the warp's pixels (0: 8 x 4 block, 1: 16 x 2 strip); persistent: resident
// blocks taking tiles from a counter instead of one block per tile
cudaError_t launch_blend_views(cudaStream_t s, int mode, const BlendViews& b, int map, bool persistent);
// adjoint of the derivative blend (grad2d accumulated; zero it first)
cudaError_t launch_blend_backward(cudaStream_t s, int mode, const BlendBwdArgs& a);
// adjoint of the projection: grad2d [n][9] -> gradients of the inputs (overwritten)
cudaError_t launch_project_backward(cudaStream_t s, const gs_gaussians& g, const CameraParams& cam,
                                    const float* grad2d, const gs_gaussian_grads& out);
// adjoint of the upscale: dout [3][sH][sW] -> dC [3][H][W], dG [9][H][W] (overwritten)
cudaError_t launch_upscale_backward(cudaStream_t s, const float* dout, int W, int H, int factor, float* dC,
                                    float* dG);
// any output size W2 x H2 with W <= W2 <= 16 W, H <= H2 <= 16 H (fractional factors);
// err (may be NULL: then the TMA-fed form is not used) records an expired
// bounded wait of the TMA-fed form
cudaError_t launch_upscale_to(cudaStream_t s, const float* C, const float* grads, int W, int H, int W2, int H2,
                              float* out, int* err = nullptr);
cudaError_t launch_upscale_backward_to(cudaStream_t s, const float* dout, int W, int H, int W2, int H2, float* dC,
                                       float* dG);
// classical bicubic comparator (cubic convolution with Keys' parameter a) of C [3][H][W]
cudaError_t launch_bicubic(cudaStream_t s, const float* C, int W, int H, int W2, int H2, float a, float* out);
cudaError_t launch_blend_stats(cudaStream_t s, int mode, const BlendArgs& a, unsigned long long* stats);

cudaError_t launch_upscale(cudaStream_t s, const float* C, const float* grads, int W, int H, int factor,
                           float* out, int* err = nullptr);

// The spline upscales of a batch of views in one launch (view v's 64 x 32
// output tiles are blocks start[v] .. start[v + 1] - 1; upscale_tiles gives
// each view's count)
struct UpscaleView {
    const float* C;
    const float* G;
    int W, H, W2, H2;
    float* out;
};
struct UpscaleViews {
    UpscaleView v[kMaxBatchViews];
    int start[kMaxBatchViews + 1];
    int V;
};
int upscale_tiles(int W2, int H2);
cudaError_t launch_upscale_views(cudaStream_t s, const UpscaleViews& b);

// Learned residual on the spline (parameters: GS_MLP_PARAMS FP32 values, W1 b1 W2 b2 W3 b3)
// spline + MLP residual at any output size W2 x H2 (tensor-core inference fused into the upscale)
cudaError_t launch_mlp_upscale(cudaStream_t s, const float* C, const float* G, int W, int H, int W2, int H2,
                               const float* params, float* out, int* err);
// training samples at output pixels [M][2]: BF16 feature rows [M][64], spline [M][3], target [M][3]
cudaError_t launch_mlp_samples(cudaStream_t s, const float* C, const float* G, int W, int H, int W2, int H2,
                               const int* pixels, long long M, const float* target_img, uint16_t* feat, float* base,
                               float* target, int* err);
// MSE loss over M samples and its gradient (grads and loss overwritten)
cudaError_t launch_mlp_grad(cudaStream_t s, const float* params, const uint16_t* feat, const float* base,
                            const float* target, long long M, float* grads, float* loss, int* err);
// one Adam step (step >= 1) on params with moments m, v
cudaError_t launch_mlp_adam(cudaStream_t s, float* params, float* m, float* v, const float* g, int step, float lr,
                            float beta1, float beta2, float eps);

}  // namespace gs
