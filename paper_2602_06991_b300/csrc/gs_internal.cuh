// gs_internal.cuh -- shared device/host internals of the Top-K feature renderer.
// Not part of the public ABI (include/gs_topk.h is).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/gs_topk.h"

namespace gs {

// ------------------------------------------------------------------------------------
// Constants of the per-pixel test (3D Gaussian Splatting conventions that Sec. 3.1 of
// the paper defers to).
// ------------------------------------------------------------------------------------
constexpr float kQMax = 9.0f;            // 3-sigma ellipse: q = d^T Sigma^-1 d <= 9
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaClamp = 0.99f;
constexpr float kTStop = 1e-4f;
constexpr float kDilation = 0.3f;        // low-pass dilation of Sigma2D (px^2)
constexpr float kFrustumClamp = 1.3f;

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;   // 2048 elements per tile
constexpr int kSortBlocks = 296;                       // 2 per SM on a 148-SM B300
constexpr int kRadixBlocks = 592;                      // radix passes: 4 per SM, one wave
constexpr int kPieceLen = 16;                          // partial rows per feature-gradient work piece
constexpr int kGradVals = 10;                          // per-instance partial 2D gradient

// Error word bits (in the workspace header).
constexpr int kErrOverflow = 1;
constexpr int kErrTimeout = 2;

// ------------------------------------------------------------------------------------
// Camera table passed by value to kernels.
// ------------------------------------------------------------------------------------
struct CamDev {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float near_z;
    float limx, limy;          // 1.3 tan(fov/2) clamp of x/z, y/z in the Jacobian
    int W, H;
    int tiles_x, tiles_y;
    int tile_off;              // first global tile id of this camera
    int row_off;               // first global tile-row index of this camera
    long long pix_off;         // first flat pixel index of this camera
};

struct CamTable {
    int n;
    int tile_w, tile_h;
    int n_tiles;               // total over cameras
    int n_rows;                // tile rows, total over cameras
    CamDev c[GS_MAX_CAMERAS];
};

__device__ __forceinline__ int cam_of_tile(const CamTable &ct, int tile)
{
    int c = 0;
#pragma unroll 1
    for (int i = 1; i < ct.n; ++i)
        if (tile >= ct.c[i].tile_off) c = i;
    return c;
}

// ------------------------------------------------------------------------------------
// Error-free transformations (Knuth TwoSum, FMA-based TwoProduct) used to carry the
// camera transform and the pixel coordinate of each Gaussian in double-float
// precision, so that d = pixel - mean2d is accurate to the float32 rounding of d.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// ------------------------------------------------------------------------------------
// Projected record layout (GS_PROJ_FLOATS = 16 floats = 4 x float4 per (camera, Gaussian))
//   r0 = (u_hi, v_hi, u_lo, v_lo)          double-float pixel position of the mean
//   r1 = (s1, m, s2, opacity)              Cholesky form of the conic:
//                                          q = (dx s1)^2 + ((dy - m dx) s2)^2
//   r2 = (r, g, b, z)                      colour and camera depth (float32, sort key)
//   r3 = (a, b, c, extent)                 conic Sigma2D^-1 = [[a, b], [b, c]]; extent is
//                                          two fp16 half-widths (x | y << 16) of the pixel
//                                          box that can reach alpha >= 1/255; 0 = culled
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void unpack_extent(float packed, float &ex, float &ey)
{
    unsigned int bits = __float_as_uint(packed);
    ex = __half2float(__ushort_as_half((unsigned short)(bits & 0xffffu)));
    ey = __half2float(__ushort_as_half((unsigned short)(bits >> 16)));
}

// Inclusive tile rectangle [tx0, tx1] x [ty0, ty1] of the pixels whose centres lie in
// the box |x + 0.5 - u| <= ex, |y + 0.5 - v| <= ey.  Returns false if empty.
__device__ __forceinline__ bool tile_rect(const CamDev &c, int tw, int th, float u, float v,
                                          float ex, float ey, int &tx0, int &tx1, int &ty0, int &ty1)
{
    float x0 = ceilf(u - ex - 0.5f), x1 = floorf(u + ex - 0.5f);
    float y0 = ceilf(v - ey - 0.5f), y1 = floorf(v + ey - 0.5f);
    x0 = fmaxf(x0, 0.0f);
    y0 = fmaxf(y0, 0.0f);
    x1 = fminf(x1, (float)(c.W - 1));
    y1 = fminf(y1, (float)(c.H - 1));
    if (!(x0 <= x1) || !(y0 <= y1)) return false;
    tx0 = (int)x0 / tw; tx1 = (int)x1 / tw;
    ty0 = (int)y0 / th; ty1 = (int)y1 / th;
    return true;
}

// Per-pixel evaluation shared by the forward walk and the backward re-walk: both must
// take identical decisions, so both use these inlined sequences (explicit _rn
// intrinsics keep the compiler from contracting them differently in the two kernels).
__device__ __forceinline__ float eval_q(float pxf, float pyf, const float4 r0, const float4 r1, float &dx, float &dy)
{
    dx = __fsub_rn(__fsub_rn(pxf, r0.x), r0.z);
    dy = __fsub_rn(__fsub_rn(pyf, r0.y), r0.w);
    float y1 = __fmul_rn(dx, r1.x);
    float y2 = __fmul_rn(__fmaf_rn(-r1.y, dx, dy), r1.z);
    return __fmaf_rn(y1, y1, __fmul_rn(y2, y2));
}

// alpha = min(0.99, o exp(-q/2)); ao is the unclamped product.
__device__ __forceinline__ float eval_alpha(float q, float o, float &G, float &ao)
{
    G = __expf(__fmul_rn(-0.5f, q));
    ao = __fmul_rn(o, G);
    return fminf(kAlphaClamp, ao);
}

// Whether a Gaussian (centre r0, Cholesky-form conic and opacity r1) can take part at
// any pixel centre of the rectangle [x0, x1] x [y0, y1]: the minimum of
// q = (dx s1)^2 + ((dy - m dx) s2)^2 over the rectangle (on its boundary when the centre
// is outside; the edge minima in closed form) against min(9, 2 ln(255 o)), the bound
// beyond which alpha < 1/255, with margins above the binning's for float32 slack.  A
// false answer is exact: no pixel in the rectangle would accept the Gaussian.
__device__ __forceinline__ bool touches_rect(const float4 r0, const float4 r1, float x0, float x1, float y0, float y1)
{
    const float u = r0.x + r0.z, v = r0.y + r0.w;
    const float s1 = r1.x, m = r1.y, s2 = r1.z;
    const float dx0 = x0 - u, dx1 = x1 - u, dy0 = y0 - v, dy1 = y1 - v;
    float qmin = 0.f;
    if (!(dx0 <= 0.f && dx1 >= 0.f && dy0 <= 0.f && dy1 >= 0.f)) {
        auto qf = [&](float dx, float dy) {
            const float y1v = dx * s1, y2v = (dy - m * dx) * s2;
            return y1v * y1v + y2v * y2v;
        };
        const float s22 = s2 * s2;
        const float ax = s1 * s1 + m * m * s22;
        auto on_vertical = [&](float dx) { return qf(dx, fminf(fmaxf(m * dx, dy0), dy1)); };
        auto on_horizontal = [&](float dy) { return qf(fminf(fmaxf(m * s22 * dy / ax, dx0), dx1), dy); };
        qmin = fminf(fminf(on_vertical(dx0), on_vertical(dx1)), fminf(on_horizontal(dy0), on_horizontal(dy1)));
    }
    float qb = fminf(kQMax, 2.0f * logf(255.0f * r1.w));
    qb = fmaxf(qb, 0.0f) * 1.004f + 0.02f;
    return qmin <= qb;
}

// Sum 16 per-lane values over the warp with 16 shuffles (reduce-scatter): on return
// lane l holds the total of value index (l >> 1) & 15; lanes l and l ^ 1 agree.
__device__ __forceinline__ float warp_reduce16(const float (&v)[16], int lane)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float a[8], b[4], c2[2];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float send = b4 ? v[i] : v[i + 8], keep = b4 ? v[i + 8] : v[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float send = b3 ? a[i] : a[i + 4], keep = b3 ? a[i + 4] : a[i];
        b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        float send = b2 ? b[i] : b[i + 2], keep = b2 ? b[i + 2] : b[i];
        c2[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    float d = (b1 ? c2[1] : c2[0]) + __shfl_xor_sync(0xffffffffu, b1 ? c2[0] : c2[1], 2);
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    return d;
}

// Sum 10 per-lane values over the warp with 12 shuffles (a reduce-scatter that halves
// 10 -> 5 -> 3 -> 2 -> 1 values per lane on lane bits 4, 3, 2, 1, padding with zeros):
// on return lane l holds the total of value vidx10(l), or of a padding slot when
// vidx10(l) < 0; lanes l and l ^ 1 agree.
__device__ __forceinline__ int vidx10(int lane)
{
    const int b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1, b1 = (lane >> 1) & 1;
    const bool real = b3 ? b2 == 0 : !(b2 && b1);
    return real ? 5 * b4 + 3 * b3 + 2 * b2 + b1 : -1;
}
__device__ __forceinline__ float warp_reduce10(const float (&v)[10], int lane)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float a[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const float send = b4 ? v[i] : v[i + 5], keep = b4 ? v[i + 5] : v[i];
        a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    // a[0..4] of half b4; pad to 6: halves {0,1,2} and {3,4,-}
    float b[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float lo = a[i], hi = i + 3 < 5 ? a[i + 3] : 0.f;
        const float send = b3 ? lo : hi, keep = b3 ? hi : lo;
        b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    // b[0..2]; pad to 4: halves {0,1} and {2,-}
    float c[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float lo = b[i], hi = i + 2 < 3 ? b[i + 2] : 0.f;
        const float send = b2 ? lo : hi, keep = b2 ? hi : lo;
        c[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    float d = (b1 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, b1 ? c[0] : c[1], 2);
    d += __shfl_xor_sync(0xffffffffu, d, 1);
    return d;
}

// Top-K kept in registers, KM slots in descending weight.  Slots [0, KM - K) hold
// +inf sentinels so that a runtime K <= KM keeps exactly its K largest in slots
// [KM - K, KM).  The new entry goes after every kept entry of weight >= it (a strict
// comparison), and from there every entry moves back one slot, so among equal weights
// the earlier contributor (depth order) stays ahead, also for entries displaced by an
// insertion in front of them.
template <int KM>
struct TopK {
    float w[KM];
    int id[KM];
    __device__ __forceinline__ void init(int K)
    {
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            w[k] = (k < KM - K) ? __int_as_float(0x7f800000) : -1.0f;
            id[k] = -1;
        }
    }
    __device__ __forceinline__ void insert(float nw, int nid)
    {
        if (!(nw > w[KM - 1])) return;
        bool shift = false;
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            const bool sw = shift || nw > w[k];
            shift = sw;
            float tw = sw ? nw : w[k];
            int ti = sw ? nid : id[k];
            nw = sw ? w[k] : nw;
            nid = sw ? id[k] : nid;
            w[k] = tw;
            id[k] = ti;
        }
    }
};

// The same Top-K kept in shared memory, slot-major ([slot][thread], B threads), so the
// per-thread registers drop by 2 KM; the smallest kept weight stays in a register for the
// early rejection.  Insertion from the tail: the new entry goes after every kept entry of
// weight >= it -- the position the register network gives -- so both hold identical sets
// in identical order.
template <int KM, int B>
struct TopKShared {
    float *w;
    int *id;
    float wmin;
    __device__ __forceinline__ void init(float *sw, int *sid, int tid, int K)
    {
        w = sw + tid;
        id = sid + tid;
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            w[k * B] = (k < KM - K) ? __int_as_float(0x7f800000) : -1.0f;
            id[k * B] = -1;
        }
        wmin = -1.0f;
    }
    __device__ __forceinline__ void insert(float nw, int nid)
    {
        if (!(nw > wmin)) return;
        int pos = KM - 1;
        while (pos > 0) {
            const float prev = w[(pos - 1) * B];
            if (!(nw > prev)) break;
            w[pos * B] = prev;
            id[pos * B] = id[(pos - 1) * B];
            --pos;
        }
        w[pos * B] = nw;
        id[pos * B] = nid;
        wmin = w[(KM - 1) * B];
    }
};

// ------------------------------------------------------------------------------------
// Workspace layout (host-computed; all offsets 256-byte aligned)
// ------------------------------------------------------------------------------------
constexpr int kHdrWalkTiles = 16;   // header word: next tile of the persistent re-walk
constexpr int kHdrN1 = 4;           // header word: instances in front of the depth cut (first sort)
constexpr int kHdrN2 = 5;           // header word: instances of unsaturated tiles behind it (second sort)
constexpr int kHdrIncomplete = 6;   // header word: tiles the first walk left unsaturated with a cut
constexpr int kHdrCutSig = 7;       // header word: the tile grid the recorded cuts belong to
constexpr int kCutLevels = 13;      // sparse-table levels over tile rows (a camera has at most 4096)
constexpr int kHdrFresh = 10;       // header word: slots the completion pass gave elements the first had none for
constexpr uint32_t kNoCut = 0xffffffffu;
constexpr float kCutMargin = 1.0625f;   // recorded cut = depth where the tile saturated x this
constexpr int kHdrWaitLimitByte = 96;   // header bytes [96, 104): bound of the pipeline waits (0: default)

// Kernel timers (gs_timer_*): a scope that brackets the launches it encloses with a CUDA
// event pair on `s`, when timing is enabled and `s` is not capturing.
struct TimerScope {
    TimerScope(int id, cudaStream_t s);
    ~TimerScope();
    int id;
    cudaStream_t s;
    bool on;
};

struct WsLayout {
    size_t header;             // 256 B: [0] error word, [1] instance count, [2] pieces, [3] multi-piece
                               // segments, [4] / [5] instances of the first / second tile sort,
                               // [6] incomplete tiles, [7] cut grid signature, [8] partial rows,
                               // [9] pairs, [10] fresh completion slots, [16] re-walk tile counter,
                               // [24..25] the wait limit (64-bit, SM cycles, 0 = default)
    size_t depth_keys[2], depth_vals[2];   // NE
    size_t elem_cnt;           // NE (tiles touched, per element)
    size_t elem_off;           // NE (first pre-sort instance of each element)
    size_t counts;             // NE (counts in depth order, scanned in place)
    size_t counts1;            // NE (per element: instances of the first, then the second tile sort)
    size_t inst_keys[2], inst_vals[2];     // Mcap
    size_t inst_elem;          // Mcap
    size_t tile_range;         // n_tiles x int2: each tile's run in the first sorted instances
    size_t tile_range2;        // n_tiles x int2: its run in the second (empty unless completed)
    size_t cut_store;          // n_tiles: the depth-cut keys recorded for the next render
    size_t cut_cur;            // n_tiles: the cut keys this render bins with (kNoCut: none)
    size_t tile_incomplete;    // n_tiles: 1 where the first walk ended unsaturated with a cut
    size_t tile_sat;           // n_tiles: per camera, 2D prefix sums of tile_incomplete
    size_t cut_rowmin, cut_rowmax;   // per tile row: the smallest and largest current cut key
    size_t cut_rowmax_st;      // kCutLevels x n_rows: range maxima of cut_rowmax over 2^l rows (per camera)
    size_t sort_hist;          // (kRadixBlocks + 1) x 256
    size_t scan_aux;           // scan block sums
    size_t inst_grad;          // Mcap x kGradVals floats (per-instance partial 2D gradients)
    size_t inst_walked;        // Mcap bytes: 1 where the re-walk wrote the instance's partials
    size_t elem_grad;          // NE x kGradVals floats (per-element sums of the instance partials)
    size_t pose_part;          // NE x 12 floats (per-element partial pose gradients)
    size_t pair_keys[2], pair_vals[2];     // N + P K
    size_t hbuf;               // P K floats: dL/dF_p . f_{idx_k}
    size_t seg_start, seg_end; // N each
    size_t pieces, piece_off;  // N each
    size_t multi, multi_off;   // N each
    size_t mflag, mlist;       // N each: ranks with a multi-piece segment (flag scan, compact list)
    size_t piece_rank;         // max_pieces_rows
    size_t piece_rows;         // max_multi_rows x D floats
    size_t loss_part;          // unused (the loss takes caller scratch)
    size_t tile_keys;          // n_fgblocks x B K uint2 slot records (pixel | run << 16, w') in sorted order
    size_t tile_runs;          // n_fgblocks x runs_stride uint2 run tables (first position, Gaussian id)
    size_t tile_u, tile_rowbase; // n_tiles each
    size_t tile_rows;          // rows_cap x D floats: partial feature-gradient rows per (tile, Gaussian)
    size_t total;
    int inst_sorted;           // buffer (0/1) holding the tile-sorted instances
    int pair_sorted;           // buffer (0/1) holding the sorted feature-gradient pairs
    int pair_bits;

    long long NE, P, PK, Mcap, n_pairs, max_multi_rows;
    long long rows_cap, max_pieces_rows;
    bool use_tiles;
    bool depth_cut;
    uint32_t cut_sig;
    long long n_fgblocks;      // feature-gradient pixel blocks (fg_block_shape) over all cameras
    int N, K, D, n_tiles, n_cams;
};

// The binned list of every tile: its run in the first sorted instances, then (for a
// tile the depth cut left unsaturated) its run in the second -- together the tile's
// instances in depth order.  Values are instance indices (inst_elem, partials).
struct TileLists {
    const uint32_t *v1, *v2;
    const int2 *r1, *r2;
};
struct TileList {
    const uint32_t *v1, *v2;
    int s1, n1, s2, n;
    __device__ __forceinline__ TileList(const TileLists &tl, int tile, bool empty)
    {
        const int2 a = tl.r1[tile], b = tl.r2[tile];
        v1 = tl.v1;
        v2 = tl.v2;
        s1 = a.x;
        s2 = b.x;
        n1 = empty ? 0 : a.y - a.x;
        n = empty ? 0 : n1 + (b.y - b.x);
    }
    __device__ __forceinline__ uint32_t at(int m) const { return m < n1 ? v1[s1 + m] : v2[s2 + (m - n1)]; }
};
// The first sort's pairs are in instance buffer L.inst_sorted, the second's in the other.
TileLists tile_lists(const WsLayout &L, void *ws);
// The forward walk's part in the depth cut (k_walk_fwd).
struct WalkCut {
    int phase;                 // 1: first walk of every tile; 2: the flagged tiles over their whole list
    const uint32_t *cut_cur;   // the cut keys this render binned with
    uint32_t *cut_store;       // the cut keys recorded for the next render
    uint32_t *incomplete;      // per tile: flagged by phase 1
    uint32_t *hdr;             // workspace header (the flagged-tile count)
};

// The argument rules every entry point applies to a gs_config (K, D, tile shape, dtype).
bool cfg_ok(const gs_config *cfg);
bool make_layout(const gs_config *cfg, const gs_camera *cams, int n_cams, int N, WsLayout &L);
bool make_camtable(const gs_config *cfg, const gs_camera *cams, int n_cams, CamTable &ct);
int bits_for(long long v);
inline int sorted_buffer(int n_bits) { return ((n_bits + 7) / 8) & 1; }

template <typename T>
__host__ __device__ __forceinline__ T *ws_ptr(void *ws, size_t off) { return (T *)((char *)ws + off); }

// ------------------------------------------------------------------------------------
// Host-side launchers implemented in the .cu files
// ------------------------------------------------------------------------------------
bool launch_vanilla(int dtype, const CamTable &ct, const WsLayout &L, int N, const float *proj, void *ws,
                    const void *feats, void *F, cudaStream_t s);
bool launch_loss_geo(long long n_pix, const float *C, const float *Cgt, const float *Dp, const float *Dgt, float wc,
                     float wd, float *dLdC, float *dLdD, float *loss, float *part, cudaStream_t s);
struct AdamTensor {
    float *param;
    const float *grad;
    float *m, *v;
    long long n;
    float lr;
    __nv_bfloat16 *pb;         // optional bf16 copy of param (nullptr: none)
};
constexpr int kAdamMaxTensors = 16;
bool launch_adam(const AdamTensor *t, int n_tensors, int step, float beta1, float beta2, float eps, cudaStream_t s);
bool launch_prune_stats(const CamTable &ct, const WsLayout &L, int N, const float *proj, const int *topk_idx,
                        void *ws, int *count, float *S, cudaStream_t s);
size_t prune_select_ws(int N);
bool launch_prune_select(int N, const int *count, const float *S, int tau, double ratio, const float *expo,
                         uint8_t *keep, void *ws, cudaStream_t s);
// LSD radix sort of (key, value) uint32 pairs on key bits [0, n_bits); stable.  The
// element count is n_host, or *n_dev clamped to n_host if n_dev is non-null.
// vals_are_index: the input values are the positions 0, 1, 2, ... (vals0 is not read).
// The arrays start 16-byte aligned.  Returns the index (0/1) of the buffer pair holding
// the sorted result.
int radix_sort_pairs(uint32_t *keys0, uint32_t *keys1, uint32_t *vals0, uint32_t *vals1,
                     long long n_host, const uint32_t *n_dev, int n_bits, uint32_t *hist,
                     cudaStream_t s, bool vals_are_index = false);
// Exclusive scan of n uint32 in -> out (may alias); *total (device) = sum if non-null.
// run_if (optional, device): when it points to zero every launch returns at once and
// neither out nor *total is written (the caller keeps them valid for that case).
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, long long n, uint32_t *total,
                        uint32_t *aux, cudaStream_t s, const uint32_t *run_if = nullptr);

void launch_preprocess(const CamTable &ct, int N, const float *mean3d, const float *cov3d, const float *opac,
                       const float *rgb, float *proj, cudaStream_t s);
void launch_project_backward(const CamTable &ct, int N, const float *mean3d, const float *cov3d, const float *proj,
                             const uint32_t *elem_off, const uint32_t *elem_cnt, const float *inst_grad, const uint8_t *walked,
                             float *elem_grad, const int *err, const gs_grads *gr, float *pose_part, cudaStream_t s);
void launch_bin_sort(const CamTable &ct, const WsLayout &L, int N, const float *proj, void *ws, cudaStream_t s);
void launch_complete_lists(const CamTable &ct, const WsLayout &L, int N, const float *proj, void *ws,
                           cudaStream_t s);
// kbuf: where the walk keeps each pixel's Top-K (gs_config.topk_layout): 0 registers,
// 1 shared memory (KM <= 16); identical results.
bool launch_walk_fwd(const CamTable &ct, const WsLayout &L, int K, int kbuf, int N, const float *proj, void *ws,
                     float *rgb_out, float *depth_out, float *T_out, int *n_out, int *idx_out, float *w_out,
                     int phase, cudaStream_t s);
bool launch_walk_bwd(const CamTable &ct, const WsLayout &L, int K, int N, const float *proj, void *ws,
                     const float *rgb_out, const float *depth_out, const int *topk_idx, const float *topk_w,
                     const float *dLdC, const float *dLdD, bool with_feature, cudaStream_t s);
// Gather-blend (a4); bf16 rows with K in {2, 4, 8, 16}, D a multiple of 64 and fewer than
// 2^24 Gaussians take the tensor-core form (gs_blend_mma.cu), the rest the CUDA-core forms.
bool launch_blend(int dtype, int K, int D, long long n_pix, long long N, const int *idx, const float *w,
                  const void *feats, void *F, const int *err, cudaStream_t s);
bool blend_mma_supported(int dtype, int K, int D, long long N);
bool launch_blend_mma(int K, int D, long long n_pix, const int *idx, const float *w, const void *feats, void *F,
                      const int *err, cudaStream_t s);
bool launch_blend_loss_mma(int K, int D, long long n_pix, const int *idx, const float *w, const void *feats,
                           const void *Fgt, const float *C, const float *Cgt, const float *Dp, const float *Dgt,
                           float wf, float wc, float wd, float invP, void *F, void *dLdF, float *dLdC, float *dLdD,
                           float *part, float *h, const int *err, cudaStream_t s);
bool launch_feature_h(const WsLayout &L, int dtype, const int *topk_idx, const void *feats, const void *dLdF,
                      void *ws, cudaStream_t s);
// hold / hold_ev (both or neither): the stream of the re-walk, made to wait (through
// hold_ev) for the block records before the CUDA-core block product is queued on s
bool launch_feature_grad(const CamTable &ct, const WsLayout &L, int dtype, int N, const int *topk_idx,
                         const float *topk_w, const void *dLdF, float *grad_feat, void *ws, cudaStream_t s,
                         cudaStream_t hold = nullptr, cudaEvent_t hold_ev = nullptr);
bool tile_grad_supported(int dtype, int D, int K);
// Feature-gradient pixel blocks: the largest of 8x8, 8x4, 4x4 whose dL/dF rows fit one
// 64 KB shared-memory stage ({0, 0}: none).
struct FgBlock {
    int bw, bh;
};
FgBlock fg_block_shape(int dtype, int D, int K);
size_t tile_runs_bytes(int B, int K);
void retile(const CamTable &ct, int bw, int bh, CamTable &out);
bool launch_h(int dtype, int K, int D, long long n_pix, long long N, const int *idx, const void *feats,
              const void *dLdF, float *h, const int *err, cudaStream_t s);
bool launch_h_mma(int K, int D, long long n_pix, const int *idx, const void *feats, const void *dLdF, float *h,
                  const int *err, cudaStream_t s);
// The fused training form also writes h = dL/dF . f per Top-K slot (into `h`) when it
// takes the pixel-group path; blend_loss_writes_h says whether it does.
bool blend_loss_writes_h(int dtype, int K, int D, long long N);
bool launch_blend_loss(const CamTable &ct, int dtype, int K, int D, long long n_pix, long long N, const int *idx,
                       const float *w, const void *feats, const void *Fgt, const float *C, const float *Cgt,
                       const float *Dp, const float *Dgt, float wf, float wc, float wd, void *F, void *dLdF,
                       float *dLdC, float *dLdD, float *loss, float *part, float *h, const int *err, cudaStream_t s);
bool launch_loss(int dtype, int D, long long n_pix, const void *F, const void *Fgt, const float *C, const float *Cgt,
                 const float *Dp, const float *Dgt, float wf, float wc, float wd, void *dLdF, float *dLdC,
                 float *dLdD, float *loss, float *part, cudaStream_t s);

}  // namespace gs
