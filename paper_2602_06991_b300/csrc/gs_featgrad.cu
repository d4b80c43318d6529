// gs_featgrad.cu -- feature part of a5: dL/df_g = sum over (pixel p, slot k) with
// idx_k(p) = g of w'_k(p) dL/dF_p, plus h_k(p) = dL/dF_p . f_g for the re-walk.
//
// This is a transposed sparse product (P x N with K entries per row)^T (P x D).  It is
// done without atomics:
//   1. Gaussians are ranked by the 3D Morton code of their mean, so Gaussians that are
//      processed together cover neighbouring pixels in every view and the dL/dF rows
//      they read stay in L2;
//   2. the (pixel, slot) pairs are sorted by that rank (own radix sort).  Each rank also
//      gets one marker entry, placed first in its segment by the stable sort, so every
//      Gaussian -- selected or not -- has a segment and gets its row written;
//   3. segments are cut into pieces of at most kPieceLen pairs (load balance: a large
//      near Gaussian can be selected by thousands of pixels); one warp reduces one piece
//      in registers, loading the Gaussian's own row once and each pixel's dL/dF row
//      once with 16-byte loads;
//   4. single-piece Gaussians write their gradient row directly; multi-piece ones write
//      piece rows that a fix-up pass sums in a fixed order.
#include "gs_internal.cuh"

namespace gs {

__device__ __forceinline__ int f2ord(float f)
{
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}

__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_bbox_init(int *bb)
{
    if (threadIdx.x < 3) bb[threadIdx.x] = 0x7fffffff;
    else if (threadIdx.x < 6) bb[threadIdx.x] = (int)0x80000000;
}

__global__ void __launch_bounds__(256) k_bbox(int N, const float *__restrict__ mean3d, int *bb)
{
    int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff}, hi[3] = {(int)0x80000000, (int)0x80000000, (int)0x80000000};
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < N; g += gridDim.x * blockDim.x)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int v = f2ord(mean3d[3 * (size_t)g + a]);
            lo[a] = min(lo[a], v);
            hi[a] = max(hi[a], v);
        }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(bb + a, lo[a]);      // min/max are order independent: deterministic
            atomicMax(bb + 3 + a, hi[a]);
        }
}

__device__ __forceinline__ uint32_t spread3(uint32_t x)   // 10 bits -> every third bit
{
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void k_morton(int N, const float *__restrict__ mean3d, const int *bb, uint32_t *keys, uint32_t *vals)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    uint32_t code = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float lo = ord2f(bb[a]), hi = ord2f(bb[3 + a]);
        float ext = hi - lo;
        float t = ext > 0.f ? (mean3d[3 * (size_t)g + a] - lo) / ext : 0.f;
        uint32_t qv = (uint32_t)fminf(fmaxf(t * 1023.f, 0.f), 1023.f);
        code |= spread3(qv) << a;
    }
    keys[g] = code;
    vals[g] = (uint32_t)g;
}

__global__ void k_rank_scatter(int N, const uint32_t *__restrict__ order, uint32_t *grank)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < N) grank[order[r]] = (uint32_t)r;
}

constexpr uint32_t kMarker = 0xffffffffu;

__global__ void k_pairs(int N, int K, long long PK, const int *__restrict__ topk_idx,
                        const float *__restrict__ topk_w, const uint32_t *__restrict__ grank, uint32_t *keys,
                        uint32_t *vals, float *wnorm)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        keys[i] = (uint32_t)i;
        vals[i] = kMarker;
    } else if (i < N + PK) {
        long long s = i - N;
        int id = topk_idx[s];
        keys[i] = id >= 0 ? grank[id] : (uint32_t)N;
        vals[i] = (uint32_t)s;
        // renormalised weight w / S (Eq. 3), summed in slot order as the blend does
        long long p = s / K;
        float S = 0.f;
        for (int k = 0; k < K; ++k) S += topk_w[p * K + k];
        wnorm[s] = S > 0.f ? topk_w[s] * (1.f / S) : 0.f;
    }
}

__global__ void k_segments(int N, long long n_host, const uint32_t *n_dev, const uint32_t *__restrict__ keys,
                           const uint32_t *__restrict__ vals, uint32_t *seg_start, uint32_t *seg_end)
{
    long long n_pairs = n_dev ? min((long long)*n_dev, n_host) : n_host;
    long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_pairs) return;
    uint32_t k = keys[m];
    if (k >= (uint32_t)N) return;
    if (vals[m] == kMarker) seg_start[k] = (uint32_t)(m + 1);
    if (m + 1 == n_pairs || keys[m + 1] != k) seg_end[k] = (uint32_t)(m + 1);
}

// Row mode: one marker entry per Gaussian id, then the pair count N + U_tot.
__global__ void k_markers(int N, uint32_t *keys, uint32_t *vals)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        keys[i] = (uint32_t)i;
        vals[i] = kMarker;
    }
}

// Pairs to sort: the N markers and one per partial row.  When the rows overflowed their
// capacity (or any earlier stage failed) no row is trusted: only the markers are sorted,
// the feature gradient comes out zero and the error word reports the overflow.
__global__ void k_pair_count(int N, const uint32_t *u_tot, uint32_t rows_cap, const int *err, uint32_t *n_pairs)
{
    const bool ok = *err == 0 && *u_tot <= rows_cap;
    *n_pairs = (uint32_t)N + (ok ? *u_tot : 0u);
}

__global__ void k_pieces(int N, const uint32_t *__restrict__ seg_start, const uint32_t *__restrict__ seg_end,
                         uint32_t *pieces, uint32_t *multi)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    uint32_t n = seg_end[r] - seg_start[r];
    uint32_t pc = n == 0 ? 1u : (n + kPieceLen - 1) / kPieceLen;
    pieces[r] = pc;
    multi[r] = pc > 1 ? pc : 0u;
}

__global__ void k_piece_rank(int N, const uint32_t *__restrict__ pieces, const uint32_t *__restrict__ piece_off,
                             const uint32_t *__restrict__ multi, const uint32_t *__restrict__ mflag_off,
                             uint32_t *piece_rank, uint32_t *mlist)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    uint32_t o = piece_off[r], n = pieces[r];
    for (uint32_t j = 0; j < n; ++j) piece_rank[o + j] = (uint32_t)r;
    if (multi[r] > 0) mlist[mflag_off[r]] = (uint32_t)r;
}

__global__ void k_multi_flags(int N, const uint32_t *__restrict__ multi, uint32_t *mflag)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < N) mflag[r] = multi[r] > 0 ? 1u : 0u;
}

template <bool BF16>
struct Row;

template <>
struct Row<false> {
    static constexpr int VEC = 4;
    __device__ __forceinline__ static void load(const void *base, size_t chunk, float (&x)[4])
    {
        float4 v = __ldg((const float4 *)base + chunk);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
};

template <>
struct Row<true> {
    static constexpr int VEC = 8;
    __device__ __forceinline__ static void load(const void *base, size_t chunk, float (&x)[8])
    {
        uint4 v = __ldg((const uint4 *)base + chunk);
        const __nv_bfloat162 *h = (const __nv_bfloat162 *)&v;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 f = __bfloat1622float2(h[i]);
            x[2 * i] = f.x;
            x[2 * i + 1] = f.y;
        }
    }
};

// One warp per piece.  CPL = 16-byte chunks per lane (row has nch <= 32 CPL chunks).
// Four pairs are in flight at a time: their dL/dF chunks are loaded together, then
// accumulated, and their four dot products with the Gaussian's own row are reduced with
// one reduce-scatter (6 shuffles for 4 dots).
template <bool BF16, int CPL, bool ROWS>
__global__ void __launch_bounds__(256) k_fgrad_main(int K, int nch, const uint32_t *__restrict__ n_pieces_dev,
                                                    const uint32_t *__restrict__ piece_rank,
                                                    const uint32_t *__restrict__ piece_off,
                                                    const uint32_t *__restrict__ pieces,
                                                    const uint32_t *__restrict__ multi_off,
                                                    const uint32_t *__restrict__ seg_start,
                                                    const uint32_t *__restrict__ seg_end,
                                                    const uint32_t *__restrict__ order,
                                                    const uint32_t *__restrict__ pair_vals,
                                                    const float *__restrict__ wnorm, const void *__restrict__ feats,
                                                    const void *__restrict__ dLdF, float *__restrict__ hbuf,
                                                    float *__restrict__ grad_f, float *__restrict__ piece_rows)
{
    // ROWS: the pairs point at float32 partial rows (one per (tile, Gaussian)), the
    // weight is 1 and no dot products are formed; ranks are Gaussian ids (order unused).
    using Rw = Row<BF16 && !ROWS>;
    constexpr int VEC = Rw::VEC;
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const long long pc = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (pc >= (long long)*n_pieces_dev) return;
    const uint32_t r = piece_rank[pc];
    const uint32_t j = (uint32_t)pc - piece_off[r];
    const uint32_t g = ROWS ? r : order[r];
    const uint32_t m0 = seg_start[r] + j * kPieceLen;
    const uint32_t m1 = min(m0 + kPieceLen, seg_end[r]);
    float f[CPL][VEC], acc[CPL][VEC];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        int ch = lane + 32 * c;
#pragma unroll
        for (int i = 0; i < VEC; ++i) { f[c][i] = 0.f; acc[c][i] = 0.f; }
        if (!ROWS && ch < nch && m1 > m0) Rw::load(feats, (size_t)g * nch + ch, f[c]);   // unselected: zero row only
    }
    uint32_t m = m0;
    for (; m + U <= m1; m += U) {
        uint32_t sv[U], pv[U];
        float wp[U], dot[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            sv[u] = pair_vals[m + u];
            pv[u] = ROWS ? sv[u] : sv[u] / (uint32_t)K;
            wp[u] = ROWS ? 1.f : __ldg(wnorm + sv[u]);
            dot[u] = 0.f;
        }
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            int ch = lane + 32 * c;
            if (ch < nch) {
                float x[U][VEC];
#pragma unroll
                for (int u = 0; u < U; ++u) Rw::load(dLdF, (size_t)pv[u] * nch + ch, x[u]);
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int i = 0; i < VEC; ++i) {
                        acc[c][i] = fmaf(wp[u], x[u][i], acc[c][i]);
                        dot[u] = fmaf(x[u][i], f[c][i], dot[u]);
                    }
            }
        }
        if (ROWS) continue;
        // reduce-scatter of 4 dots: lane l ends with dot (l >> 3) & 3 (lanes 0, 8, 16, 24)
        const bool b4 = lane & 16, b3 = lane & 8;
        float a0 = (b4 ? dot[2] : dot[0]) + __shfl_xor_sync(0xffffffffu, b4 ? dot[0] : dot[2], 16);
        float a1 = (b4 ? dot[3] : dot[1]) + __shfl_xor_sync(0xffffffffu, b4 ? dot[1] : dot[3], 16);
        float d = (b3 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, b3 ? a0 : a1, 8);
        d += __shfl_xor_sync(0xffffffffu, d, 4);
        d += __shfl_xor_sync(0xffffffffu, d, 2);
        d += __shfl_xor_sync(0xffffffffu, d, 1);
        if ((lane & 7) == 0) hbuf[sv[(lane >> 3) & 3]] = d;
    }
    for (; m < m1; ++m) {
        const uint32_t sv = pair_vals[m];
        const uint32_t pv = ROWS ? sv : sv / (uint32_t)K;
        const float wp = ROWS ? 1.f : __ldg(wnorm + sv);
        float dot = 0.f;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            int ch = lane + 32 * c;
            if (ch < nch) {
                float x[VEC];
                Rw::load(dLdF, (size_t)pv * nch + ch, x);
#pragma unroll
                for (int i = 0; i < VEC; ++i) {
                    acc[c][i] = fmaf(wp, x[i], acc[c][i]);
                    dot = fmaf(x[i], f[c][i], dot);
                }
            }
        }
        if (ROWS) continue;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (lane == 0) hbuf[sv] = dot;
    }
    float *dst = pieces[r] == 1 ? grad_f + (size_t)g * nch * VEC
                                : piece_rows + (size_t)(multi_off[r] + j) * nch * VEC;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        int ch = lane + 32 * c;
        if (ch < nch) {
            float4 *d4 = (float4 *)(dst + (size_t)ch * VEC);
#pragma unroll
            for (int i = 0; i < VEC / 4; ++i)
                d4[i] = make_float4(acc[c][4 * i], acc[c][4 * i + 1], acc[c][4 * i + 2], acc[c][4 * i + 3]);
        }
    }
}

// Gaussians whose segment was cut into several pieces: one CTA per such Gaussian (from
// the compact list).  Its 1024 threads are 8 row groups x 128 float4 columns; each
// group sums every 8th piece row with two accumulators, and the 8 group sums are
// combined in shared memory in a fixed order -- deterministic, and a Gaussian selected
// by most of the frame (thousands of piece rows) is summed 8 ways in parallel.
constexpr int kFixCols = 128, kFixGroups = 8;
__global__ void __launch_bounds__(kFixCols *kFixGroups) k_fgrad_fixup(int D4, const uint32_t *__restrict__ n_multi_dev,
                                                                      const uint32_t *__restrict__ mlist,
                                                                      const uint32_t *__restrict__ multi,
                                                                      const uint32_t *__restrict__ multi_off,
                                                                      const uint32_t *__restrict__ order,
                                                                      const float4 *__restrict__ piece_rows,
                                                                      float4 *__restrict__ grad_f)
{
    __shared__ float4 part[kFixGroups][kFixCols];
    const int col = threadIdx.x % kFixCols, grp = threadIdx.x / kFixCols;
    const uint32_t n_multi = *n_multi_dev;
    for (uint32_t i = blockIdx.x; i < n_multi; i += gridDim.x) {
        const uint32_t r = mlist[i];
        const uint32_t n = multi[r], base = multi_off[r], g = order ? order[r] : r;
        for (int c0 = 0; c0 < D4; c0 += kFixCols) {
            const int c = c0 + col;
            float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
            if (c < D4) {
                uint32_t k = grp;
                for (; k + kFixGroups < n; k += 2 * kFixGroups) {
                    float4 v = __ldg(piece_rows + (size_t)(base + k) * D4 + c);
                    float4 w = __ldg(piece_rows + (size_t)(base + k + kFixGroups) * D4 + c);
                    a0.x += v.x; a0.y += v.y; a0.z += v.z; a0.w += v.w;
                    a1.x += w.x; a1.y += w.y; a1.z += w.z; a1.w += w.w;
                }
                if (k < n) {
                    float4 v = __ldg(piece_rows + (size_t)(base + k) * D4 + c);
                    a0.x += v.x; a0.y += v.y; a0.z += v.z; a0.w += v.w;
                }
            }
            part[grp][col] = make_float4(a0.x + a1.x, a0.y + a1.y, a0.z + a1.z, a0.w + a1.w);
            __syncthreads();
            if (grp == 0 && c < D4) {
                float4 t = part[0][col];
#pragma unroll
                for (int q = 1; q < kFixGroups; ++q) {
                    float4 v = part[q][col];
                    t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w;
                }
                grad_f[(size_t)g * D4 + c] = t;
            }
            __syncthreads();
        }
    }
}

template <bool BF16, bool ROWS>
static bool fgrad_main(int cpl, unsigned blocks, cudaStream_t s, int K, int nch, const uint32_t *np,
                       const uint32_t *pr, const uint32_t *po, const uint32_t *pcs, const uint32_t *mo,
                       const uint32_t *ss, const uint32_t *se, const uint32_t *ord, const uint32_t *pv,
                       const float *wn, const void *feats, const void *dLdF, float *h, float *gf, float *rows)
{
    switch (cpl) {
    case 1: k_fgrad_main<BF16, 1, ROWS><<<blocks, 256, 0, s>>>(K, nch, np, pr, po, pcs, mo, ss, se, ord, pv, wn, feats, dLdF, h, gf, rows); return true;
    case 2: k_fgrad_main<BF16, 2, ROWS><<<blocks, 256, 0, s>>>(K, nch, np, pr, po, pcs, mo, ss, se, ord, pv, wn, feats, dLdF, h, gf, rows); return true;
    case 4: k_fgrad_main<BF16, 4, ROWS><<<blocks, 256, 0, s>>>(K, nch, np, pr, po, pcs, mo, ss, se, ord, pv, wn, feats, dLdF, h, gf, rows); return true;
    case 8: k_fgrad_main<BF16, 8, ROWS><<<blocks, 256, 0, s>>>(K, nch, np, pr, po, pcs, mo, ss, se, ord, pv, wn, feats, dLdF, h, gf, rows); return true;
    }
    return false;
}

static int cpl_for(int nch) { return nch <= 32 ? 1 : nch <= 64 ? 2 : nch <= 128 ? 4 : 8; }

bool launch_tile_grad(const CamTable &ct, const WsLayout &L, int dtype, const int *topk_idx, const float *topk_w,
                      const void *dLdF, void *ws, cudaStream_t s);

// Tile-major path: T1-T3 in gs_tilegrad.cu, then the per-Gaussian reduction of the
// partial rows (row mode of the segmented reduction).
static bool feature_grad_tiles(const CamTable &ct, const WsLayout &L, int dtype, int N, const int *topk_idx,
                               const float *topk_w, const void *feats, const void *dLdF, float *grad_feat, void *ws,
                               cudaStream_t s)
{
    uint32_t *hdr = ws_ptr<uint32_t>(ws, L.header);
    uint32_t *n_pieces = hdr + 2, *n_multi = hdr + 3, *u_tot = hdr + 8, *n_pairs_dev = hdr + 9;
    uint32_t *hist = ws_ptr<uint32_t>(ws, L.sort_hist);
    uint32_t *aux = ws_ptr<uint32_t>(ws, L.scan_aux);
    uint32_t *pk[2] = {ws_ptr<uint32_t>(ws, L.pair_keys[0]), ws_ptr<uint32_t>(ws, L.pair_keys[1])};
    uint32_t *pv[2] = {ws_ptr<uint32_t>(ws, L.pair_vals[0]), ws_ptr<uint32_t>(ws, L.pair_vals[1])};
    uint32_t *seg_start = ws_ptr<uint32_t>(ws, L.seg_start), *seg_end = ws_ptr<uint32_t>(ws, L.seg_end);
    uint32_t *pieces = ws_ptr<uint32_t>(ws, L.pieces), *piece_off = ws_ptr<uint32_t>(ws, L.piece_off);
    uint32_t *multi = ws_ptr<uint32_t>(ws, L.multi), *multi_off = ws_ptr<uint32_t>(ws, L.multi_off);
    uint32_t *mflag = ws_ptr<uint32_t>(ws, L.mflag), *mlist = ws_ptr<uint32_t>(ws, L.mlist);
    uint32_t *piece_rank = ws_ptr<uint32_t>(ws, L.piece_rank);
    float *prow = ws_ptr<float>(ws, L.piece_rows);
    float *trows = ws_ptr<float>(ws, L.tile_rows);
    const unsigned nbN = (unsigned)((N + 255) / 256);

    // h = dL/dF . f per slot for the re-walk, then the per-block partial rows
    if (!launch_h(dtype, L.K, L.D, L.P, topk_idx, feats, dLdF, ws_ptr<float>(ws, L.hbuf), (const int *)hdr, s))
        return false;
    if (!launch_tile_grad(ct, L, dtype, topk_idx, topk_w, dLdF, ws, s)) return false;
    k_markers<<<nbN, 256, 0, s>>>(N, pk[0], pv[0]);
    k_pair_count<<<1, 1, 0, s>>>(N, u_tot, (uint32_t)L.rows_cap, (const int *)hdr, n_pairs_dev);
    const long long n_host = N + L.rows_cap;
    int pcur = radix_sort_pairs(pk[0], pk[1], pv[0], pv[1], n_host, n_pairs_dev, L.pair_bits, hist, s);
    k_segments<<<(unsigned)((n_host + 255) / 256), 256, 0, s>>>(N, n_host, n_pairs_dev, pk[pcur], pv[pcur], seg_start,
                                                                seg_end);
    k_pieces<<<nbN, 256, 0, s>>>(N, seg_start, seg_end, pieces, multi);
    exclusive_scan_u32(pieces, piece_off, N, n_pieces, aux, s);
    exclusive_scan_u32(multi, multi_off, N, nullptr, aux, s);
    k_multi_flags<<<nbN, 256, 0, s>>>(N, multi, mflag);
    exclusive_scan_u32(mflag, mflag, N, n_multi, aux, s);
    k_piece_rank<<<nbN, 256, 0, s>>>(N, pieces, piece_off, multi, mflag, piece_rank, mlist);
    const int nch = L.D / 4;
    unsigned blocks = (unsigned)((L.max_pieces_rows * 32 + 255) / 256);
    if (!fgrad_main<false, true>(cpl_for(nch), blocks, s, L.K, nch, n_pieces, piece_rank, piece_off, pieces,
                                 multi_off, seg_start, seg_end, nullptr, pv[pcur], nullptr, nullptr, trows, nullptr,
                                 grad_feat, prow))
        return false;
    k_fgrad_fixup<<<148 * 2, kFixCols * kFixGroups, 0, s>>>(L.D / 4, n_multi, mlist, multi, multi_off, nullptr,
                                                            (const float4 *)prow, (float4 *)grad_feat);
    return true;
}

bool launch_feature_grad(const CamTable &ct, const WsLayout &L, int dtype, int N, const float *mean3d,
                         const int *topk_idx, const float *topk_w, const void *feats, const void *dLdF,
                         float *grad_feat, void *ws, cudaStream_t s)
{
    if (L.use_tiles)
        return feature_grad_tiles(ct, L, dtype, N, topk_idx, topk_w, feats, dLdF, grad_feat, ws, s);
    uint32_t *hdr = ws_ptr<uint32_t>(ws, L.header);
    uint32_t *n_pieces = hdr + 2;
    uint32_t *n_multi = hdr + 3;
    int *bb = (int *)(hdr + 4);
    uint32_t *hist = ws_ptr<uint32_t>(ws, L.sort_hist);
    uint32_t *aux = ws_ptr<uint32_t>(ws, L.scan_aux);
    uint32_t *rk[2] = {ws_ptr<uint32_t>(ws, L.rank_keys[0]), ws_ptr<uint32_t>(ws, L.rank_keys[1])};
    uint32_t *rv[2] = {ws_ptr<uint32_t>(ws, L.rank_vals[0]), ws_ptr<uint32_t>(ws, L.rank_vals[1])};
    uint32_t *grank = ws_ptr<uint32_t>(ws, L.grank);
    uint32_t *pk[2] = {ws_ptr<uint32_t>(ws, L.pair_keys[0]), ws_ptr<uint32_t>(ws, L.pair_keys[1])};
    uint32_t *pv[2] = {ws_ptr<uint32_t>(ws, L.pair_vals[0]), ws_ptr<uint32_t>(ws, L.pair_vals[1])};
    float *hbuf = ws_ptr<float>(ws, L.hbuf);
    float *wnorm = ws_ptr<float>(ws, L.wnorm);
    uint32_t *seg_start = ws_ptr<uint32_t>(ws, L.seg_start), *seg_end = ws_ptr<uint32_t>(ws, L.seg_end);
    uint32_t *pieces = ws_ptr<uint32_t>(ws, L.pieces), *piece_off = ws_ptr<uint32_t>(ws, L.piece_off);
    uint32_t *multi = ws_ptr<uint32_t>(ws, L.multi), *multi_off = ws_ptr<uint32_t>(ws, L.multi_off);
    uint32_t *mflag = ws_ptr<uint32_t>(ws, L.mflag), *mlist = ws_ptr<uint32_t>(ws, L.mlist);
    uint32_t *piece_rank = ws_ptr<uint32_t>(ws, L.piece_rank);
    float *rows = ws_ptr<float>(ws, L.piece_rows);

    const unsigned nbN = (unsigned)((N + 255) / 256);
    // 1. Morton rank
    k_bbox_init<<<1, 32, 0, s>>>(bb);
    k_bbox<<<min((int)nbN, 148 * 4), 256, 0, s>>>(N, mean3d, bb);
    k_morton<<<nbN, 256, 0, s>>>(N, mean3d, bb, rk[0], rv[0]);
    int rcur = radix_sort_pairs(rk[0], rk[1], rv[0], rv[1], N, nullptr, 30, hist, s);
    const uint32_t *order = rv[rcur];
    k_rank_scatter<<<nbN, 256, 0, s>>>(N, order, grank);
    // 2. pairs sorted by rank (plus the renormalised weight of every slot)
    long long n_pairs = L.n_pairs;
    k_pairs<<<(unsigned)((n_pairs + 255) / 256), 256, 0, s>>>(N, L.K, L.PK, topk_idx, topk_w, grank, pk[0], pv[0],
                                                              wnorm);
    int pcur = radix_sort_pairs(pk[0], pk[1], pv[0], pv[1], n_pairs, nullptr, L.pair_bits, hist, s);
    k_segments<<<(unsigned)((n_pairs + 255) / 256), 256, 0, s>>>(N, n_pairs, nullptr, pk[pcur], pv[pcur], seg_start,
                                                                 seg_end);
    // 3. pieces, and the compact list of Gaussians cut into several pieces
    k_pieces<<<nbN, 256, 0, s>>>(N, seg_start, seg_end, pieces, multi);
    exclusive_scan_u32(pieces, piece_off, N, n_pieces, aux, s);
    exclusive_scan_u32(multi, multi_off, N, nullptr, aux, s);
    k_multi_flags<<<nbN, 256, 0, s>>>(N, multi, mflag);
    exclusive_scan_u32(mflag, mflag, N, n_multi, aux, s);
    k_piece_rank<<<nbN, 256, 0, s>>>(N, pieces, piece_off, multi, mflag, piece_rank, mlist);
    // 4. reduce
    const int vec = dtype == GS_BF16 ? 8 : 4;
    const int nch = L.D / vec;
    const int cpl = cpl_for(nch);
    unsigned blocks = (unsigned)((L.max_pieces * 32 + 255) / 256);
    bool ok = dtype == GS_BF16
                  ? fgrad_main<true, false>(cpl, blocks, s, L.K, nch, n_pieces, piece_rank, piece_off, pieces, multi_off,
                                     seg_start, seg_end, order, pv[pcur], wnorm, feats, dLdF, hbuf, grad_feat, rows)
                  : fgrad_main<false, false>(cpl, blocks, s, L.K, nch, n_pieces, piece_rank, piece_off, pieces, multi_off,
                                      seg_start, seg_end, order, pv[pcur], wnorm, feats, dLdF, hbuf, grad_feat, rows);
    if (!ok) return false;
    k_fgrad_fixup<<<148 * 2, kFixCols * kFixGroups, 0, s>>>(L.D / 4, n_multi, mlist, multi, multi_off, order,
                                                            (const float4 *)rows, (float4 *)grad_feat);
    return true;
}

}  // namespace gs
