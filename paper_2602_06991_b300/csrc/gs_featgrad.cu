// gs_featgrad.cu -- feature part of a5: dL/df_g = sum over (pixel p, slot k) with
// idx_k(p) = g of w'_k(p) dL/dF_p (Eqs. 3-4), and h_k(p) = dL/dF_p . f_g for the re-walk.
//
// This is a transposed sparse product (P x N with K entries per row)^T (P x D), done
// without atomics in four stages:
//   h      per slot, by the pixel-group kernel of gs_blend.cu (launch_h);
//   T1-T3  per pixel block, the partial row of every (block, selected Gaussian) pair
//          (gs_tilegrad.cu);
//   T4     per Gaussian, the sum of its partial rows (here): the (Gaussian, row) pairs
//          are sorted by Gaussian with the library's radix sort; every Gaussian has a
//          marker entry placed first in its segment by the stable sort, so segments are
//          found without a search.  Segments are cut into pieces of at most kPieceLen
//          rows (a Gaussian near the camera can be selected in thousands of blocks); one
//          warp sums one piece in registers with 16-byte loads.  Single-piece Gaussians
//          write their gradient row directly, multi-piece ones write piece rows that a
//          fix-up pass sums in a fixed order, and Gaussians selected nowhere get a zero
//          row from a streaming fill.  Every order is fixed: the result is deterministic.
#include "gs_internal.cuh"

namespace gs {

constexpr uint32_t kMarker = 0xffffffffu;

// One marker entry per Gaussian id ahead of the partial-row pairs.
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

// Segment [seg_start, seg_end) of sorted positions holding Gaussian k's rows.
__global__ void k_segments(int N, long long n_host, const uint32_t *n_dev, const uint32_t *__restrict__ keys,
                           const uint32_t *__restrict__ vals, uint32_t *seg_start, uint32_t *seg_end)
{
    long long n_pairs = min((long long)*n_dev, n_host);
    long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_pairs) return;
    uint32_t k = keys[m];
    if (k >= (uint32_t)N) return;
    if (vals[m] == kMarker) seg_start[k] = (uint32_t)(m + 1);
    if (m + 1 == n_pairs || keys[m + 1] != k) seg_end[k] = (uint32_t)(m + 1);
}

// Pieces per Gaussian (0 for a Gaussian selected nowhere) and the piece count of
// multi-piece ones.
__global__ void k_pieces(int N, const uint32_t *__restrict__ seg_start, const uint32_t *__restrict__ seg_end,
                         uint32_t *pieces, uint32_t *multi)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    uint32_t n = seg_end[r] - seg_start[r];
    uint32_t pc = (n + kPieceLen - 1) / kPieceLen;
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

// Zero gradient rows of the Gaussians selected nowhere: one thread per float4 of the
// N x D gradient, a grid-stride streaming fill.
// Zero rows for the Gaussians no pixel selected: one warp per row, grid-stride over the
// Gaussians, 16-byte stores.
__global__ void __launch_bounds__(256) k_zero_unselected(int N, int D4, const uint32_t *__restrict__ seg_start,
                                                         const uint32_t *__restrict__ seg_end,
                                                         float4 *__restrict__ grad_f)
{
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < N; g += nwarps) {
        if (seg_end[g] != seg_start[g]) continue;          // warp-uniform
        float4 *row = grad_f + g * D4;
        for (int c = lane; c < D4; c += 32) row[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// One warp per piece of a Gaussian's segment: the sum of its partial rows (float32,
// D = 4 nch), CPL 16-byte chunks per lane, four rows in flight at a time.
template <int CPL>
__global__ void __launch_bounds__(256) k_rows_main(int nch, const uint32_t *__restrict__ n_pieces_dev,
                                                   const uint32_t *__restrict__ piece_rank,
                                                   const uint32_t *__restrict__ piece_off,
                                                   const uint32_t *__restrict__ pieces,
                                                   const uint32_t *__restrict__ multi_off,
                                                   const uint32_t *__restrict__ seg_start,
                                                   const uint32_t *__restrict__ seg_end,
                                                   const uint32_t *__restrict__ pair_vals,
                                                   const float4 *__restrict__ rows, float4 *__restrict__ grad_f,
                                                   float4 *__restrict__ piece_rows)
{
    constexpr int U = 4;
    const int lane = threadIdx.x & 31;
    const long long pc = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (pc >= (long long)*n_pieces_dev) return;
    const uint32_t g = piece_rank[pc];
    const uint32_t j = (uint32_t)pc - piece_off[g];
    const uint32_t m0 = seg_start[g] + j * kPieceLen;
    const uint32_t m1 = min(m0 + kPieceLen, seg_end[g]);
    float4 acc[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t m = m0;
    for (; m + U <= m1; m += U) {
        uint32_t rv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) rv[u] = pair_vals[m + u];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int ch = lane + 32 * c;
            if (ch < nch) {
                float4 x[U];
#pragma unroll
                for (int u = 0; u < U; ++u) x[u] = __ldg(rows + (size_t)rv[u] * nch + ch);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    acc[c].x += x[u].x; acc[c].y += x[u].y; acc[c].z += x[u].z; acc[c].w += x[u].w;
                }
            }
        }
    }
    for (; m < m1; ++m) {
        const uint32_t rv = pair_vals[m];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int ch = lane + 32 * c;
            if (ch < nch) {
                const float4 x = __ldg(rows + (size_t)rv * nch + ch);
                acc[c].x += x.x; acc[c].y += x.y; acc[c].z += x.z; acc[c].w += x.w;
            }
        }
    }
    float4 *dst = pieces[g] == 1 ? grad_f + (size_t)g * nch : piece_rows + (size_t)(multi_off[g] + j) * nch;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int ch = lane + 32 * c;
        if (ch < nch) dst[ch] = acc[c];
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
                                                                      const float4 *__restrict__ piece_rows,
                                                                      float4 *__restrict__ grad_f)
{
    __shared__ float4 part[kFixGroups][kFixCols];
    const int col = threadIdx.x % kFixCols, grp = threadIdx.x / kFixCols;
    const uint32_t n_multi = *n_multi_dev;
    for (uint32_t i = blockIdx.x; i < n_multi; i += gridDim.x) {
        const uint32_t r = mlist[i];
        const uint32_t n = multi[r], base = multi_off[r], g = r;
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

bool launch_tile_grad(const CamTable &ct, const WsLayout &L, int dtype, const int *topk_idx, const float *topk_w,
                      const void *dLdF, void *ws, cudaStream_t s, cudaStream_t hold, cudaEvent_t hold_ev);

// h = dL/dF . f per slot, read by the re-walk.
bool launch_feature_h(const WsLayout &L, int dtype, const int *topk_idx, const void *feats, const void *dLdF,
                      void *ws, cudaStream_t s)
{
    if (!L.use_tiles) return false;
    return launch_h(dtype, L.K, L.D, L.P, L.N, topk_idx, feats, dLdF, ws_ptr<float>(ws, L.hbuf),
                    ws_ptr<const int>(ws, L.header), s);
}

// The feature gradient proper: per-block partial rows, then per-Gaussian sums.  It
// reads only the Top-K record and dL/dF, so it may run beside the re-walk.
bool launch_feature_grad(const CamTable &ct, const WsLayout &L, int dtype, int N, const int *topk_idx,
                         const float *topk_w, const void *dLdF, float *grad_feat, void *ws, cudaStream_t s,
                         cudaStream_t hold, cudaEvent_t hold_ev)
{
    if (!L.use_tiles) return false;
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
    float4 *prow = ws_ptr<float4>(ws, L.piece_rows);
    const float4 *trows = ws_ptr<float4>(ws, L.tile_rows);
    const unsigned nbN = (unsigned)((N + 255) / 256);

    // per-block partial rows
    if (!launch_tile_grad(ct, L, dtype, topk_idx, topk_w, dLdF, ws, s, hold, hold_ev)) return false;
    // T4: (Gaussian, row) pairs sorted by Gaussian, segments, pieces
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
    const int D4 = L.D / 4;
    k_zero_unselected<<<148 * 8, 256, 0, s>>>(N, D4, seg_start, seg_end, (float4 *)grad_feat);
    const int cpl = D4 <= 32 ? 1 : D4 <= 64 ? 2 : D4 <= 128 ? 4 : 8;
    const unsigned blocks = (unsigned)((L.max_pieces_rows * 32 + 255) / 256);
#define GS_RM(C)                                                                                                    \
    k_rows_main<C><<<blocks, 256, 0, s>>>(D4, n_pieces, piece_rank, piece_off, pieces, multi_off, seg_start, seg_end, \
                                          pv[pcur], trows, (float4 *)grad_feat, prow)
    switch (cpl) {
    case 1: GS_RM(1); break;
    case 2: GS_RM(2); break;
    case 4: GS_RM(4); break;
    default: GS_RM(8); break;
    }
#undef GS_RM
    k_fgrad_fixup<<<148 * 2, kFixCols * kFixGroups, 0, s>>>(D4, n_multi, mlist, multi, multi_off, prow,
                                                            (float4 *)grad_feat);
    return true;
}

}  // namespace gs
