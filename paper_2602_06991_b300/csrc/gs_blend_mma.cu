// gs_blend_mma.cu -- a4 for bf16 feature rows on the tensor cores: the gather-blend of
// Eqs. 3-4, and its training form with the loss gradient and the re-walk's per-slot
// terms h = dL/dF . f.
//
// With bf16 rows the CUDA-core blend is bound by instruction issue, not by HBM: per
// pixel it converts and multiplies K rows of D values and again for h, while moving only
// 2 D bytes per stream.  Over a group of 16 consecutive flat pixels the blend is a small
// dense product,
//     F[16 x D]  = W[16 x U] R[U x D]         (W: renormalised weights w'; R: the group's
//     h[16 x U]  = dL/dF[16 x D] R^T[D x U]     U distinct rows, ascending Gaussian id),
// which one warp computes with mma.m16n8k16 (bf16 operands, float32 accumulation).
// Precision: the rows and dL/dF are bf16 already (products exact in float32); the
// float32 weights are split exactly into three bf16 terms (w = hi + mid + lo), so F is
// the float32-weighted sum of the bf16 rows with float32 accumulation, as the CUDA-core
// form computes it (only the summation order differs).
//
// Per warp (16 pixels): the K slots of each pixel are loaded, S and w' formed in slot
// order; the (id, slot) keys are sorted in registers (bitonic) to give the distinct rows
// and each slot's rank; W is built densely and split into A fragments.  The rows are then
// staged 64 columns at a time into padded shared memory (cp.async, double-buffered, one
// row per lane) and multiplied (ldmatrix.trans for the B fragments).  Training form:
// pass 1 writes F (bf16) and reduces |F|^2, F.Fgt, |Fgt|^2 per pixel in the accumulator
// layout (a quad of lanes per pixel row); pass 2 recomputes F, forms dL/dF = a Fgt + b F,
// writes it, and feeds it -- already in the A-fragment layout -- to the h product.
// A group with more than kMmaRows distinct rows is split in halves (down to single
// pixels, whose K rows always fit); the blend-only and the training kernels split alike,
// so their F are bit-identical.
#include "gs_internal.cuh"
#include "gs_mma.cuh"

#include <algorithm>

namespace gs {

constexpr int kMmaPix = 16;                     // pixels per warp (the M of the MMA)
constexpr int kMmaRows = 32;                    // distinct rows per (sub)group
constexpr int kMmaCols = 64;                    // columns per staged chunk
constexpr int kMmaPitch = kMmaCols * 2 + 16;    // bytes per staged row: conflict-free ldmatrix
constexpr int kMmaWarps = 4;                    // warps per CTA

// Per warp.  The tables of a (sub)group (dense W, w' per slot, then h) are used only
// before and after its chunk loop, the pixel chunk buffers only inside it, so they share
// memory: 14.2 KB per warp, four 4-warp CTAs per SM.
struct MmaWarpSmem {
    unsigned char rows[2][kMmaRows * kMmaPitch];    // staged row chunks (double buffer)
    union {
        unsigned char pix[2][kMmaPix * kMmaPitch];  // the 16 pixels' chunk: target rows in, F / dL/dF out
        struct {
            float wt[kMmaPix][kMmaRows];            // dense W, then h by (pixel, rank)
            float wslot[kMmaPix * 16];              // w' per slot
        };
    };
    int ids[kMmaRows];                              // distinct ids, ascending
    unsigned char rank[kMmaPix * 16];               // rank of each slot's id (0xff: none)
};
static_assert(sizeof(MmaWarpSmem) * kMmaWarps * 4 <= 227 * 1024, "four CTAs per SM");

size_t blend_mma_smem() { return sizeof(MmaWarpSmem) * kMmaWarps; }

// Loads the K slots of the pixels [lo, hi) of the warp's 16 (the others count as empty),
// forms w' in slot order, sorts the (id, slot) keys, and fills ids, rank and the dense W.
// Returns U, the number of distinct rows (the tables are only filled when U <= kMmaRows).
template <int K>
__device__ __forceinline__ int mma_table(long long p0, long long n_pix, int lo, int hi, const int *__restrict__ idx,
                                         const float *__restrict__ wts, bool bad, int lane, MmaWarpSmem &sm)
{
    // (wts == nullptr: ids and ranks only, W stays zero)
    constexpr int SPL = K / 2;
    constexpr int KPT = SPL;                      // keys per lane in the sort (a power of two)
    constexpr int NS = 32 * KPT;
    constexpr uint32_t kNone = 0xffffffffu;
    const int pl = lane >> 1;
    const long long p = p0 + pl;
    const bool live = !bad && pl >= lo && pl < hi && p < n_pix;
    int id[SPL];
    float w[SPL];
#pragma unroll
    for (int j = 0; j < SPL; ++j) {
        id[j] = -1;
        w[j] = 0.f;
    }
    if (live) {
        const long long base = p * K + (lane & 1) * SPL;
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
            id[j] = __ldg(idx + base + j);
            w[j] = wts ? __ldg(wts + base + j) : 0.f;
        }
    }
    // S over the pixel's K slots in slot order: the even lane holds slots [0, K/2), its odd
    // neighbour continues from its partial sum
    float a = 0.f;
    if (!(lane & 1)) {
#pragma unroll
        for (int j = 0; j < SPL; ++j) a += w[j];
    }
    float S = __shfl_sync(0xffffffffu, a, lane & ~1);
    if (lane & 1) {
#pragma unroll
        for (int j = 0; j < SPL; ++j) S += w[j];
    }
    S = __shfl_sync(0xffffffffu, S, lane | 1);
    const float inv = S > 0.f ? 1.f / S : 0.f;
    uint32_t key[KPT];
#pragma unroll
    for (int j = 0; j < SPL; ++j) {
        const int s = lane * SPL + j;
        sm.wslot[s] = id[j] >= 0 ? w[j] * inv : 0.f;
        key[j] = id[j] >= 0 ? (((uint32_t)id[j] << 8) | (uint32_t)s) : kNone;
    }
    // bitonic sort of the 32 KPT keys, element e = lane KPT + r
#pragma unroll
    for (int size = 2; size <= NS; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= KPT) {
                const int lm = stride / KPT;
                const bool lower = (lane & lm) == 0;
#pragma unroll
                for (int r = 0; r < KPT; ++r) {
                    const bool up = ((lane * KPT + r) & size) == 0;
                    const uint32_t o = __shfl_xor_sync(0xffffffffu, key[r], lm);
                    key[r] = (lower == up) ? min(key[r], o) : max(key[r], o);
                }
            } else {
#pragma unroll
                for (int r = 0; r < KPT; ++r) {
                    if ((r & stride) == 0) {
                        const bool up = ((lane * KPT + r) & size) == 0;
                        const uint32_t x = key[r], y = key[r | stride];
                        key[r] = up ? min(x, y) : max(x, y);
                        key[r | stride] = up ? max(x, y) : min(x, y);
                    }
                }
            }
        }
    }
    const uint32_t before = __shfl_up_sync(0xffffffffu, key[KPT - 1], 1);
    bool st[KPT];
    int starts = 0;
#pragma unroll
    for (int r = 0; r < KPT; ++r) {
        const uint32_t pk = r ? key[r - 1] : before;
        st[r] = key[r] != kNone && ((lane == 0 && r == 0) || (pk >> 8) != (key[r] >> 8));
        starts += st[r];
    }
    int inc = starts;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    const int U = __shfl_sync(0xffffffffu, inc, 31);
    if (U > kMmaRows) return U;
    // dense W (zero), then one entry per valid slot; rank of every slot
    for (int i = lane; i < kMmaPix * kMmaRows; i += 32) (&sm.wt[0][0])[i] = 0.f;
    for (int i = lane; i < kMmaPix * 16; i += 32) sm.rank[i] = 0xff;
    __syncwarp();
    int u = inc - starts - 1;
#pragma unroll
    for (int r = 0; r < KPT; ++r) {
        if (key[r] != kNone) {
            if (st[r]) {
                ++u;
                sm.ids[u] = (int)(key[r] >> 8);
            }
            const int s = (int)(key[r] & 255u);
            sm.wt[s / K][u] = sm.wslot[s];
            sm.rank[s] = (unsigned char)u;
        }
    }
    __syncwarp();
    return U;
}

// Stages columns [c0, c0 + 64) of the group's rows 0..nrows-1 into buffer `buf` (one
// row per lane, eight 16-byte copies); rows at or past U are zero-filled.
__device__ __forceinline__ void mma_stage(const __nv_bfloat16 *__restrict__ feats, int D, int c0, int nrows, int U,
                                          int lane, MmaWarpSmem &sm, int buf)
{
    if (lane < nrows) {
        const bool real = lane < U;
        const __nv_bfloat16 *src = feats + (real ? (size_t)sm.ids[lane] * D + c0 : 0);
        const uint32_t dst = smem_addr(sm.rows[buf] + lane * kMmaPitch);
#pragma unroll
        for (int q = 0; q < 8; ++q) cp_async_16(dst + 16 * q, src + (real ? 8 * q : 0), real ? 16 : 0);
    }
    cp_async_commit_group();
}

// Stages columns [c0, c0 + 64) of the 16 pixels' target rows into pix[buf] (four 16-byte
// copies per lane, whole 128-byte lines); pixels past n_pix are zero-filled.  Joins the
// copy group of the next mma_stage call.
__device__ __forceinline__ void mma_stage_pix(const __nv_bfloat16 *__restrict__ src_rows, long long p0, long long n_pix,
                                              int D, int c0, int lane, MmaWarpSmem &sm, int buf)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = 4 * i + (lane >> 3), q = lane & 7;
        const bool real = p0 + r < n_pix;
        const __nv_bfloat16 *src = src_rows + (real ? (size_t)(p0 + r) * D + c0 + 8 * q : 0);
        cp_async_16(smem_addr(sm.pix[buf] + r * kMmaPitch + 16 * q), src, real ? 16 : 0);
    }
}

// The accumulator-layout values of the chunk's 16 pixel rows from pix[buf]: v[j][0] the
// lane's pair of row g, v[j][1] of row g + 8, n-tile j (ldmatrix: four 8 x 8 blocks per
// 16 columns).
__device__ __forceinline__ void mma_pix_load(const MmaWarpSmem &sm, int buf, int lane, uint32_t (&v)[8][2])
{
    const uint32_t base = smem_addr(sm.pix[buf]);
    const int mi = lane >> 3, mr = lane & 7;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int r = mr + 8 * (mi & 1), c = 16 * m + 8 * (mi >> 1);
        ldsm_x4(base + r * kMmaPitch + 2 * c, v[2 * m][0], v[2 * m][1], v[2 * m + 1][0], v[2 * m + 1][1]);
    }
}

// Writes the accumulator-layout pairs v of the chunk to pix[buf] (stmatrix), then the
// rows [lo, hi) of the 16 pixels to dst with whole-line 16-byte stores.
__device__ __forceinline__ void mma_pix_store(const uint32_t (&v)[8][2], MmaWarpSmem &sm, int buf, int lane,
                                              __nv_bfloat16 *__restrict__ dst, long long p0, long long n_pix, int lo,
                                              int hi, int D, int c0)
{
    const uint32_t base = smem_addr(sm.pix[buf]);
    const int mi = lane >> 3, mr = lane & 7;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int r = mr + 8 * (mi & 1), c = 16 * m + 8 * (mi >> 1);
        stsm_x4(base + r * kMmaPitch + 2 * c, v[2 * m][0], v[2 * m][1], v[2 * m + 1][0], v[2 * m + 1][1]);
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = 4 * i + (lane >> 3), q = lane & 7;
        if (r >= lo && r < hi && p0 + r < n_pix) {
            const uint4 x = *(const uint4 *)(sm.pix[buf] + r * kMmaPitch + 16 * q);
            *(uint4 *)(dst + (size_t)(p0 + r) * D + c0 + 8 * q) = x;
        }
    }
}

// acc (8 n-tiles of 8 columns) = W R for one staged 64-column chunk
template <int KS>
__device__ __forceinline__ void mma_blend_chunk(const uint32_t (&afr)[2][3][4], const MmaWarpSmem &sm, int buf,
                                                int lane, float (&acc)[8][4])
{
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[j][v] = 0.f;
    const uint32_t base = smem_addr(sm.rows[buf]);
    const int mi = lane >> 3, mr = lane & 7;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
        uint32_t b[4][4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            // matrices: rows 16ks + {0-7, 8-15} x columns 16m + {0-7, 8-15}, transposed
            const int r = 16 * ks + mr + 8 * (mi & 1), c = 16 * m + 8 * (mi >> 1);
            ldsm_x4_t(base + r * kMmaPitch + 2 * c, b[m][0], b[m][1], b[m][2], b[m][3]);
        }
        // each accumulator takes the three terms in order; the eight accumulators of a
        // term are independent, so consecutive products do not wait on each other
#pragma unroll
        for (int sp = 0; sp < 3; ++sp)
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                mma16816(acc[2 * m], afr[ks][sp], b[m][0], b[m][1]);
                mma16816(acc[2 * m + 1], afr[ks][sp], b[m][2], b[m][3]);
            }
    }
}

// A fragments of W (three bf16 splits) for k-steps 0..KS-1
__device__ __forceinline__ void mma_weight_frags(const MmaWarpSmem &sm, int KS, int lane, uint32_t (&afr)[2][3][4])
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
        if (ks >= KS) break;
        float v[8];
        const int c = 16 * ks + 2 * t;
        v[0] = sm.wt[g][c];         v[1] = sm.wt[g][c + 1];
        v[2] = sm.wt[g + 8][c];     v[3] = sm.wt[g + 8][c + 1];
        v[4] = sm.wt[g][c + 8];     v[5] = sm.wt[g][c + 9];
        v[6] = sm.wt[g + 8][c + 8]; v[7] = sm.wt[g + 8][c + 9];
        float hh[8], mm[8], ll[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) split3(v[i], hh[i], mm[i], ll[i]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            afr[ks][0][q] = pack_bf16(hh[2 * q], hh[2 * q + 1]);
            afr[ks][1][q] = pack_bf16(mm[2 * q], mm[2 * q + 1]);
            afr[ks][2][q] = pack_bf16(ll[2 * q], ll[2 * q + 1]);
        }
    }
}

template <int K>
__device__ __forceinline__ void mma_group_tail(long long p0, long long n_pix, int lo, int hi, int KS,
                                               const float (&hacc)[4][4], float cosa, float cosb,
                                               const float *__restrict__ C, const float *__restrict__ Cgt,
                                               const float *__restrict__ Dp, const float *__restrict__ Dgt, float wf,
                                               float wc, float wd, float invP, float *__restrict__ dLdC,
                                               float *__restrict__ dLdD, float *__restrict__ part,
                                               float *__restrict__ h, int lane, MmaWarpSmem &sm);

// One (sub)group [lo, hi) of the warp's pixels.  LOSS: the training form.
template <int K, bool LOSS>
__device__ __forceinline__ void mma_group(long long p0, long long n_pix, int lo, int hi, int U, int D,
                          const __nv_bfloat16 *__restrict__ feats, const __nv_bfloat16 *__restrict__ Fgt,
                          const float *__restrict__ C, const float *__restrict__ Cgt, const float *__restrict__ Dp,
                          const float *__restrict__ Dgt, float wf, float wc, float wd, float invP,
                          __nv_bfloat16 *__restrict__ F, __nv_bfloat16 *__restrict__ dLdF, float *__restrict__ dLdC,
                          float *__restrict__ dLdD, float *__restrict__ part, float *__restrict__ h, int lane,
                          MmaWarpSmem &sm)
{
    const int g = lane >> 2;
    const int KS = U <= 16 ? 1 : 2;               // 16-row k-steps
    const int nrows = 16 * KS;
    uint32_t afr[2][3][4];
    mma_weight_frags(sm, KS, lane, afr);
    __syncwarp();                                 // W is read: the pixel buffers it shares memory with are free
    const int nchunk = D / kMmaCols;
    const int steps = LOSS ? 2 * nchunk : nchunk;
    // per-pixel sums F.F, F.G, G.G of the first pass.  K >= 16 (wider weight tables, two
    // k-steps in most groups): as the diagonals of the 16 x 16 products F F^T, F G^T, G G^T
    // on the tensor cores (two 8-pixel n-tiles each), which issues fewer instructions than
    // the 12 FMAs per value pair; K < 16: FMAs per lane, summed over the quad (fewer
    // registers, one more resident CTA per SM -- measured faster there)
    constexpr bool kTcSums = K >= 16;
    float ffc[2][4], fgc[2][4], ggc[2][4];
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int v = 0; v < 4; ++v) ffc[n][v] = fgc[n][v] = ggc[n][v] = 0.f;
    float ffa = 0.f, fga = 0.f, gga = 0.f, ffb = 0.f, fgb = 0.f, ggb = 0.f;
    float caa = 0.f, cba = 0.f, cab = 0.f, cbb = 0.f, cosa = 0.f, cosb = 0.f;
    float hacc[4][4];
#pragma unroll
    for (int n = 0; n < 4; ++n)
#pragma unroll
        for (int v = 0; v < 4; ++v) hacc[n][v] = 0.f;

    if (LOSS) mma_stage_pix(Fgt, p0, n_pix, D, 0, lane, sm, 0);
    mma_stage(feats, D, 0, nrows, U, lane, sm, 0);
    for (int step = 0; step < steps; ++step) {
        const int buf = step & 1;
        const int ch = step % nchunk;
        const bool pass2 = LOSS && step >= nchunk;
        if (LOSS && step == nchunk) {
            // end of pass 1: the diagonals -- pixel g's entry of n-tile 0 and pixel g + 8's
            // of n-tile 1 sit in lane 4 g + g / 2 -- for the whole quad, then the loss
            // coefficients
            if constexpr (kTcSums) {
                const int src = 4 * g + (g >> 1);
                auto diag = [&](const float (&c)[2][4], float &va, float &vb) {
                    va = __shfl_sync(0xffffffffu, (g & 1) ? c[0][1] : c[0][0], src);
                    vb = __shfl_sync(0xffffffffu, (g & 1) ? c[1][3] : c[1][2], src);
                };
                diag(ffc, ffa, ffb);
                diag(fgc, fga, fgb);
                diag(ggc, gga, ggb);
            } else {
#pragma unroll
                for (int o = 1; o < 4; o <<= 1) {
                    ffa += __shfl_xor_sync(0xffffffffu, ffa, o);
                    fga += __shfl_xor_sync(0xffffffffu, fga, o);
                    gga += __shfl_xor_sync(0xffffffffu, gga, o);
                    ffb += __shfl_xor_sync(0xffffffffu, ffb, o);
                    fgb += __shfl_xor_sync(0xffffffffu, fgb, o);
                    ggb += __shfl_xor_sync(0xffffffffu, ggb, o);
                }
            }
            auto coef = [&](float ff, float fg, float gg, float &ca, float &cb, float &cs) {
                const float nf = sqrtf(ff), ng = sqrtf(gg);
                const bool ok = nf > 0.f && ng > 0.f;
                cs = ok ? fg / (nf * ng) : 0.f;
                ca = ok ? -wf * invP / (nf * ng) : 0.f;
                cb = ok ? wf * invP * cs / ff : 0.f;
            };
            coef(ffa, fga, gga, caa, cba, cosa);
            coef(ffb, fgb, ggb, cab, cbb, cosb);
        }
        if (step + 1 < steps) {
            const int cn = ((step + 1) % nchunk) * kMmaCols;
            if (LOSS) mma_stage_pix(Fgt, p0, n_pix, D, cn, lane, sm, buf ^ 1);
            mma_stage(feats, D, cn, nrows, U, lane, sm, buf ^ 1);
            cp_async_wait_group<1>();
        } else {
            cp_async_wait_group<0>();
        }
        __syncwarp();
        const int c0 = ch * kMmaCols;
        // the chunk's target values (the loss reads them in both passes)
        uint32_t gt[8][2];
        if (LOSS) mma_pix_load(sm, buf, lane, gt);
        float acc[8][4];
        if (KS == 1) mma_blend_chunk<1>(afr, sm, buf, lane, acc);
        else mma_blend_chunk<2>(afr, sm, buf, lane, acc);
        uint32_t fo[8][2];                        // F as stored (bf16 pairs)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            fo[j][0] = pack_bf16(acc[j][0], acc[j][1]);
            fo[j][1] = pack_bf16(acc[j][2], acc[j][3]);
        }
        if (!pass2) {
            // the loss sees F as stored: F (bf16, the A layout of its accumulators) against
            // G^T and F^T (B fragments read from the staged rows of the chunk)
            const uint32_t pb = smem_addr(sm.pix[buf]);
            const int mi = lane >> 3, mr = lane & 7;
            if (LOSS && kTcSums) {
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4(pb + (mr + 8 * (mi >> 1)) * kMmaPitch + 2 * (16 * m + 8 * (mi & 1)), b0, b1, b2, b3);
                    const uint32_t af[4] = {fo[2 * m][0], fo[2 * m][1], fo[2 * m + 1][0], fo[2 * m + 1][1]};
                    const uint32_t ag[4] = {gt[2 * m][0], gt[2 * m][1], gt[2 * m + 1][0], gt[2 * m + 1][1]};
                    mma16816(fgc[0], af, b0, b1);
                    mma16816(fgc[1], af, b2, b3);
                    mma16816(ggc[0], ag, b0, b1);
                    mma16816(ggc[1], ag, b2, b3);
                }
                __syncwarp();                     // every lane has read the target values
            } else if (LOSS) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float a0 = bf_lo(fo[j][0]), a1 = bf_hi(fo[j][0]), b0 = bf_lo(fo[j][1]), b1 = bf_hi(fo[j][1]);
                    const float g0 = bf_lo(gt[j][0]), g1 = bf_hi(gt[j][0]), g2 = bf_lo(gt[j][1]), g3 = bf_hi(gt[j][1]);
                    ffa = fmaf(a0, a0, fmaf(a1, a1, ffa));
                    fga = fmaf(a0, g0, fmaf(a1, g1, fga));
                    gga = fmaf(g0, g0, fmaf(g1, g1, gga));
                    ffb = fmaf(b0, b0, fmaf(b1, b1, ffb));
                    fgb = fmaf(b0, g2, fmaf(b1, g3, fgb));
                    ggb = fmaf(g2, g2, fmaf(g3, g3, ggb));
                }
                __syncwarp();                     // every lane has read the target values
            }
            mma_pix_store(fo, sm, buf, lane, F, p0, n_pix, lo, hi, D, c0);
            if (LOSS && kTcSums) {
#pragma unroll
                for (int m = 0; m < 4; ++m) {     // the buffer now holds F as stored
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4(pb + (mr + 8 * (mi >> 1)) * kMmaPitch + 2 * (16 * m + 8 * (mi & 1)), b0, b1, b2, b3);
                    const uint32_t af[4] = {fo[2 * m][0], fo[2 * m][1], fo[2 * m + 1][0], fo[2 * m + 1][1]};
                    mma16816(ffc[0], af, b0, b1);
                    mma16816(ffc[1], af, b2, b3);
                }
            }
        } else {
            // dL/dF = a Fgt + b F (F as stored), written in bf16; as stored it is the A
            // operand of h = dL/dF R^T (k-step m covers n-tiles 2m, 2m + 1)
            uint32_t dfr[8][2];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float d0 = fmaf(caa, bf_lo(gt[j][0]), cba * bf_lo(fo[j][0]));
                const float d1 = fmaf(caa, bf_hi(gt[j][0]), cba * bf_hi(fo[j][0]));
                const float d2 = fmaf(cab, bf_lo(gt[j][1]), cbb * bf_lo(fo[j][1]));
                const float d3 = fmaf(cab, bf_hi(gt[j][1]), cbb * bf_hi(fo[j][1]));
                dfr[j][0] = pack_bf16(d0, d1);
                dfr[j][1] = pack_bf16(d2, d3);
            }
            const uint32_t base = smem_addr(sm.rows[buf]);
            const int mi = lane >> 3, mr = lane & 7;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const uint32_t a[4] = {dfr[2 * m][0], dfr[2 * m][1], dfr[2 * m + 1][0], dfr[2 * m + 1][1]};
#pragma unroll
                for (int nb = 0; nb < 2; ++nb) {
                    if (nb >= KS) break;
                    // matrices: rows 16nb + {0-7, 8-15} x columns 16m + {0-7, 8-15}
                    const int r = 16 * nb + mr + 8 * (mi >> 1), c = 16 * m + 8 * (mi & 1);
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4(base + r * kMmaPitch + 2 * c, b0, b1, b2, b3);
                    mma16816(hacc[2 * nb], a, b0, b1);
                    mma16816(hacc[2 * nb + 1], a, b2, b3);
                }
            }
            __syncwarp();                         // every lane has read the target values
            mma_pix_store(dfr, sm, buf, lane, dLdF, p0, n_pix, lo, hi, D, c0);
        }
        __syncwarp();                             // both buffers of the step are free again
    }
    if constexpr (LOSS) mma_group_tail<K>(p0, n_pix, lo, hi, KS, hacc, cosa, cosb, C, Cgt, Dp, Dgt, wf, wc, wd, invP,
                                           dLdC, dLdD, part, h, lane, sm);
}

// The training form's per-slot h (from the h accumulators) and the colour / depth terms
// and loss share of the (sub)group's pixels.
template <int K>
__device__ __forceinline__ void mma_group_tail(long long p0, long long n_pix, int lo, int hi, int KS,
                                               const float (&hacc)[4][4], float cosa, float cosb,
                                               const float *__restrict__ C, const float *__restrict__ Cgt,
                                               const float *__restrict__ Dp, const float *__restrict__ Dgt, float wf,
                                               float wc, float wd, float invP, float *__restrict__ dLdC,
                                               float *__restrict__ dLdD, float *__restrict__ part,
                                               float *__restrict__ h, int lane, MmaWarpSmem &sm)
{
    constexpr int SPL = K / 2;
    const int g = lane >> 2, t = lane & 3;
    // h by (pixel, rank) into the W table, then one h per slot
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        if (n >= 2 * KS) break;
        const int c = 8 * n + 2 * t;
        sm.wt[g][c] = hacc[n][0];
        sm.wt[g][c + 1] = hacc[n][1];
        sm.wt[g + 8][c] = hacc[n][2];
        sm.wt[g + 8][c + 1] = hacc[n][3];
    }
    __syncwarp();
    {
        const int pl = lane >> 1;
        const long long p = p0 + pl;
        if (pl >= lo && pl < hi && p < n_pix) {
#pragma unroll
            for (int j = 0; j < SPL; ++j) {
                const int s = lane * SPL + j;
                const int rk = sm.rank[s];
                h[p * K + (lane & 1) * SPL + j] = rk != 0xff ? sm.wt[pl][rk] : 0.f;
            }
        }
    }
    __syncwarp();
    // colour / depth terms and the pixel's loss share: lane i < 16 takes pixel p0 + i
    const float cs_a = __shfl_sync(0xffffffffu, cosa, 4 * (lane & 7));
    const float cs_b = __shfl_sync(0xffffffffu, cosb, 4 * (lane & 7));
    if (lane < kMmaPix && lane >= lo && lane < hi && p0 + lane < n_pix) {
        const long long p = p0 + lane;
        const float cosv = lane < 8 ? cs_a : cs_b;
        float lc = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float d = C[3 * p + i] - Cgt[3 * p + i];
            lc += fabsf(d);
            dLdC[3 * p + i] = wc * invP / 3.f * (float)((d > 0.f) - (d < 0.f));
        }
        const float dd = Dp[p] - Dgt[p];
        dLdD[p] = wd * invP * (float)((dd > 0.f) - (dd < 0.f));
        part[p] = (wf * (1.f - cosv) + wc * lc / 3.f + wd * fabsf(dd)) * invP;
    }
}

template <int K, bool LOSS>
__global__ void __launch_bounds__(kMmaWarps * 32, (LOSS && K >= 16) ? 3 : 4) k_blend_mma(long long n_pix, int D, const int *__restrict__ idx,
                                                              const float *__restrict__ wts,
                                                              const __nv_bfloat16 *__restrict__ feats,
                                                              const __nv_bfloat16 *__restrict__ Fgt,
                                                              const float *__restrict__ C, const float *__restrict__ Cgt,
                                                              const float *__restrict__ Dp,
                                                              const float *__restrict__ Dgt, float wf, float wc,
                                                              float wd, float invP, __nv_bfloat16 *__restrict__ F,
                                                              __nv_bfloat16 *__restrict__ dLdF,
                                                              float *__restrict__ dLdC, float *__restrict__ dLdD,
                                                              float *__restrict__ part, float *__restrict__ h,
                                                              const int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_mma[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    MmaWarpSmem &sm = ((MmaWarpSmem *)smem_mma)[wib];
    const long long p0 = ((long long)blockIdx.x * kMmaWarps + wib) * kMmaPix;
    if (p0 >= n_pix) return;                          // whole warp
    if (LOSS) {
        // start this warp's target rows on their way to L2 while the table is built
        const long long pend = min(p0 + kMmaPix, n_pix);
        const char *a = (const char *)(Fgt + (size_t)p0 * D);
        const long long lines = ((pend - p0) * D * 2 + 127) / 128;
        for (long long l = lane; l < lines; l += 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(a + 128 * l));
    }
    const bool bad = err && *err != 0;
    // the whole group, or halves of it until the distinct rows fit
    int lo = 0, span = kMmaPix;
    while (lo < kMmaPix) {
        const int hi = min(lo + span, kMmaPix);
        const int U = mma_table<K>(p0, n_pix, lo, hi, idx, wts, bad, lane, sm);
        if (U > kMmaRows && hi - lo > 1) {
            span = (hi - lo) >> 1;
            continue;
        }
        mma_group<K, LOSS>(p0, n_pix, lo, hi, U, D, feats, Fgt, C, Cgt, Dp, Dgt, wf, wc, wd, invP, F, dLdF, dLdC,
                           dLdD, part, h, lane, sm);
        lo = hi;
    }
}

// h = dL/dF . f per Top-K slot from a given bf16 dL/dF (gs_backward when the loss's h is
// not reused): the same tensor-core product as the training form's second pass -- the
// same A values (dL/dF as stored), B fragments and MMA sequence over the columns for
// every (pixel, row) element -- so the two give bit-identical h.
template <int K>
__global__ void __launch_bounds__(kMmaWarps * 32, 4) k_h_mma(long long n_pix, int D, const int *__restrict__ idx,
                                                          const __nv_bfloat16 *__restrict__ feats,
                                                          const __nv_bfloat16 *__restrict__ dLdF,
                                                          float *__restrict__ h, const int *__restrict__ err)
{
    constexpr int SPL = K / 2;
    extern __shared__ __align__(16) unsigned char smem_mma[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    MmaWarpSmem &sm = ((MmaWarpSmem *)smem_mma)[wib];
    const long long p0 = ((long long)blockIdx.x * kMmaWarps + wib) * kMmaPix;
    if (p0 >= n_pix) return;                          // whole warp
    const bool bad = err && *err != 0;
    const int nchunk = D / kMmaCols;
    int lo = 0, span = kMmaPix;
    while (lo < kMmaPix) {
        const int hi = min(lo + span, kMmaPix);
        const int U = mma_table<K>(p0, n_pix, lo, hi, idx, nullptr, bad, lane, sm);
        if (U > kMmaRows && hi - lo > 1) {
            span = (hi - lo) >> 1;
            continue;
        }
        const int KS = U <= 16 ? 1 : 2;
        float hacc[4][4];
#pragma unroll
        for (int n = 0; n < 4; ++n)
#pragma unroll
            for (int v = 0; v < 4; ++v) hacc[n][v] = 0.f;
        mma_stage_pix(dLdF, p0, n_pix, D, 0, lane, sm, 0);
        mma_stage(feats, D, 0, 16 * KS, U, lane, sm, 0);
        for (int ch = 0; ch < nchunk; ++ch) {
            const int buf = ch & 1;
            if (ch + 1 < nchunk) {
                mma_stage_pix(dLdF, p0, n_pix, D, (ch + 1) * kMmaCols, lane, sm, buf ^ 1);
                mma_stage(feats, D, (ch + 1) * kMmaCols, 16 * KS, U, lane, sm, buf ^ 1);
                cp_async_wait_group<1>();
            } else {
                cp_async_wait_group<0>();
            }
            __syncwarp();
            const uint32_t base = smem_addr(sm.rows[buf]);
            const int mi = lane >> 3, mr = lane & 7;
            uint32_t dv[8][2];                    // dL/dF of the chunk in the A-operand layout
            mma_pix_load(sm, buf, lane, dv);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const uint32_t a[4] = {dv[2 * m][0], dv[2 * m][1], dv[2 * m + 1][0], dv[2 * m + 1][1]};
#pragma unroll
                for (int nb = 0; nb < 2; ++nb) {
                    if (nb >= KS) break;
                    const int r = 16 * nb + mr + 8 * (mi >> 1), cc = 16 * m + 8 * (mi & 1);
                    uint32_t b0, b1, b2, b3;
                    ldsm_x4(base + r * kMmaPitch + 2 * cc, b0, b1, b2, b3);
                    mma16816(hacc[2 * nb], a, b0, b1);
                    mma16816(hacc[2 * nb + 1], a, b2, b3);
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            if (n >= 2 * KS) break;
            const int c = 8 * n + 2 * t;
            sm.wt[g][c] = hacc[n][0];
            sm.wt[g][c + 1] = hacc[n][1];
            sm.wt[g + 8][c] = hacc[n][2];
            sm.wt[g + 8][c + 1] = hacc[n][3];
        }
        __syncwarp();
        const int pl = lane >> 1;
        const long long p = p0 + pl;
        if (pl >= lo && pl < hi && p < n_pix) {
#pragma unroll
            for (int j = 0; j < SPL; ++j) {
                const int rk = sm.rank[lane * SPL + j];
                h[p * K + (lane & 1) * SPL + j] = rk != 0xff ? sm.wt[pl][rk] : 0.f;
            }
        }
        __syncwarp();
        lo = hi;
    }
}

bool blend_mma_supported(int dtype, int K, int D, long long N)
{
    return dtype == GS_BF16 && (K == 2 || K == 4 || K == 8 || K == 16) && D % kMmaCols == 0 && D <= 1024 &&
           N < (1ll << 24);
}

template <int K, bool LOSS>
static void blend_mma_k(long long n_pix, int D, const int *idx, const float *w, const void *feats, const void *Fgt,
                        const float *C, const float *Cgt, const float *Dp, const float *Dgt, float wf, float wc,
                        float wd, float invP, void *F, void *dLdF, float *dLdC, float *dLdD, float *part, float *h,
                        const int *err, cudaStream_t s)
{
    const size_t sm = blend_mma_smem();
    cudaFuncSetAttribute(k_blend_mma<K, LOSS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const long long per_cta = (long long)kMmaWarps * kMmaPix;
    const unsigned blocks = (unsigned)((n_pix + per_cta - 1) / per_cta);
    k_blend_mma<K, LOSS><<<blocks, kMmaWarps * 32, sm, s>>>(
        n_pix, D, idx, w, (const __nv_bfloat16 *)feats, (const __nv_bfloat16 *)Fgt, C, Cgt, Dp, Dgt, wf, wc, wd, invP,
        (__nv_bfloat16 *)F, (__nv_bfloat16 *)dLdF, dLdC, dLdD, part, h, err);
}

// F only (gs_feature_blend)
bool launch_blend_mma(int K, int D, long long n_pix, const int *idx, const float *w, const void *feats, void *F,
                      const int *err, cudaStream_t s)
{
    if (n_pix <= 0) return true;
#define GS_BM(KV) blend_mma_k<KV, false>(n_pix, D, idx, w, feats, nullptr, nullptr, nullptr, nullptr, nullptr, 0.f, 0.f, \
                                         0.f, 0.f, F, nullptr, nullptr, nullptr, nullptr, nullptr, err, s)
    switch (K) {
    case 2: GS_BM(2); return true;
    case 4: GS_BM(4); return true;
    case 8: GS_BM(8); return true;
    case 16: GS_BM(16); return true;
    }
#undef GS_BM
    return false;
}

// F, the loss gradients, the per-pixel loss shares and h (gs_feature_blend_loss)
bool launch_blend_loss_mma(int K, int D, long long n_pix, const int *idx, const float *w, const void *feats,
                           const void *Fgt, const float *C, const float *Cgt, const float *Dp, const float *Dgt,
                           float wf, float wc, float wd, float invP, void *F, void *dLdF, float *dLdC, float *dLdD,
                           float *part, float *h, const int *err, cudaStream_t s)
{
    if (n_pix <= 0) return true;
#define GS_BLM(KV) blend_mma_k<KV, true>(n_pix, D, idx, w, feats, Fgt, C, Cgt, Dp, Dgt, wf, wc, wd, invP, F, dLdF, \
                                         dLdC, dLdD, part, h, err, s)
    switch (K) {
    case 2: GS_BLM(2); return true;
    case 4: GS_BLM(4); return true;
    case 8: GS_BLM(8); return true;
    case 16: GS_BLM(16); return true;
    }
#undef GS_BLM
    return false;
}

// h = dL/dF . f per slot from a given dL/dF (the re-walk's feature term)
bool launch_h_mma(int K, int D, long long n_pix, const int *idx, const void *feats, const void *dLdF, float *h,
                  const int *err, cudaStream_t s)
{
    if (n_pix <= 0) return true;
    const size_t sm = blend_mma_smem();
    const long long per_cta = (long long)kMmaWarps * kMmaPix;
    const unsigned blocks = (unsigned)((n_pix + per_cta - 1) / per_cta);
#define GS_HM(KV)                                                                                                   \
    cudaFuncSetAttribute(k_h_mma<KV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);                        \
    k_h_mma<KV><<<blocks, kMmaWarps * 32, sm, s>>>(n_pix, D, idx, (const __nv_bfloat16 *)feats,                      \
                                                   (const __nv_bfloat16 *)dLdF, h, err)
    switch (K) {
    case 2: GS_HM(2); return true;
    case 4: GS_HM(4); return true;
    case 8: GS_HM(8); return true;
    case 16: GS_HM(16); return true;
    }
#undef GS_HM
    return false;
}

}  // namespace gs
