// gs_blend.cu -- a4: the K-row gather-blend of Eqs. 3-4, and the training loss.
//
// Gather-blend: F[p] = sum_k (w_k / S_p) f_{idx_k}.  This is a weighted gather with
// 2 K D flops per pixel against at least 4 D bytes written, far below the tensor-core
// ridge, so it runs on the CUDA cores and is shaped for HBM: a group of lanes owns one
// pixel (a full warp when the row has >= 32 16-byte chunks), every lane moves whole
// 16-byte chunks (float4, or 8 bf16), all K row loads of a chunk are issued before the
// FMAs, and the output row is written with 16-byte coalesced stores.  Rows reused by
// neighbouring pixels are served by L2.
#include "gs_internal.cuh"

namespace gs {

template <bool BF16>
struct Chunk;

template <>
struct Chunk<false> {                 // 4 floats
    static constexpr int VEC = 4;
    __device__ __forceinline__ static void load(const void *base, size_t chunk, float (&x)[4])
    {
        float4 v = __ldg((const float4 *)base + chunk);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
    __device__ __forceinline__ static void store(void *base, size_t chunk, const float (&x)[4])
    {
        ((float4 *)base)[chunk] = make_float4(x[0], x[1], x[2], x[3]);
    }
};

template <>
struct Chunk<true> {                  // 8 bf16
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
    __device__ __forceinline__ static void store(void *base, size_t chunk, const float (&x)[8])
    {
        uint4 v;
        __nv_bfloat162 *h = (__nv_bfloat162 *)&v;
#pragma unroll
        for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
        ((uint4 *)base)[chunk] = v;
    }
};

template <int KM, bool BF16>
__global__ void __launch_bounds__(256) k_blend(long long n_pix, int K, int nch, int lpp_log2,
                                               const int *__restrict__ idx, const float *__restrict__ wts,
                                               const void *__restrict__ feats, void *__restrict__ F,
                                               const int *__restrict__ err)
{
    using Ch = Chunk<BF16>;
    constexpr int VEC = Ch::VEC;
    const int lane = threadIdx.x & 31;
    const int lpp = 1 << lpp_log2;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long p = warp * (32 >> lpp_log2) + (lane >> lpp_log2);
    const int sub = lane & (lpp - 1);
    if (p >= n_pix) return;
    const bool bad = err && *err;
    int ids[KM];
    float ws[KM];
    float S = 0.f;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        ids[k] = -1;
        ws[k] = 0.f;
        if (k < K && !bad) {
            ids[k] = __ldg(idx + p * K + k);
            ws[k] = __ldg(wts + p * K + k);
            S += ws[k];
        }
    }
    const float inv = S > 0.f ? 1.f / S : 0.f;
#pragma unroll
    for (int k = 0; k < KM; ++k) ws[k] = ids[k] >= 0 ? ws[k] * inv : 0.f;
    for (int ch = sub; ch < nch; ch += lpp) {
        float x[KM][VEC];
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            if (ids[k] >= 0) {
                Ch::load(feats, (size_t)ids[k] * nch + ch, x[k]);
            } else {
#pragma unroll
                for (int i = 0; i < VEC; ++i) x[k][i] = 0.f;
            }
        }
        float acc[VEC];
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc[i] = 0.f;
#pragma unroll
        for (int k = 0; k < KM; ++k)
#pragma unroll
            for (int i = 0; i < VEC; ++i) acc[i] = fmaf(ws[k], x[k][i], acc[i]);
        Ch::store(F, (size_t)p * nch + ch, acc);
    }
}


// ------------------------------------------------------------------------------------
// Pixel-group form of the gather-blend.  Neighbouring pixels select mostly the same
// Gaussians, so a warp takes G consecutive pixels (G K <= 32 (id, w) pairs, one per
// lane), finds the distinct ids among them with a warp match, and loads each distinct
// row once for the whole group: every lane holds CPL 16-byte chunks of the row and
// adds it, with each pixel's renormalised weight (0 where the pixel did not select
// it), into G register accumulators.  The row traffic from L2 drops from G K rows to
// the group's distinct rows.  A pixel's terms are summed in the order of first
// occurrence in the group, so F depends only on the grouping (always G consecutive
// flat pixels), never on the tile shape; the blend-only and the fused kernels group
// identically and give bit-identical F.
// ------------------------------------------------------------------------------------
// pixels per warp of the group kernels, for the device code and the launch grids alike
__host__ __device__ constexpr int group_pixels(int KM) { return KM <= 8 ? 4 : 2; }
template <int KM>
struct Group {
    static constexpr int G = group_pixels(KM);            // pixels per warp (KM <= 16)
};

struct GroupTable {
    float w[32][4];                                       // distinct id x pixel
    int id[32];
    signed char slot[32][4];                              // slot of the id in each pixel, -1 if absent
};

// Loads the group's (id, w') pairs, builds the distinct-id table of this warp and
// returns the number of distinct ids.  Lane l holds pixel l / KM, slot l % KM.
template <int KM, int G, bool WITH_W = true>
__device__ __forceinline__ int group_table(long long p0, long long n_pix, int K, const int *__restrict__ idx,
                                           const float *__restrict__ wts, bool bad, int lane, GroupTable &t)
{
    const int gl = lane / KM, kl = lane - gl * KM;
    const long long pl = p0 + gl;
    int id = -1;
    float wn = 0.f;
    if (gl < G && kl < K && pl < n_pix && !bad) {
        id = __ldg(idx + pl * K + kl);
        if (WITH_W) {
            // S in slot order, exactly as the per-pixel kernels sum it
            float S = 0.f;
            for (int k = 0; k < K; ++k) S += __ldg(wts + pl * K + k);
            const float inv = S > 0.f ? 1.f / S : 0.f;
            wn = id >= 0 ? __ldg(wts + pl * K + kl) * inv : 0.f;
        }
    }
    const unsigned same = __match_any_sync(0xffffffffu, id);
    const int first = __ffs(same) - 1;
    const unsigned lead = __ballot_sync(0xffffffffu, id >= 0 && first == lane);
    const int U = __popc(lead);
    if (lane < U) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            t.w[lane][g] = 0.f;
            t.slot[lane][g] = -1;
        }
    }
    __syncwarp();
    if (id >= 0) {
        const int r = __popc(lead & ((1u << first) - 1u));
        t.w[r][gl] = wn;
        t.slot[r][gl] = (signed char)kl;
        if (first == lane) t.id[r] = id;
    }
    __syncwarp();
    return U;
}

// acc[g] = sum over the distinct rows u of w'[u][g] f_u, for chunks lane + 32 c.
// Two rows are in flight: the next row's loads are issued before this row's FMAs.
template <int G, bool BF16, int CPL>
__device__ __forceinline__ void group_accumulate(int U, int nch, int lane, const void *__restrict__ feats,
                                                 const GroupTable &t, float (&acc)[G][CPL][Chunk<BF16>::VEC])
{
    using Ch = Chunk<BF16>;
    constexpr int VEC = Ch::VEC;
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[g][c][v] = 0.f;
    auto load_row = [&](int u, float (&x)[CPL][VEC]) {
        const size_t base = (size_t)t.id[u] * nch;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int ch = lane + 32 * c;
            if (ch < nch) Ch::load(feats, base + ch, x[c]);
            else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) x[c][v] = 0.f;
            }
        }
    };
    auto add_row = [&](int u, const float (&x)[CPL][VEC]) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const float wg = t.w[u][g];
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[g][c][v] = fmaf(wg, x[c][v], acc[g][c][v]);
        }
    };
    float xa[CPL][VEC], xb[CPL][VEC];
    if (U > 0) load_row(0, xa);
    for (int u = 0; u < U; u += 2) {
        if (u + 1 < U) load_row(u + 1, xb);
        add_row(u, xa);
        if (u + 1 < U) {
            if (u + 2 < U) load_row(u + 2, xa);
            add_row(u + 1, xb);
        }
    }
}

template <int KM, bool BF16, int CPL>
__global__ void __launch_bounds__(256, 2) k_blend_group(long long n_pix, int K, int nch, const int *__restrict__ idx,
                                                     const float *__restrict__ wts, const void *__restrict__ feats,
                                                     void *__restrict__ F, const int *__restrict__ err)
{
    using Ch = Chunk<BF16>;
    constexpr int VEC = Ch::VEC;
    constexpr int G = Group<KM>::G;
    __shared__ GroupTable s_t[8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long p0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * G;
    if (p0 >= n_pix) return;                         // whole warp leaves together
    const bool bad = err && *err;
    GroupTable &t = s_t[wib];
    const int U = group_table<KM, G>(p0, n_pix, K, idx, wts, bad, lane, t);
    float acc[G][CPL][VEC];
    group_accumulate<G, BF16, CPL>(U, nch, lane, feats, t, acc);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (p0 + g >= n_pix) break;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int ch = lane + 32 * c;
            if (ch < nch) Ch::store(F, (size_t)(p0 + g) * nch + ch, acc[g][c]);
        }
    }
}

// The group form serves K <= 16 and nch >= 32 16-byte chunks while the G accumulator
// rows fit in 64 registers per lane (G CPL VEC <= 64): float32 rows D 128..512 at
// K <= 8 and D 128..1024 at K <= 16; bf16 rows D 256..512 at K <= 8 and 256..1024 at
// K <= 16.  Other widths and K keep the per-pixel kernels.
template <int KM, bool BF16, int CPL>
struct GroupFits {
    static constexpr bool value = Group<KM>::G * CPL * Chunk<BF16>::VEC <= 64;
};

static int group_cpl(int dtype, int K, int nch)
{
    if (K > 16 || nch < 32) return 0;
    const int need = (nch + 31) / 32;
    const int cpl = need <= 1 ? 1 : need <= 2 ? 2 : need <= 4 ? 4 : need <= 8 ? 8 : 16;
    const int G = K <= 8 ? 4 : 2;
    const int vec = dtype == GS_BF16 ? 8 : 4;
    return G * cpl * vec <= 64 ? cpl : 0;
}

template <int KM, bool BF16>
static void blend_group_launch(int cpl, unsigned blocks, cudaStream_t s, long long n_pix, int K, int nch,
                               const int *idx, const float *w, const void *feats, void *F, const int *err)
{
    switch (cpl) {
    case 1: k_blend_group<KM, BF16, 1><<<blocks, 256, 0, s>>>(n_pix, K, nch, idx, w, feats, F, err); break;
    case 2: k_blend_group<KM, BF16, 2><<<blocks, 256, 0, s>>>(n_pix, K, nch, idx, w, feats, F, err); break;
    case 4:
        if constexpr (GroupFits<KM, BF16, 4>::value)
            k_blend_group<KM, BF16, 4><<<blocks, 256, 0, s>>>(n_pix, K, nch, idx, w, feats, F, err);
        break;
    case 8:
        if constexpr (GroupFits<KM, BF16, 8>::value)
            k_blend_group<KM, BF16, 8><<<blocks, 256, 0, s>>>(n_pix, K, nch, idx, w, feats, F, err);
        break;
    }
}

static int lpp_log2_for(int nch)
{
    int l = 0;
    while (l < 5 && (2 << l) <= nch) ++l;
    return l;
}

template <bool BF16>
static bool blend_k(int KM, int K, int nch, long long n_pix, const int *idx, const float *w, const void *feats,
                    void *F, const int *err, cudaStream_t s)
{
    int l = lpp_log2_for(nch);
    long long warps = (n_pix + (32 >> l) - 1) / (32 >> l);
    unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    switch (KM) {
    case 4: k_blend<4, BF16><<<blocks, 256, 0, s>>>(n_pix, K, nch, l, idx, w, feats, F, err); return true;
    case 8: k_blend<8, BF16><<<blocks, 256, 0, s>>>(n_pix, K, nch, l, idx, w, feats, F, err); return true;
    case 16: k_blend<16, BF16><<<blocks, 256, 0, s>>>(n_pix, K, nch, l, idx, w, feats, F, err); return true;
    case 32: k_blend<32, BF16><<<blocks, 256, 0, s>>>(n_pix, K, nch, l, idx, w, feats, F, err); return true;
    }
    return false;
}

bool launch_blend(int dtype, int K, int D, long long n_pix, long long N, const int *idx, const float *w,
                  const void *feats, void *F, const int *err, cudaStream_t s)
{
    if (n_pix <= 0) return true;
    if (blend_mma_supported(dtype, K, D, N)) return launch_blend_mma(K, D, n_pix, idx, w, feats, F, err, s);
    int KM = K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32;
    const int nch = dtype == GS_BF16 ? D / 8 : D / 4;
    const int cpl = group_cpl(dtype, K, nch);
    if (cpl) {
        const int G = group_pixels(KM);
        const long long warps = (n_pix + G - 1) / G;
        const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
        if (dtype == GS_BF16) {
            switch (KM) {
            case 4: blend_group_launch<4, true>(cpl, blocks, s, n_pix, K, nch, idx, w, feats, F, err); break;
            case 8: blend_group_launch<8, true>(cpl, blocks, s, n_pix, K, nch, idx, w, feats, F, err); break;
            default: blend_group_launch<16, true>(cpl, blocks, s, n_pix, K, nch, idx, w, feats, F, err); break;
            }
        } else {
            switch (KM) {
            case 4: blend_group_launch<4, false>(cpl, blocks, s, n_pix, K, nch, idx, w, feats, F, err); break;
            case 8: blend_group_launch<8, false>(cpl, blocks, s, n_pix, K, nch, idx, w, feats, F, err); break;
            default: blend_group_launch<16, false>(cpl, blocks, s, n_pix, K, nch, idx, w, feats, F, err); break;
            }
        }
        return true;
    }
    if (dtype == GS_BF16) return blend_k<true>(KM, K, nch, n_pix, idx, w, feats, F, err, s);
    return blend_k<false>(KM, K, nch, n_pix, idx, w, feats, F, err, s);
}

// ------------------------------------------------------------------------------------
// h_k(p) = dL/dF_p . f_{idx_k(p)} for every Top-K slot (the feature term of dL/dw used
// by the re-walk of a5).  Pixel-group form: a warp holds the dL/dF rows of its G pixels
// in registers, loads each distinct selected row once, forms the G partial dot products
// per lane and reduces them over the warp with one reduce-scatter (lane l ends with the
// total of pixel (l >> 3) & 3).  Per-pixel form (other widths, K > 16): a group of lanes
// per pixel, one reduction per slot.
// ------------------------------------------------------------------------------------
template <int G, bool BF16, int CPL>
__device__ __forceinline__ void group_h(int U, int nch, int K, int lane, long long p0, const void *__restrict__ feats,
                                        const GroupTable &t, const float (&d)[G][CPL][Chunk<BF16>::VEC],
                                        float *__restrict__ h)
{
    using Ch = Chunk<BF16>;
    constexpr int VEC = Ch::VEC;
    auto load_row = [&](int u, float (&x)[CPL][VEC]) {
        const size_t base = (size_t)t.id[u] * nch;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int ch = lane + 32 * c;
            if (ch < nch) Ch::load(feats, base + ch, x[c]);
            else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) x[c][v] = 0.f;
            }
        }
    };
    auto dot_row = [&](int u, const float (&x)[CPL][VEC]) {
        float pd[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) pd[g] = 0.f;
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int v = 0; v < VEC; ++v) pd[g] = fmaf(d[g][c][v], x[c][v], pd[g]);
        // reduce-scatter of 4 values: lane l ends with the total of value (l >> 3) & 3
        const bool b4 = lane & 16, b3 = lane & 8;
        float a0 = (b4 ? pd[2] : pd[0]) + __shfl_xor_sync(0xffffffffu, b4 ? pd[0] : pd[2], 16);
        float a1 = (b4 ? pd[3] : pd[1]) + __shfl_xor_sync(0xffffffffu, b4 ? pd[1] : pd[3], 16);
        float r = (b3 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, b3 ? a0 : a1, 8);
        r += __shfl_xor_sync(0xffffffffu, r, 4);
        r += __shfl_xor_sync(0xffffffffu, r, 2);
        r += __shfl_xor_sync(0xffffffffu, r, 1);
        const int g = (lane >> 3) & 3;
        if ((lane & 7) == 0 && g < G) {
            const int k = t.slot[u][g];
            if (k >= 0) h[(p0 + g) * K + k] = r;
        }
    };
    float xa[CPL][VEC], xb[CPL][VEC];
    if (U > 0) load_row(0, xa);
    for (int u = 0; u < U; u += 2) {
        if (u + 1 < U) load_row(u + 1, xb);
        dot_row(u, xa);
        if (u + 1 < U) {
            if (u + 2 < U) load_row(u + 2, xa);
            dot_row(u + 1, xb);
        }
    }
}

template <int KM, bool BF16, int CPL>
__global__ void __launch_bounds__(256, 2) k_h_group(long long n_pix, int K, int nch, const int *__restrict__ idx,
                                                 const void *__restrict__ feats, const void *__restrict__ dLdF,
                                                 float *__restrict__ h, const int *__restrict__ err)
{
    using Ch = Chunk<BF16>;
    constexpr int VEC = Ch::VEC;
    constexpr int G = Group<KM>::G;
    __shared__ GroupTable s_t[8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long p0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * G;
    if (p0 >= n_pix) return;                         // whole warp leaves together
    const bool bad = err && *err;
    GroupTable &t = s_t[wib];
    const int U = group_table<KM, G, false>(p0, n_pix, K, idx, nullptr, bad, lane, t);
    float d[G][CPL][VEC];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int ch = lane + 32 * c;
            if (p0 + g < n_pix && ch < nch) Ch::load(dLdF, (size_t)(p0 + g) * nch + ch, d[g][c]);
            else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) d[g][c][v] = 0.f;
            }
        }
    group_h<G, BF16, CPL>(U, nch, K, lane, p0, feats, t, d, h);
}

template <bool BF16>
__global__ void __launch_bounds__(256) k_h_pixel(long long n_pix, int K, int nch, int lpp_log2,
                                                 const int *__restrict__ idx, const void *__restrict__ feats,
                                                 const void *__restrict__ dLdF, float *__restrict__ h,
                                                 const int *__restrict__ err)
{
    using Ch = Chunk<BF16>;
    constexpr int VEC = Ch::VEC;
    const int lane = threadIdx.x & 31;
    const int lpp = 1 << lpp_log2;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long p = warp * (32 >> lpp_log2) + (lane >> lpp_log2);
    const int sub = lane & (lpp - 1);
    const bool live = p < n_pix;
    if (!live) p = n_pix - 1;                        // keep every lane in the shuffles
    const bool bad = err && *err;
    for (int k = 0; k < K; ++k) {
        const int id = bad ? -1 : __ldg(idx + p * K + k);
        float part = 0.f;
        if (id >= 0) {
            for (int ch = sub; ch < nch; ch += lpp) {
                float a[VEC], b[VEC];
                Ch::load(dLdF, (size_t)p * nch + ch, a);
                Ch::load(feats, (size_t)id * nch + ch, b);
#pragma unroll
                for (int v = 0; v < VEC; ++v) part = fmaf(a[v], b[v], part);
            }
        }
        for (int o = 1; o < lpp; o <<= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (live && sub == 0 && id >= 0) h[p * K + k] = part;
    }
}

bool launch_h(int dtype, int K, int D, long long n_pix, long long N, const int *idx, const void *feats,
              const void *dLdF, float *h, const int *err, cudaStream_t s)
{
    if (n_pix <= 0) return true;
    if (blend_mma_supported(dtype, K, D, N)) return launch_h_mma(K, D, n_pix, idx, feats, dLdF, h, err, s);
    const int KM = K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32;
    const int nch = dtype == GS_BF16 ? D / 8 : D / 4;
    const int cpl = group_cpl(dtype, K, nch);
    if (cpl) {
        const int G = group_pixels(KM);
        const long long warps = (n_pix + G - 1) / G;
        const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
#define GS_HG(KMV, BF)                                                                                            \
    switch (cpl) {                                                                                                \
    case 1: k_h_group<KMV, BF, 1><<<blocks, 256, 0, s>>>(n_pix, K, nch, idx, feats, dLdF, h, err); break;          \
    case 2: k_h_group<KMV, BF, 2><<<blocks, 256, 0, s>>>(n_pix, K, nch, idx, feats, dLdF, h, err); break;          \
    case 4:                                                                                                       \
        if constexpr (GroupFits<KMV, BF, 4>::value)                                                                \
            k_h_group<KMV, BF, 4><<<blocks, 256, 0, s>>>(n_pix, K, nch, idx, feats, dLdF, h, err);                 \
        break;                                                                                                    \
    case 8:                                                                                                       \
        if constexpr (GroupFits<KMV, BF, 8>::value)                                                                \
            k_h_group<KMV, BF, 8><<<blocks, 256, 0, s>>>(n_pix, K, nch, idx, feats, dLdF, h, err);                 \
        break;                                                                                                    \
    }
        if (dtype == GS_BF16) {
            switch (KM) { case 4: GS_HG(4, true); break; case 8: GS_HG(8, true); break; default: GS_HG(16, true); }
        } else {
            switch (KM) { case 4: GS_HG(4, false); break; case 8: GS_HG(8, false); break; default: GS_HG(16, false); }
        }
#undef GS_HG
        return true;
    }
    const int l = lpp_log2_for(nch);
    const long long warps = (n_pix + (32 >> l) - 1) / (32 >> l);
    const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    if (dtype == GS_BF16) k_h_pixel<true><<<blocks, 256, 0, s>>>(n_pix, K, nch, l, idx, feats, dLdF, h, err);
    else k_h_pixel<false><<<blocks, 256, 0, s>>>(n_pix, K, nch, l, idx, feats, dLdF, h, err);
    return true;
}

// ------------------------------------------------------------------------------------
// Loss: w_feat (1 - cos(F, Fgt)) + w_rgb |C - Cgt|_1 / 3 + w_depth |D - Dgt|, averaged
// over pixels.  Per-pixel values go to `part`, then a fixed-order two-level sum.
// ------------------------------------------------------------------------------------
template <bool BF16>
__global__ void __launch_bounds__(256) k_loss(long long n_pix, int nch, int lpp_log2, const void *__restrict__ F,
                                              const void *__restrict__ Fgt, const float *__restrict__ C,
                                              const float *__restrict__ Cgt, const float *__restrict__ Dp,
                                              const float *__restrict__ Dgt, float wf, float wc, float wd,
                                              void *__restrict__ dLdF, float *__restrict__ dLdC,
                                              float *__restrict__ dLdD, float *__restrict__ part)
{
    using Ch = Chunk<BF16>;
    constexpr int VEC = Ch::VEC;
    const int lane = threadIdx.x & 31;
    const int lpp = 1 << lpp_log2;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long p = warp * (32 >> lpp_log2) + (lane >> lpp_log2);
    const int sub = lane & (lpp - 1);
    const bool live = p < n_pix;
    if (!live) p = n_pix - 1;                    // keep every lane in the shuffles
    float ff = 0.f, fg = 0.f, gg = 0.f;
    for (int ch = sub; ch < nch; ch += lpp) {
        float a[VEC], b[VEC];
        Ch::load(F, (size_t)p * nch + ch, a);
        Ch::load(Fgt, (size_t)p * nch + ch, b);
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
            ff = fmaf(a[i], a[i], ff);
            fg = fmaf(a[i], b[i], fg);
            gg = fmaf(b[i], b[i], gg);
        }
    }
    for (int o = 1; o < lpp; o <<= 1) {
        ff += __shfl_xor_sync(0xffffffffu, ff, o);
        fg += __shfl_xor_sync(0xffffffffu, fg, o);
        gg += __shfl_xor_sync(0xffffffffu, gg, o);
    }
    if (!live) return;
    const float invP = 1.f / (float)n_pix;
    float nf = sqrtf(ff), ng = sqrtf(gg);
    bool ok = nf > 0.f && ng > 0.f;
    float cosv = ok ? fg / (nf * ng) : 0.f;
    float ca = ok ? -wf * invP / (nf * ng) : 0.f;          // coefficient of Fgt
    float cb = ok ? wf * invP * cosv / ff : 0.f;           // coefficient of F
    for (int ch = sub; ch < nch; ch += lpp) {
        float a[VEC], b[VEC], gdx[VEC];
        Ch::load(F, (size_t)p * nch + ch, a);
        Ch::load(Fgt, (size_t)p * nch + ch, b);
#pragma unroll
        for (int i = 0; i < VEC; ++i) gdx[i] = fmaf(ca, b[i], cb * a[i]);
        Ch::store(dLdF, (size_t)p * nch + ch, gdx);
    }
    if (sub == 0) {
        float l = wf * (1.f - cosv);
        float lc = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float d = C[3 * p + i] - Cgt[3 * p + i];
            lc += fabsf(d);
            dLdC[3 * p + i] = wc * invP / 3.f * (float)((d > 0.f) - (d < 0.f));
        }
        float dd = Dp[p] - Dgt[p];
        dLdD[p] = wd * invP * (float)((dd > 0.f) - (dd < 0.f));
        part[p] = (l + wc * lc / 3.f + wd * fabsf(dd)) * invP;
    }
}

__global__ void __launch_bounds__(1024) k_sum_fixed(const float *__restrict__ in, long long n, float *out)
{
    // fixed-order: each thread a contiguous slice, then a tree over threads
    __shared__ float sm[1024];
    long long per = (n + gridDim.x * 1024ll - 1) / (gridDim.x * 1024ll);
    long long b = ((long long)blockIdx.x * 1024 + threadIdx.x) * per, e = min(b + per, n);
    float s = 0.f;
    for (long long i = b; i < e; ++i) s += in[i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sm[0];
}

// ------------------------------------------------------------------------------------
// Fused training form: gather-blend (Eqs. 3-4) and the loss gradient in one pass with
// the k_blend layout (a group of lanes per pixel, many small CTAs): each pixel's F row
// is built in registers, the target row is read, |F|^2, F.Fgt, |Fgt|^2 are reduced
// over the pixel's lanes, and F and dL/dF are written -- F is never read back.
// ------------------------------------------------------------------------------------
template <int KM, bool BF16, int CPL>
__global__ void __launch_bounds__(256) k_blend_loss(long long n_pix, int K, int nch, int lpp_log2,
                                                    const int *__restrict__ idx, const float *__restrict__ wts,
                                                    const void *__restrict__ feats, const void *__restrict__ Fgt,
                                                    const float *__restrict__ C, const float *__restrict__ Cgt,
                                                    const float *__restrict__ Dp, const float *__restrict__ Dgt,
                                                    float wf, float wc, float wd, float invP, void *__restrict__ F,
                                                    void *__restrict__ dLdF, float *__restrict__ dLdC,
                                                    float *__restrict__ dLdD, float *__restrict__ part,
                                                    const int *__restrict__ err)
{
    using Ch = Chunk<BF16>;
    constexpr int VEC = Ch::VEC;
    const int lane = threadIdx.x & 31;
    const int lpp = 1 << lpp_log2;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    long long p = warp * (32 >> lpp_log2) + (lane >> lpp_log2);
    const int sub = lane & (lpp - 1);
    const bool live = p < n_pix;
    if (!live) p = n_pix - 1;                      // keep every lane in the shuffles
    const bool bad = *err != 0;
    int ids[KM];
    float ws[KM], S = 0.f;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        ids[k] = -1;
        ws[k] = 0.f;
        if (k < K && !bad) {
            ids[k] = __ldg(idx + p * K + k);
            ws[k] = __ldg(wts + p * K + k);
            S += ws[k];
        }
    }
    const float inv = S > 0.f ? 1.f / S : 0.f;
#pragma unroll
    for (int k = 0; k < KM; ++k) ws[k] = ids[k] >= 0 ? ws[k] * inv : 0.f;
    float f[CPL][VEC], g[CPL][VEC];
    float ff = 0.f, fg = 0.f, gg = 0.f;
#pragma unroll
    for (int cc = 0; cc < CPL; ++cc) {
        const int ch = sub + cc * lpp;
#pragma unroll
        for (int v = 0; v < VEC; ++v) { f[cc][v] = 0.f; g[cc][v] = 0.f; }
        if (ch < nch) {
            float x[KM][VEC];
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                if (ids[k] >= 0) Ch::load(feats, (size_t)ids[k] * nch + ch, x[k]);
                else {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) x[k][v] = 0.f;
                }
            }
            Ch::load(Fgt, (size_t)p * nch + ch, g[cc]);
#pragma unroll
            for (int k = 0; k < KM; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) f[cc][v] = fmaf(ws[k], x[k][v], f[cc][v]);
            if (live) Ch::store(F, (size_t)p * nch + ch, f[cc]);
            if (BF16) {            // the loss sees F as stored
#pragma unroll
                for (int v = 0; v < VEC; ++v) f[cc][v] = __bfloat162float(__float2bfloat16(f[cc][v]));
            }
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                ff = fmaf(f[cc][v], f[cc][v], ff);
                fg = fmaf(f[cc][v], g[cc][v], fg);
                gg = fmaf(g[cc][v], g[cc][v], gg);
            }
        }
    }
    for (int o = 1; o < lpp; o <<= 1) {
        ff += __shfl_xor_sync(0xffffffffu, ff, o);
        fg += __shfl_xor_sync(0xffffffffu, fg, o);
        gg += __shfl_xor_sync(0xffffffffu, gg, o);
    }
    if (!live) return;
    const float nf = sqrtf(ff), ng = sqrtf(gg);
    const bool ok = nf > 0.f && ng > 0.f;
    const float cosv = ok ? fg / (nf * ng) : 0.f;
    const float ca = ok ? -wf * invP / (nf * ng) : 0.f;
    const float cb = ok ? wf * invP * cosv / ff : 0.f;
#pragma unroll
    for (int cc = 0; cc < CPL; ++cc) {
        const int ch = sub + cc * lpp;
        if (ch < nch) {
            float gdx[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) gdx[v] = fmaf(ca, g[cc][v], cb * f[cc][v]);
            Ch::store(dLdF, (size_t)p * nch + ch, gdx);
        }
    }
    if (sub == 0) {
        float lc = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float d = C[3 * p + i] - Cgt[3 * p + i];
            lc += fabsf(d);
            dLdC[3 * p + i] = wc * invP / 3.f * (float)((d > 0.f) - (d < 0.f));
        }
        float dd = Dp[p] - Dgt[p];
        dLdD[p] = wd * invP * (float)((dd > 0.f) - (dd < 0.f));
        part[p] = (wf * (1.f - cosv) + wc * lc / 3.f + wd * fabsf(dd)) * invP;
    }
}


// Fused training form in the pixel-group layout: the G rows of F are built in
// registers as in k_blend_group, then pixel by pixel the target row is read, |F|^2,
// F.Fgt and |Fgt|^2 are reduced over the warp, and F and dL/dF are written.
template <int KM, bool BF16, int CPL>
__global__ void __launch_bounds__(256, 2) k_blend_loss_group(long long n_pix, int K, int nch,
                                                          const int *__restrict__ idx, const float *__restrict__ wts,
                                                          const void *__restrict__ feats, const void *__restrict__ Fgt,
                                                          const float *__restrict__ C, const float *__restrict__ Cgt,
                                                          const float *__restrict__ Dp, const float *__restrict__ Dgt,
                                                          float wf, float wc, float wd, float invP,
                                                          void *__restrict__ F, void *__restrict__ dLdF,
                                                          float *__restrict__ dLdC, float *__restrict__ dLdD,
                                                          float *__restrict__ part, float *__restrict__ h,
                                                          const int *__restrict__ err)
{
    using Ch = Chunk<BF16>;
    constexpr int VEC = Ch::VEC;
    constexpr int G = Group<KM>::G;
    __shared__ GroupTable s_t[8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long p0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * G;
    if (p0 >= n_pix) return;
    {
        // start the target rows on their way to L2 while the blend gathers feature rows
        const long long pend = min(p0 + G, n_pix);
        const char *a = (const char *)Fgt + (size_t)p0 * nch * 16;
        const long long lines = ((pend - p0) * nch * 16 + 127) / 128;
        for (long long l = lane; l < lines; l += 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(a + 128 * l));
    }
    const bool bad = *err != 0;
    GroupTable &t = s_t[wib];
    const int U = group_table<KM, G>(p0, n_pix, K, idx, wts, bad, lane, t);
    float acc[G][CPL][VEC];
    group_accumulate<G, BF16, CPL>(U, nch, lane, feats, t, acc);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const long long p = p0 + g;
        if (p >= n_pix) {                           // warp-uniform
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[g][c][v] = 0.f;
            continue;
        }
        float gt[CPL][VEC];
        float ff = 0.f, fg = 0.f, gg = 0.f;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int ch = lane + 32 * c;
#pragma unroll
            for (int v = 0; v < VEC; ++v) gt[c][v] = 0.f;
            if (ch < nch) {
                Ch::load(Fgt, (size_t)p * nch + ch, gt[c]);
                Ch::store(F, (size_t)p * nch + ch, acc[g][c]);
                if (BF16) {            // the loss sees F as stored
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[g][c][v] = __bfloat162float(__float2bfloat16(acc[g][c][v]));
                }
            }
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                ff = fmaf(acc[g][c][v], acc[g][c][v], ff);
                fg = fmaf(acc[g][c][v], gt[c][v], fg);
                gg = fmaf(gt[c][v], gt[c][v], gg);
            }
        }
        for (int o = 1; o < 32; o <<= 1) {
            ff += __shfl_xor_sync(0xffffffffu, ff, o);
            fg += __shfl_xor_sync(0xffffffffu, fg, o);
            gg += __shfl_xor_sync(0xffffffffu, gg, o);
        }
        const float nf = sqrtf(ff), ng = sqrtf(gg);
        const bool ok = nf > 0.f && ng > 0.f;
        const float cosv = ok ? fg / (nf * ng) : 0.f;
        const float ca = ok ? -wf * invP / (nf * ng) : 0.f;
        const float cb = ok ? wf * invP * cosv / ff : 0.f;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int ch = lane + 32 * c;
            if (ch < nch) {
                float gdx[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) gdx[v] = fmaf(ca, gt[c][v], cb * acc[g][c][v]);
                Ch::store(dLdF, (size_t)p * nch + ch, gdx);
                // acc now holds dL/dF as stored, for h below
#pragma unroll
                for (int v = 0; v < VEC; ++v)
                    acc[g][c][v] = BF16 ? __bfloat162float(__float2bfloat16(gdx[v])) : gdx[v];
            } else {
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[g][c][v] = 0.f;
            }
        }
        if (lane == g) {
            float lc = 0.f;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float d = C[3 * p + i] - Cgt[3 * p + i];
                lc += fabsf(d);
                dLdC[3 * p + i] = wc * invP / 3.f * (float)((d > 0.f) - (d < 0.f));
            }
            float dd = Dp[p] - Dgt[p];
            dLdD[p] = wd * invP * (float)((dd > 0.f) - (dd < 0.f));
            part[p] = (wf * (1.f - cosv) + wc * lc / 3.f + wd * fabsf(dd)) * invP;
        }
    }
    // the re-walk's per-slot terms h = dL/dF . f, from rows the blend just read (L2)
    if (h) group_h<G, BF16, CPL>(U, nch, K, lane, p0, feats, t, acc, h);
}

template <int KM, bool BF16>
static void blend_loss_group_launch(int cpl, unsigned blocks, cudaStream_t s, long long n_pix, int K, int nch,
                                    const int *idx, const float *w, const void *feats, const void *Fgt, const float *C,
                                    const float *Cgt, const float *Dp, const float *Dgt, float wf, float wc, float wd,
                                    float invP, void *F, void *dLdF, float *dLdC, float *dLdD, float *part, float *h,
                                    const int *err)
{
#define GS_BLGC(CP)                                                                                                   \
    k_blend_loss_group<KM, BF16, CP><<<blocks, 256, 0, s>>>(n_pix, K, nch, idx, w, feats, Fgt, C, Cgt, Dp, Dgt, wf, wc, \
                                                            wd, invP, F, dLdF, dLdC, dLdD, part, h, err)
    switch (cpl) {
    case 1: GS_BLGC(1); break;
    case 2: GS_BLGC(2); break;
    case 4:
        if constexpr (GroupFits<KM, BF16, 4>::value) GS_BLGC(4);
        break;
    case 8:
        if constexpr (GroupFits<KM, BF16, 8>::value) GS_BLGC(8);
        break;
    }
#undef GS_BLGC
}

template <int KM, bool BF16>
static bool blend_loss_cpl(int cpl, unsigned blocks, long long n_pix, int K, int nch, int l, const int *idx,
                           const float *w, const void *feats, const void *Fgt, const float *C, const float *Cgt,
                           const float *Dp, const float *Dgt, float wf, float wc, float wd, float invP, void *F,
                           void *dLdF, float *dLdC, float *dLdD, float *part, const int *err, cudaStream_t s)
{
#define GS_BL(CP) k_blend_loss<KM, BF16, CP><<<blocks, 256, 0, s>>>(n_pix, K, nch, l, idx, w, feats, Fgt, C, Cgt, Dp, \
                                                                   Dgt, wf, wc, wd, invP, F, dLdF, dLdC, dLdD,   \
                                                                   part, err)
    switch (cpl) {
    case 1: GS_BL(1); return true;
    case 2: GS_BL(2); return true;
    case 4: GS_BL(4); return true;
    case 8: GS_BL(8); return true;
    }
#undef GS_BL
    return false;
}

bool blend_loss_writes_h(int dtype, int K, int D, long long N)
{
    return blend_mma_supported(dtype, K, D, N) || group_cpl(dtype, K, dtype == GS_BF16 ? D / 8 : D / 4) != 0;
}

bool launch_blend_loss(const CamTable &ct, int dtype, int K, int D, long long n_pix, long long N, const int *idx,
                       const float *w, const void *feats, const void *Fgt, const float *C, const float *Cgt,
                       const float *Dp, const float *Dgt, float wf, float wc, float wd, void *F, void *dLdF,
                       float *dLdC, float *dLdD, float *loss, float *part, float *h, const int *err, cudaStream_t s)
{
    (void)ct;
    if (n_pix <= 0) return true;
    if (blend_mma_supported(dtype, K, D, N)) {
        if (!launch_blend_loss_mma(K, D, n_pix, idx, w, feats, Fgt, C, Cgt, Dp, Dgt, wf, wc, wd, 1.f / (float)n_pix, F,
                                   dLdF, dLdC, dLdD, part, h, err, s))
            return false;
        float *part2 = part + n_pix;
        k_sum_fixed<<<kSortBlocks, 1024, 0, s>>>(part, n_pix, part2);
        k_sum_fixed<<<1, 1024, 0, s>>>(part2, kSortBlocks, loss);
        return true;
    }
    const int KM = K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32;
    const int nch = dtype == GS_BF16 ? D / 8 : D / 4;
    const int l = lpp_log2_for(nch);
    const int lpp = 1 << l;
    const int cpl_need = (nch + lpp - 1) / lpp;
    const int cpl = cpl_need <= 1 ? 1 : cpl_need <= 2 ? 2 : cpl_need <= 4 ? 4 : 8;
    const long long warps = (n_pix + (32 >> l) - 1) / (32 >> l);
    const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    const float invP = 1.f / (float)n_pix;
    bool ok = true;
    const int gcpl = group_cpl(dtype, K, nch);
    if (gcpl) {
        const int G = group_pixels(KM);
        const long long gw = (n_pix + G - 1) / G;
        const unsigned gblocks = (unsigned)((gw * 32 + 255) / 256);
#define GS_BLG(KMV, BF)                                                                                          \
    blend_loss_group_launch<KMV, BF>(gcpl, gblocks, s, n_pix, K, nch, idx, w, feats, Fgt, C, Cgt, Dp, Dgt, wf, wc, \
                                     wd, invP, F, dLdF, dLdC, dLdD, part, h, err)
        if (dtype == GS_BF16) {
            switch (KM) { case 4: GS_BLG(4, true); break; case 8: GS_BLG(8, true); break; default: GS_BLG(16, true); }
        } else {
            switch (KM) { case 4: GS_BLG(4, false); break; case 8: GS_BLG(8, false); break; default: GS_BLG(16, false); }
        }
#undef GS_BLG
    } else {
#define GS_BK(KMV, BF) ok = blend_loss_cpl<KMV, BF>(cpl, blocks, n_pix, K, nch, l, idx, w, feats, Fgt, C, Cgt, Dp, Dgt, \
                                                    wf, wc, wd, invP, F, dLdF, dLdC, dLdD, part, err, s)
    if (dtype == GS_BF16) {
        switch (KM) { case 4: GS_BK(4, true); break; case 8: GS_BK(8, true); break; case 16: GS_BK(16, true); break; default: GS_BK(32, true); }
    } else {
        switch (KM) { case 4: GS_BK(4, false); break; case 8: GS_BK(8, false); break; case 16: GS_BK(16, false); break; default: GS_BK(32, false); }
    }
#undef GS_BK
    }
    if (!ok) return false;
    float *part2 = part + n_pix;
    k_sum_fixed<<<kSortBlocks, 1024, 0, s>>>(part, n_pix, part2);
    k_sum_fixed<<<1, 1024, 0, s>>>(part2, kSortBlocks, loss);
    return true;
}

bool launch_loss(int dtype, int D, long long n_pix, const void *F, const void *Fgt, const float *C, const float *Cgt,
                 const float *Dp, const float *Dgt, float wf, float wc, float wd, void *dLdF, float *dLdC,
                 float *dLdD, float *loss, float *part, cudaStream_t s)
{
    if (n_pix <= 0) return true;
    int nch = dtype == GS_BF16 ? D / 8 : D / 4;
    int l = lpp_log2_for(nch);
    long long warps = (n_pix + (32 >> l) - 1) / (32 >> l);
    unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    if (dtype == GS_BF16)
        k_loss<true><<<blocks, 256, 0, s>>>(n_pix, nch, l, F, Fgt, C, Cgt, Dp, Dgt, wf, wc, wd, dLdF, dLdC, dLdD, part);
    else
        k_loss<false><<<blocks, 256, 0, s>>>(n_pix, nch, l, F, Fgt, C, Cgt, Dp, Dgt, wf, wc, wd, dLdF, dLdC, dLdD, part);
    float *part2 = part + n_pix;
    k_sum_fixed<<<kSortBlocks, 1024, 0, s>>>(part, n_pix, part2);
    k_sum_fixed<<<1, 1024, 0, s>>>(part2, kSortBlocks, loss);
    return true;
}

}  // namespace gs
