// gs_tilegrad.cu -- feature part of a5, tile-major: every dL/dF row is read from HBM
// once.
//
//   dL/df_g = sum over (pixel p, slot k) with idx_k(p) = g of w'_k(p) dL/dF_p     (Eqs. 3-4)
//   h_k(p)  = dL/dF_p . f_{idx_k(p)}     (needed by the re-walk for dL/dw of Top-K members)
//
// Stage T1 (k_tile_slots): one CTA per screen tile sorts the tile's (Gaussian, slot)
//   keys in shared memory (bitonic: deterministic), stores them, and counts the distinct
//   Gaussians U_t selected in the tile.
// Stage T2: exclusive scan of U_t over tiles gives every (tile, Gaussian) its partial
//   row -- deterministic, no atomics.  A (tile, Gaussian) selection is always one of the
//   binning instances, so the row count is bounded by the instance count.
// Stage T3 (k_tile_accum): one 512-thread CTA per tile and per SM.  Each warp takes an
//   equal contiguous share of the tile's sorted slots and processes whole rows (16 B
//   per lane per 128-column chunk, all chunks of a row at once): it sums w' dL/dF over
//   the slots of each Gaussian in registers and forms the slot dot products h (one
//   reduce-scatter per 8 slots).  A Gaussian whose slots straddle warps is finished in
//   fixed order from shared-memory edge rows.  The tile's dL/dF rows are read from HBM
//   once and then re-read K times from L2 while the CTA lives: one CTA per SM keeps
//   148 x 512 KB of rows resident in the 126 MB L2.  (Staging 256-byte column slices in
//   shared memory with TMA was measured slower: the slices are too narrow to amortise
//   the per-slot work.)
// Stage T4: the partial rows are reduced per Gaussian by the sort-by-Gaussian segmented
//   reduction of gs_featgrad.cu in row mode (weight 1, no h).
#include "gs_internal.cuh"

namespace gs {

constexpr unsigned long long kKeyInvalid = ~0ull;

// ------------------------------------------------------------------------------------
// T1: per-tile sort of (Gaussian id << 16 | slot) keys
// ------------------------------------------------------------------------------------
constexpr int kSortNT = 1024;

template <int TW, int TH>
__global__ void __launch_bounds__(kSortNT) k_tile_slots(CamTable ct, int K, int nsort, const int *__restrict__ topk_idx,
                                                        const int *__restrict__ err,
                                                        unsigned long long *__restrict__ tile_keys,
                                                        uint32_t *__restrict__ tile_u)
{
    constexpr int B = TW * TH;
    extern __shared__ unsigned long long s_keys[];           // nsort (power of two >= B K)
    __shared__ uint32_t s_red[kSortNT / 32];
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int c = cam_of_tile(ct, tile);
    const CamDev &cam = ct.c[c];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const bool bad = *err != 0;
    for (int i = tid; i < nsort; i += kSortNT) {
        unsigned long long key = kKeyInvalid;
        int pl = i / K, k = i - pl * K;
        if (i < B * K && !bad) {
            int px = tx * TW + (pl % TW), py = ty * TH + (pl / TW);
            if (px < cam.W && py < cam.H) {
                long long p = cam.pix_off + (long long)py * cam.W + px;
                int id = topk_idx[p * K + k];
                if (id >= 0) key = ((unsigned long long)(uint32_t)id << 16) | (unsigned long long)i;
            }
        }
        s_keys[i] = key;
    }
    __syncthreads();
    for (int size = 2; size <= nsort; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < nsort / 2; i += kSortNT) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool up = (lo & size) == 0;
                unsigned long long a = s_keys[lo], b = s_keys[hi];
                if ((a > b) == up) {
                    s_keys[lo] = b;
                    s_keys[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    const int nslots = B * K;
    uint32_t cnt = 0;
    for (int i = tid; i < nslots; i += kSortNT) {
        unsigned long long key = s_keys[i];
        tile_keys[(size_t)tile * nslots + i] = key;
        if (key != kKeyInvalid && (i == 0 || (s_keys[i - 1] >> 16) != (key >> 16))) ++cnt;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = cnt;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kSortNT / 32; ++w) t += s_red[w];
        tile_u[tile] = t;
    }
}

// ------------------------------------------------------------------------------------
// T3: per-tile accumulation, whole rows per slot, re-reads served by L2
// ------------------------------------------------------------------------------------
constexpr int kAccNT = 512;
constexpr int kAccNW = kAccNT / 32;

template <bool BF16>
struct Row16;
template <>
struct Row16<false> {     // 16 bytes = 4 floats
    static constexpr int VEC = 4;
    __device__ __forceinline__ static void load(const void *base, size_t chunk, float (&x)[4])
    {
        float4 v = __ldg((const float4 *)base + chunk);
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
};
template <>
struct Row16<true> {      // 16 bytes = 8 bf16
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

// Dynamic shared memory: edge rows [kAccNW][2][D] f32, then per sorted position (B K):
// pixel (u16), run (u16), weight (f32), h (f32); per run: start (u16, + 1), id (u32).
size_t tile_accum_smem(int B, int K, int D)
{
    size_t n = (size_t)B * K;
    return (size_t)kAccNW * 2 * D * 4 + 2 * n * 2 + 16 + 4 * n * 2 + 2 * (n + 1) + 16 + 4 * n + 64;
}

template <int TW, int TH, bool BF16, int CPL>
__global__ void __launch_bounds__(kAccNT, 1) k_tile_accum(CamTable ct, int K, int D, const float *__restrict__ topk_w,
                                                          const unsigned long long *__restrict__ tile_keys,
                                                          const uint32_t *__restrict__ row_base,
                                                          const uint32_t *__restrict__ tile_u, uint32_t rows_cap,
                                                          const void *__restrict__ feats,
                                                          const void *__restrict__ dLdF, float *__restrict__ rows,
                                                          uint32_t *__restrict__ pair_keys,
                                                          uint32_t *__restrict__ pair_vals, int N,
                                                          float *__restrict__ hbuf, int *err)
{
    constexpr int B = TW * TH;
    using Rw = Row16<BF16>;
    constexpr int VEC = Rw::VEC;
    // slots whose rows are in flight together: 32 registers of row data per lane
    constexpr int DEPTH = CPL * VEC >= 32 ? 1 : 32 / (CPL * VEC);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_scan[kAccNW];
    __shared__ int s_nu, s_nvalid;
    const int nslots = B * K;
    const int nch = D / VEC;                           // 16-byte chunks per row
    float *s_edge = (float *)smem_raw;                 // [kAccNW][2][D]
    uint16_t *s_pl = (uint16_t *)(s_edge + (size_t)kAccNW * 2 * D);
    uint16_t *s_run = s_pl + nslots;
    float *s_wn = (float *)(((uintptr_t)(s_run + nslots) + 15) & ~(uintptr_t)15);
    float *s_h = s_wn + nslots;
    uint16_t *s_ustart = (uint16_t *)(s_h + nslots);
    uint32_t *s_uid = (uint32_t *)(((uintptr_t)(s_ustart + nslots + 1) + 15) & ~(uintptr_t)15);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    const int c = cam_of_tile(ct, tile);
    const CamDev &cam = ct.c[c];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const uint32_t U = tile_u[tile];
    const uint32_t rb = row_base[tile];
    if (*err != 0 || U == 0) return;
    if (rb + U > rows_cap) {
        if (tid == 0) atomicOr(err, kErrOverflow);
        return;
    }
    auto pixel_of = [&](int pl) -> long long {
        return cam.pix_off + (long long)(ty * TH + pl / TW) * cam.W + tx * TW + pl % TW;
    };
    // renormalised weights per slot (Eq. 3), staged in s_h
    for (int pl = tid; pl < B; pl += kAccNT) {
        const int px = tx * TW + (pl % TW), py = ty * TH + (pl / TW);
        if (px < cam.W && py < cam.H) {
            const long long p = pixel_of(pl);
            float S = 0.f;
            for (int k = 0; k < K; ++k) S += topk_w[p * K + k];
            const float inv = S > 0.f ? 1.f / S : 0.f;
            for (int k = 0; k < K; ++k) s_h[pl * K + k] = topk_w[p * K + k] * inv;
        }
    }
    __syncthreads();
    // sorted positions: each thread a contiguous block of PPT positions; run starts by a
    // block scan of (starts << 16 | valid) counts
    const int PPT = (nslots + kAccNT - 1) / kAccNT;
    const int i_lo = min(tid * PPT, nslots), i_hi = min(i_lo + PPT, nslots);
    const unsigned long long *keys = tile_keys + (size_t)tile * nslots;
    {
        uint32_t n_start = 0, n_valid = 0;
        unsigned long long prev = i_lo > 0 ? keys[i_lo - 1] : kKeyInvalid;
        for (int i = i_lo; i < i_hi; ++i) {
            const unsigned long long key = keys[i];
            const bool valid = key != kKeyInvalid;
            const int sl = (int)(key & 0xffffull);
            s_pl[i] = valid ? (uint16_t)(sl / K) : (uint16_t)0;
            s_wn[i] = valid ? s_h[sl] : 0.f;
            n_valid += valid;
            n_start += valid && (i == 0 || (prev >> 16) != (key >> 16));
            prev = key;
        }
        uint32_t packed = (n_start << 16) | n_valid, inc = packed;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_scan[warp] = inc;
        __syncthreads();                                  // also: every staged weight has been read
        uint32_t before = inc - packed;
        for (int w = 0; w < warp; ++w) before += s_scan[w];
        if (tid == kAccNT - 1) {
            uint32_t tot = before + packed;
            s_nu = (int)(tot >> 16);
            s_nvalid = (int)(tot & 0xffffu);
        }
        int u = (int)(before >> 16) - 1;
        prev = i_lo > 0 ? keys[i_lo - 1] : kKeyInvalid;
        for (int i = i_lo; i < i_hi; ++i) {
            const unsigned long long key = keys[i];
            if (key != kKeyInvalid && (i == 0 || (prev >> 16) != (key >> 16))) {
                ++u;
                s_ustart[u] = (uint16_t)i;
                s_uid[u] = (uint32_t)(key >> 16);
            }
            s_run[i] = (uint16_t)(u < 0 ? 0 : u);
            s_h[i] = 0.f;
            prev = key;
        }
    }
    __syncthreads();
    const int nu = s_nu, nvalid = s_nvalid;
    if (tid == 0) s_ustart[nu] = (uint16_t)nvalid;
    __syncthreads();

    // warp w owns sorted positions [a, b)
    const int R = (nvalid + kAccNW - 1) / kAccNW;
    const int a = min(warp * R, nvalid), b = min(a + R, nvalid);
    float acc[CPL][VEC], f[CPL][VEC];
    int cur = -1, seg0 = a;
    auto flush = [&](int end) {
        // segment [seg0, end) of run cur: whole run -> its partial row; cut -> edge row
        const bool cutL = seg0 == a && a > s_ustart[cur];
        const bool cutR = end == b && b < s_ustart[cur + 1];
        float *dst = !cutL && !cutR ? rows + (size_t)(rb + cur) * D
                                    : s_edge + ((size_t)warp * 2 + (cutL ? 0 : 1)) * D;
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) {
            const int ch = lane + 32 * cc;
            if (ch < nch) {
                float4 *d4 = (float4 *)(dst + (size_t)ch * VEC);
#pragma unroll
                for (int v = 0; v < VEC / 4; ++v)
                    d4[v] = make_float4(acc[cc][4 * v], acc[cc][4 * v + 1], acc[cc][4 * v + 2], acc[cc][4 * v + 3]);
            }
        }
    };
    for (int j0 = 0; j0 < R; j0 += 8) {
        float dot[8];
#pragma unroll
        for (int h4 = 0; h4 < 8; h4 += DEPTH) {
            // issue the row loads of DEPTH slots before any of their arithmetic
            float x[DEPTH][CPL][VEC];
#pragma unroll
            for (int q = 0; q < DEPTH; ++q) {
                const int i = a + j0 + h4 + q;
                const long long p = i < b ? pixel_of(s_pl[i]) : 0;
#pragma unroll
                for (int cc = 0; cc < CPL; ++cc) {
                    const int ch = lane + 32 * cc;
                    if (i < b && ch < nch) Rw::load(dLdF, (size_t)p * nch + ch, x[q][cc]);
                    else {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) x[q][cc][v] = 0.f;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < DEPTH; ++q) {
                const int i = a + j0 + h4 + q;
                dot[h4 + q] = 0.f;
                if (i < b) {
                    const int run = s_run[i];
                    if (run != cur) {
                        if (cur >= 0) flush(i);
                        cur = run;
                        seg0 = i;
                        const uint32_t id = s_uid[run];
#pragma unroll
                        for (int cc = 0; cc < CPL; ++cc) {
                            const int ch = lane + 32 * cc;
#pragma unroll
                            for (int v = 0; v < VEC; ++v) { acc[cc][v] = 0.f; f[cc][v] = 0.f; }
                            if (ch < nch) Rw::load(feats, (size_t)id * nch + ch, f[cc]);
                        }
                    }
                    const float wp = s_wn[i];
#pragma unroll
                    for (int cc = 0; cc < CPL; ++cc)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            acc[cc][v] = fmaf(wp, x[q][cc][v], acc[cc][v]);
                            dot[h4 + q] = fmaf(x[q][cc][v], f[cc][v], dot[h4 + q]);
                        }
                }
            }
        }
        // reduce-scatter of 8 dots over the warp: lane l ends with dot (l >> 2) & 7
        const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
        float ra[4], rbv[2];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            ra[q] = (b4 ? dot[q + 4] : dot[q]) + __shfl_xor_sync(0xffffffffu, b4 ? dot[q] : dot[q + 4], 16);
#pragma unroll
        for (int q = 0; q < 2; ++q)
            rbv[q] = (b3 ? ra[q + 2] : ra[q]) + __shfl_xor_sync(0xffffffffu, b3 ? ra[q] : ra[q + 2], 8);
        float d = (b2 ? rbv[1] : rbv[0]) + __shfl_xor_sync(0xffffffffu, b2 ? rbv[0] : rbv[1], 4);
        d += __shfl_xor_sync(0xffffffffu, d, 2);
        d += __shfl_xor_sync(0xffffffffu, d, 1);
        const int q = (lane >> 2) & 7;
        if (!(lane & 3) && a + j0 + q < b) s_h[a + j0 + q] = d;
    }
    if (cur >= 0) flush(b);
    __syncthreads();
    // the warp where a cut run starts adds the edge rows of the following warps
    if (b > a) {
        const int last = s_run[b - 1];
        const bool cutR = b < s_ustart[last + 1];
        const bool startsHere = s_ustart[last] >= a;
        if (cutR && startsHere) {
            const int w_end = (s_ustart[last + 1] - 1) / R;
            for (int ch = lane; ch < nch; ch += 32) {
                float t[VEC];
                const float *e = s_edge + ((size_t)warp * 2 + 1) * D + (size_t)ch * VEC;
#pragma unroll
                for (int v = 0; v < VEC; ++v) t[v] = e[v];
                for (int w = warp + 1; w <= w_end; ++w) {
                    const float *e2 = s_edge + ((size_t)w * 2 + 0) * D + (size_t)ch * VEC;
#pragma unroll
                    for (int v = 0; v < VEC; ++v) t[v] += e2[v];
                }
                float4 *d4 = (float4 *)(rows + (size_t)(rb + last) * D + (size_t)ch * VEC);
#pragma unroll
                for (int v = 0; v < VEC / 4; ++v) d4[v] = make_float4(t[4 * v], t[4 * v + 1], t[4 * v + 2], t[4 * v + 3]);
            }
        }
    }
    // h per slot, and the (Gaussian, partial row) pairs of the per-Gaussian reduction
    for (int i = tid; i < nvalid; i += kAccNT) {
        const int sl = (int)(keys[i] & 0xffffull);
        const int pl = s_pl[i], k = sl - pl * K;
        hbuf[pixel_of(pl) * K + k] = s_h[i];
    }
    for (int u = tid; u < nu; u += kAccNT) {
        pair_keys[N + rb + u] = s_uid[u];
        pair_vals[N + rb + u] = rb + u;
    }
}

// ------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------
int tile_sort_len(int slots)
{
    int n = 1;
    while (n < slots) n <<= 1;
    return n;
}

bool tile_grad_supported(int dtype, int D, int K, int tw, int th)
{
    const int nch = D / (dtype == GS_BF16 ? 8 : 4);
    return nch <= 32 * 8 && tw * th * K <= 65535 && tile_accum_smem(tw * th, K, D) <= 200 * 1024 &&
           8 * (size_t)tile_sort_len(tw * th * K) <= 200 * 1024;
}

template <int TW, int TH, bool BF16, int CPLV>
static void accum_one(unsigned grid, size_t sm, cudaStream_t s, const CamTable &ct, const WsLayout &L,
                      const float *tw, const unsigned long long *keys, const uint32_t *rbase, const uint32_t *tu,
                      const void *feats, const void *dLdF, float *rows, uint32_t *pk, uint32_t *pv, float *hbuf,
                      int *err)
{
    cudaFuncSetAttribute(k_tile_accum<TW, TH, BF16, CPLV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_tile_accum<TW, TH, BF16, CPLV><<<grid, kAccNT, sm, s>>>(ct, L.K, L.D, tw, keys, rbase, tu, (uint32_t)L.rows_cap,
                                                              feats, dLdF, rows, pk, pv, L.N, hbuf, err);
}

template <int TW, int TH, bool BF16>
static void accum_launch(int cpl, unsigned grid, size_t sm, cudaStream_t s, const CamTable &ct, const WsLayout &L,
                         const float *tw, const unsigned long long *keys, const uint32_t *rbase, const uint32_t *tu,
                         const void *feats, const void *dLdF, float *rows, uint32_t *pk, uint32_t *pv, float *hbuf,
                         int *err)
{
    // (D <= 1024 caps bf16 rows at 4 chunks per lane; float32 rows at 8)
    switch (cpl) {
    case 1: accum_one<TW, TH, BF16, 1>(grid, sm, s, ct, L, tw, keys, rbase, tu, feats, dLdF, rows, pk, pv, hbuf, err); break;
    case 2: accum_one<TW, TH, BF16, 2>(grid, sm, s, ct, L, tw, keys, rbase, tu, feats, dLdF, rows, pk, pv, hbuf, err); break;
    case 4: accum_one<TW, TH, BF16, 4>(grid, sm, s, ct, L, tw, keys, rbase, tu, feats, dLdF, rows, pk, pv, hbuf, err); break;
    default: accum_one<TW, TH, BF16, (BF16 ? 4 : 8)>(grid, sm, s, ct, L, tw, keys, rbase, tu, feats, dLdF, rows, pk, pv, hbuf, err); break;
    }
}

template <int TW, int TH>
static bool tile_launch(const CamTable &ct, const WsLayout &L, int dtype, const int *topk_idx, const float *topk_w,
                        const void *feats, const void *dLdF, void *ws, cudaStream_t s)
{
    constexpr int B = TW * TH;
    uint32_t *hdr = ws_ptr<uint32_t>(ws, L.header);
    int *err = (int *)hdr;
    unsigned long long *keys = ws_ptr<unsigned long long>(ws, L.tile_keys);
    uint32_t *tile_u = ws_ptr<uint32_t>(ws, L.tile_u);
    uint32_t *row_base = ws_ptr<uint32_t>(ws, L.tile_rowbase);
    float *rows = ws_ptr<float>(ws, L.tile_rows);
    uint32_t *pk = ws_ptr<uint32_t>(ws, L.pair_keys[0]);
    uint32_t *pv = ws_ptr<uint32_t>(ws, L.pair_vals[0]);
    float *hbuf = ws_ptr<float>(ws, L.hbuf);
    uint32_t *aux = ws_ptr<uint32_t>(ws, L.scan_aux);
    const int nsort = tile_sort_len(B * L.K);
    const size_t sm1 = sizeof(unsigned long long) * nsort;
    cudaFuncSetAttribute(k_tile_slots<TW, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    k_tile_slots<TW, TH><<<ct.n_tiles, kSortNT, sm1, s>>>(ct, L.K, nsort, topk_idx, err, keys, tile_u);
    exclusive_scan_u32(tile_u, row_base, ct.n_tiles, hdr + 8, aux, s);
    const size_t sm3 = tile_accum_smem(B, L.K, L.D);
    const int nch = L.D / (dtype == GS_BF16 ? 8 : 4);
    const int cpl = nch <= 32 ? 1 : nch <= 64 ? 2 : nch <= 128 ? 4 : 8;
    if (dtype == GS_BF16)
        accum_launch<TW, TH, true>(cpl, ct.n_tiles, sm3, s, ct, L, topk_w, keys, row_base, tile_u, feats, dLdF, rows,
                                   pk, pv, hbuf, err);
    else
        accum_launch<TW, TH, false>(cpl, ct.n_tiles, sm3, s, ct, L, topk_w, keys, row_base, tile_u, feats, dLdF, rows,
                                    pk, pv, hbuf, err);
    return true;
}

// Stages T1-T3; leaves the (Gaussian, row) pairs after N marker slots in pair buffer 0,
// the partial rows, hbuf, and U_tot in header word 8.
bool launch_tile_grad(const CamTable &ct, const WsLayout &L, int dtype, const int *topk_idx, const float *topk_w,
                      const void *feats, const void *dLdF, void *ws, cudaStream_t s)
{
    if (ct.tile_w == 16 && ct.tile_h == 16) return tile_launch<16, 16>(ct, L, dtype, topk_idx, topk_w, feats, dLdF, ws, s);
    if (ct.tile_w == 32 && ct.tile_h == 8) return tile_launch<32, 8>(ct, L, dtype, topk_idx, topk_w, feats, dLdF, ws, s);
    if (ct.tile_w == 16 && ct.tile_h == 8) return tile_launch<16, 8>(ct, L, dtype, topk_idx, topk_w, feats, dLdF, ws, s);
    if (ct.tile_w == 8 && ct.tile_h == 8) return tile_launch<8, 8>(ct, L, dtype, topk_idx, topk_w, feats, dLdF, ws, s);
    return false;
}

}  // namespace gs
