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
// Stage T3 (k_tile_accum): one CTA per tile streams the tile's dL/dF rows through shared
//   memory in 256-byte column chunks with TMA (cp.async.bulk.tensor.2d, one box per tile
//   row, two stages on mbarriers with bounded waits).  Each half-warp owns one distinct
//   Gaussian of the tile: it sums w' dL/dF over that Gaussian's slots in registers (one
//   partial row per (tile, Gaussian)) and forms the slot dot products h, reduced with one
//   shuffle per slot (reduce-scatter over 8 slots).
// Stage T4: the partial rows are reduced per Gaussian by the sort-by-Gaussian segmented
//   reduction of gs_featgrad.cu in row mode (weight 1, no h).
#include "gs_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <mutex>

namespace gs {

constexpr unsigned long long kKeyInvalid = ~0ull;
constexpr int kChunkBytes = 256;          // columns staged per pass, per pixel row
constexpr int kStages = 2;

// ------------------------------------------------------------------------------------
// T1: per-tile sort of (Gaussian id << 16 | slot) keys
// ------------------------------------------------------------------------------------
template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) k_tile_slots(CamTable ct, int K, int nsort, const int *__restrict__ topk_idx,
                                                        const int *__restrict__ err,
                                                        unsigned long long *__restrict__ tile_keys,
                                                        uint32_t *__restrict__ tile_u)
{
    constexpr int B = TW * TH;
    extern __shared__ unsigned long long s_keys[];           // nsort (power of two >= B K)
    __shared__ uint32_t s_red[B / 32];
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int c = cam_of_tile(ct, tile);
    const CamDev &cam = ct.c[c];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const bool bad = *err != 0;
    for (int i = tid; i < nsort; i += B) {
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
            for (int i = tid; i < nsort / 2; i += B) {
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
    for (int i = tid; i < nslots; i += B) {
        unsigned long long key = s_keys[i];
        tile_keys[(size_t)tile * nslots + i] = key;
        if (key != kKeyInvalid && (i == 0 || (s_keys[i - 1] >> 16) != (key >> 16))) ++cnt;
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = cnt;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0;
        for (int w = 0; w < B / 32; ++w) t += s_red[w];
        tile_u[tile] = t;
    }
}

// ------------------------------------------------------------------------------------
// T3: per-tile accumulation with TMA-staged dL/dF chunks
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Bounded wait on the phase with the given parity; false if the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t addr = smem_u32(bar);
    for (uint32_t it = 0; it < (1u << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

template <bool BF16>
struct Chunk16;
template <>
struct Chunk16<false> {     // 16 bytes = 4 floats
    static constexpr int VEC = 4;
    __device__ __forceinline__ static void cvt(const uint4 &v, float (&x)[4])
    {
        x[0] = __uint_as_float(v.x); x[1] = __uint_as_float(v.y); x[2] = __uint_as_float(v.z); x[3] = __uint_as_float(v.w);
    }
};
template <>
struct Chunk16<true> {      // 16 bytes = 8 bf16
    static constexpr int VEC = 8;
    __device__ __forceinline__ static void cvt(const uint4 &v, float (&x)[8])
    {
        const __nv_bfloat162 *h = (const __nv_bfloat162 *)&v;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 f = __bfloat1622float2(h[i]);
            x[2 * i] = f.x;
            x[2 * i + 1] = f.y;
        }
    }
};

// Dynamic shared memory, in order: [kStages][B pixels][256 B] staged dL/dF (1024-byte
// aligned), kStages mbarriers, edge partials [B/16][2][256 B as float32 accumulators x2],
// then per sorted position (B K): slot (u16), pixel (u16), run index (u16), weight (f32),
// h (f32); per run: start (u16, + 1) and Gaussian id (u32).
size_t tile_accum_smem(int B, int K)
{
    size_t n = (size_t)B * K;
    size_t e = (size_t)(B / 16) * 2 * 128 * sizeof(float);
    return 1024 + (size_t)kStages * B * kChunkBytes + 64 + e + 2 * n * 3 + 16 + 4 * n * 2 + 2 * (n + 1) + 16 + 4 * n + 64;
}

template <int TW, int TH, bool BF16>
__global__ void __launch_bounds__(TW *TH) k_tile_accum(const __grid_constant__ CUtensorMap dmap, CamTable ct, int K,
                                                        int D, const float *__restrict__ topk_w,
                                                        const unsigned long long *__restrict__ tile_keys,
                                                        const uint32_t *__restrict__ row_base,
                                                        const uint32_t *__restrict__ tile_u, uint32_t rows_cap,
                                                        const void *__restrict__ feats, float *__restrict__ rows,
                                                        uint32_t *__restrict__ pair_keys,
                                                        uint32_t *__restrict__ pair_vals, int N,
                                                        float *__restrict__ hbuf, int *err)
{
    constexpr int B = TW * TH;
    constexpr int NW = B / 32;
    constexpr int NH = B / 16;                        // half-warps
    using Ch = Chunk16<BF16>;
    constexpr int VEC = Ch::VEC;
    constexpr int ELEM = BF16 ? 2 : 4;
    constexpr int CE = kChunkBytes / ELEM;           // elements per staged chunk
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint32_t s_scan[NW];
    __shared__ int s_nu, s_nvalid;
    const int nslots = B * K;
    // TMA destinations must be 128-byte aligned: align explicitly (the launch adds slack)
    unsigned char *stage = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(stage + (size_t)kStages * B * kChunkBytes);
    float *s_edge = (float *)(bars + 8);                               // [NH][2][CE]
    uint16_t *s_slot = (uint16_t *)(s_edge + NH * 2 * CE);
    uint16_t *s_pl = s_slot + nslots;
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
    // renormalised weights of this thread's pixel, indexed by slot (Eq. 3); staged in s_h
    {
        const int px = tx * TW + (tid % TW), py = ty * TH + (tid / TW);
        if (px < cam.W && py < cam.H) {
            const long long p = cam.pix_off + (long long)py * cam.W + px;
            float S = 0.f;
            for (int k = 0; k < K; ++k) S += topk_w[p * K + k];
            const float inv = S > 0.f ? 1.f / S : 0.f;
            for (int k = 0; k < K; ++k) s_h[tid * K + k] = topk_w[p * K + k] * inv;
        }
    }
    __syncthreads();
    // sorted positions: slot, pixel, weight; run starts via a block scan over K-long runs
    {
        const unsigned long long *keys = tile_keys + (size_t)tile * nslots;
        uint32_t n_start = 0, n_valid = 0;
        unsigned long long prev = tid > 0 ? keys[tid * K - 1] : kKeyInvalid;
        for (int j = 0; j < K; ++j) {
            const int i = tid * K + j;
            const unsigned long long key = keys[i];
            const bool valid = key != kKeyInvalid;
            const int sl = (int)(key & 0xffffull);
            s_slot[i] = (uint16_t)sl;
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
        __syncthreads();                                  // also: every s_h weight has been read
        uint32_t before = inc - packed;
        for (int w = 0; w < warp; ++w) before += s_scan[w];
        if (tid == B - 1) {
            uint32_t tot = before + packed;
            s_nu = (int)(tot >> 16);
            s_nvalid = (int)(tot & 0xffffu);
        }
        int u = (int)(before >> 16) - 1;
        prev = tid > 0 ? keys[tid * K - 1] : kKeyInvalid;
        for (int j = 0; j < K; ++j) {
            const int i = tid * K + j;
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
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int nu = s_nu, nvalid = s_nvalid;
    if (tid == 0) s_ustart[nu] = (uint16_t)nvalid;
    const int n_chunks = (D * ELEM) / kChunkBytes;   // host guarantees an exact multiple
    const long long p_row0 = cam.pix_off + (long long)(ty * TH) * cam.W + tx * TW;

    auto issue = [&](int ch) {
        const int s = ch % kStages;
        mbar_expect_tx(&bars[s], (uint32_t)(B * kChunkBytes));
#pragma unroll 1
        for (int r = 0; r < TH; ++r)
            tma_load_2d(stage + (size_t)s * B * kChunkBytes + (size_t)r * TW * kChunkBytes, &dmap, ch * CE,
                        (int)(p_row0 + (long long)r * cam.W), &bars[s]);
    };
    if (tid == 0) {
        issue(0);
        if (n_chunks > 1) issue(1);
    }
    __syncthreads();
    // balanced split: half-warp hw owns sorted positions [a, b)
    const int half = lane >> 4, hl = lane & 15, hw = warp * 2 + half;
    const int R = (nvalid + NH - 1) / NH;
    const int a = min(hw * R, nvalid), b = min(a + R, nvalid);
    for (int ch = 0; ch < n_chunks; ++ch) {
        const int s = ch % kStages;
        const bool ok = mbar_wait(&bars[s], (uint32_t)((ch / kStages) & 1));
        if (__syncthreads_and(ok) == 0) {
            if (tid == 0) atomicOr(err, kErrTimeout);
            // the copies in flight get one more bounded wait before the CTA exits
            for (int t = ch + 1; t < n_chunks && t < ch + kStages; ++t)
                mbar_wait(&bars[t % kStages], (uint32_t)((t / kStages) & 1));
            return;
        }
        const unsigned char *buf = stage + (size_t)s * B * kChunkBytes;
        const int colv = ch * CE + hl * VEC;             // first element of this lane's 16 B
        float acc[VEC], f[VEC];
        int cur = -1, seg0 = a;
        auto flush = [&](int end) {
            // segment [seg0, end) of run cur: whole run -> its partial row; cut -> edge buffer
            const bool cutL = seg0 == a && a > s_ustart[cur];
            const bool cutR = end == b && b < s_ustart[cur + 1];
            float *dst = !cutL && !cutR ? rows + (size_t)(rb + cur) * D + colv
                                        : s_edge + ((size_t)hw * 2 + (cutL ? 0 : 1)) * CE + hl * VEC;
            float4 *d4 = (float4 *)dst;
#pragma unroll
            for (int v = 0; v < VEC / 4; ++v)
                d4[v] = make_float4(acc[4 * v], acc[4 * v + 1], acc[4 * v + 2], acc[4 * v + 3]);
        };
        for (int j0 = 0; j0 < R; j0 += 8) {
            float dot[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                dot[q] = 0.f;
                const int i = a + j0 + q;
                if (i < b) {
                    const int run = s_run[i];
                    if (run != cur) {
                        if (cur >= 0) flush(i);
                        cur = run;
                        seg0 = i;
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
                        const uint4 fv = __ldg((const uint4 *)((const char *)feats + ((size_t)s_uid[run] * D + colv) * ELEM));
                        Ch::cvt(fv, f);
                    }
                    const float wp = s_wn[i];
                    const uint4 xv = *(const uint4 *)(buf + (size_t)s_pl[i] * kChunkBytes + hl * 16);
                    float x[VEC];
                    Ch::cvt(xv, x);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        acc[v] = fmaf(wp, x[v], acc[v]);
                        dot[q] = fmaf(x[v], f[v], dot[q]);
                    }
                }
            }
            // reduce-scatter of 8 dots over the 16 lanes of this half-warp:
            // lane hl ends with dot (hl >> 1) & 7 (lanes hl and hl ^ 1 agree)
            const bool b3 = hl & 8, b2 = hl & 4, b1 = hl & 2;
            float ra[4], rbv[2];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                ra[q] = (b3 ? dot[q + 4] : dot[q]) + __shfl_xor_sync(0xffffffffu, b3 ? dot[q] : dot[q + 4], 8);
#pragma unroll
            for (int q = 0; q < 2; ++q)
                rbv[q] = (b2 ? ra[q + 2] : ra[q]) + __shfl_xor_sync(0xffffffffu, b2 ? ra[q] : ra[q + 2], 4);
            float d = (b1 ? rbv[1] : rbv[0]) + __shfl_xor_sync(0xffffffffu, b1 ? rbv[0] : rbv[1], 2);
            d += __shfl_xor_sync(0xffffffffu, d, 1);
            const int q = (hl >> 1) & 7;
            if (!(hl & 1) && a + j0 + q < b) s_h[a + j0 + q] += d;
        }
        if (cur >= 0) flush(b);
        __syncthreads();                                  // edges written; stage consumed
        // the half-warp where a cut run starts adds the pieces of the following half-warps
        if (b > a) {
            const int last = s_run[b - 1];
            const bool cutR = b < s_ustart[last + 1];
            const bool startsHere = s_ustart[last] >= a;
            if (cutR && startsHere) {
                const int h_end = (s_ustart[last + 1] - 1) / R;
                float t[VEC];
                const float *e = s_edge + ((size_t)hw * 2 + 1) * CE + hl * VEC;
#pragma unroll
                for (int v = 0; v < VEC; ++v) t[v] = e[v];
                for (int h = hw + 1; h <= h_end; ++h) {
                    const float *e2 = s_edge + ((size_t)h * 2 + 0) * CE + hl * VEC;
#pragma unroll
                    for (int v = 0; v < VEC; ++v) t[v] += e2[v];
                }
                float4 *d4 = (float4 *)(rows + (size_t)(rb + last) * D + colv);
#pragma unroll
                for (int v = 0; v < VEC / 4; ++v) d4[v] = make_float4(t[4 * v], t[4 * v + 1], t[4 * v + 2], t[4 * v + 3]);
            }
        }
        __syncthreads();                                  // edges read before the next chunk
        if (tid == 0 && ch + kStages < n_chunks) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(ch + kStages);
        }
    }
    // h per slot, and the (Gaussian, partial row) pairs of the per-Gaussian reduction
    for (int i = tid; i < nvalid; i += B) {
        const int sl = s_slot[i];
        const int pl = s_pl[i], k = sl - pl * K;
        const long long p = cam.pix_off + (long long)(ty * TH + pl / TW) * cam.W + tx * TW + pl % TW;
        hbuf[p * K + k] = s_h[i];
    }
    for (int u = tid; u < nu; u += B) {
        pair_keys[N + rb + u] = s_uid[u];
        pair_vals[N + rb + u] = rb + u;
    }
}

// ------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

int tile_sort_len(int slots)
{
    int n = 1;
    while (n < slots) n <<= 1;
    return n;
}

bool tile_grad_supported(int dtype, int D, int K, int tw, int th)
{
    const int elem = dtype == GS_BF16 ? 2 : 4;
    return (D * elem) % kChunkBytes == 0 && tw * th * K <= 65535 && tile_accum_smem(tw * th, K) <= 227 * 1024;
}

template <int TW, int TH>
static bool tile_launch(const CamTable &ct, const WsLayout &L, int dtype, const CUtensorMap &map, const int *topk_idx,
                        const float *topk_w, const void *feats, void *ws, cudaStream_t s)
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
    k_tile_slots<TW, TH><<<ct.n_tiles, B, sm1, s>>>(ct, L.K, nsort, topk_idx, err, keys, tile_u);
    exclusive_scan_u32(tile_u, row_base, ct.n_tiles, hdr + 8, aux, s);
    const size_t sm3 = tile_accum_smem(B, L.K);
    if (dtype == GS_BF16) {
        cudaFuncSetAttribute(k_tile_accum<TW, TH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
        k_tile_accum<TW, TH, true><<<ct.n_tiles, B, sm3, s>>>(map, ct, L.K, L.D, topk_w, keys, row_base, tile_u,
                                                              (uint32_t)L.rows_cap, feats, rows, pk, pv, L.N, hbuf,
                                                              err);
    } else {
        cudaFuncSetAttribute(k_tile_accum<TW, TH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
        k_tile_accum<TW, TH, false><<<ct.n_tiles, B, sm3, s>>>(map, ct, L.K, L.D, topk_w, keys, row_base, tile_u,
                                                               (uint32_t)L.rows_cap, feats, rows, pk, pv, L.N, hbuf,
                                                               err);
    }
    return true;
}

// Stages T1-T3; leaves the (Gaussian, row) pairs after N marker slots in pair buffer 0,
// the partial rows, hbuf, and U_tot in header word 8.
bool launch_tile_grad(const CamTable &ct, const WsLayout &L, int dtype, const int *topk_idx, const float *topk_w,
                      const void *feats, const void *dLdF, void *ws, cudaStream_t s)
{
    auto enc = get_encode();
    if (!enc) return false;
    CUtensorMap map;
    const int elem = dtype == GS_BF16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)L.D, (cuuint64_t)L.P};
    cuuint64_t strides[1] = {(cuuint64_t)L.D * elem};
    cuuint32_t box[2] = {(cuuint32_t)(kChunkBytes / elem), (cuuint32_t)ct.tile_w};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, dtype == GS_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                     const_cast<void *>(dLdF), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    if (ct.tile_w == 16 && ct.tile_h == 16) return tile_launch<16, 16>(ct, L, dtype, map, topk_idx, topk_w, feats, ws, s);
    if (ct.tile_w == 32 && ct.tile_h == 8) return tile_launch<32, 8>(ct, L, dtype, map, topk_idx, topk_w, feats, ws, s);
    if (ct.tile_w == 16 && ct.tile_h == 8) return tile_launch<16, 8>(ct, L, dtype, map, topk_idx, topk_w, feats, ws, s);
    if (ct.tile_w == 8 && ct.tile_h == 8) return tile_launch<8, 8>(ct, L, dtype, map, topk_idx, topk_w, feats, ws, s);
    return false;
}

}  // namespace gs
