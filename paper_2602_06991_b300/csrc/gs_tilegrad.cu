// gs_tilegrad.cu -- feature part of a5, block-major: every dL/dF row is read from HBM
// once and re-read only from shared memory.
//
//   dL/df_g = sum over (pixel p, slot k) with idx_k(p) = g of w'_k(p) dL/dF_p     (Eqs. 3-4)
//
// (h_k(p) = dL/dF_p . f_{idx_k(p)}, needed by the re-walk, comes from the fused blend +
// loss kernel or from k_h_group in gs_blend.cu.)
//
// The screen is cut into small pixel blocks (8x8, 8x4 or 4x4, the largest whose dL/dF
// rows fit one 64 KB shared-memory stage with at most 512 slots; blocks of 32 or more
// pixels whose rows fit half a stage take that, so two CTAs share an SM), independent of the
// binning tile.
// Stage T1 (k_tile_slots_warp, or k_tile_slots for very large scenes): per block, the
//   (Gaussian, slot) keys are sorted (bitonic: deterministic) and, in sorted order, one
//   record per slot (pixel, run, renormalised weight) and one entry per run of equal
//   Gaussians (first position, id) are written; U_b = the number of runs.
// Stage T2: exclusive scan of U_b over blocks gives every (block, Gaussian) its partial
//   row -- deterministic, no atomics.
// Stage T3 (k_block_accum): a persistent CTA per SM walks blocks.  A producer warp
//   streams each block's dL/dF rows (tensor-map TMA boxes), records and run table (bulk
//   copies) into a ring of shared-memory stages, completing on mbarriers, while eight
//   consumer warps reduce the stages already full: each consumer owns whole runs and sums
//   w' dL/dF over a run's slots in slot order, whole rows at a time (16 B per lane per
//   128-column chunk) read from shared memory, then writes the run's partial row.
// Stage T4: the partial rows are reduced per Gaussian by the sort-by-Gaussian segmented
//   reduction of gs_featgrad.cu in row mode.
// For bf16 dL/dF (D a multiple of 64, blocks of 16 or 32 pixels) T3 is k_block_mma, the
// same partial rows as a tensor-core product per block.
#include "gs_internal.cuh"
#include "gs_mma.cuh"

#include <cuda.h>
#include <mutex>
#include <string.h>

namespace gs {

constexpr unsigned long long kKeyInvalid = ~0ull;
constexpr int kStageMax = 64 * 1024;            // bytes of dL/dF rows per block stage

FgBlock fg_block_shape(int dtype, int D, int K)
{
    // the rows of a block (in 256-element TMA box rows) fit one 64 KB stage and its slots
    // number at most 512
    const int row = (D < 256 ? D : (D + 255) / 256 * 256) * (dtype == GS_BF16 ? 2 : 4);
    // blocks of at least 32 pixels in stages of half the maximum first (two CTAs per SM:
    // more consumer warps for rows of many short runs), else the largest that fits
    if (64 * row <= kStageMax / 2 && 64 * K <= 512) return {8, 8};
    if (32 * row <= kStageMax / 2 && 32 * K <= 512) return {8, 4};
    if (64 * row <= kStageMax && 64 * K <= 512) return {8, 8};
    if (32 * row <= kStageMax && 32 * K <= 512) return {8, 4};
    if (16 * row <= kStageMax && 16 * K <= 512) return {4, 4};
    return {0, 0};
}

void retile(const CamTable &ct, int bw, int bh, CamTable &out)
{
    out = ct;
    out.tile_w = bw;
    out.tile_h = bh;
    int off = 0, rows = 0;
    for (int c = 0; c < ct.n; ++c) {
        CamDev &d = out.c[c];
        d.tiles_x = (d.W + bw - 1) / bw;
        d.tiles_y = (d.H + bh - 1) / bh;
        d.tile_off = off;
        d.row_off = rows;
        off += d.tiles_x * d.tiles_y;
        rows += d.tiles_y;
    }
    out.n_tiles = off;
    out.n_rows = rows;
}

// ------------------------------------------------------------------------------------
// T1: per-block sort of (Gaussian id << 16 | slot) keys, then the block's slot records
// and run table, so that T3 reads everything it needs as two contiguous arrays.
//   rec[i]  (sorted position i < B K): x = pixel | run << 16, y = bits of w' (Eq. 3)
//   runs[u] (u < U_b): x = first sorted position, y = Gaussian id;  runs[U_b].x = the
//           number of valid positions
// ------------------------------------------------------------------------------------
static __host__ __device__ __forceinline__ int runs_stride(int nslots) { return (nslots + 2) & ~1; }

template <int TW, int TH>
__global__ void __launch_bounds__(1024) k_tile_slots(CamTable ct, int K, int nsort, const int *__restrict__ topk_idx,
                                                     const float *__restrict__ topk_w, const int *__restrict__ err,
                                                     uint2 *__restrict__ rec, uint2 *__restrict__ runs,
                                                     uint32_t *__restrict__ tile_u)
{
    constexpr int B = TW * TH;
    extern __shared__ unsigned long long s_keys[];           // nsort (power of two >= B K), then B K floats
    __shared__ uint32_t s_red[32];
    __shared__ uint32_t s_total;
    const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int nslots = B * K;
    float *s_w = (float *)(s_keys + nsort);                  // w per slot, then w' in place
    const int tile = blockIdx.x;
    const int c = cam_of_tile(ct, tile);
    const CamDev &cam = ct.c[c];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const bool bad = *err != 0;
    for (int i = tid; i < nsort; i += NT) {
        unsigned long long key = kKeyInvalid;
        int pl = i / K, k = i - pl * K;
        if (i < nslots) s_w[i] = 0.f;
        if (i < nslots && !bad) {
            int px = tx * TW + (pl % TW), py = ty * TH + (pl / TW);
            if (px < cam.W && py < cam.H) {
                long long p = cam.pix_off + (long long)py * cam.W + px;
                int id = topk_idx[p * K + k];
                s_w[i] = topk_w[p * K + k];
                if (id >= 0) key = ((unsigned long long)(uint32_t)id << 16) | (unsigned long long)i;
            }
        }
        s_keys[i] = key;
    }
    __syncthreads();
    // renormalised weights w' = w / S per pixel (S in slot order)
    for (int pl = tid; pl < B; pl += NT) {
        float S = 0.f;
        for (int k = 0; k < K; ++k) S += s_w[pl * K + k];
        const float inv = S > 0.f ? 1.f / S : 0.f;
        for (int k = 0; k < K; ++k) s_w[pl * K + k] *= inv;
    }
    for (int size = 2; size <= nsort; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            for (int i = tid; i < nsort / 2; i += NT) {
                int lo = 2 * i - (i & (stride - 1));
                int hi = lo + stride;
                bool up = (lo & size) == 0;
                unsigned long long a = s_keys[lo], b = s_keys[hi];
                if ((a > b) == up) {
                    s_keys[lo] = b;
                    s_keys[hi] = a;
                }
            }
        }
    }
    __syncthreads();
    // run index of every sorted position: each thread a contiguous group of positions,
    // a block scan of the run-start counts
    const int PPT = (nslots + NT - 1) / NT;
    const int i_lo = min(tid * PPT, nslots), i_hi = min(i_lo + PPT, nslots);
    uint32_t cnt = 0;
    for (int i = i_lo; i < i_hi; ++i) {
        const unsigned long long key = s_keys[i];
        cnt += key != kKeyInvalid && (i == 0 || (s_keys[i - 1] >> 16) != (key >> 16));
    }
    uint32_t inc = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_red[warp] = inc;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0;
        for (int w = 0; w < NT / 32; ++w) {
            const uint32_t v = s_red[w];
            s_red[w] = t;
            t += v;
        }
        s_total = t;
    }
    __syncthreads();
    int u = (int)(s_red[warp] + inc - cnt) - 1;               // runs started before i_lo, minus 1
    uint2 *brec = rec + (size_t)tile * nslots;
    uint2 *bruns = runs + (size_t)tile * runs_stride(nslots);
    for (int i = i_lo; i < i_hi; ++i) {
        const unsigned long long key = s_keys[i];
        uint2 r = make_uint2(0u, 0u);
        if (key != kKeyInvalid) {
            if (i == 0 || (s_keys[i - 1] >> 16) != (key >> 16)) {
                ++u;
                bruns[u] = make_uint2((uint32_t)i, (uint32_t)(key >> 16));
            }
            const int sl = (int)(key & 0xffffull);
            r = make_uint2((uint32_t)(sl / K) | ((uint32_t)u << 16), __float_as_uint(s_w[sl]));
        } else if (i == 0 || s_keys[i - 1] != kKeyInvalid) {
            bruns[s_total] = make_uint2((uint32_t)i, 0u);      // end of the valid positions
        }
        brec[i] = r;
    }
    if (tid == 0) {
        tile_u[tile] = s_total;
        if (s_keys[nslots - 1] != kKeyInvalid) bruns[s_total] = make_uint2((uint32_t)nslots, 0u);
    }
}

// T1, warp form (fewer than 2^22 Gaussians, at most 512 slots): one warp per block.
// The slots' 32-bit keys (id << 9 | slot) are sorted in registers by a bitonic network
// (KPT keys per lane, element e = lane KPT + r; strides below KPT inside a lane, the
// others across lanes by shuffles), so no shared-memory round trip or block barrier
// sits in the sort.  Same order, records and runs as k_tile_slots.
template <int TW, int TH, int KPT>
__global__ void __launch_bounds__(128) k_tile_slots_warp(CamTable ct, int K, const int *__restrict__ topk_idx,
                                                         const float *__restrict__ topk_w, const int *__restrict__ err,
                                                         uint2 *__restrict__ rec, uint2 *__restrict__ runs,
                                                         uint32_t *__restrict__ tile_u)
{
    constexpr int B = TW * TH;
    constexpr int NS = 32 * KPT;
    constexpr uint32_t kNone = 0xffffffffu;
    __shared__ float s_w[4][NS];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int tile = blockIdx.x * 4 + wib;
    if (tile >= ct.n_tiles) return;                          // whole warp
    const int nslots = B * K;
    float *w = s_w[wib];
    const int c = cam_of_tile(ct, tile);
    const CamDev &cam = ct.c[c];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const bool bad = *err != 0;
    uint32_t key[KPT];
#pragma unroll
    for (int r = 0; r < KPT; ++r) {
        const int i = lane * KPT + r;
        key[r] = kNone;
        if (i < nslots) {
            float wi = 0.f;
            const int pl = i / K, k = i - pl * K;
            const int px = tx * TW + (pl % TW), py = ty * TH + (pl / TW);
            if (!bad && px < cam.W && py < cam.H) {
                const long long p = cam.pix_off + (long long)py * cam.W + px;
                const int id = topk_idx[p * K + k];
                wi = topk_w[p * K + k];
                if (id >= 0) key[r] = ((uint32_t)id << 9) | (uint32_t)i;
            }
            w[i] = wi;
        }
    }
    __syncwarp();
    // renormalised weights w' = w / S per pixel (S in slot order)
    for (int pl = lane; pl < B; pl += 32) {
        float S = 0.f;
        for (int k = 0; k < K; ++k) S += w[pl * K + k];
        const float inv = S > 0.f ? 1.f / S : 0.f;
        for (int k = 0; k < K; ++k) w[pl * K + k] *= inv;
    }
    __syncwarp();
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
                        const uint32_t a = key[r], b = key[r | stride];
                        key[r] = up ? min(a, b) : max(a, b);
                        key[r | stride] = up ? max(a, b) : min(a, b);
                    }
                }
            }
        }
    }
    // run starts (valid keys sort first), their exclusive scan over the lanes
    const uint32_t before_lane = __shfl_up_sync(0xffffffffu, key[KPT - 1], 1);
    bool st[KPT];
    int starts = 0, valid = 0;
#pragma unroll
    for (int r = 0; r < KPT; ++r) {
        const uint32_t pk = r ? key[r - 1] : before_lane;
        const bool v = key[r] != kNone;
        st[r] = v && ((lane == 0 && r == 0) || (pk >> 9) != (key[r] >> 9));
        starts += st[r];
        valid += v;
    }
    int inc = starts, vtot = valid;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
        vtot += __shfl_xor_sync(0xffffffffu, vtot, o);
    }
    const int U = __shfl_sync(0xffffffffu, inc, 31);
    int u = inc - starts - 1;
    uint2 *brec = rec + (size_t)tile * nslots;
    uint2 *bruns = runs + (size_t)tile * runs_stride(nslots);
#pragma unroll
    for (int r = 0; r < KPT; ++r) {
        const int e = lane * KPT + r;
        if (e < nslots) {
            uint2 rr = make_uint2(0u, 0u);
            if (key[r] != kNone) {
                if (st[r]) {
                    ++u;
                    bruns[u] = make_uint2((uint32_t)e, key[r] >> 9);
                }
                const int sl = (int)(key[r] & 511u);
                rr = make_uint2((uint32_t)(sl / K) | ((uint32_t)u << 16), __float_as_uint(w[sl]));
            }
            brec[e] = rr;
        }
    }
    if (lane == 0) {
        tile_u[tile] = (uint32_t)U;
        bruns[U] = make_uint2((uint32_t)vtot, 0u);
    }
}

// ------------------------------------------------------------------------------------
// T3: per-block accumulation from shared-memory stages filled by TMA
// ------------------------------------------------------------------------------------
constexpr int kBlkNT = 256;
constexpr int kBlkNW = kBlkNT / 32;
constexpr int kTmaInner = 256;                       // elements per TMA box row (box limit)
constexpr long long kWaitCycles = 2000000000ll;      // default bound of an mbarrier wait (~1 s)

struct TmaMaps {
    CUtensorMap m[GS_MAX_CAMERAS];                   // dL/dF of each camera as [H][W][D]
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Waits for the phase with the given parity to complete; false once more than `limit`
// SM clock cycles have passed.  The elapsed time is checked before every probe, so a
// limit of a few cycles runs out on the first check whether or not the phase is done.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit)
{
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        if (clock64() - t0 > limit) return false;
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
    }
}
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"((unsigned long long)src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

template <bool BF16>
struct SRow;
template <>
struct SRow<false> {      // 16 bytes = 4 floats, from shared memory
    static constexpr int VEC = 4;
    __device__ __forceinline__ static void load(const unsigned char *p, float (&x)[4])
    {
        const float4 v = *(const float4 *)p;
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    }
};
template <>
struct SRow<true> {       // 16 bytes = 8 bf16
    static constexpr int VEC = 8;
    __device__ __forceinline__ static void load(const unsigned char *p, float (&x)[8])
    {
        const uint4 v = *(const uint4 *)p;
        const __nv_bfloat162 *h = (const __nv_bfloat162 *)&v;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 f = __bfloat1622float2(h[i]);
            x[2 * i] = f.x;
            x[2 * i + 1] = f.y;
        }
    }
};

// Row geometry of a stage: a block's dL/dF rows arrive as ncol TMA boxes of
// [TH][TW][inner] elements (inner = min(D, 256)); chunk ch (16 bytes) of pixel pl sits at
// (ch / cpb) * B * inner * esz + pl * inner * esz + (ch % cpb) * 16, cpb = inner esz / 16.
static int tma_inner(int D) { return D < kTmaInner ? D : kTmaInner; }
static int tma_ncol(int D) { return (D + kTmaInner - 1) / kTmaInner; }

// One stage: the rows, the block's records (B K uint2) and run table (runs_stride uint2),
// 128-byte aligned.  Dynamic shared memory: kStages stages.
constexpr int kStages = 3;

static size_t stage_bytes(int B, int K, int dtype, int D)
{
    const size_t rows = (size_t)tma_ncol(D) * B * tma_inner(D) * (dtype == GS_BF16 ? 2 : 4);
    const size_t b = rows + 8 * (size_t)B * K + 8 * (size_t)runs_stride(B * K);
    return (b + 127) & ~(size_t)127;
}

size_t block_accum_smem(int B, int K, int D, int dtype) { return 128 + kStages * stage_bytes(B, K, dtype, D); }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// Warp-specialised pipeline: warp kBlkNW (the producer) fills the kStages stages with
// TMA and bulk copies, one block after another, once the consumers have released a
// stage; warps 0..kBlkNW-1 (the consumers) each own whole runs (runs w, w + kBlkNW, ...)
// of the block in a full stage: a run -- one Gaussian's slots in the block, at most B --
// is summed by one warp in slot order and written as its partial row, so the result does
// not depend on the warp count and needs no cross-warp merge; no CTA-wide barrier sits
// between blocks.
template <int TW, int TH, bool BF16, int CPL>
__global__ void __launch_bounds__(kBlkNT + 32, 1) k_block_accum(const __grid_constant__ TmaMaps maps, CamTable cb,
                                                                int K, int D, int st_sz,
                                                                const uint2 *__restrict__ rec,
                                                                const uint2 *__restrict__ runs,
                                                                const uint32_t *__restrict__ row_base,
                                                                const uint32_t *__restrict__ tile_u,
                                                                uint32_t rows_cap, float *__restrict__ rows,
                                                                uint32_t *__restrict__ pair_keys,
                                                                uint32_t *__restrict__ pair_vals, int N, int *err,
                                                                const unsigned long long *__restrict__ wait_limit)
{
    constexpr int B = TW * TH;
    using Rw = SRow<BF16>;
    constexpr int VEC = Rw::VEC;
    constexpr int ESZ = BF16 ? 2 : 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t s_full[kStages], s_empty[kStages];
    __shared__ uint32_t s_meta[kStages][2];          // (U, row base) of the block in each stage
    __shared__ int s_bad, s_issued, s_done[kBlkNW];
    __shared__ long long s_limit;
    const int nslots = B * K;
    const int rstride = runs_stride(nslots);
    const int nch = D / VEC;                           // 16-byte chunks per row
    const int inner = D < kTmaInner ? D : kTmaInner;
    const int ncol = (D + kTmaInner - 1) / kTmaInner;
    const int cpb = inner * ESZ / 16;                  // chunks per box row
    const int pix_bytes = inner * ESZ;
    const int col_bytes = B * pix_bytes;
    const int rows_sz = ncol * col_bytes;
    // 128-byte aligned base, offset within the shared array (the pointer stays a
    // shared-memory pointer, so the stage reads compile to shared loads)
    unsigned char *base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_blocks = cb.n_tiles;
    const int G = gridDim.x;
    const int my_n = (int)((n_blocks - (int)blockIdx.x + G - 1) / G);
    const uint32_t stage_tx = (uint32_t)(rows_sz + 8 * nslots + 8 * rstride);

    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&s_full[i], 1);
            mbar_init(&s_empty[i], kBlkNW);
        }
        fence_mbar_init();
        s_bad = *err != 0;
        s_issued = 0;
        // the pipeline waits' bound (0: the default); the final drain keeps the default
        const unsigned long long wl = *wait_limit;
        s_limit = wl == 0ull || wl > (unsigned long long)kWaitCycles ? kWaitCycles : (long long)wl;
    }
    if (tid < kBlkNW) s_done[tid] = 0;
    __syncthreads();
    const bool bad = s_bad != 0;
    const long long limit = s_limit;

    if (warp == kBlkNW) {
        // producer
        if (lane == 0 && !bad) {
            // (U, row base) of the next two blocks are loaded ahead, so no global round
            // trip delays a copy
            uint32_t U0 = 0, rb0 = 0, U1 = 0, rb1 = 0;
            if (my_n > 0) { U0 = tile_u[blockIdx.x]; rb0 = row_base[blockIdx.x]; }
            if (my_n > 1) { U1 = tile_u[blockIdx.x + G]; rb1 = row_base[blockIdx.x + G]; }
            int j = 0;
            for (; j < my_n; ++j) {
                const int sidx = j % kStages;
                const int blk = blockIdx.x + j * G;
                uint32_t U2 = 0, rb2 = 0;
                if (j + 2 < my_n) { U2 = tile_u[blk + 2 * G]; rb2 = row_base[blk + 2 * G]; }
                if (j >= kStages && !mbar_wait(&s_empty[sidx], ((j / kStages) - 1) & 1, limit)) {
                    atomicOr(err, kErrTimeout);
                    break;
                }
                s_meta[sidx][0] = U0;
                s_meta[sidx][1] = rb0;
                U0 = U1; rb0 = rb1; U1 = U2; rb1 = rb2;
                unsigned char *st = base + (size_t)sidx * st_sz;
                const int c = cam_of_tile(cb, blk);
                const CamDev &cam = cb.c[c];
                const int lt = blk - cam.tile_off;
                const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
                fence_async_shared();
                mbar_expect_tx(&s_full[sidx], stage_tx);
                for (int col = 0; col < ncol; ++col)
                    tma_load_3d(st + (size_t)col * col_bytes, &maps.m[c], col * inner, tx * TW, ty * TH,
                                &s_full[sidx]);
                bulk_load(st + rows_sz, rec + (size_t)blk * nslots, 8u * nslots, &s_full[sidx]);
                bulk_load(st + rows_sz + 8 * nslots, runs + (size_t)blk * rstride, 8u * rstride, &s_full[sidx]);
            }
            s_issued = j;
        }
    } else if (!bad) {
        // consumers
        int coff[CPL];                               // stage offset of each lane chunk
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) {
            const int ch = lane + 32 * cc;
            coff[cc] = (ch / cpb) * col_bytes + (ch % cpb) * 16;
        }
        int j = 0;
        for (; j < my_n; ++j) {
            const int sidx = j % kStages;
            if (!mbar_wait(&s_full[sidx], (j / kStages) & 1, limit)) {
                if (lane == 0) atomicOr(err, kErrTimeout);
                break;
            }
            const uint32_t U = s_meta[sidx][0], rb = s_meta[sidx][1];
            const bool over = U > 0 && rb + U > rows_cap;
            if (over && warp == 0 && lane == 0) atomicOr(err, kErrOverflow);
            if (!over) {
                const unsigned char *st = base + (size_t)sidx * st_sz;
                const uint2 *s_rec = (const uint2 *)(st + rows_sz);
                const uint2 *s_runs = (const uint2 *)(st + rows_sz + 8 * nslots);
                for (int u = warp; u < (int)U; u += kBlkNW) {
                    const int i0 = (int)s_runs[u].x, i1 = (int)s_runs[u + 1].x;
                    float acc[CPL][VEC];
#pragma unroll
                    for (int cc = 0; cc < CPL; ++cc)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[cc][v] = 0.f;
                    for (int i = i0; i < i1; ++i) {
                        const uint2 r = s_rec[i];
                        const float wp = __uint_as_float(r.y);
                        const unsigned char *px = st + (size_t)(r.x & 0xffffu) * pix_bytes;
#pragma unroll
                        for (int cc = 0; cc < CPL; ++cc) {
                            if (lane + 32 * cc < nch) {
                                float x[VEC];
                                Rw::load(px + coff[cc], x);
#pragma unroll
                                for (int v = 0; v < VEC; ++v) acc[cc][v] = fmaf(wp, x[v], acc[cc][v]);
                            }
                        }
                    }
                    float *dst = rows + (size_t)(rb + u) * D;
#pragma unroll
                    for (int cc = 0; cc < CPL; ++cc) {
                        const int ch = lane + 32 * cc;
                        if (ch < nch) {
                            float4 *d4 = (float4 *)(dst + (size_t)ch * VEC);
#pragma unroll
                            for (int v = 0; v < VEC / 4; ++v)
                                d4[v] = make_float4(acc[cc][4 * v], acc[cc][4 * v + 1], acc[cc][4 * v + 2],
                                                    acc[cc][4 * v + 3]);
                        }
                    }
                    if (lane == 0) {
                        pair_keys[N + rb + u] = s_runs[u].y;
                        pair_vals[N + rb + u] = rb + u;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_empty[sidx]);   // this warp is done with the stage
        }
        if (lane == 0) s_done[warp] = j;
    }
    __syncthreads();
    // copies still in flight (only after a timed-out wait): wait for them with the
    // default bound whatever the pipeline's limit, so no copy lands after the CTA exits
    if (tid == 0) {
        int done = my_n;
        for (int w = 0; w < kBlkNW; ++w) done = min(done, s_done[w]);
        if (bad) done = 0;
        for (int jj = done; jj < s_issued; ++jj) mbar_wait(&s_full[jj % kStages], (jj / kStages) & 1, kWaitCycles);
    }
}

// ------------------------------------------------------------------------------------
// T3 for bf16 dL/dF on the tensor cores.  A block's partial rows are a small dense
// product: P[U_b x D] = W^T[U_b x B] dL/dF[B x D], W^T[u][p] = w' of pixel p's slot that
// selected run u's Gaussian (0 elsewhere; at K = 8 most entries are filled).  One warp
// per block: W^T built from the sorted slot records, its float32 weights split exactly
// into three bf16 terms (A fragments, 16 runs x 16 pixels per MMA tile); the block's
// dL/dF rows staged 64 columns at a time by cp.async into padded shared memory
// (double-buffered, one pixel row per lane) and read with ldmatrix.trans; mma.m16n8k16
// with float32 accumulation; runs in batches of 32.  Each partial row is a fixed
// sequence of MMAs, so the result is deterministic.
// ------------------------------------------------------------------------------------
constexpr int kBmRuns = 32;                      // runs per batch (two 16-row MMA tiles)
constexpr int kBmCols = 64;                      // columns per staged chunk
constexpr int kBmPitch = kBmCols * 2 + 16;       // bytes per staged row: conflict-free ldmatrix
constexpr int kBmWarps = 4;

template <int B>
struct BlockMmaSmem {
    unsigned char rows[2][B * kBmPitch];         // the block's dL/dF rows, one chunk (double buffer)
    float wt[kBmRuns][B];                        // W^T of a batch of runs
};

template <int TW, int TH>
__device__ __forceinline__ void block_mma_one(const CamTable &cb, int K, int D, const __nv_bfloat16 *__restrict__ dLdF,
                                              const uint2 *__restrict__ rec, const uint2 *__restrict__ runs,
                                              const uint32_t *__restrict__ row_base,
                                              const uint32_t *__restrict__ tile_u, uint32_t rows_cap,
                                              float *__restrict__ rows, uint32_t *__restrict__ pair_keys,
                                              uint32_t *__restrict__ pair_vals, int N, int *err, int blk, int lane,
                                              BlockMmaSmem<TW * TH> &sm);

template <int TW, int TH>
__global__ void __launch_bounds__(kBmWarps * 32, 3) k_block_mma(CamTable cb, int K, int D, const __nv_bfloat16 *__restrict__ dLdF,
                                                          const uint2 *__restrict__ rec, const uint2 *__restrict__ runs,
                                                          const uint32_t *__restrict__ row_base,
                                                          const uint32_t *__restrict__ tile_u, uint32_t rows_cap,
                                                          float *__restrict__ rows, uint32_t *__restrict__ pair_keys,
                                                          uint32_t *__restrict__ pair_vals, int N, int *err)
{
    constexpr int B = TW * TH;
    static_assert(B % 16 == 0 && B <= 32, "pixel blocks of 16 or 32");
    extern __shared__ __align__(16) unsigned char smem_bm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    BlockMmaSmem<B> &sm = ((BlockMmaSmem<B> *)smem_bm)[wib];
    if (*err) return;
    const int blk = blockIdx.x * kBmWarps + wib;
    if (blk >= cb.n_tiles) return;               // whole warp
    block_mma_one<TW, TH>(cb, K, D, dLdF, rec, runs, row_base, tile_u, rows_cap, rows, pair_keys, pair_vals, N, err,
                          blk, lane, sm);
}

// One feature-gradient block of k_block_mma (a warp).
template <int TW, int TH>
__device__ __forceinline__ void block_mma_one(const CamTable &cb, int K, int D, const __nv_bfloat16 *__restrict__ dLdF,
                                              const uint2 *__restrict__ rec, const uint2 *__restrict__ runs,
                                              const uint32_t *__restrict__ row_base,
                                              const uint32_t *__restrict__ tile_u, uint32_t rows_cap,
                                              float *__restrict__ rows, uint32_t *__restrict__ pair_keys,
                                              uint32_t *__restrict__ pair_vals, int N, int *err, int blk, int lane,
                                              BlockMmaSmem<TW * TH> &sm)
{
    constexpr int B = TW * TH;
    constexpr int KSP = B / 16;                  // 16-pixel k-steps
    const int g = lane >> 2, t = lane & 3;
    const int nslots = B * K;
    const int rstride = (nslots + 2) & ~1;       // runs_stride
    const uint32_t U = tile_u[blk], rb = row_base[blk];
    if (U == 0) return;
    if (rb + U > rows_cap) {
        if (lane == 0) atomicOr(err, kErrOverflow);
        return;
    }
    const uint2 *brec = rec + (size_t)blk * nslots;
    const uint2 *bruns = runs + (size_t)blk * rstride;
    // the block's pixels in the flat pixel space (lane < B stages pixel row `lane`)
    const int c = cam_of_tile(cb, blk);
    const CamDev &cam = cb.c[c];
    const int lt = blk - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    long long my_pix = -1;
    if (lane < B) {
        const int px = tx * TW + lane % TW, py = ty * TH + lane / TW;
        if (px < cam.W && py < cam.H) my_pix = cam.pix_off + (long long)py * cam.W + px;
    }
    auto stage = [&](int c0, int buf) {
        if (lane < B) {
            const bool real = my_pix >= 0;
            const __nv_bfloat16 *src = dLdF + (real ? (size_t)my_pix * D + c0 : 0);
            const uint32_t dst = smem_addr(sm.rows[buf] + lane * kBmPitch);
#pragma unroll
            for (int q = 0; q < 8; ++q) cp_async_16(dst + 16 * q, src + (real ? 8 * q : 0), real ? 16 : 0);
        }
        cp_async_commit_group();
    };
    const int nchunk = D / kBmCols;
    const int mi = lane >> 3, mr = lane & 7;
    for (uint32_t u0 = 0; u0 < U; u0 += kBmRuns) {
        const int nr = (int)min((uint32_t)kBmRuns, U - u0);
        const int MT = nr <= 16 ? 1 : 2;         // 16-run MMA tiles
        // W^T of this batch from the sorted slot records of its runs
        for (int i = lane; i < kBmRuns * B; i += 32) (&sm.wt[0][0])[i] = 0.f;
        __syncwarp();
        const int i0 = (int)bruns[u0].x, i1 = (int)bruns[u0 + nr].x;
        for (int i = i0 + lane; i < i1; i += 32) {
            const uint2 r = brec[i];
            sm.wt[(int)(r.x >> 16) - (int)u0][r.x & 0xffffu] = __uint_as_float(r.y);
        }
        __syncwarp();
        uint32_t afr[2][KSP][3][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            if (mt >= MT) break;
#pragma unroll
            for (int ks = 0; ks < KSP; ++ks) {
                const int r0 = 16 * mt + g, cc = 16 * ks + 2 * t;
                const float v[8] = {sm.wt[r0][cc], sm.wt[r0][cc + 1], sm.wt[r0 + 8][cc], sm.wt[r0 + 8][cc + 1],
                                    sm.wt[r0][cc + 8], sm.wt[r0][cc + 9], sm.wt[r0 + 8][cc + 8], sm.wt[r0 + 8][cc + 9]};
                float hh[8], mm[8], ll[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) split3(v[e], hh[e], mm[e], ll[e]);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    afr[mt][ks][0][q] = pack_bf16(hh[2 * q], hh[2 * q + 1]);
                    afr[mt][ks][1][q] = pack_bf16(mm[2 * q], mm[2 * q + 1]);
                    afr[mt][ks][2][q] = pack_bf16(ll[2 * q], ll[2 * q + 1]);
                }
            }
        }
        stage(0, 0);
        for (int ch = 0; ch < nchunk; ++ch) {
            const int buf = ch & 1;
            if (ch + 1 < nchunk) {
                stage((ch + 1) * kBmCols, buf ^ 1);
                cp_async_wait_group<1>();
            } else {
                cp_async_wait_group<0>();
            }
            __syncwarp();
            float acc[2][8][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int j = 0; j < 8; ++j)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[mt][j][v] = 0.f;
            const uint32_t base = smem_addr(sm.rows[buf]);
#pragma unroll
            for (int ks = 0; ks < KSP; ++ks) {
                uint32_t b[4][4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    // pixels 16ks + {0-7, 8-15} x columns 16m + {0-7, 8-15}, transposed
                    const int r = 16 * ks + mr + 8 * (mi & 1), cc = 16 * m + 8 * (mi >> 1);
                    ldsm_x4_t(base + r * kBmPitch + 2 * cc, b[m][0], b[m][1], b[m][2], b[m][3]);
                }
                // per accumulator the three terms in order, independent products between
#pragma unroll
                for (int sp = 0; sp < 3; ++sp)
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        if (mt >= MT) break;
#pragma unroll
                        for (int m = 0; m < 4; ++m) {
                            mma16816(acc[mt][2 * m], afr[mt][ks][sp], b[m][0], b[m][1]);
                            mma16816(acc[mt][2 * m + 1], afr[mt][ks][sp], b[m][2], b[m][3]);
                        }
                    }
            }
            // partial rows (float32): run 16 mt + g (+ 8), columns 8 j + 2 t (+ 1)
            const int c0 = ch * kBmCols;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                if (mt >= MT) break;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int u = 16 * mt + g + 8 * half;
                    if (u < nr) {
                        float *dst = rows + (size_t)(rb + u0 + u) * D + c0 + 2 * t;
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            *(float2 *)(dst + 8 * j) = make_float2(acc[mt][j][2 * half], acc[mt][j][2 * half + 1]);
                    }
                }
            }
            __syncwarp();                        // the buffer is free for the next stage
        }
        for (int u = lane; u < nr; u += 32) {
            pair_keys[N + rb + u0 + u] = bruns[u0 + u].y;
            pair_vals[N + rb + u0 + u] = rb + u0 + u;
        }
        __syncwarp();
    }
}

bool block_mma_supported(int dtype, int D, int B) { return dtype == GS_BF16 && D % kBmCols == 0 && (B == 16 || B == 32); }

// ------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------
int tile_sort_len(int slots)
{
    int n = 1;
    while (n < slots) n <<= 1;
    return n;
}

bool tile_grad_supported(int dtype, int D, int K)
{
    const FgBlock fb = fg_block_shape(dtype, D, K);
    if (fb.bw == 0) return false;
    const int B = fb.bw * fb.bh;
    return B * K <= 65535 && block_accum_smem(B, K, D, dtype) <= 227 * 1024 &&
           (8 + 4) * (size_t)tile_sort_len(B * K) <= 200 * 1024;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// dL/dF of camera c viewed as [H][W][D], boxes of [bh][bw][min(D, 256)] elements
static bool make_maps(const CamTable &cb, int dtype, int D, const void *dLdF, TmaMaps &maps)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const int esz = dtype == GS_BF16 ? 2 : 4;
    memset(&maps, 0, sizeof(maps));
    for (int c = 0; c < cb.n; ++c) {
        const CamDev &cam = cb.c[c];
        void *gbase = (void *)((const char *)dLdF + (size_t)cam.pix_off * D * esz);
        const cuuint64_t dims[3] = {(cuuint64_t)D, (cuuint64_t)cam.W, (cuuint64_t)cam.H};
        const cuuint64_t strides[2] = {(cuuint64_t)D * esz, (cuuint64_t)D * esz * cam.W};
        const cuuint32_t box[3] = {(cuuint32_t)tma_inner(D), (cuuint32_t)cb.tile_w, (cuuint32_t)cb.tile_h};
        const cuuint32_t estr[3] = {1, 1, 1};
        const CUresult r = enc(&maps.m[c], dtype == GS_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                               3, gbase, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

template <int TW, int TH, bool BF16, int CPLV>
static void accum_one(unsigned grid, size_t sm, cudaStream_t s, const TmaMaps &maps, const CamTable &cb,
                      const WsLayout &L, int st_sz, const uint2 *rec, const uint2 *runs, const uint32_t *rbase,
                      const uint32_t *tu, float *rows, uint32_t *pk, uint32_t *pv, int *err,
                      const unsigned long long *wl)
{
    cudaFuncSetAttribute(k_block_accum<TW, TH, BF16, CPLV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    // persistent: as many CTAs as fit on the SMs (grid arrives as blocks, capped at one per SM)
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_block_accum<TW, TH, BF16, CPLV>, kBlkNT + 32, sm);
    grid = std::max(1u, std::min(grid * (unsigned)std::max(1, occ), (unsigned)cb.n_tiles));
    k_block_accum<TW, TH, BF16, CPLV><<<grid, kBlkNT + 32, sm, s>>>(maps, cb, L.K, L.D, st_sz, rec, runs, rbase, tu,
                                                               (uint32_t)L.rows_cap, rows, pk, pv, L.N, err, wl);
}

template <int TW, int TH, bool BF16>
static void accum_launch(int cpl, unsigned grid, size_t sm, cudaStream_t s, const TmaMaps &maps, const CamTable &cb,
                         const WsLayout &L, int st_sz, const uint2 *rec, const uint2 *runs, const uint32_t *rbase,
                         const uint32_t *tu, float *rows, uint32_t *pk, uint32_t *pv, int *err,
                         const unsigned long long *wl)
{
    // (D <= 1024 caps bf16 rows at 4 chunks per lane; float32 rows at 8)
    switch (cpl) {
    case 1: accum_one<TW, TH, BF16, 1>(grid, sm, s, maps, cb, L, st_sz, rec, runs, rbase, tu, rows, pk, pv, err, wl); break;
    case 2: accum_one<TW, TH, BF16, 2>(grid, sm, s, maps, cb, L, st_sz, rec, runs, rbase, tu, rows, pk, pv, err, wl); break;
    case 4: accum_one<TW, TH, BF16, 4>(grid, sm, s, maps, cb, L, st_sz, rec, runs, rbase, tu, rows, pk, pv, err, wl); break;
    default:
        accum_one<TW, TH, BF16, (BF16 ? 4 : 8)>(grid, sm, s, maps, cb, L, st_sz, rec, runs, rbase, tu, rows, pk, pv,
                                                 err, wl);
        break;
    }
}

static int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 148;
    return n;
}

template <int TW, int TH>
static bool tile_launch(const CamTable &cb, const WsLayout &L, int dtype, const int *topk_idx, const float *topk_w,
                        const void *dLdF, void *ws, cudaStream_t s, cudaStream_t hold, cudaEvent_t hold_ev)
{
    constexpr int B = TW * TH;
    uint32_t *hdr = ws_ptr<uint32_t>(ws, L.header);
    int *err = (int *)hdr;
    uint2 *rec = ws_ptr<uint2>(ws, L.tile_keys);
    uint2 *runs = ws_ptr<uint2>(ws, L.tile_runs);
    uint32_t *tile_u = ws_ptr<uint32_t>(ws, L.tile_u);
    uint32_t *row_base = ws_ptr<uint32_t>(ws, L.tile_rowbase);
    float *rows = ws_ptr<float>(ws, L.tile_rows);
    uint32_t *pk = ws_ptr<uint32_t>(ws, L.pair_keys[0]);
    uint32_t *pv = ws_ptr<uint32_t>(ws, L.pair_vals[0]);
    uint32_t *aux = ws_ptr<uint32_t>(ws, L.scan_aux);
    const int nsort = tile_sort_len(B * L.K);
    if (L.N < (1 << 22) && nsort <= 512) {
        const unsigned g = (unsigned)((cb.n_tiles + 3) / 4);
#define GS_TSW(KP) k_tile_slots_warp<TW, TH, KP><<<g, 128, 0, s>>>(cb, L.K, topk_idx, topk_w, err, rec, runs, tile_u)
        switch (std::max(32, nsort) / 32) {
        case 1: GS_TSW(1); break;
        case 2: GS_TSW(2); break;
        case 4: GS_TSW(4); break;
        case 8: GS_TSW(8); break;
        default: GS_TSW(16); break;
        }
#undef GS_TSW
    } else {
        const size_t sm1 = (sizeof(unsigned long long) + sizeof(float)) * nsort;
        const int nt1 = std::min(1024, std::max(32, nsort / 2));
        cudaFuncSetAttribute(k_tile_slots<TW, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
        k_tile_slots<TW, TH><<<cb.n_tiles, nt1, sm1, s>>>(cb, L.K, nsort, topk_idx, topk_w, err, rec, runs, tile_u);
    }
    exclusive_scan_u32(tile_u, row_base, cb.n_tiles, hdr + 8, aux, s);
    if constexpr (B == 16 || B == 32) {
        if (block_mma_supported(dtype, L.D, B)) {
            const size_t smb = sizeof(BlockMmaSmem<B>) * kBmWarps;
            cudaFuncSetAttribute(k_block_mma<TW, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smb);
            const unsigned gb = (unsigned)((cb.n_tiles + kBmWarps - 1) / kBmWarps);
            TimerScope tm(GS_TIMER_BLOCK_GRAD, s);
            k_block_mma<TW, TH><<<gb, kBmWarps * 32, smb, s>>>(cb, L.K, L.D, (const __nv_bfloat16 *)dLdF, rec, runs,
                                                               row_base, tile_u, (uint32_t)L.rows_cap, rows, pk, pv,
                                                               L.N, err);
            return true;
        }
    }
    TmaMaps maps;
    if (!make_maps(cb, dtype, L.D, dLdF, maps)) return false;
    // The re-walk on the other stream holds until the block records are written, so it
    // becomes ready together with the block product queued next: the product's CTAs (one
    // per SM) are placed first and the re-walk's persistent CTAs fill the rest of each SM.
    // Launched earlier, the re-walk takes every SM's registers and the product starts only
    // as it drains.  (The tensor-core product, many CTAs per SM, is not held: it would take
    // the SMs from the re-walk instead.)
    if (hold && hold_ev && hold != s) {
        if (cudaEventRecord(hold_ev, s) != cudaSuccess || cudaStreamWaitEvent(hold, hold_ev, 0) != cudaSuccess)
            return false;
    }
    const size_t sm3 = block_accum_smem(B, L.K, L.D, dtype);
    const int st_sz = (int)stage_bytes(B, L.K, dtype, L.D);
    const int nch = L.D / (dtype == GS_BF16 ? 8 : 4);
    const int cpl = nch <= 32 ? 1 : nch <= 64 ? 2 : nch <= 128 ? 4 : 8;
    const unsigned grid = (unsigned)std::max(1, std::min(cb.n_tiles, sm_count()));
    const unsigned long long *wl = ws_ptr<const unsigned long long>(ws, L.header + kHdrWaitLimitByte);
    TimerScope tm(GS_TIMER_BLOCK_GRAD, s);
    if (dtype == GS_BF16)
        accum_launch<TW, TH, true>(cpl, grid, sm3, s, maps, cb, L, st_sz, rec, runs, row_base, tile_u, rows, pk, pv,
                                   err, wl);
    else
        accum_launch<TW, TH, false>(cpl, grid, sm3, s, maps, cb, L, st_sz, rec, runs, row_base, tile_u, rows, pk, pv,
                                    err, wl);
    return true;
}

// Stages T1-T3 on the feature-gradient blocks of ct's cameras; leaves the (Gaussian,
// row) pairs after N marker slots in pair buffer 0, the partial rows, and U_tot in
// header word 8.
bool launch_tile_grad(const CamTable &ct, const WsLayout &L, int dtype, const int *topk_idx, const float *topk_w,
                      const void *dLdF, void *ws, cudaStream_t s, cudaStream_t hold, cudaEvent_t hold_ev)
{
    const FgBlock fb = fg_block_shape(dtype, L.D, L.K);
    CamTable cb;
    retile(ct, fb.bw, fb.bh, cb);
    if (fb.bw == 8 && fb.bh == 8) return tile_launch<8, 8>(cb, L, dtype, topk_idx, topk_w, dLdF, ws, s, hold, hold_ev);
    if (fb.bw == 8 && fb.bh == 4) return tile_launch<8, 4>(cb, L, dtype, topk_idx, topk_w, dLdF, ws, s, hold, hold_ev);
    if (fb.bw == 4 && fb.bh == 4) return tile_launch<4, 4>(cb, L, dtype, topk_idx, topk_w, dLdF, ws, s, hold, hold_ev);
    return false;
}

size_t tile_runs_bytes(int B, int K) { return 8 * (size_t)runs_stride(B * K); }

}  // namespace gs
