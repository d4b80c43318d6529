// gs_bin.cu -- a2: tile binning and (tile, depth) ordering.
//
// Order of work (chosen so the sort over the large instance set needs only the tile
// bits):
//   1. sort the (camera, Gaussian) elements by float32 depth (32-bit keys, N-sized);
//   2. count the tiles of each element's footprint box that its ellipse reaches (one run
//      of tiles per tile row, from the ellipse's x-range over the row), in depth order,
//      and scan;
//   3. emit one instance per such (element, tile), in depth order, keyed by global tile id;
//   4. stable radix sort of the instances by tile id -> within a tile, depth order
//      (ties keep element order, i.e. ascending Gaussian id within a camera);
//   5. per-tile [start, end) ranges (a search per tile over the sorted keys).
// The instance count is only known on the device; every launch after step 2 reads it
// from the workspace header, so nothing synchronises with the host.
#include "gs_internal.cuh"

namespace gs {

__global__ void k_depth_keys(long long NE, const float4 *__restrict__ proj, uint32_t *keys, uint32_t *vals)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NE) return;
    float4 r2 = proj[4 * e + 2], r3 = proj[4 * e + 3];
    bool live = __float_as_uint(r3.w) != 0u;
    keys[e] = live ? __float_as_uint(r2.w) : 0xffffffffu;   // positive floats order as integers
    vals[e] = (uint32_t)e;
}

__device__ __forceinline__ uint32_t tiles_of(const CamTable &ct, const float4 *proj, uint32_t e, int N,
                                             int &c, int &tx0, int &tx1, int &ty0, int &ty1)
{
    c = (int)(e / (uint32_t)N);
    float4 r3 = proj[4 * (size_t)e + 3];
    if (__float_as_uint(r3.w) == 0u) return 0;
    float4 r0 = proj[4 * (size_t)e];
    float ex, ey;
    unpack_extent(r3.w, ex, ey);
    if (!tile_rect(ct.c[c], ct.tile_w, ct.tile_h, r0.x, r0.y, ex, ey, tx0, tx1, ty0, ty1)) return 0;
    return (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
}

// The tiles of a footprint box that the Gaussian's opacity-cut ellipse q(dx, dy) <= qb
// reaches (qb and q as in the walks' touches_rect), one row of tiles at a time.  With
// q = (s1 dx)^2 + (s2 (dy - m dx))^2 and A = s1^2 + s2^2 m^2, the ellipse's section at
// offset dy spans
//     dx = (s2^2 m dy -/+ sqrt(A qb - (s1 s2 dy)^2)) / A,   |dy| <= sqrt(A qb) / (s1 s2);
// its right end is largest at dy = m sqrt(qb) / s1 and its left end smallest at the
// opposite offset.  So over the band of a tile row's pixel centres the ellipse covers one
// x-interval -- its ends are those two offsets clamped into the band -- and the tiles
// whose pixel-centre columns meet it form one run.  A tile outside the run has no pixel
// centre with q <= qb, so no walk would accept the Gaussian there.  Only correctly
// rounded single operations are used (never contracted into FMAs), so the counting and
// the emitting kernels derive identical runs.
struct RowCull {
    float u, v, s2m, A, s12, qb, dymax, dys;
    bool ok;
    __device__ __forceinline__ RowCull(const float4 r0, const float4 r1)
    {
        u = __fadd_rn(r0.x, r0.z);
        v = __fadd_rn(r0.y, r0.w);
        const float s1 = r1.x, m = r1.y, s2 = r1.z;
        // 2 ln(255 o) through the hardware log2 (one instruction, the same result in both
        // kernels; its error is far inside the 0.4% + 0.02 margin)
        const float q = fminf(kQMax, __fmul_rn(1.38629436f, __log2f(__fmul_rn(255.0f, r1.w))));
        qb = __fadd_rn(__fmul_rn(fmaxf(q, 0.0f), 1.004f), 0.02f);
        ok = s1 > 0.f && s2 > 0.f && isfinite(m) && isfinite(s1) && isfinite(s2);
        const float s22 = __fmul_rn(s2, s2), s1s2 = __fmul_rn(s1, s2);
        s2m = __fmul_rn(s22, m);
        A = __fadd_rn(__fmul_rn(s1, s1), __fmul_rn(s2m, m));
        s12 = __fmul_rn(s1s2, s1s2);
        dymax = ok ? __fdiv_rn(__fsqrt_rn(__fmul_rn(A, qb)), s1s2) : 0.f;
        dys = ok ? __fdiv_rn(__fmul_rn(m, __fsqrt_rn(qb)), s1) : 0.f;
    }
    __device__ __forceinline__ float root(float dy) const
    {
        return __fsqrt_rn(fmaxf(__fsub_rn(__fmul_rn(A, qb), __fmul_rn(s12, __fmul_rn(dy, dy))), 0.f));
    }
    // The run [a, b] of tile columns (within [tx0, tx1]) that the ellipse reaches in tile
    // row ty; false for none.
    __device__ __forceinline__ bool run(const CamDev &cam, int tw, int th, int ty, int tx0, int tx1, int &a,
                                        int &b) const
    {
        if (!ok) {
            a = tx0;
            b = tx1;
            return true;
        }
        const float lo = fmaxf(__fsub_rn((float)(ty * th) + 0.5f, v), -dymax);
        const float hi = fminf(__fsub_rn((float)min((ty + 1) * th, cam.H) - 0.5f, v), dymax);
        if (!(lo <= hi)) return false;
        const float yr = fminf(fmaxf(dys, lo), hi), yl = fminf(fmaxf(-dys, lo), hi);
        const float xmax = __fdiv_rn(__fadd_rn(__fmul_rn(s2m, yr), root(yr)), A);
        const float xmin = __fdiv_rn(__fsub_rn(__fmul_rn(s2m, yl), root(yl)), A);
        // columns tx with pixel centres [tx tw + 0.5, (tx + 1) tw - 0.5] meeting
        // [u + xmin, u + xmax], widened by 0.01 px
        const float X0 = __fsub_rn(__fadd_rn(u, xmin), 0.01f), X1 = __fadd_rn(__fadd_rn(u, xmax), 0.01f);
        const float af = __fsub_rn(ceilf(__fdiv_rn(__fadd_rn(X0, 0.5f), (float)tw)), 1.0f);
        const float bf = floorf(__fdiv_rn(__fsub_rn(X1, 0.5f), (float)tw));
        a = (int)fminf(fmaxf(af, (float)tx0), (float)(tx1 + 1));
        b = (int)fmaxf(fminf(bf, (float)tx1), (float)(tx0 - 1));
        return a <= b;
    }
};

// Instances of each element, in depth order: the tiles of its footprint box that its
// ellipse reaches (RowCull runs), counted by depth rank.
__global__ void __launch_bounds__(256) k_count_tiles(CamTable ct, int N, long long NE, const float4 *__restrict__ proj,
                                                     const uint32_t *__restrict__ sorted_e, uint32_t *counts,
                                                     uint32_t *elem_cnt)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= NE) return;
    const uint32_t e = sorted_e[r];
    int c, tx0, tx1, ty0, ty1;
    const uint32_t box = tiles_of(ct, proj, e, N, c, tx0, tx1, ty0, ty1);
    uint32_t n = 0;
    if (box > 0) {
        const RowCull rc(proj[4 * (size_t)e], proj[4 * (size_t)e + 1]);
        const CamDev &cam = ct.c[c];
        for (int ty = ty0; ty <= ty1; ++ty) {
            int a, b;
            if (rc.run(cam, ct.tile_w, ct.tile_h, ty, tx0, tx1, a, b)) n += (uint32_t)(b - a + 1);
        }
    }
    counts[r] = n;
    elem_cnt[e] = n;
}

// Writes the instances counted by k_count_tiles: one warp per 32 consecutive depth ranks,
// element by element, one lane per tile row (its run, placed by a warp prefix over the
// rows), so the writes of an element are consecutive.  (An instance's sort value is its
// own index, which the tile sort generates; the re-walk's walked flags are cleared by
// k_clear_walked.)
__global__ void __launch_bounds__(256) k_duplicate(CamTable ct, int N, long long NE, const float4 *__restrict__ proj,
                                                   const uint32_t *__restrict__ sorted_e,
                                                   const uint32_t *__restrict__ offsets, uint32_t mcap,
                                                   uint32_t *inst_keys, uint32_t *inst_elem,
                                                   uint32_t *elem_off, uint32_t *elem_cnt, int *err)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    uint32_t e = 0, o = 0, n = 0;
    int c = 0, tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
    if (r < NE) {
        e = sorted_e[r];
        o = offsets[r];
        elem_off[e] = o;
        n = elem_cnt[e];                          // the instances counted by k_count_tiles
        if (n > 0) tiles_of(ct, proj, e, N, c, tx0, tx1, ty0, ty1);
        if (n > 0 && (unsigned long long)o + n > mcap) {
            // instances past the capacity are dropped; the render is reported as failed
            atomicOr(err, kErrOverflow);
            elem_cnt[e] = o < mcap ? mcap - o : 0u;
        }
    }
    for (int j = 0; j < 32; ++j) {
        const uint32_t nj = __shfl_sync(0xffffffffu, n, j);
        if (nj == 0) continue;
        const uint32_t ej = __shfl_sync(0xffffffffu, e, j), oj = __shfl_sync(0xffffffffu, o, j);
        const int cj = __shfl_sync(0xffffffffu, c, j);
        const int x0 = __shfl_sync(0xffffffffu, tx0, j), x1 = __shfl_sync(0xffffffffu, tx1, j);
        const int y0 = __shfl_sync(0xffffffffu, ty0, j), y1 = __shfl_sync(0xffffffffu, ty1, j);
        const CamDev &cam = ct.c[cj];
        const RowCull rc(proj[4 * (size_t)ej], proj[4 * (size_t)ej + 1]);
        uint32_t base = oj;
        for (int ry = y0; ry <= y1; ry += 32) {
            const int ty = ry + lane;
            int a = 0, b = -1;
            const bool any = ty <= y1 && rc.run(cam, ct.tile_w, ct.tile_h, ty, x0, x1, a, b);
            const uint32_t cnt = any ? (uint32_t)(b - a + 1) : 0u;
            uint32_t incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            const uint32_t at = base + incl - cnt;
            const uint32_t key0 = (uint32_t)(cam.tile_off + ty * cam.tiles_x + a);
            for (uint32_t k = 0; k < cnt; ++k) {
                if (at + k < mcap) {
                    inst_keys[at + k] = key0 + k;
                    inst_elem[at + k] = ej;
                }
            }
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

// Clears the walked flags of the instances [0, min(*n_dev, mcap)), 16 bytes per store
// (the re-walk sets the flags of the instances it reaches).
__global__ void __launch_bounds__(256) k_clear_walked(const uint32_t *n_dev, uint32_t mcap, uint8_t *walked)
{
    const long long n = min(*n_dev, mcap);
    const long long n16 = n / 16;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride)
        ((uint4 *)walked)[i] = make_uint4(0u, 0u, 0u, 0u);
    const long long tail = n16 * 16 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tail < n) walked[tail] = 0;
}

// Per-tile [start, end) of the sorted instances: one warp per tile finds the first
// position whose key is >= its tile id by a 32-way search over the sorted keys (a few
// dependent steps instead of a pass over every instance); that position ends the
// previous tile's range.  Empty tiles get start == end.
__global__ void __launch_bounds__(256) k_tile_ranges(const uint32_t *__restrict__ keys, const uint32_t *n_dev,
                                                     uint32_t mcap, int2 *ranges, uint32_t n_tiles)
{
    const uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n_tiles) return;                       // whole warp
    const uint32_t n = min(*n_dev, mcap);
    uint32_t lo = 0, hi = n;                        // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t pos = lo + (uint32_t)lane * step;
        const bool valid = pos < hi;
        const unsigned less = __ballot_sync(0xffffffffu, valid && keys[pos] < t);
        const unsigned probes = __ballot_sync(0xffffffffu, valid);
        const int c = __popc(less);
        if (c == 0) {
            hi = lo;
            break;
        }
        const uint32_t nlo = lo + (uint32_t)(c - 1) * step + 1;
        hi = c < __popc(probes) ? lo + (uint32_t)c * step : hi;
        lo = nlo;
    }
    const uint32_t pos = lo + (uint32_t)lane;
    const uint32_t first = lo + (uint32_t)__popc(__ballot_sync(0xffffffffu, pos < hi && keys[pos] < t));
    if (lane == 0) {
        ranges[t].x = (int)first;
        if (t > 0) ranges[t - 1].y = (int)first;
        if (t + 1 == n_tiles) ranges[t].y = (int)n;
    }
}

int bits_for(long long v)
{
    int b = 0;
    while ((1ll << b) < v) ++b;
    return b < 1 ? 1 : b;
}

void launch_bin_sort(const CamTable &ct, const WsLayout &L, int N, const float *proj_f, void *ws, cudaStream_t s)
{
    const float4 *proj = (const float4 *)proj_f;
    long long NE = L.NE;
    uint32_t *hdr = ws_ptr<uint32_t>(ws, L.header);
    int *err = (int *)hdr;
    uint32_t *n_inst = hdr + 1;
    uint32_t *dk[2] = {ws_ptr<uint32_t>(ws, L.depth_keys[0]), ws_ptr<uint32_t>(ws, L.depth_keys[1])};
    uint32_t *dv[2] = {ws_ptr<uint32_t>(ws, L.depth_vals[0]), ws_ptr<uint32_t>(ws, L.depth_vals[1])};
    uint32_t *ik[2] = {ws_ptr<uint32_t>(ws, L.inst_keys[0]), ws_ptr<uint32_t>(ws, L.inst_keys[1])};
    uint32_t *iv[2] = {ws_ptr<uint32_t>(ws, L.inst_vals[0]), ws_ptr<uint32_t>(ws, L.inst_vals[1])};
    uint32_t *hist = ws_ptr<uint32_t>(ws, L.sort_hist);
    uint32_t *aux = ws_ptr<uint32_t>(ws, L.scan_aux);
    uint32_t *counts = ws_ptr<uint32_t>(ws, L.counts);
    uint32_t *elem_cnt = ws_ptr<uint32_t>(ws, L.elem_cnt);
    uint32_t *elem_off = ws_ptr<uint32_t>(ws, L.elem_off);
    uint32_t *inst_elem = ws_ptr<uint32_t>(ws, L.inst_elem);
    int2 *ranges = ws_ptr<int2>(ws, L.tile_range);

    if (NE <= 0) {
        cudaMemsetAsync(ranges, 0, sizeof(int2) * (size_t)L.n_tiles, s);
        cudaMemsetAsync(n_inst, 0, sizeof(uint32_t), s);
        return;
    }
    unsigned nb = (unsigned)((NE + 255) / 256);
    k_depth_keys<<<nb, 256, 0, s>>>(NE, proj, dk[0], dv[0]);
    int dcur = radix_sort_pairs(dk[0], dk[1], dv[0], dv[1], NE, nullptr, 32, hist, s);
    k_count_tiles<<<nb, 256, 0, s>>>(ct, N, NE, proj, dv[dcur], counts, elem_cnt);
    exclusive_scan_u32(counts, counts, NE, n_inst, aux, s);
    k_duplicate<<<nb, 256, 0, s>>>(ct, N, NE, proj, dv[dcur], counts, (uint32_t)L.Mcap, ik[0], inst_elem,
                                  elem_off, elem_cnt, err);
    k_clear_walked<<<148 * 8, 256, 0, s>>>(n_inst, (uint32_t)L.Mcap, ws_ptr<uint8_t>(ws, L.inst_walked));
    int icur = radix_sort_pairs(ik[0], ik[1], iv[0], iv[1], L.Mcap, n_inst, bits_for(L.n_tiles), hist, s, true);
    (void)icur;   // equals L.inst_sorted
    k_tile_ranges<<<(unsigned)(((long long)L.n_tiles * 32 + 255) / 256), 256, 0, s>>>(
        ik[L.inst_sorted], n_inst, (uint32_t)L.Mcap, ranges, (uint32_t)L.n_tiles);
}

}  // namespace gs
