// gs_bin.cu -- a2: tile binning and (tile, depth) ordering.
//
// Order of work (chosen so the sort over the large instance set needs only the tile
// bits):
//   1. sort the (camera, Gaussian) elements by float32 depth (32-bit keys, N-sized);
//   2. count the tiles each element's footprint box overlaps, in depth order, and scan;
//   3. emit one instance per (element, tile), in depth order, keyed by global tile id;
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

__global__ void k_count_tiles(CamTable ct, int N, long long NE, const float4 *__restrict__ proj,
                              const uint32_t *__restrict__ sorted_e, uint32_t *counts, uint32_t *elem_cnt)
{
    long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= NE) return;
    uint32_t e = sorted_e[r];
    int c, a, b, d, f;
    uint32_t n = tiles_of(ct, proj, e, N, c, a, b, d, f);
    counts[r] = n;
    elem_cnt[e] = n;
}

// One warp per 32 consecutive depth ranks: each lane works out its element's tile
// rectangle, then the warp writes the instances element by element, lanes striding over
// the rectangle, so large footprints are written in parallel and coalesced.
// (An instance's sort value is its own index, which the tile sort generates; the
// re-walk's walked flags are cleared by k_clear_walked.)
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
        n = tiles_of(ct, proj, e, N, c, tx0, tx1, ty0, ty1);
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
        const int y0 = __shfl_sync(0xffffffffu, ty0, j);
        const int w = x1 - x0 + 1;
        const CamDev &cam = ct.c[cj];
        for (uint32_t t = lane; t < nj; t += 32) {
            uint32_t oo = oj + t;
            if (oo >= mcap) break;
            int ty = y0 + (int)(t / (uint32_t)w), tx = x0 + (int)(t % (uint32_t)w);
            inst_keys[oo] = (uint32_t)(cam.tile_off + ty * cam.tiles_x + tx);
            inst_elem[oo] = ej;
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
    k_duplicate<<<nb, 256, 0, s>>>(ct, N, NE, proj, dv[dcur], counts, (uint32_t)L.Mcap, ik[0], inst_elem, elem_off,
                                  elem_cnt, err);
    k_clear_walked<<<148 * 8, 256, 0, s>>>(n_inst, (uint32_t)L.Mcap, ws_ptr<uint8_t>(ws, L.inst_walked));
    int icur = radix_sort_pairs(ik[0], ik[1], iv[0], iv[1], L.Mcap, n_inst, bits_for(L.n_tiles), hist, s, true);
    (void)icur;   // equals L.inst_sorted
    k_tile_ranges<<<(unsigned)(((long long)L.n_tiles * 32 + 255) / 256), 256, 0, s>>>(
        ik[L.inst_sorted], n_inst, (uint32_t)L.Mcap, ranges, (uint32_t)L.n_tiles);
}

}  // namespace gs
