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
    float u, v, s2m, invA, Aqb, s12, dymax, dys;
    int ok;
    RowCull() = default;
    __device__ __forceinline__ RowCull(const float4 r0, const float4 r1)
    {
        u = __fadd_rn(r0.x, r0.z);
        v = __fadd_rn(r0.y, r0.w);
        const float s1 = r1.x, m = r1.y, s2 = r1.z;
        // 2 ln(255 o) through the hardware log2 (one instruction, the same result in both
        // kernels; its error is far inside the 0.4% + 0.02 margin)
        const float q = fminf(kQMax, __fmul_rn(1.38629436f, __log2f(__fmul_rn(255.0f, r1.w))));
        const float qb = __fadd_rn(__fmul_rn(fmaxf(q, 0.0f), 1.004f), 0.02f);
        ok = (s1 > 0.f && s2 > 0.f && isfinite(m) && isfinite(s1) && isfinite(s2)) ? 1 : 0;
        const float s22 = __fmul_rn(s2, s2), s1s2 = __fmul_rn(s1, s2);
        s2m = __fmul_rn(s22, m);
        const float A = __fadd_rn(__fmul_rn(s1, s1), __fmul_rn(s2m, m));
        invA = __frcp_rn(A);
        Aqb = __fmul_rn(A, qb);
        s12 = __fmul_rn(s1s2, s1s2);
        dymax = ok ? __fdiv_rn(__fsqrt_rn(Aqb), s1s2) : 0.f;
        dys = ok ? __fdiv_rn(__fmul_rn(m, __fsqrt_rn(qb)), s1) : 0.f;
    }
    // lane j's record, in every lane
    __device__ __forceinline__ RowCull from_lane(int j) const
    {
        RowCull o;
        o.u = __shfl_sync(0xffffffffu, u, j);
        o.v = __shfl_sync(0xffffffffu, v, j);
        o.s2m = __shfl_sync(0xffffffffu, s2m, j);
        o.invA = __shfl_sync(0xffffffffu, invA, j);
        o.Aqb = __shfl_sync(0xffffffffu, Aqb, j);
        o.s12 = __shfl_sync(0xffffffffu, s12, j);
        o.dymax = __shfl_sync(0xffffffffu, dymax, j);
        o.dys = __shfl_sync(0xffffffffu, dys, j);
        o.ok = __shfl_sync(0xffffffffu, ok, j);
        return o;
    }
    // sqrt(A qb - (s1 s2 dy)^2) as x rsqrt(x): the hardware reciprocal square root (a few
    // ulp, far inside the margins, and the same instructions in both kernels)
    __device__ __forceinline__ float root(float dy) const
    {
        const float x = __fsub_rn(Aqb, __fmul_rn(s12, __fmul_rn(dy, dy)));
        return x > 0.f ? __fmul_rn(x, rsqrtf(x)) : 0.f;
    }
    // The run [a, b] of tile columns (within [tx0, tx1]) that the ellipse reaches in tile
    // row ty; false for none.  itw = 1 / tile width (exact: a power of two).
    __device__ __forceinline__ bool run(const CamDev &cam, int th, float itw, int ty, int tx0, int tx1, int &a,
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
        const float xmax = __fmul_rn(__fadd_rn(__fmul_rn(s2m, yr), root(yr)), invA);
        const float xmin = __fmul_rn(__fsub_rn(__fmul_rn(s2m, yl), root(yl)), invA);
        // columns tx with pixel centres [tx tw + 0.5, (tx + 1) tw - 0.5] meeting
        // [u + xmin, u + xmax], widened by 0.01 px
        const float X0 = __fsub_rn(__fadd_rn(u, xmin), 0.01f), X1 = __fadd_rn(__fadd_rn(u, xmax), 0.01f);
        const float af = __fsub_rn(ceilf(__fmul_rn(__fadd_rn(X0, 0.5f), itw)), 1.0f);
        const float bf = floorf(__fmul_rn(__fsub_rn(X1, 0.5f), itw));
        a = (int)fminf(fmaxf(af, (float)tx0), (float)(tx1 + 1));
        b = (int)fmaxf(fminf(bf, (float)tx1), (float)(tx0 - 1));
        return a <= b;
    }
};

// Instances of each element, in depth order: the tiles of its footprint box that its
// ellipse reaches (RowCull runs) -- n, the element's instance slots -- and n1, those in
// front of their tile's depth cut (key <= cut; all of them without cuts), by depth rank.
// An element behind the largest cut of every row of its box has no instance in front of
// any cut: it gets no slots here (n = 0, no run is computed), and slots only if the
// completion pass emits some of its instances.
__global__ void __launch_bounds__(256) k_count_tiles(CamTable ct, int N, long long NE, const float4 *__restrict__ proj,
                                                     const uint32_t *__restrict__ sorted_e,
                                                     const uint32_t *__restrict__ sorted_key,
                                                     const uint32_t *__restrict__ cut,
                                                     const uint32_t *__restrict__ rowmin,
                                                     const uint32_t *__restrict__ rowmax,
                                                     const uint32_t *__restrict__ rowmax_st, int use_cut,
                                                     uint32_t *counts, uint32_t *counts1, uint32_t *elem_cnt)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= NE) return;
    const uint32_t e = sorted_e[r];
    int c, tx0, tx1, ty0, ty1;
    const uint32_t box = tiles_of(ct, proj, e, N, c, tx0, tx1, ty0, ty1);
    uint32_t n = 0, n1 = 0;
    bool any = box > 0;
    const uint32_t key = sorted_key[r];
    if (any && use_cut) {
        // the largest cut over the box's rows: two lookups in the sparse table
        const int row0 = ct.c[c].row_off, len = ty1 - ty0 + 1;
        const int l = 31 - __clz(len);
        const uint32_t *st = rowmax_st + (size_t)l * ct.n_rows;
        any = key <= max(__ldg(st + row0 + ty0), __ldg(st + row0 + ty1 - (1 << l) + 1));
    }
    if (any) {
        const RowCull rc(proj[4 * (size_t)e], proj[4 * (size_t)e + 1]);
        const CamDev &cam = ct.c[c];
        const float itw = __frcp_rn((float)ct.tile_w);
        for (int ty = ty0; ty <= ty1; ++ty) {
            int a, b;
            if (!rc.run(cam, ct.tile_h, itw, ty, tx0, tx1, a, b)) continue;
            n += (uint32_t)(b - a + 1);
            if (use_cut) {
                const int row = cam.row_off + ty;
                if (key <= __ldg(rowmin + row)) {
                    n1 += (uint32_t)(b - a + 1);          // in front of every cut of the row
                } else if (key <= __ldg(rowmax + row)) {
                    const uint32_t *cr = cut + cam.tile_off + ty * cam.tiles_x;
                    for (int x = a; x <= b; ++x) n1 += key <= __ldg(cr + x) ? 1u : 0u;
                }
            }
        }
        if (!use_cut) n1 = n;
    }
    counts[r] = n;
    counts1[r] = n1;
    elem_cnt[e] = n;
}

// Second binning pass, after the first walk: per element, its instances in tiles that
// walk left unsaturated and behind their cut (key > cut).  Elements whose footprint box
// holds no such tile (a summed-area table of the flags) are skipped at once; with no
// unsaturated tile nothing is written, and the scan and emission after it skip as well.
__global__ void __launch_bounds__(256) k_count_tiles2(CamTable ct, int N, long long NE, const float4 *__restrict__ proj,
                                                      const uint32_t *__restrict__ sorted_e,
                                                      const uint32_t *__restrict__ sorted_key,
                                                      const uint32_t *__restrict__ cut,
                                                      const uint32_t *__restrict__ incomplete,
                                                      const uint32_t *__restrict__ sat, const uint32_t *hdr,
                                                      const uint32_t *__restrict__ elem_cnt, uint32_t *counts2,
                                                      uint32_t *fresh2)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= NE || hdr[kHdrIncomplete] == 0) return;   // (nothing flagged: counts and their scan are skipped)
    uint32_t n2 = 0;
    {
        const uint32_t e = sorted_e[r];
        int c, tx0, tx1, ty0, ty1;
        if (tiles_of(ct, proj, e, N, c, tx0, tx1, ty0, ty1) > 0) {
            const CamDev &cam = ct.c[c];
            const uint32_t *S = sat + cam.tile_off;
            const int W = cam.tiles_x;
            auto at = [&](int x, int y) { return (x < 0 || y < 0) ? 0u : __ldg(S + y * W + x); };
            const uint32_t inbox = at(tx1, ty1) - at(tx0 - 1, ty1) - at(tx1, ty0 - 1) + at(tx0 - 1, ty0 - 1);
            if (inbox > 0) {
                const RowCull rc(proj[4 * (size_t)e], proj[4 * (size_t)e + 1]);
                const uint32_t key = sorted_key[r];
                const float itw = __frcp_rn((float)ct.tile_w);
                for (int ty = ty0; ty <= ty1; ++ty) {
                    int a, b;
                    if (!rc.run(cam, ct.tile_h, itw, ty, tx0, tx1, a, b)) continue;
                    const int t0 = cam.tile_off + ty * W;
                    for (int x = a; x <= b; ++x)
                        n2 += (__ldg(incomplete + t0 + x) != 0u && key > __ldg(cut + t0 + x)) ? 1u : 0u;
                }
            }
        }
    }
    counts2[r] = n2;
    fresh2[r] = (n2 > 0 && elem_cnt[sorted_e[r]] == 0) ? n2 : 0u;
}

// Per camera, the inclusive 2D prefix sums of the unsaturated-tile flags over its tile
// grid (one block per camera: rows, then columns).
__global__ void __launch_bounds__(1024) k_incomplete_sat(CamTable ct, const uint32_t *__restrict__ incomplete,
                                                         const uint32_t *hdr, uint32_t *sat)
{
    if (hdr[kHdrIncomplete] == 0) return;
    const CamDev &cam = ct.c[blockIdx.x];
    const int W = cam.tiles_x, H = cam.tiles_y;
    const uint32_t *f = incomplete + cam.tile_off;
    uint32_t *S = sat + cam.tile_off;
    for (int y = threadIdx.x; y < H; y += blockDim.x) {
        uint32_t run = 0;
        for (int x = 0; x < W; ++x) {
            run += f[y * W + x] != 0u ? 1u : 0u;
            S[y * W + x] = run;
        }
    }
    __syncthreads();
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        uint32_t run = 0;
        for (int y = 0; y < H; ++y) {
            run += S[y * W + x];
            S[y * W + x] = run;
        }
    }
}

// Writes the instances of one binning pass: one warp per 32 consecutive depth ranks,
// element by element, one lane per tile row to find the row runs, then the element's
// instance slots walked flat by the warp.  Slot t of element e is instance o(e) + t (its
// position among all the element's instances, whichever pass sorts it); the pass keeps
// the slots whose tile passes its test -- PASS 1: in front of the tile's cut; PASS 2:
// behind it in a tile the first walk left unsaturated -- and writes them compacted
// (ballot prefix) from the element's offset among that pass's instances: key = tile,
// value = instance, and the instance's element.  (The re-walk's walked flags are cleared
// by k_clear_walked.)
template <int PASS>
__global__ void __launch_bounds__(256) k_duplicate(CamTable ct, int N, long long NE, const float4 *__restrict__ proj,
                                                   const uint32_t *__restrict__ sorted_e,
                                                   const uint32_t *__restrict__ sorted_key,
                                                   const uint32_t *__restrict__ cut,
                                                   const uint32_t *__restrict__ incomplete, int use_cut,
                                                   const uint32_t *__restrict__ offsets,
                                                   const uint32_t *__restrict__ pass_off, const uint32_t *hdr,
                                                   uint32_t mcap, uint32_t *keys_out, uint32_t *vals_out,
                                                   uint32_t *inst_elem, uint32_t *elem_off, uint32_t *elem_cnt,
                                                   uint8_t *walked, int *err)
{
    if (PASS == 2 && hdr[kHdrIncomplete] == 0) return;
    // PASS 2, an element the first pass gave no slots: its emitted instances take fresh
    // slots after the first pass's, in emission order (offsets: the scanned counts of those)
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const uint32_t pass_total = PASS == 1 ? hdr[kHdrN1] : hdr[kHdrN2];
    uint32_t e = 0, o = 0, n = 0, po = 0, pn = 0, key = 0;
    int fresh = 0;
    int c = 0, tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;
    RowCull own = {};                             // this lane's element's record
    if (r < NE) {
        e = sorted_e[r];
        key = sorted_key[r];
        if (PASS == 1) {
            o = offsets[r];
            elem_off[e] = o;
        } else {
            o = elem_off[e];
        }
        n = elem_cnt[e];                          // the instance slots counted by k_count_tiles
        po = pass_off[r];
        pn = (r + 1 < NE ? pass_off[r + 1] : pass_total) - po;
        if (PASS == 2 && n == 0 && pn > 0) {
            fresh = 1;
            o = hdr[1] + offsets[r];
            elem_off[e] = o;
            elem_cnt[e] = pn;
            if ((unsigned long long)o + pn > mcap) atomicOr(err, kErrOverflow);
        }
        if (pn > 0) {
            tiles_of(ct, proj, e, N, c, tx0, tx1, ty0, ty1);
            own = RowCull(proj[4 * (size_t)e], proj[4 * (size_t)e + 1]);
        }
        if (PASS == 1 && n > 0 && (unsigned long long)o + n > mcap) {
            // instances past the capacity are dropped; the render is reported as failed
            atomicOr(err, kErrOverflow);
            elem_cnt[e] = o < mcap ? mcap - o : 0u;
        }
    }
    const uint32_t lt_mask = (1u << lane) - 1u;
    const float itw = __frcp_rn((float)ct.tile_w);
    for (int j = 0; j < 32; ++j) {
        if (__shfl_sync(0xffffffffu, pn, j) == 0) continue;
        const uint32_t ej = __shfl_sync(0xffffffffu, e, j), oj = __shfl_sync(0xffffffffu, o, j);
        const uint32_t kj = __shfl_sync(0xffffffffu, key, j);
        uint32_t pbase = __shfl_sync(0xffffffffu, po, j);
        const uint32_t pstart = pbase;
        const bool fj = __shfl_sync(0xffffffffu, fresh, j) != 0;
        const int cj = __shfl_sync(0xffffffffu, c, j);
        const int x0 = __shfl_sync(0xffffffffu, tx0, j), x1 = __shfl_sync(0xffffffffu, tx1, j);
        const int y0 = __shfl_sync(0xffffffffu, ty0, j), y1 = __shfl_sync(0xffffffffu, ty1, j);
        const CamDev &cam = ct.c[cj];
        const RowCull rc = own.from_lane(j);
        uint32_t base = oj;
        for (int ry = y0; ry <= y1; ry += 32) {
            const int ty = ry + lane;
            int a = 0, b = -1;
            const bool any = ty <= y1 && rc.run(cam, ct.tile_h, itw, ty, x0, x1, a, b);
            const uint32_t cnt = any ? (uint32_t)(b - a + 1) : 0u;
            uint32_t incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
            const int tile_row0 = cam.tile_off + ry * cam.tiles_x;
            // slot t's row is the number of rows whose inclusive count is <= t
            for (uint32_t t0 = 0; t0 < tot; t0 += 32) {
                const uint32_t t = t0 + lane;
                int row = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1)
                    if (__shfl_sync(0xffffffffu, incl, row + step - 1) <= t) row += step;
                const uint32_t first = __shfl_sync(0xffffffffu, incl - cnt, row);
                const int ar = __shfl_sync(0xffffffffu, a, row);
                const uint32_t tile = (uint32_t)(tile_row0 + row * cam.tiles_x + ar + (int)(t - first));
                bool keep = t < tot;
                if (keep && use_cut) {
                    const uint32_t ck = __ldg(cut + tile);
                    keep = PASS == 1 ? kj <= ck : (__ldg(incomplete + tile) != 0u && kj > ck);
                }
                const uint32_t kept = __ballot_sync(0xffffffffu, keep);
                const uint32_t pos = pbase + __popc(kept & lt_mask);
                const uint32_t slot = fj ? oj + (pos - pstart) : base + t;
                if (keep && slot < mcap && pos < mcap) {
                    keys_out[pos] = tile;
                    vals_out[pos] = slot;
                    inst_elem[slot] = ej;
                    if (fj) walked[slot] = 0;         // (beyond the first pass's cleared slots)
                }
                pbase += __popc(kept);
            }
            base += tot;
        }
    }
}

// The cut keys this render bins with: the recorded ones when depth cuts are on and the
// workspace's record belongs to this tile grid, else none (and the record is reset).
// Clears the second sort's ranges.
// Also the smallest and largest cut key of each tile row (rowmin / rowmax, preset to
// all ones / zero): an element at or in front of a row's smallest cut is in front of the
// cut in every tile of that row, one behind its largest in none.
__global__ void __launch_bounds__(256) k_cut_prepare(CamTable ct, const uint32_t *hdr, uint32_t sig, int enabled,
                                                     uint32_t *cut_store, uint32_t *cut_cur, int2 *ranges2,
                                                     uint32_t *rowmin, uint32_t *rowmax)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = t < (uint32_t)ct.n_tiles;
    uint32_t cut = kNoCut;
    int row = -1;
    if (live) {
        const bool recorded = hdr[kHdrCutSig] == sig;
        if (!recorded) cut_store[t] = kNoCut;
        cut = (enabled && recorded) ? cut_store[t] : kNoCut;
        cut_cur[t] = cut;
        ranges2[t] = make_int2(0, 0);
        const int c = cam_of_tile(ct, (int)t);
        row = ct.c[c].row_off + ((int)t - ct.c[c].tile_off) / ct.c[c].tiles_x;
    }
    // one atomic per distinct row of the warp
    const unsigned same = __match_any_sync(0xffffffffu, row);
    const uint32_t mn = __reduce_min_sync(same, cut), mx = __reduce_max_sync(same, cut);
    if (live && (__ffs(same) - 1) == (int)(threadIdx.x & 31)) {
        atomicMin(rowmin + row, mn);
        atomicMax(rowmax + row, mx);
    }
}

// Range maxima of the row maxima, per camera: level l holds the largest over rows
// [i, i + 2^l) of the camera (clipped at its last row).  One block per camera.
__global__ void __launch_bounds__(256) k_cut_rowmax_table(CamTable ct, const uint32_t *__restrict__ rowmax,
                                                          uint32_t *st)
{
    const CamDev &cam = ct.c[blockIdx.x];
    const int r0 = cam.row_off, H = cam.tiles_y;
    for (int i = threadIdx.x; i < H; i += blockDim.x) st[r0 + i] = rowmax[r0 + i];
    for (int l = 1; l < kCutLevels; ++l) {
        __syncthreads();
        const uint32_t *prev = st + (size_t)(l - 1) * ct.n_rows;
        uint32_t *cur = st + (size_t)l * ct.n_rows;
        const int half = 1 << (l - 1);
        for (int i = threadIdx.x; i < H; i += blockDim.x)
            cur[r0 + i] = i + half < H ? max(prev[r0 + i], prev[r0 + i + half]) : prev[r0 + i];
    }
}

__global__ void k_store_u32(uint32_t *dst, uint32_t v) { *dst = v; }

// Copies the first min(*n_dev, mcap) (key, value) pairs.
__global__ void __launch_bounds__(256) k_copy_pairs(const uint32_t *n_dev, uint32_t mcap,
                                                    const uint32_t *__restrict__ ks, const uint32_t *__restrict__ vs,
                                                    uint32_t *__restrict__ kd, uint32_t *__restrict__ vd)
{
    const uint32_t n = min(*n_dev, mcap);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        kd[i] = ks[i];
        vd[i] = vs[i];
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

TileLists tile_lists(const WsLayout &L, void *ws)
{
    TileLists tl;
    tl.v1 = ws_ptr<uint32_t>(ws, L.inst_vals[L.inst_sorted]);
    tl.v2 = ws_ptr<uint32_t>(ws, L.inst_vals[1 - L.inst_sorted]);
    tl.r1 = ws_ptr<int2>(ws, L.tile_range);
    tl.r2 = ws_ptr<int2>(ws, L.tile_range2);
    return tl;
}

// The first binning pass.  Instances are counted and given their slots (o(e) + t) as
// without cuts; only those in front of their tile's cut are written and sorted.  Sorted
// pairs end in buffer L.inst_sorted.
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
    uint32_t *counts1 = ws_ptr<uint32_t>(ws, L.counts1);
    uint32_t *elem_cnt = ws_ptr<uint32_t>(ws, L.elem_cnt);
    uint32_t *elem_off = ws_ptr<uint32_t>(ws, L.elem_off);
    uint32_t *inst_elem = ws_ptr<uint32_t>(ws, L.inst_elem);
    uint32_t *cut_cur = ws_ptr<uint32_t>(ws, L.cut_cur);
    int2 *ranges = ws_ptr<int2>(ws, L.tile_range);

    cudaMemsetAsync(hdr + kHdrN1, 0, 3 * sizeof(uint32_t), s);     // N1, N2, incomplete tiles
    cudaMemsetAsync(hdr + kHdrFresh, 0, sizeof(uint32_t), s);       // fresh slots of the completion
    uint32_t *rowmin = ws_ptr<uint32_t>(ws, L.cut_rowmin), *rowmax = ws_ptr<uint32_t>(ws, L.cut_rowmax);
    cudaMemsetAsync(rowmin, 0xff, sizeof(uint32_t) * (size_t)ct.n_rows, s);
    cudaMemsetAsync(rowmax, 0, sizeof(uint32_t) * (size_t)ct.n_rows, s);
    k_cut_prepare<<<(unsigned)((L.n_tiles + 255) / 256), 256, 0, s>>>(
        ct, hdr, L.cut_sig, L.depth_cut ? 1 : 0, ws_ptr<uint32_t>(ws, L.cut_store), cut_cur,
        ws_ptr<int2>(ws, L.tile_range2), rowmin, rowmax);
    uint32_t *rowmax_st = ws_ptr<uint32_t>(ws, L.cut_rowmax_st);
    k_cut_rowmax_table<<<ct.n, 256, 0, s>>>(ct, rowmax, rowmax_st);
    k_store_u32<<<1, 1, 0, s>>>(hdr + kHdrCutSig, L.cut_sig);
    if (NE <= 0) {
        cudaMemsetAsync(ranges, 0, sizeof(int2) * (size_t)L.n_tiles, s);
        cudaMemsetAsync(n_inst, 0, sizeof(uint32_t), s);
        return;
    }
    unsigned nb = (unsigned)((NE + 255) / 256);
    k_depth_keys<<<nb, 256, 0, s>>>(NE, proj, dk[0], dv[0]);
    int dcur = radix_sort_pairs(dk[0], dk[1], dv[0], dv[1], NE, nullptr, 32, hist, s);
    const int use_cut = L.depth_cut ? 1 : 0;
    {
        TimerScope tm(GS_TIMER_BINNING, s);
        k_count_tiles<<<nb, 256, 0, s>>>(ct, N, NE, proj, dv[dcur], dk[dcur], cut_cur, rowmin, rowmax, rowmax_st,
                                         use_cut, counts, counts1, elem_cnt);
        exclusive_scan_u32(counts, counts, NE, n_inst, aux, s);
        exclusive_scan_u32(counts1, counts1, NE, hdr + kHdrN1, aux, s);
        k_duplicate<1><<<nb, 256, 0, s>>>(ct, N, NE, proj, dv[dcur], dk[dcur], cut_cur, nullptr, use_cut, counts,
                                          counts1, hdr, (uint32_t)L.Mcap, ik[0], iv[0], inst_elem, elem_off, elem_cnt,
                                          nullptr, err);
        k_clear_walked<<<148 * 8, 256, 0, s>>>(n_inst, (uint32_t)L.Mcap, ws_ptr<uint8_t>(ws, L.inst_walked));
    }
    {
        TimerScope tm(GS_TIMER_TILE_SORT, s);
        int icur = radix_sort_pairs(ik[0], ik[1], iv[0], iv[1], L.Mcap, hdr + kHdrN1, bits_for(L.n_tiles), hist, s);
        (void)icur;   // equals L.inst_sorted
    }
    k_tile_ranges<<<(unsigned)(((long long)L.n_tiles * 32 + 255) / 256), 256, 0, s>>>(
        ik[L.inst_sorted], hdr + kHdrN1, (uint32_t)L.Mcap, ranges, (uint32_t)L.n_tiles);
}

// The second binning pass, after the first walk has flagged the tiles it left
// unsaturated with a cut: their instances behind the cut, sorted by (tile, depth) into
// buffer 1 - L.inst_sorted (ping-ponging through the instance-partial array, which is
// unused until the backward), with their runs in tile_range2.  Device-side counts make
// every launch a no-op when no tile was flagged.
void launch_complete_lists(const CamTable &ct, const WsLayout &L, int N, const float *proj_f, void *ws,
                           cudaStream_t s)
{
    if (!L.depth_cut || L.NE <= 0) return;
    const float4 *proj = (const float4 *)proj_f;
    const long long NE = L.NE;
    uint32_t *hdr = ws_ptr<uint32_t>(ws, L.header);
    int *err = (int *)hdr;
    const int dcur = sorted_buffer(32);
    const uint32_t *dk = ws_ptr<uint32_t>(ws, L.depth_keys[dcur]);
    const uint32_t *dv = ws_ptr<uint32_t>(ws, L.depth_vals[dcur]);
    const int tb = 1 - L.inst_sorted;
    uint32_t *ik = ws_ptr<uint32_t>(ws, L.inst_keys[tb]);
    uint32_t *iv = ws_ptr<uint32_t>(ws, L.inst_vals[tb]);
    uint32_t *scratch = ws_ptr<uint32_t>(ws, L.inst_grad);            // 10 Mcap words, free until the backward
    uint32_t *counts2 = ws_ptr<uint32_t>(ws, L.counts1);
    uint32_t *sat = ws_ptr<uint32_t>(ws, L.tile_sat);
    const uint32_t *cut_cur = ws_ptr<uint32_t>(ws, L.cut_cur);
    const uint32_t *incomplete = ws_ptr<uint32_t>(ws, L.tile_incomplete);
    const unsigned nb = (unsigned)((NE + 255) / 256);
    k_incomplete_sat<<<ct.n, 1024, 0, s>>>(ct, incomplete, hdr, sat);
    uint32_t *fresh2 = ws_ptr<uint32_t>(ws, L.counts);                 // (the first pass's offsets are in elem_off)
    k_count_tiles2<<<nb, 256, 0, s>>>(ct, N, NE, proj, dv, dk, cut_cur, incomplete, sat, hdr,
                                      ws_ptr<uint32_t>(ws, L.elem_cnt), counts2, fresh2);
    // with no flagged tile the scan is skipped too: the second sort's count stays the zero
    // binning set
    exclusive_scan_u32(counts2, counts2, NE, hdr + kHdrN2, ws_ptr<uint32_t>(ws, L.scan_aux), s, hdr + kHdrIncomplete);
    exclusive_scan_u32(fresh2, fresh2, NE, hdr + kHdrFresh, ws_ptr<uint32_t>(ws, L.scan_aux), s, hdr + kHdrIncomplete);
    k_duplicate<2><<<nb, 256, 0, s>>>(ct, N, NE, proj, dv, dk, cut_cur, incomplete, 1, fresh2, counts2, hdr,
                                      (uint32_t)L.Mcap, ik, iv, ws_ptr<uint32_t>(ws, L.inst_elem),
                                      ws_ptr<uint32_t>(ws, L.elem_off), ws_ptr<uint32_t>(ws, L.elem_cnt),
                                      ws_ptr<uint8_t>(ws, L.inst_walked), err);
    uint32_t *scratch_v = scratch + ((L.Mcap + 3) & ~3ll);              // 16-byte aligned
    const int cur = radix_sort_pairs(ik, scratch, iv, scratch_v, L.Mcap, hdr + kHdrN2, bits_for(L.n_tiles),
                                     ws_ptr<uint32_t>(ws, L.sort_hist), s);
    if (cur == 1)
        k_copy_pairs<<<148 * 4, 256, 0, s>>>(hdr + kHdrN2, (uint32_t)L.Mcap, scratch, scratch_v, ik, iv);
    k_tile_ranges<<<(unsigned)(((long long)L.n_tiles * 32 + 255) / 256), 256, 0, s>>>(
        ik, hdr + kHdrN2, (uint32_t)L.Mcap, ws_ptr<int2>(ws, L.tile_range2), (uint32_t)L.n_tiles);
}

}  // namespace gs
