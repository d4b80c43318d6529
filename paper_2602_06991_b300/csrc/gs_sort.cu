// gs_sort.cu -- the library's own device radix sort and exclusive scan.
//
// Radix sort: least-significant-digit, 8-bit digits, reduce-then-scan per pass:
//   upsweep   : each block counts the digits of its contiguous range of tiles;
//   scan      : one block turns the (digit-major, block-minor) counts into offsets;
//   downsweep : each block ranks its keys stably (warp ballots + per-warp counters),
//               reorders each tile by digit in shared memory and writes every digit's
//               run to consecutive final positions.
// No block waits on another, so nothing can spin.  Stability makes the multi-pass
// sort correct and keeps equal keys in input order (used to keep depth order within
// a tile, and to put each Gaussian's marker entry first in its segment).
#include "gs_internal.cuh"

namespace gs {

__device__ __forceinline__ long long sort_count(long long n_host, const uint32_t *n_dev)
{
    if (n_dev) {
        long long m = (long long)(*n_dev);
        return m < n_host ? m : n_host;
    }
    return n_host;
}

__device__ __forceinline__ void block_tiles(long long n, long long &t0, long long &t1)
{
    long long n_tiles = (n + kSortTile - 1) / kSortTile;
    long long tpb = (n_tiles + gridDim.x - 1) / gridDim.x;
    t0 = (long long)blockIdx.x * tpb;
    t1 = t0 + tpb;
    if (t1 > n_tiles) t1 = n_tiles;
}

__global__ void __launch_bounds__(kSortThreads) k_rs_upsweep(const uint32_t *__restrict__ keys, long long n_host,
                                                             const uint32_t *n_dev, int shift,
                                                             uint32_t *__restrict__ hist)
{
    if (n_dev && *n_dev == 0u) return;           // an empty device-counted sort: nothing to do
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t cnt[W][256];
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < W * 256; i += kSortThreads) (&cnt[0][0])[i] = 0;
    __syncthreads();
    long long n = sort_count(n_host, n_dev), t0, t1;
    block_tiles(n, t0, t1);
    long long e0 = t0 * kSortTile, e1 = t1 * kSortTile;
    if (e1 > n) e1 = n;
    for (long long i = e0 + tid; i < e1; i += kSortThreads) {
        uint32_t d = (__ldg(keys + i) >> shift) & 255u;
        atomicAdd(&cnt[warp][d], 1u);
    }
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) s += cnt[w][tid];
    hist[(size_t)blockIdx.x * 256 + tid] = s;          // block-major: coalesced
}

// Offsets of a pass, step 1: one CTA per digit d scans that digit's counts over the
// G blocks (hist[b][d] becomes the exclusive prefix over blocks 0..b-1; each thread
// takes a contiguous run of blocks) and writes the digit total to hist[G][d].  The
// downsweep adds the prefix of the digit totals.
__global__ void __launch_bounds__(512) k_rs_scan(uint32_t *hist, int G, const uint32_t *n_dev)
{
    if (n_dev && *n_dev == 0u) return;
    __shared__ uint32_t warp_sums[16];
    const int d = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (G + 511) / 512;
    const int b0 = min(t * per, G), b1 = min(b0 + per, G);
    uint32_t v = 0;
    for (int b = b0; b < b1; ++b) v += hist[(size_t)b * 256 + d];
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += warp_sums[w];
    uint32_t run = inc - v + before;
    for (int b = b0; b < b1; ++b) {
        const uint32_t x = hist[(size_t)b * 256 + d];
        hist[(size_t)b * 256 + d] = run;
        run += x;
    }
    if (t == 511) hist[(size_t)G * 256 + d] = run;   // the last run ends at block G
}

// Exclusive scan in place of len uint32 by one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_single(uint32_t *data, int len, uint32_t *total,
                                                      const uint32_t *run_if = nullptr)
{
    if (run_if && *run_if == 0u) return;
    __shared__ uint32_t warp_sums[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int per = (len + 1023) / 1024;
    int b = tid * per, e = min(b + per, len);
    uint32_t s = 0;
    for (int i = b; i < e; ++i) s += data[i];
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        warp_sums[lane] = v;          // inclusive
    }
    __syncthreads();
    uint32_t run = x - s + (warp > 0 ? warp_sums[warp - 1] : 0u);
    for (int i = b; i < e; ++i) {
        uint32_t v = data[i];
        data[i] = run;
        run += v;
    }
    if (total && tid == 1023) *total = run;
}

// Asynchronous 16-byte global -> shared copy (cp.async, L2 only) of the first `bytes`
// (0..16) of the chunk; the rest of the destination is zero-filled, and nothing past
// `bytes` is read.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Downsweep of a pass: per tile of kSortTile keys, stable ranks (the warp's lanes of equal
// digit found by nine ballots -- validity and the 8 digit bits -- and per-warp digit
// counters), then the tile is reordered by digit in shared memory and
// written out in that order, so each digit's run of the tile goes to consecutive
// addresses (coalesced) instead of one scattered store per key.  The next tile's keys
// and values are copied into shared memory (cp.async) while the current one is ranked
// and written, so the global load latency of a tile is hidden behind the previous
// tile's work; the current tile's buffer is then reused for its reordering.
// vin == nullptr: the values are the keys' input positions (0, 1, 2, ...), generated
// here instead of read.
__global__ void __launch_bounds__(kSortThreads) k_rs_downsweep(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                               uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                               long long n_host, const uint32_t *n_dev, int shift,
                                                               const uint32_t *__restrict__ hist)
{
    if (n_dev && *n_dev == 0u) return;
    constexpr int W = kSortThreads / 32;
    constexpr int kChunks = kSortTile / 4;           // 16-byte chunks per tile and array
    __shared__ uint32_t s_base[256];     // global position of this block's next key of each digit
    __shared__ uint32_t s_tot[W];
    __shared__ uint32_t s_start[256];    // first position of each digit in the reordered tile
    __shared__ uint32_t s_wsum[W];
    __shared__ uint32_t s_wcnt[W][257];
    __shared__ __align__(16) uint32_t s_k[2][kSortTile], s_v[2][kSortTile];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    {
        // digit base = exclusive prefix over digits of the digit totals
        uint32_t tot = hist[(size_t)gridDim.x * 256 + tid];
        uint32_t inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_tot[warp] = inc;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += s_tot[w];
        s_base[tid] = hist[(size_t)blockIdx.x * 256 + tid] + inc - tot + before;
        __syncthreads();
    }
    long long n = sort_count(n_host, n_dev), t0, t1;
    block_tiles(n, t0, t1);
    // the copies of tile t into buffer b: chunk c covers keys [4c, 4c + 4) of the tile
    auto issue = [&](long long t, int b) {
        const long long first = t * kSortTile;
        for (int c = tid; c < kChunks; c += kSortThreads) {
            const long long e = first + 4ll * c;
            const long long left = n - e;
            const int bytes = left >= 4 ? 16 : left > 0 ? (int)left * 4 : 0;
            const long long src = bytes > 0 ? e : 0;          // a valid address even when nothing is read
            cp_async16(&s_k[b][4 * c], kin + src, bytes);
            if (vin) cp_async16(&s_v[b][4 * c], vin + src, bytes);
        }
        cp_async_commit();
    };
    if (t0 < t1) issue(t0, 0);
    int buf = 0;
    for (long long t = t0; t < t1; ++t, buf ^= 1) {
        if (t + 1 < t1) {
            issue(t + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        for (int i = tid; i < W * 257; i += kSortThreads) (&s_wcnt[0][0])[i] = 0;
        __syncthreads();
        uint32_t k[kSortItems], v[kSortItems], lr[kSortItems];
        int dg[kSortItems];
        const int wloc = warp * 32 * kSortItems;
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            const int loc = wloc + i * 32 + lane;
            const bool valid = t * kSortTile + loc < n;
            k[i] = s_k[buf][loc];
            v[i] = vin ? s_v[buf][loc] : (uint32_t)(t * kSortTile + loc);
            dg[i] = valid ? (int)((k[i] >> shift) & 255u) : 256;
        }
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            // lanes holding the same digit: the validity and the 8 digit bits, one ballot each
            const bool valid = dg[i] < 256;
            const uint32_t vm = __ballot_sync(0xffffffffu, valid);
            uint32_t peers = valid ? vm : ~vm;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const bool bit = (dg[i] >> b) & 1;
                const uint32_t bm = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bm : ~bm;
            }
            int leader = __ffs(peers) - 1;
            uint32_t before = s_wcnt[warp][dg[i]];
            __syncwarp();
            if (lane == leader) s_wcnt[warp][dg[i]] = before + __popc(peers);
            __syncwarp();
            lr[i] = before + __popc(peers & lt_mask);
        }
        __syncthreads();
        uint32_t run = 0;
        {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint32_t c = s_wcnt[w][tid];
                s_wcnt[w][tid] = run;
                run += c;
            }
            // exclusive prefix of the tile's digit counts over the digits
            uint32_t inc = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) s_wsum[warp] = inc;
            __syncthreads();
            uint32_t before = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) before += w < warp ? s_wsum[w] : 0u;
            s_start[tid] = inc - run + before;
        }
        __syncthreads();
        // every thread has read its items of this buffer (barriers above): reorder in place
#pragma unroll
        for (int i = 0; i < kSortItems; ++i) {
            if (dg[i] < 256) {
                const uint32_t lp = s_start[dg[i]] + s_wcnt[warp][dg[i]] + lr[i];
                s_k[buf][lp] = k[i];
                s_v[buf][lp] = v[i];
            }
        }
        __syncthreads();
        const long long rem = n - t * kSortTile;
        const int cnt = rem < kSortTile ? (int)rem : kSortTile;
        for (int j = tid; j < cnt; j += kSortThreads) {
            const uint32_t kk = s_k[buf][j];
            const int d = (int)((kk >> shift) & 255u);
            const uint32_t pos = s_base[d] + (uint32_t)j - s_start[d];
            kout[pos] = kk;
            vout[pos] = s_v[buf][j];
        }
        __syncthreads();
        s_base[tid] += run;
    }
}

int radix_sort_pairs(uint32_t *keys0, uint32_t *keys1, uint32_t *vals0, uint32_t *vals1,
                     long long n_host, const uint32_t *n_dev, int n_bits, uint32_t *hist, cudaStream_t s,
                     bool vals_are_index)
{
    // the four arrays start 16-byte aligned (the downsweep copies 16-byte chunks)
    if (n_host <= 0 || n_bits <= 0) return 0;
    int passes = (n_bits + 7) / 8;
    long long n_tiles = (n_host + kSortTile - 1) / kSortTile;
    int G = (int)(n_tiles < kRadixBlocks ? n_tiles : kRadixBlocks);
    uint32_t *kb[2] = {keys0, keys1}, *vb[2] = {vals0, vals1};
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_rs_upsweep<<<G, kSortThreads, 0, s>>>(kb[cur], n_host, n_dev, shift, hist);
        k_rs_scan<<<256, 512, 0, s>>>(hist, G, n_dev);
        const uint32_t *vin = (p == 0 && vals_are_index) ? nullptr : vb[cur];
        k_rs_downsweep<<<G, kSortThreads, 0, s>>>(kb[cur], vin, kb[cur ^ 1], vb[cur ^ 1], n_host, n_dev, shift, hist);
        cur ^= 1;
    }
    return cur;
}

// ------------------------------------------------------------------------------------
// Exclusive scan of uint32 (reduce, scan block sums, downsweep), tiles of 4096.
// ------------------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *warp_sums, uint32_t &block_total)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        warp_sums[lane] = v;
    }
    __syncthreads();
    block_total = warp_sums[31];
    uint32_t r = inc - x + (warp > 0 ? warp_sums[warp - 1] : 0u);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in, long long n,
                                                              long long per_block, uint32_t *aux,
                                                              const uint32_t *run_if)
{
    if (run_if && *run_if == 0u) return;
    __shared__ uint32_t warp_sums[32];
    long long b0 = (long long)blockIdx.x * per_block, b1 = min(b0 + per_block, n);
    uint32_t s = 0;
    for (long long i = b0 + threadIdx.x; i < b1; i += kScanThreads) s += in[i];
    uint32_t tot;
    block_excl_scan(s, warp_sums, tot);
    if (threadIdx.x == 0) aux[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t *in, uint32_t *out, long long n,
                                                            long long per_block, const uint32_t *aux,
                                                            const uint32_t *run_if)
{
    if (run_if && *run_if == 0u) return;
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t tile[kScanTile];
    const int tid = threadIdx.x;
    long long b0 = (long long)blockIdx.x * per_block, b1 = min(b0 + per_block, n);
    uint32_t carry = aux[blockIdx.x];
    for (long long t = b0; t < b1; t += kScanTile) {
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            long long idx = t + i * kScanThreads + tid;
            tile[i * kScanThreads + tid] = idx < b1 ? in[idx] : 0u;
        }
        __syncthreads();
        uint32_t v[kScanItems], s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) { v[i] = tile[tid * kScanItems + i]; s += v[i]; }
        uint32_t tot;
        uint32_t run = block_excl_scan(s, warp_sums, tot) + carry;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) { tile[tid * kScanItems + i] = run; run += v[i]; }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            long long idx = t + i * kScanThreads + tid;
            if (idx < b1) out[idx] = tile[i * kScanThreads + tid];
        }
        carry += tot;
        __syncthreads();
    }
}

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, long long n, uint32_t *total, uint32_t *aux, cudaStream_t s,
                        const uint32_t *run_if)
{
    if (n <= 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
        return;
    }
    long long n_tiles = (n + kScanTile - 1) / kScanTile;
    int G = (int)(n_tiles < kSortBlocks ? n_tiles : kSortBlocks);
    long long tiles_per_block = (n_tiles + G - 1) / G;
    long long per_block = tiles_per_block * kScanTile;
    G = (int)((n + per_block - 1) / per_block);
    k_scan_reduce<<<G, kScanThreads, 0, s>>>(in, n, per_block, aux, run_if);
    k_scan_single<<<1, 1024, 0, s>>>(aux, G, total, run_if);
    k_scan_down<<<G, kScanThreads, 0, s>>>(in, out, n, per_block, aux, run_if);
}

}  // namespace gs
