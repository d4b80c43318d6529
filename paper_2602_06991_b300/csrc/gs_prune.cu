// gs_prune.cu -- consistency-pruning statistics and survival selection (Sec. 3.3).
//
// Statistics of one rendered view, accumulated by the caller over the views of a
// pruning window:
//   count[g] += the number of pixels whose Top-K set (Eq. 2) holds g -- a warp-
//               aggregated integer histogram of topk_idx (integer sums: exact);
//   S[g]      = max(S[g], max over every pixel where g contributes of w_g), Eq. 8 --
//               a re-walk of the tile lists with the walk's own contributor rule,
//               the per-(tile, Gaussian) maximum reduced over the tile's pixels in
//               fixed order, then one integer atomicMax per instance on the float's
//               bit pattern (w >= 0, so the integer order is the float order and the
//               result is exact and order-independent).
// Selection (Eq. 9): the candidates G_prune are the Gaussians with count < tau; m =
// floor(ratio |G_prune| + 1/2) of them survive, drawn by weighted sampling without
// replacement with probability S_i / sum S -- an exponential race: candidate i
// finishes at e_i / S_i for caller-given e_i ~ Exp(1); the library's radix sort orders
// the finishing times (stable: equal times by id) and the m earliest survive.
#include "gs_internal.cuh"

#include <math.h>

namespace gs {

__global__ void __launch_bounds__(256) k_topk_count(long long PK, const int *__restrict__ topk_idx,
                                                    const int *__restrict__ err, int *__restrict__ count)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int id = -1;
    if (i < PK && *err == 0) id = topk_idx[i];
    // one atomic per distinct id of the warp
    const unsigned same = __match_any_sync(0xffffffffu, id);
    if (id >= 0 && (__ffs(same) - 1) == lane) atomicAdd(count + id, __popc(same));
}

// Re-walk with the forward walk's staging and contributor rule; per staged Gaussian the
// warps' maxima of w go to shared memory and the CTA's maximum to S (atomicMax on bits).
template <int TW, int TH>
__global__ void __launch_bounds__(TW *TH) k_walk_maxw(CamTable ct, int N, const float4 *__restrict__ proj,
                                                      TileLists tl, const uint32_t *__restrict__ inst_elem,
                                                      const int *__restrict__ err, unsigned *__restrict__ S_bits)
{
    constexpr int B = TW * TH;
    constexpr int NW = B / 32;
    __shared__ float4 s_r0[B], s_r1[B];
    __shared__ int s_g[B];
    __shared__ float s_max[NW][B];
    __shared__ int s_jend[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    const int c = cam_of_tile(ct, tile);
    const CamDev &cam = ct.c[c];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int px = tx * TW + (tid % TW), py = ty * TH + (tid / TW);
    bool done = !(px < cam.W && py < cam.H);
    const TileList lst(tl, tile, *err != 0);
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    float T = 1.f;
    const int cN = c * N;
    for (int b0 = 0; b0 < lst.n; b0 += B) {
        if (__syncthreads_count(!done) == 0) break;
        const int m = b0 + tid;
        if (m < lst.n) {
            const uint32_t e = inst_elem[lst.at(m)];
            const float4 *r = proj + 4 * (size_t)e;
            s_r0[tid] = r[0];
            s_r1[tid] = r[1];
            s_g[tid] = (int)e - cN;
        }
        __syncthreads();
        const int cnt = min(B, lst.n - b0);
        int j_end = cnt;
        for (int j = 0; j < cnt; ++j) {
            if (__all_sync(0xffffffffu, done)) {
                j_end = j;
                break;
            }
            float w = 0.f;
            if (!done) {
                float dx, dy;
                const float4 r1 = s_r1[j];
                const float q = eval_q(pxf, pyf, s_r0[j], r1, dx, dy);
                if (q <= kQMax) {
                    float G, ao;
                    const float alpha = eval_alpha(q, r1.w, G, ao);
                    if (alpha >= kAlphaMin) {
                        const float test_T = __fmul_rn(T, __fsub_rn(1.f, alpha));
                        if (test_T < kTStop) {
                            done = true;
                        } else {
                            w = __fmul_rn(alpha, T);
                            T = test_T;
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w = fmaxf(w, __shfl_xor_sync(0xffffffffu, w, o));
            if (lane == 0) s_max[warp][j] = w;
        }
        if (lane == 0) s_jend[warp] = j_end;
        __syncthreads();
        for (int j = tid; j < cnt; j += B) {
            float mx = 0.f;
#pragma unroll
            for (int w = 0; w < NW; ++w) mx = fmaxf(mx, j < s_jend[w] ? s_max[w][j] : 0.f);
            if (mx > 0.f) atomicMax(S_bits + s_g[j], __float_as_uint(mx));
        }
    }
}

template <int TW, int TH>
static void walk_maxw_k(const CamTable &ct, const WsLayout &L, int N, const float4 *proj, void *ws, unsigned *S,
                        cudaStream_t s)
{
    k_walk_maxw<TW, TH><<<ct.n_tiles, TW * TH, 0, s>>>(ct, N, proj, tile_lists(L, ws), ws_ptr<uint32_t>(ws, L.inst_elem),
                                                       ws_ptr<int>(ws, L.header), S);
}

bool launch_prune_stats(const CamTable &ct, const WsLayout &L, int N, const float *proj, const int *topk_idx,
                        void *ws, int *count, float *S, cudaStream_t s)
{
    const int *err = ws_ptr<int>(ws, L.header);
    if (L.PK > 0)
        k_topk_count<<<(unsigned)((L.PK + 255) / 256), 256, 0, s>>>(L.PK, topk_idx, err, count);
    if (N == 0) return true;
    const float4 *p4 = (const float4 *)proj;
    unsigned *Sb = (unsigned *)S;
    if (ct.tile_w == 16 && ct.tile_h == 16) walk_maxw_k<16, 16>(ct, L, N, p4, ws, Sb, s);
    else if (ct.tile_w == 32 && ct.tile_h == 8) walk_maxw_k<32, 8>(ct, L, N, p4, ws, Sb, s);
    else if (ct.tile_w == 16 && ct.tile_h == 8) walk_maxw_k<16, 8>(ct, L, N, p4, ws, Sb, s);
    else if (ct.tile_w == 8 && ct.tile_h == 8) walk_maxw_k<8, 8>(ct, L, N, p4, ws, Sb, s);
    else return false;
    return true;
}

// ------------------------------------------------------------------------------------
// Selection (Eq. 9)
// ------------------------------------------------------------------------------------
// Candidate finishing times as sortable keys: a non-negative float's bits order as the
// float; +inf (S = 0) after every finite time; non-candidates (0xffffffff) last.
__global__ void __launch_bounds__(256) k_prune_keys(int N, const int *__restrict__ count, const float *__restrict__ S,
                                                    int tau, const float *__restrict__ expo, uint32_t *keys,
                                                    uint32_t *vals, uint32_t *n_cand)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool cand = false;
    if (g < N) {
        cand = count[g] < tau;
        uint32_t key = 0xffffffffu;
        if (cand) {
            const float sg = S[g];
            key = sg > 0.f ? __float_as_uint(__fdiv_rn(expo[g], sg)) : 0x7f800000u;
        }
        keys[g] = key;
        vals[g] = (uint32_t)g;
    }
    const unsigned b = __ballot_sync(0xffffffffu, cand);
    if (lane == 0 && b) atomicAdd(n_cand, (uint32_t)__popc(b));
}

// keep: the m earliest candidates (sorted positions < m) and every non-candidate
// (positions >= |G_prune|), m = floor(ratio |G_prune| + 1/2).
__global__ void __launch_bounds__(256) k_prune_keep(int N, const uint32_t *__restrict__ vals,
                                                    const uint32_t *__restrict__ n_cand_dev, double ratio,
                                                    uint8_t *__restrict__ keep)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const uint32_t n_cand = *n_cand_dev;
    const long long m = (long long)floor(ratio * (double)n_cand + 0.5);
    keep[vals[r]] = ((long long)r < m || r >= (int)n_cand) ? 1 : 0;
}

size_t prune_select_ws(int N)
{
    auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t u = sizeof(uint32_t);
    return a(256) + 4 * a(u * (size_t)(N > 0 ? N : 1)) + a(u * 256 * (kRadixBlocks + 1));
}

bool launch_prune_select(int N, const int *count, const float *S, int tau, double ratio, const float *expo,
                         uint8_t *keep, void *ws, cudaStream_t s)
{
    if (N <= 0) return true;
    auto a = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t u = sizeof(uint32_t), vec = a(u * (size_t)N);
    uint32_t *hdr = (uint32_t *)ws;
    uint32_t *k0 = (uint32_t *)((char *)ws + a(256));
    uint32_t *k1 = (uint32_t *)((char *)k0 + vec);
    uint32_t *v0 = (uint32_t *)((char *)k1 + vec);
    uint32_t *v1 = (uint32_t *)((char *)v0 + vec);
    uint32_t *hist = (uint32_t *)((char *)v1 + vec);         // (kRadixBlocks + 1) x 256
    cudaMemsetAsync(hdr, 0, 256, s);
    const unsigned nb = (unsigned)((N + 255) / 256);
    k_prune_keys<<<nb, 256, 0, s>>>(N, count, S, tau, expo, k0, v0, hdr);
    const int cur = radix_sort_pairs(k0, k1, v0, v1, N, nullptr, 32, hist, s);
    k_prune_keep<<<nb, 256, 0, s>>>(N, cur ? v1 : v0, hdr, ratio, keep);
    return true;
}

}  // namespace gs
