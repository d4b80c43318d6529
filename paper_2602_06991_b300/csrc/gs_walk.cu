// gs_walk.cu -- a3: front-to-back walk with per-pixel Top-K (forward) and the re-walk
// of the adjoint (geometry part of a5).
//
// Forward (Eqs. 1-2): one CTA per screen tile, one thread per pixel.  The tile's
// depth-ordered instance list is staged through shared memory in batches of one
// record per thread; each pixel evaluates alpha with the double-float offset and the
// Cholesky-form conic, accumulates colour and depth (Eq. 1) and keeps its Top-K
// (Eq. 2) by insertion, in registers or (gs_config.topk_layout = 1, fewer registers)
// in shared memory, with identical results.  A batch loop ends as soon as every pixel
// of the tile has stopped.
//
// Backward: the same walk is recomputed (not stored) with the very same inlined
// evaluation, so contributor sets and transmittances match the forward bit for bit.
// Its CTAs are persistent (tiles come from a counter) and each warp skips the staged
// Gaussians whose ellipse misses its pixel rectangle, as the forward walk does.
// For contributor i with upstream dL/dC, dL/dD and the feature term,
//   dL/dw_i = dL/dC . c_i + dL/dD z_i + [i in K] (h_i - H) / S,
//   dL/dalpha_i = dL/dw_i T_i - (sum_{m>i} dL/dw_m w_m) / (1 - alpha_i),
// where h_i = dL/dF . f_i (written by the fused blend + loss, or by k_h_group), H = sum_k w'_k h_k,
// and the suffix sum is total - prefix with total = dL/dC . C + dL/dD . D (the
// feature terms sum to zero over the Top-K set).  Per-Gaussian partials are reduced
// across the tile's pixels (warp reduce-scatter, then a fixed-order sum over warps)
// and written once per walked (Gaussian, tile) instance, which is flagged; instances
// past the point where every pixel of the tile stopped are never written (their flags,
// cleared at binning, stay 0).  No atomics, deterministic.
#include "gs_internal.cuh"

#include <algorithm>
#include <type_traits>

namespace gs {

// KB: the Top-K buffer in registers (0), in shared memory with per-thread insertion (1),
// or in shared memory with warp-level insertion (2); identical results.
// wc.phase 1: every tile over its first list; records the tile's depth cut for the next
// render and flags the tiles it leaves unsaturated behind a cut.  Phase 2: the flagged
// tiles again, over their whole (completed) list.
template <int TW, int TH, int KM, int KB>
__global__ void __launch_bounds__(TW *TH) k_walk_fwd(CamTable ct, int K, int N, const float4 *__restrict__ proj,
                                                     TileLists tl, const uint32_t *__restrict__ inst_elem,
                                                     WalkCut wc, const int *__restrict__ err,
                                                     float *__restrict__ rgb_out, float *__restrict__ depth_out,
                                                     float *__restrict__ T_out, int *__restrict__ n_out,
                                                     int *__restrict__ idx_out, float *__restrict__ w_out)
{
    constexpr int B = TW * TH;
    __shared__ float4 s_r0[B], s_r1[B], s_r2[B];
    __shared__ int s_g[B];
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    if (wc.phase == 2 && (wc.hdr[kHdrIncomplete] == 0u || wc.incomplete[tile] == 0u)) return;   // whole CTA
    const int c = cam_of_tile(ct, tile);
    const CamDev &cam = ct.c[c];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int px = tx * TW + (tid % TW), py = ty * TH + (tid / TW);
    const bool inside = px < cam.W && py < cam.H;
    // pixel-centre rectangle of this warp: all TW columns, its 32 / TW rows
    const int lane = tid & 31;
    const float wx0 = (float)(tx * TW) + 0.5f, wx1 = (float)(tx * TW + TW) - 0.5f;
    const float wy0 = (float)(ty * TH + (tid - lane) / TW) + 0.5f;
    const float wy1 = wy0 + (float)(32 / TW - 1);
    const TileList lst(tl, tile, *err != 0);
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, Dd = 0.f;
    int nc = 0;
    constexpr int KMS = KB ? KM : 1;
    __shared__ float s_kw[KMS * B];
    __shared__ int s_kid[KMS * B];
    using Buf = typename std::conditional<KB == 0, TopK<KM>, TopKShared<KM, B>>::type;
    Buf tk;
    if constexpr (KB == 0) tk.init(K);
    else tk.init(s_kw, s_kid, tid, K);
    bool done = !inside;
    const int cN = c * N;
    int last_b0 = 0;
    for (int b0 = 0; b0 < lst.n; b0 += B) {
        if (__syncthreads_count(done) == B) break;
        last_b0 = b0;
        int m = b0 + tid;
        if (m < lst.n) {
            uint32_t e = inst_elem[lst.at(m)];
            const float4 *r = proj + 4 * (size_t)e;
            s_r0[tid] = r[0];
            s_r1[tid] = r[1];
            s_r2[tid] = r[2];
            s_g[tid] = (int)e - cN;
        }
        __syncthreads();
        const int cnt = min(B, lst.n - b0);
        for (int jc = 0; jc < cnt && __any_sync(0xffffffffu, !done); jc += 32) {
            // Gaussians of this chunk that can reach a pixel of this warp's rows
            const int jl = jc + lane;
            unsigned live = __ballot_sync(0xffffffffu, jl < cnt && touches_rect(s_r0[jl], s_r1[jl], wx0, wx1, wy0, wy1));
            if constexpr (KB == 2) {
                // warp-level insertion: the lanes step through the staged Gaussians together,
                // and each pixel that takes one into its Top-K is inserted by the warp, lane
                // k < KM holding slot k of that pixel (a ballot finds the position, a
                // shuffle shifts the slots behind it)
                while (live) {
                    if (__all_sync(0xffffffffu, done)) break;
                    const int j = jc + __ffs(live) - 1;
                    live &= live - 1;
                    float w = 0.f;
                    bool take = false;
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
                                    const float4 r2 = s_r2[j];
                                    C0 = fmaf(w, r2.x, C0);
                                    C1 = fmaf(w, r2.y, C1);
                                    C2 = fmaf(w, r2.z, C2);
                                    Dd = fmaf(w, r2.w, Dd);
                                    T = test_T;
                                    ++nc;
                                    take = w > tk.wmin;
                                }
                            }
                        }
                    }
                    unsigned ins = __ballot_sync(0xffffffffu, take);
                    const int gid = s_g[j];
                    while (ins) {
                        const int ql = __ffs(ins) - 1;
                        ins &= ins - 1;
                        const float nw = __shfl_sync(0xffffffffu, w, ql);
                        const int col = tid - lane + ql;
                        float sw = -1.0f;
                        int sid = -1;
                        if (lane < KM) {
                            sw = s_kw[lane * B + col];
                            sid = s_kid[lane * B + col];
                        }
                        // slots that stay ahead: weight >= the new one (sorted descending)
                        const int pos = __popc(__ballot_sync(0xffffffffu, lane < KM && !(nw > sw)));
                        const float upw = __shfl_up_sync(0xffffffffu, sw, 1);
                        const int upi = __shfl_up_sync(0xffffffffu, sid, 1);
                        float nv = sw;
                        if (lane < KM && lane >= pos) {
                            nv = lane == pos ? nw : upw;
                            s_kw[lane * B + col] = nv;
                            s_kid[lane * B + col] = lane == pos ? gid : upi;
                        }
                        const float nmin = __shfl_sync(0xffffffffu, nv, KM - 1);
                        if (lane == ql) tk.wmin = nmin;
                    }
                }
            } else {
            while (live && !done) {
            const int j = jc + __ffs(live) - 1;
            live &= live - 1;
            float dx, dy;
            const float4 r1 = s_r1[j];
            float q = eval_q(pxf, pyf, s_r0[j], r1, dx, dy);
            if (q > kQMax) continue;
            float G, ao;
            float alpha = eval_alpha(q, r1.w, G, ao);
            if (alpha < kAlphaMin) continue;
            float test_T = __fmul_rn(T, __fsub_rn(1.f, alpha));
            if (test_T < kTStop) {
                done = true;
                break;
            }
            float w = __fmul_rn(alpha, T);
            const float4 r2 = s_r2[j];
            C0 = fmaf(w, r2.x, C0);
            C1 = fmaf(w, r2.y, C1);
            C2 = fmaf(w, r2.z, C2);
            Dd = fmaf(w, r2.w, Dd);
            T = test_T;
            ++nc;
            tk.insert(w, s_g[j]);
            }
            }
        }
    }
    // the depth cut for the next render: where the tile saturated (the last staged
    // Gaussian's depth, with the margin), or none; in phase 1 an unsaturated tile whose
    // list was cut is flagged for completion
    const bool saturated = __syncthreads_count(done) == B;
    if (tid == 0 && *err == 0) {
        uint32_t rec = kNoCut;
        if (saturated && lst.n > 0) rec = __float_as_uint(s_r2[min(B, lst.n - last_b0) - 1].w * kCutMargin);
        wc.cut_store[tile] = rec;
        if (wc.phase == 1) {
            const bool inc = !saturated && wc.cut_cur[tile] != kNoCut;
            wc.incomplete[tile] = inc ? 1u : 0u;
            if (inc) atomicAdd(wc.hdr + kHdrIncomplete, 1u);
        }
    }
    if constexpr (KB == 2) __syncwarp();          // the slots other lanes wrote
    if (!inside) return;
    const long long p = cam.pix_off + (long long)py * cam.W + px;
    rgb_out[3 * p] = C0;
    rgb_out[3 * p + 1] = C1;
    rgb_out[3 * p + 2] = C2;
    depth_out[p] = Dd;
    T_out[p] = T;
    n_out[p] = nc;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        if (k >= KM - K) {
            int slot = k - (KM - K);
            float wk;
            int ik;
            if constexpr (KB == 0) {
                wk = tk.w[k];
                ik = tk.id[k];
            } else {
                wk = tk.w[k * B];
                ik = tk.id[k * B];
            }
            idx_out[p * K + slot] = ik;
            w_out[p * K + slot] = wk > 0.f ? wk : 0.f;
        }
    }
}

// PPT vertically adjacent pixels per thread: a thread sums its pixels' contributions to
// a staged Gaussian in registers, so each warp-level reduction covers 32 PPT pixels.
constexpr int kBwdPPT = 2;                       // 4 was measured slower (more registers, fewer warps)
// pixels per thread of a TW x TH tile: kBwdPPT while that leaves at least one warp
__host__ __device__ constexpr int bwd_ppt(int tw, int th) { return tw * th / kBwdPPT >= 32 ? kBwdPPT : tw * th / 32; }

template <int TW, int TH, int KM>
__global__ void __launch_bounds__(TW *TH / bwd_ppt(TW, TH)) k_walk_bwd(CamTable ct, int K, int N, const float4 *__restrict__ proj,
                                                              TileLists tl,
                                                              const uint32_t *__restrict__ inst_elem,
                                                              const int *__restrict__ err,
                                                              const float *__restrict__ rgb_out,
                                                              const float *__restrict__ depth_out,
                                                              const int *__restrict__ topk_idx,
                                                              const float *__restrict__ topk_w,
                                                              const float *__restrict__ hbuf,
                                                              const float *__restrict__ dLdC,
                                                              const float *__restrict__ dLdD,
                                                              float *__restrict__ inst_grad,
                                                              uint8_t *__restrict__ inst_walked,
                                                              unsigned *__restrict__ tile_counter)
{
    constexpr int PPT = bwd_ppt(TW, TH);
    constexpr int NT = TW * TH / PPT;
    constexpr int NW = NT / 32;
    constexpr int BB = 64;                       // Gaussians per staged batch
    __shared__ float4 s_r0[BB], s_r1[BB], s_r2[BB], s_r3[BB];
    __shared__ int s_g[BB];
    __shared__ uint32_t s_o[BB];
    __shared__ float s_red[NW][BB][kGradVals];
    __shared__ unsigned long long s_wrote[NW];   // per warp: the staged Gaussians it reduced
    __shared__ int s_tile;
    // the tile's Top-K ids as a set (open addressing), and per staged Gaussian whether it
    // is in it: a Gaussian in no pixel's Top-K of the tile has no feature term anywhere
    // in it, so its pixels skip the slot match
    constexpr int kHset = 1024;
    __shared__ int s_hset[kHset];
    __shared__ unsigned char s_inu[BB];
    __shared__ int s_hfull;
    auto hslot = [](int id) { return (int)(((uint32_t)id * 2654435761u) >> 22); };
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // persistent: each CTA takes the next unprocessed tile until none is left
    for (;;) {
        if (tid == 0) s_tile = (int)atomicAdd(tile_counter, 1u);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= ct.n_tiles) break;               // block-uniform
        const int c = cam_of_tile(ct, tile);
        const CamDev &cam = ct.c[c];
        const int lt = tile - cam.tile_off;
        const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
        const TileList lst(tl, tile, *err != 0);
        const int px = tx * TW + (tid % TW);
        const float pxf = (float)px + 0.5f;
        // pixel-centre rectangle of this warp: all TW columns, its thread rows x PPT rows
        const float wx0 = (float)(tx * TW) + 0.5f, wx1 = (float)(tx * TW + TW) - 0.5f;
        const float wy0 = (float)(ty * TH + ((tid - lane) / TW) * PPT) + 0.5f;
        const float wy1 = (float)(ty * TH + ((tid - lane + 31) / TW) * PPT + PPT - 1) + 0.5f;

        float pyf[PPT], dC0[PPT], dC1[PPT], dC2[PPT], dD[PPT], total[PPT], T[PPT], prefix[PPT];
        int kid[PPT][KM];
        float kfp[PPT][KM];
        bool pdone[PPT];
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
            const int py = ty * TH + (tid / TW) * PPT + r;
            pyf[r] = (float)py + 0.5f;
            const bool inside = px < cam.W && py < cam.H;
            pdone[r] = !inside;
            T[r] = 1.f;
            prefix[r] = 0.f;
            dC0[r] = dC1[r] = dC2[r] = dD[r] = total[r] = 0.f;
#pragma unroll
            for (int k = 0; k < KM; ++k) { kid[r][k] = -2; kfp[r][k] = 0.f; }
            if (inside) {
                const long long p = cam.pix_off + (long long)py * cam.W + px;
                dC0[r] = dLdC[3 * p]; dC1[r] = dLdC[3 * p + 1]; dC2[r] = dLdC[3 * p + 2];
                dD[r] = dLdD[p];
                total[r] = dC0[r] * rgb_out[3 * p] + dC1[r] * rgb_out[3 * p + 1] + dC2[r] * rgb_out[3 * p + 2] +
                           dD[r] * depth_out[p];
                float S = 0.f;
#pragma unroll
                for (int k = 0; k < KM; ++k)
                    if (k < K) S += topk_w[p * K + k];
                const float inv = S > 0.f ? 1.f / S : 0.f;
                float H = 0.f;
#pragma unroll
                for (int k = 0; k < KM; ++k) {
                    if (k < K) {
                        const int id = topk_idx[p * K + k];
                        if (id >= 0) {
                            kid[r][k] = id;
                            kfp[r][k] = hbuf ? hbuf[p * K + k] : 0.f;    // no feature loss: no term
                            H += topk_w[p * K + k] * inv * kfp[r][k];
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < KM; ++k) kfp[r][k] = (kfp[r][k] - H) * inv;
            }
        }
        for (int i = tid; i < kHset; i += NT) s_hset[i] = -1;
        if (tid == 0) s_hfull = 0;
        __syncthreads();
        // (the ids are read again from topk_idx, so the loop stays rolled and the
        // registers holding kid are not touched)
#pragma unroll 1
        for (int q = 0; q < PPT * K; ++q) {
            const int r = q / K, k = q - r * K;
            const int py = ty * TH + (tid / TW) * PPT + r;
            if (px >= cam.W || py >= cam.H) continue;
            const int id = topk_idx[(cam.pix_off + (long long)py * cam.W + px) * K + k];
            if (id < 0) continue;
            {
                int h = hslot(id);
                for (int n = 0;; ++n) {
                    const int old = atomicCAS(&s_hset[h], -1, id);
                    if (old == -1 || old == id) break;
                    h = (h + 1) & (kHset - 1);
                    if (n == 63) {                      // crowded: every Gaussian counts as a member
                        s_hfull = 1;
                        break;
                    }
                }
            }
        }
        __syncthreads();
        auto all_done = [&]() {
            bool d = true;
#pragma unroll
            for (int r = 0; r < PPT; ++r) d = d && pdone[r];
            return d;
        };
        const int cN = c * N;
        for (int b0 = 0; b0 < lst.n; b0 += BB) {
            // every pixel stopped: the remaining instances of this tile contribute nothing
            // (their walked flags stay 0, so the per-element sums skip them)
            if (__syncthreads_count(!all_done()) == 0) break;
            for (int t = tid; t < BB; t += NT) {
                if (b0 + t < lst.n) {
                    const uint32_t o = lst.at(b0 + t);
                    const uint32_t e = inst_elem[o];
                    const float4 *rr = proj + 4 * (size_t)e;
                    s_r0[t] = rr[0];
                    s_r1[t] = rr[1];
                    s_r2[t] = rr[2];
                    s_r3[t] = rr[3];
                    const int g = (int)e - cN;
                    s_g[t] = g;
                    s_o[t] = o;
                    bool inu = s_hfull != 0;
                    if (!inu) {
                        int h = hslot(g);
                        for (int n = 0; n < 64; ++n) {
                            const int v = s_hset[h];
                            if (v == g || n == 63) {
                                inu = true;
                                break;
                            }
                            if (v == -1) break;
                            h = (h + 1) & (kHset - 1);
                        }
                    }
                    s_inu[t] = inu ? 1 : 0;
                }
            }
            __syncthreads();
            const int cnt = min(BB, lst.n - b0);
            // only the staged Gaussians that can reach a pixel of this warp's rectangle (the
            // exact ellipse-rectangle test of the forward walk), in list order; a warp whose
            // pixels have all stopped leaves the batch.  The per-tile sum below counts the
            // entries a warp reduced (its mask), all others are zero for it.
            static_assert(BB == 64, "two 32-bit ballots per batch");
            const unsigned m0 = __ballot_sync(0xffffffffu, lane < cnt && touches_rect(s_r0[lane], s_r1[lane], wx0, wx1, wy0, wy1));
            const unsigned m1 = __ballot_sync(0xffffffffu, lane + 32 < cnt &&
                                                               touches_rect(s_r0[lane + 32], s_r1[lane + 32], wx0, wx1, wy0, wy1));
            unsigned long long live = ((unsigned long long)m1 << 32) | m0;
            unsigned long long wrote = 0ull;
            while (live) {
                if (__all_sync(0xffffffffu, all_done())) break;
                const int j = __ffsll((long long)live) - 1;
                live &= live - 1;
                float v[kGradVals];
#pragma unroll
                for (int i = 0; i < kGradVals; ++i) v[i] = 0.f;
                bool contrib = false;
                const float4 r0 = s_r0[j], r1 = s_r1[j];
#pragma unroll
                for (int r = 0; r < PPT; ++r) {
                    if (pdone[r]) continue;
                    float dx, dy;
                    const float q = eval_q(pxf, pyf[r], r0, r1, dx, dy);
                    if (q > kQMax) continue;
                    float G, ao;
                    const float alpha = eval_alpha(q, r1.w, G, ao);
                    if (alpha < kAlphaMin) continue;
                    const float test_T = __fmul_rn(T[r], __fsub_rn(1.f, alpha));
                    if (test_T < kTStop) {
                        pdone[r] = true;
                        continue;
                    }
                    contrib = true;
                    const float w = __fmul_rn(alpha, T[r]);
                    const float4 r2 = s_r2[j];
                    const int gid = s_g[j];
                    float fp = 0.f;
                    if (s_inu[j]) {                     // the same for the whole CTA
#pragma unroll
                        for (int k = 0; k < KM; ++k) fp = (kid[r][k] == gid) ? kfp[r][k] : fp;
                    }
                    const float gi = dC0[r] * r2.x + dC1[r] * r2.y + dC2[r] * r2.z + dD[r] * r2.w + fp;
                    prefix[r] = fmaf(gi, w, prefix[r]);
                    const float suffix = total[r] - prefix[r];
                    const float dalpha = gi * T[r] - __fdividef(suffix, 1.f - alpha);
                    v[6] += w * dC0[r]; v[7] += w * dC1[r]; v[8] += w * dC2[r]; v[9] += w * dD[r];
                    if (ao < kAlphaClamp) {
                        const float4 r3 = s_r3[j];
                        v[5] += dalpha * G;
                        const float dq = -0.5f * alpha * dalpha;
                        v[2] += dq * dx * dx;
                        v[3] += dq * 2.f * dx * dy;
                        v[4] += dq * dy * dy;
                        v[0] += -2.f * dq * (r3.x * dx + r3.y * dy);
                        v[1] += -2.f * dq * (r3.y * dx + r3.z * dy);
                    }
                    T[r] = test_T;
                }
                if (__any_sync(0xffffffffu, contrib)) {
                    const float d = warp_reduce10(v, lane);
                    const int vi = vidx10(lane);
                    if (!(lane & 1) && vi >= 0) s_red[warp][j][vi] = d;
                    wrote |= 1ull << j;
                }
            }
            if (lane == 0) s_wrote[warp] = wrote;
            __syncthreads();
            for (int i = tid; i < cnt * kGradVals; i += NT) {
                const int j = i / kGradVals, vi = i - j * kGradVals;
                float sum = 0.f;
#pragma unroll
                for (int w = 0; w < NW; ++w) sum += ((s_wrote[w] >> j) & 1ull) ? s_red[w][j][vi] : 0.f;
                inst_grad[(size_t)kGradVals * s_o[j] + vi] = sum;
                if (vi == 0) inst_walked[s_o[j]] = 1;
            }
        }
        __syncthreads();                         // shared state is free for the next tile
    }
}

template <int TW, int TH>
static bool walk_fwd_k(int KM, int kbuf, dim3 grid, cudaStream_t s, const CamTable &ct, int K, int N,
                       const float4 *proj, const TileLists &tl, const uint32_t *ie, const WalkCut &wc, const int *err,
                       float *a, float *b, float *cc, int *d, int *e, float *f)
{
    constexpr int B = TW * TH;
#define GS_WF(KMV, KBV) k_walk_fwd<TW, TH, KMV, KBV><<<grid, B, 0, s>>>(ct, K, N, proj, tl, ie, wc, err, a, b, cc, d, e, f)
    if (kbuf == 1) {
        switch (KM) {
        case 4: GS_WF(4, 1); return true;
        case 8: GS_WF(8, 1); return true;
        case 16: GS_WF(16, 1); return true;
        }
        return false;                        // (KM = 32 has no shared form: the buffer would not fit)
    }
    if (kbuf == 2) {
        switch (KM) {
        case 4: GS_WF(4, 2); return true;
        case 8: GS_WF(8, 2); return true;
        case 16: GS_WF(16, 2); return true;
        }
        return false;
    }

    switch (KM) {
    case 4: GS_WF(4, 0); return true;
    case 8: GS_WF(8, 0); return true;
    case 16: GS_WF(16, 0); return true;
    case 32: GS_WF(32, 0); return true;
    }
#undef GS_WF
    return false;
}

template <int TW, int TH>
static bool walk_bwd_k(int KM, dim3 grid, cudaStream_t s, const CamTable &ct, int K, int N, const float4 *proj,
                       const TileLists &tl, const uint32_t *ie, const int *err, const float *C,
                       const float *Dp, const int *ti, const float *tw, const float *h, const float *dC,
                       const float *dD, float *ig, uint8_t *wk, unsigned *ctr)
{
    constexpr int B = TW * TH / bwd_ppt(TW, TH);
    auto go = [&](auto kern) {
        // persistent grid: the resident CTAs per SM times the SMs (a tile counter hands
        // out the tiles, so uneven tiles balance across CTAs)
        int dev = 0, sms = 148, occ = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, B, 0);
        const long long want = (long long)sms * std::max(1, occ);
        const unsigned g = (unsigned)std::min<long long>(want, grid.x);
        cudaMemsetAsync(ctr, 0, sizeof(unsigned), s);
        kern<<<g, B, 0, s>>>(ct, K, N, proj, tl, ie, err, C, Dp, ti, tw, h, dC, dD, ig, wk, ctr);
    };
    switch (KM) {
    case 4: go(k_walk_bwd<TW, TH, 4>); return true;
    case 8: go(k_walk_bwd<TW, TH, 8>); return true;
    case 16: go(k_walk_bwd<TW, TH, 16>); return true;
    case 32: go(k_walk_bwd<TW, TH, 32>); return true;
    }
    return false;
}

static int k_bucket(int K) { return K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16 : 32; }

bool launch_walk_fwd(const CamTable &ct, const WsLayout &L, int K, int kbuf, int N, const float *proj_f, void *ws,
                     float *rgb_out, float *depth_out, float *T_out, int *n_out, int *idx_out, float *w_out,
                     int phase, cudaStream_t s)
{
    TimerScope tm(phase == 1 ? GS_TIMER_WALK_FWD : -1, s);
    const float4 *proj = (const float4 *)proj_f;
    const int *err = ws_ptr<int>(ws, L.header);
    const TileLists tl = tile_lists(L, ws);
    const uint32_t *ie = ws_ptr<uint32_t>(ws, L.inst_elem);
    WalkCut wc;
    wc.phase = phase;
    wc.cut_cur = ws_ptr<uint32_t>(ws, L.cut_cur);
    wc.cut_store = ws_ptr<uint32_t>(ws, L.cut_store);
    wc.incomplete = ws_ptr<uint32_t>(ws, L.tile_incomplete);
    wc.hdr = ws_ptr<uint32_t>(ws, L.header);
    dim3 grid(ct.n_tiles);
    int KM = k_bucket(K);
#define GS_FWD(TW, TH) walk_fwd_k<TW, TH>(KM, kbuf, grid, s, ct, K, N, proj, tl, ie, wc, err, rgb_out, depth_out, T_out, n_out, idx_out, w_out)
    if (ct.tile_w == 16 && ct.tile_h == 16) return GS_FWD(16, 16);
    if (ct.tile_w == 32 && ct.tile_h == 8) return GS_FWD(32, 8);
    if (ct.tile_w == 16 && ct.tile_h == 8) return GS_FWD(16, 8);
    if (ct.tile_w == 8 && ct.tile_h == 8) return GS_FWD(8, 8);
#undef GS_FWD
    return false;
}

bool launch_walk_bwd(const CamTable &ct, const WsLayout &L, int K, int N, const float *proj_f, void *ws,
                     const float *rgb_out, const float *depth_out, const int *topk_idx, const float *topk_w,
                     const float *dLdC, const float *dLdD, bool with_feature, cudaStream_t s)
{
    TimerScope tm(GS_TIMER_WALK_BWD, s);
    const float4 *proj = (const float4 *)proj_f;
    const int *err = ws_ptr<int>(ws, L.header);
    const TileLists tl = tile_lists(L, ws);
    const uint32_t *ie = ws_ptr<uint32_t>(ws, L.inst_elem);
    const float *h = with_feature ? ws_ptr<float>(ws, L.hbuf) : nullptr;
    float *ig = ws_ptr<float>(ws, L.inst_grad);
    uint8_t *wk = ws_ptr<uint8_t>(ws, L.inst_walked);
    unsigned *ctr = ws_ptr<unsigned>(ws, L.header) + kHdrWalkTiles;
    dim3 grid(ct.n_tiles);
    int KM = k_bucket(K);
#define GS_BWD(TW, TH) walk_bwd_k<TW, TH>(KM, grid, s, ct, K, N, proj, tl, ie, err, rgb_out, depth_out, topk_idx, topk_w, h, dLdC, dLdD, ig, wk, ctr)
    if (ct.tile_w == 16 && ct.tile_h == 16) return GS_BWD(16, 16);
    if (ct.tile_w == 32 && ct.tile_h == 8) return GS_BWD(32, 8);
    if (ct.tile_w == 16 && ct.tile_h == 8) return GS_BWD(16, 8);
    if (ct.tile_w == 8 && ct.tile_h == 8) return GS_BWD(8, 8);
#undef GS_BWD
    return false;
}

}  // namespace gs
