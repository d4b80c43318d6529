// gs_vanilla.cu -- the full alpha-blending feature baseline the paper compares Top-K
// rendering against (Sec. 3.2, Tab. 4 "vanilla"; Feature3DGS renders features this
// way): F(p) = sum over every contributor i of w_i f_i, Eq. 1 applied to the D-wide
// feature rows, no Top-K and no renormalisation.
//
// One CTA per screen tile, one pixel per thread.  A pixel's D accumulators cannot stay
// in registers for D = 512, so the columns are processed in chunks of DC: for each
// chunk the tile's depth-ordered list is walked again (alpha, T and the contributor
// rule are recomputed exactly as the Top-K walk does), each staged Gaussian's DC-column
// slice of its feature row is loaded into shared memory once for the tile's pixels,
// and every pixel adds w_i times the slice for its contributors.  The cost grows with
// the contributors per pixel times D -- the bottleneck Top-K rendering removes.
#include "gs_internal.cuh"

namespace gs {

constexpr int kVanDC = 64;                       // feature columns per pass

template <int TW, int TH, bool BF16>
__global__ void __launch_bounds__(TW *TH) k_walk_vanilla(CamTable ct, int N, int D, const float4 *__restrict__ proj,
                                                         TileLists tl, const uint32_t *__restrict__ inst_elem,
                                                         const int *__restrict__ err,
                                                         const void *__restrict__ feats, void *__restrict__ F)
{
    constexpr int B = TW * TH;
    constexpr int DC = kVanDC;
    __shared__ float4 s_r0[B], s_r1[B];
    extern __shared__ float4 s_f4[];              // [B][DC / 4]
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int c = cam_of_tile(ct, tile);
    const CamDev &cam = ct.c[c];
    const int lt = tile - cam.tile_off;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int px = tx * TW + (tid % TW), py = ty * TH + (tid / TW);
    const bool inside = px < cam.W && py < cam.H;
    const TileList lst(tl, tile, *err != 0);
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const int cN = c * N;
    const long long p = inside ? cam.pix_off + (long long)py * cam.W + px : 0;
    for (int c0 = 0; c0 < D; c0 += DC) {
        const int dc = min(DC, D - c0);                       // a multiple of 8
        float acc[DC];
#pragma unroll
        for (int v = 0; v < DC; ++v) acc[v] = 0.f;
        float T = 1.f;
        bool done = !inside;
        for (int b0 = 0; b0 < lst.n; b0 += B) {
            if (__syncthreads_count(!done) == 0) break;
            const int m = b0 + tid;
            if (m < lst.n) {
                const uint32_t e = inst_elem[lst.at(m)];
                const float4 *r = proj + 4 * (size_t)e;
                s_r0[tid] = r[0];
                s_r1[tid] = r[1];
                const size_t g = (size_t)((int)e - cN);
                float4 *dst = s_f4 + (size_t)tid * (DC / 4);
                if (BF16) {
                    const uint4 *src = (const uint4 *)((const __nv_bfloat16 *)feats + g * D + c0);
                    for (int q = 0; q < dc / 8; ++q) {
                        const uint4 u = __ldg(src + q);
                        const __nv_bfloat162 *h = (const __nv_bfloat162 *)&u;
                        const float2 a = __bfloat1622float2(h[0]), b = __bfloat1622float2(h[1]);
                        const float2 cc = __bfloat1622float2(h[2]), d = __bfloat1622float2(h[3]);
                        dst[2 * q] = make_float4(a.x, a.y, b.x, b.y);
                        dst[2 * q + 1] = make_float4(cc.x, cc.y, d.x, d.y);
                    }
                } else {
                    const float4 *src = (const float4 *)((const float *)feats + g * D + c0);
                    for (int q = 0; q < dc / 4; ++q) dst[q] = __ldg(src + q);
                }
            }
            __syncthreads();
            const int cnt = min(B, lst.n - b0);
            for (int j = 0; j < cnt && !done; ++j) {
                float dx, dy;
                const float4 r1 = s_r1[j];
                const float q = eval_q(pxf, pyf, s_r0[j], r1, dx, dy);
                if (q > kQMax) continue;
                float G, ao;
                const float alpha = eval_alpha(q, r1.w, G, ao);
                if (alpha < kAlphaMin) continue;
                const float test_T = __fmul_rn(T, __fsub_rn(1.f, alpha));
                if (test_T < kTStop) {
                    done = true;
                    break;
                }
                const float w = __fmul_rn(alpha, T);
                const float4 *fr = s_f4 + (size_t)j * (DC / 4);
#pragma unroll
                for (int q4 = 0; q4 < DC / 4; ++q4) {
                    const float4 f = fr[q4];
                    acc[4 * q4] = fmaf(w, f.x, acc[4 * q4]);
                    acc[4 * q4 + 1] = fmaf(w, f.y, acc[4 * q4 + 1]);
                    acc[4 * q4 + 2] = fmaf(w, f.z, acc[4 * q4 + 2]);
                    acc[4 * q4 + 3] = fmaf(w, f.w, acc[4 * q4 + 3]);
                }
                T = test_T;
            }
        }
        if (inside) {
            if (BF16) {
                uint4 *dst = (uint4 *)((__nv_bfloat16 *)F + (size_t)p * D + c0);
#pragma unroll
                for (int q = 0; q < DC / 8; ++q) {
                    if (q < dc / 8) {
                        uint4 u;
                        __nv_bfloat162 *h = (__nv_bfloat162 *)&u;
#pragma unroll
                        for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(acc[8 * q + 2 * i], acc[8 * q + 2 * i + 1]);
                        dst[q] = u;
                    }
                }
            } else {
                float4 *dst = (float4 *)((float *)F + (size_t)p * D + c0);
#pragma unroll
                for (int q = 0; q < DC / 4; ++q)
                    if (q < dc / 4) dst[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
            }
        }
    }
}

template <int TW, int TH>
static void vanilla_k(int dtype, const CamTable &ct, const WsLayout &L, int N, const float4 *proj, void *ws,
                      const void *feats, void *F, cudaStream_t s)
{
    constexpr int B = TW * TH;
    const size_t sm = sizeof(float) * B * kVanDC;
    const TileLists tl = tile_lists(L, ws);
    const uint32_t *ie = ws_ptr<uint32_t>(ws, L.inst_elem);
    const int *err = ws_ptr<int>(ws, L.header);
    if (dtype == GS_BF16) {
        cudaFuncSetAttribute(k_walk_vanilla<TW, TH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_walk_vanilla<TW, TH, true><<<ct.n_tiles, B, sm, s>>>(ct, N, L.D, proj, tl, ie, err, feats, F);
    } else {
        cudaFuncSetAttribute(k_walk_vanilla<TW, TH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_walk_vanilla<TW, TH, false><<<ct.n_tiles, B, sm, s>>>(ct, N, L.D, proj, tl, ie, err, feats, F);
    }
}

bool launch_vanilla(int dtype, const CamTable &ct, const WsLayout &L, int N, const float *proj, void *ws,
                    const void *feats, void *F, cudaStream_t s)
{
    const float4 *p4 = (const float4 *)proj;
    if (ct.tile_w == 16 && ct.tile_h == 16) vanilla_k<16, 16>(dtype, ct, L, N, p4, ws, feats, F, s);
    else if (ct.tile_w == 32 && ct.tile_h == 8) vanilla_k<32, 8>(dtype, ct, L, N, p4, ws, feats, F, s);
    else if (ct.tile_w == 16 && ct.tile_h == 8) vanilla_k<16, 8>(dtype, ct, L, N, p4, ws, feats, F, s);
    else if (ct.tile_w == 8 && ct.tile_h == 8) vanilla_k<8, 8>(dtype, ct, L, N, p4, ws, feats, F, s);
    else return false;
    return true;
}

}  // namespace gs
