// gs_hybrid.cu -- pieces of the hybrid field optimisation schedule (Sec. 3.4): the
// geometric loss of the geometry-only iterations and a fused Adam step.
//
// Geometry-only iterations render colour and depth, take Eq. 6's L1 terms and run the
// adjoint without its feature part (gs_backward with dL_dF = NULL); semantic iterations
// run the full Top-K step.  The parameters are then updated by Adam, all tensors in one
// launch.
#include "gs_internal.cuh"

namespace gs {

__global__ void k_sum_fixed(const float *__restrict__ in, long long n, float *out);

// w_rgb |C - Cgt|_1 / 3 + w_depth |D - Dgt| per pixel (averaged), and its gradient.
__global__ void __launch_bounds__(256) k_loss_geo(long long n_pix, const float *__restrict__ C,
                                                  const float *__restrict__ Cgt, const float *__restrict__ Dp,
                                                  const float *__restrict__ Dgt, float wc, float wd, float invP,
                                                  float *__restrict__ dLdC, float *__restrict__ dLdD,
                                                  float *__restrict__ part)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pix) return;
    float lc = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float d = C[3 * p + i] - Cgt[3 * p + i];
        lc += fabsf(d);
        dLdC[3 * p + i] = wc * invP / 3.f * (float)((d > 0.f) - (d < 0.f));
    }
    const float dd = Dp[p] - Dgt[p];
    dLdD[p] = wd * invP * (float)((dd > 0.f) - (dd < 0.f));
    part[p] = (wc * lc / 3.f + wd * fabsf(dd)) * invP;
}

bool launch_loss_geo(long long n_pix, const float *C, const float *Cgt, const float *Dp, const float *Dgt, float wc,
                     float wd, float *dLdC, float *dLdD, float *loss, float *part, cudaStream_t s)
{
    if (n_pix <= 0) return true;
    k_loss_geo<<<(unsigned)((n_pix + 255) / 256), 256, 0, s>>>(n_pix, C, Cgt, Dp, Dgt, wc, wd, 1.f / (float)n_pix,
                                                                dLdC, dLdD, part);
    float *part2 = part + n_pix;
    k_sum_fixed<<<kSortBlocks, 1024, 0, s>>>(part, n_pix, part2);
    k_sum_fixed<<<1, 1024, 0, s>>>(part2, kSortBlocks, loss);
    return true;
}

// ------------------------------------------------------------------------------------
// Fused Adam: the tensors' elements form one index space, walked grid-stride in groups of
// four (float4 where a tensor's base and length allow it).
// ------------------------------------------------------------------------------------
struct AdamTable {
    AdamTensor t[kAdamMaxTensors];
    long long start[kAdamMaxTensors + 1];          // in groups of 4 elements
    int n;
};

__device__ __forceinline__ void adam_one(float &p, float g, float &m, float &v, float lr, float b1, float b2,
                                         float c1, float c2, float eps)
{
    m = fmaf(b1, m, (1.f - b1) * g);
    v = fmaf(b2, v, (1.f - b2) * g * g);
    p -= lr * (m * c1) / (sqrtf(v * c2) + eps);
}

__global__ void __launch_bounds__(256) k_adam(const __grid_constant__ AdamTable tab, float b1, float b2, float c1,
                                              float c2, float eps)
{
    const long long total = tab.start[tab.n];
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < tab.n && q >= tab.start[k + 1]) ++k;
        const AdamTensor &t = tab.t[k];
        const long long i0 = 4 * (q - tab.start[k]);
        const bool vec = ((((uintptr_t)t.param) | ((uintptr_t)t.grad) | ((uintptr_t)t.m) | ((uintptr_t)t.v)) & 15) == 0 &&
                         i0 + 4 <= t.n;
        if (vec) {
            float4 p = *(float4 *)(t.param + i0), m = *(float4 *)(t.m + i0), v = *(float4 *)(t.v + i0);
            const float4 g = __ldg((const float4 *)(t.grad + i0));
            adam_one(p.x, g.x, m.x, v.x, t.lr, b1, b2, c1, c2, eps);
            adam_one(p.y, g.y, m.y, v.y, t.lr, b1, b2, c1, c2, eps);
            adam_one(p.z, g.z, m.z, v.z, t.lr, b1, b2, c1, c2, eps);
            adam_one(p.w, g.w, m.w, v.w, t.lr, b1, b2, c1, c2, eps);
            *(float4 *)(t.param + i0) = p;
            *(float4 *)(t.m + i0) = m;
            *(float4 *)(t.v + i0) = v;
            if (t.pb) {                 // 4 bf16 = 8 bytes (the copy is 8-byte aligned)
                __nv_bfloat162 lo = __floats2bfloat162_rn(p.x, p.y), hi = __floats2bfloat162_rn(p.z, p.w);
                uint2 u;
                u.x = *(const uint32_t *)&lo;
                u.y = *(const uint32_t *)&hi;
                *(uint2 *)(t.pb + i0) = u;
            }
        } else {
            for (long long i = i0; i < i0 + 4 && i < t.n; ++i) {
                float p = t.param[i], m = t.m[i], v = t.v[i];
                adam_one(p, t.grad[i], m, v, t.lr, b1, b2, c1, c2, eps);
                t.param[i] = p;
                t.m[i] = m;
                t.v[i] = v;
                if (t.pb) t.pb[i] = __float2bfloat16_rn(p);
            }
        }
    }
}

bool launch_adam(const AdamTensor *t, int n_tensors, int step, float beta1, float beta2, float eps, cudaStream_t s)
{
    AdamTable tab;
    tab.n = n_tensors;
    long long acc = 0;
    for (int i = 0; i < n_tensors; ++i) {
        tab.t[i] = t[i];
        tab.start[i] = acc;
        acc += (t[i].n + 3) / 4;
    }
    tab.start[n_tensors] = acc;
    for (int i = n_tensors; i < kAdamMaxTensors; ++i) {
        tab.t[i] = AdamTensor{nullptr, nullptr, nullptr, nullptr, 0, 0.f, nullptr};
        tab.start[i + 1] = acc;
    }
    // bias corrections in double on the host
    const float c1 = (float)(1.0 / (1.0 - pow((double)beta1, (double)step)));
    const float c2 = (float)(1.0 / (1.0 - pow((double)beta2, (double)step)));
    const long long blocks = std::min<long long>((acc + 255) / 256, 148LL * 16);
    if (blocks > 0) k_adam<<<(unsigned)blocks, 256, 0, s>>>(tab, beta1, beta2, c1, c2, eps);
    return true;
}

}  // namespace gs
