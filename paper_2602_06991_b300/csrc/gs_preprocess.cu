// gs_preprocess.cu -- a1: EWA projection of each (camera, Gaussian) and its adjoint.
//
// The projection is the one of 3D Gaussian Splatting, which the paper's geometric
// rendering follows (Sec. 3.1): p = R mu + t, J the Jacobian of the pinhole map with
// x/z, y/z clamped to 1.3 tan(fov/2), Sigma2D = (J R) Sigma3D (J R)^T + 0.3 I.
//
// B300 specifics: one thread per (camera, Gaussian); the camera transform and the
// pixel position of the mean are carried in double-float (FMA-based error-free
// transforms) so that the per-pixel offset d = pixel - mean2d, formed later in the
// walk, carries only its own float32 rounding; FP64 units are not used (they are slow
// on this part).  The 2x2 determinant uses Kahan's FMA scheme, and the conic is also
// stored in Cholesky form so the walk evaluates q as a sum of two squares.
#include "gs_internal.cuh"

namespace gs {

// a . b + t (3 terms) in double-float.
__device__ __forceinline__ void dot3_df(const float *a, float b0, float b1, float b2, float t, float &hi, float &lo)
{
    float p0, e0, p1, e1, p2, e2, s, t1, t2, t3;
    two_prod(a[0], b0, p0, e0);
    two_prod(a[1], b1, p1, e1);
    two_prod(a[2], b2, p2, e2);
    two_sum(p0, p1, s, t1);
    two_sum(s, p2, s, t2);
    two_sum(s, t, s, t3);
    float l = __fadd_rn(__fadd_rn(__fadd_rn(e0, e1), __fadd_rn(e2, t1)), __fadd_rn(t2, t3));
    fast_two_sum(s, l, hi, lo);
}

// f * (xh + xl) / (zh + zl) + c in double-float.
__device__ __forceinline__ void proj_df(float f, float c, float xh, float xl, float zh, float zl, float &hi, float &lo)
{
    float q1 = __fdiv_rn(xh, zh);
    float r = __fmaf_rn(-q1, zh, xh);                  // exact: xh - q1 zh
    r = __fadd_rn(r, __fmaf_rn(-q1, zl, xl));
    float q2 = __fdiv_rn(r, zh);
    float p, e, s, t;
    two_prod(f, q1, p, e);
    e = __fmaf_rn(f, q2, e);
    two_sum(p, c, s, t);
    fast_two_sum(s, __fadd_rn(t, e), hi, lo);
}

struct Geo {
    float x, y, z;             // camera-space mean (float32)
    float rx, ry;              // clamped x/z, y/z
    bool clx, cly;
    float T[2][3];             // J R
    float S[3][3];             // Sigma3D
    float A, B, C;             // Sigma2D
};

__device__ __forceinline__ void load_cov(const float *c6, float S[3][3])
{
    S[0][0] = c6[0]; S[0][1] = c6[1]; S[0][2] = c6[2];
    S[1][0] = c6[1]; S[1][1] = c6[3]; S[1][2] = c6[4];
    S[2][0] = c6[2]; S[2][1] = c6[4]; S[2][2] = c6[5];
}

__device__ __forceinline__ void ewa(const CamDev &cam, float x, float y, float z, const float *c6, Geo &g)
{
    g.x = x; g.y = y; g.z = z;
    float rx = x / z, ry = y / z;
    g.clx = rx < -cam.limx || rx > cam.limx;
    g.cly = ry < -cam.limy || ry > cam.limy;
    g.rx = fminf(fmaxf(rx, -cam.limx), cam.limx);
    g.ry = fminf(fmaxf(ry, -cam.limy), cam.limy);
    float j00 = cam.fx / z, j02 = -cam.fx * g.rx / z;
    float j11 = cam.fy / z, j12 = -cam.fy * g.ry / z;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        g.T[0][j] = j00 * cam.R[0 * 3 + j] + j02 * cam.R[2 * 3 + j];
        g.T[1][j] = j11 * cam.R[1 * 3 + j] + j12 * cam.R[2 * 3 + j];
    }
    load_cov(c6, g.S);
    float TS[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            TS[i][j] = g.T[i][0] * g.S[0][j] + g.T[i][1] * g.S[1][j] + g.T[i][2] * g.S[2][j];
    g.A = TS[0][0] * g.T[0][0] + TS[0][1] * g.T[0][1] + TS[0][2] * g.T[0][2] + kDilation;
    g.B = TS[0][0] * g.T[1][0] + TS[0][1] * g.T[1][1] + TS[0][2] * g.T[1][2];
    g.C = TS[1][0] * g.T[1][0] + TS[1][1] * g.T[1][1] + TS[1][2] * g.T[1][2] + kDilation;
}

__device__ __forceinline__ void cam_point(const CamDev &cam, const float *mu, float &xh, float &xl, float &yh,
                                          float &yl, float &zh, float &zl)
{
    dot3_df(cam.R + 0, mu[0], mu[1], mu[2], cam.t[0], xh, xl);
    dot3_df(cam.R + 3, mu[0], mu[1], mu[2], cam.t[1], yh, yl);
    dot3_df(cam.R + 6, mu[0], mu[1], mu[2], cam.t[2], zh, zl);
}

__global__ void __launch_bounds__(256) k_preprocess(CamTable ct, int N, const float *__restrict__ mean3d,
                                                    const float *__restrict__ cov3d, const float *__restrict__ opac,
                                                    const float *__restrict__ rgb, float4 *__restrict__ proj)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)ct.n * N) return;
    int c = (int)(e / N), g = (int)(e - (long long)c * N);
    const CamDev &cam = ct.c[c];
    float mu[3] = {mean3d[3 * (size_t)g], mean3d[3 * (size_t)g + 1], mean3d[3 * (size_t)g + 2]};
    float xh, xl, yh, yl, zh, zl;
    cam_point(cam, mu, xh, xl, yh, yl, zh, zl);
    float4 *out = proj + 4 * (size_t)e;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float o = opac[g];
    // A Gaussian can only pass alpha >= 1/255 if its opacity does (the 2D factor is <= 1).
    bool culled = !(zh > cam.near_z) || !(o >= kAlphaMin * (1.0f - 1e-5f));
    Geo geo;
    float det = 0.f;
    if (!culled) {
        ewa(cam, xh, yh, zh, cov3d + 6 * (size_t)g, geo);
        // Kahan: A C - B^2 with one rounding of the final sum
        float w = __fmul_rn(geo.B, geo.B);
        float err = __fmaf_rn(-geo.B, geo.B, w);
        float f = __fmaf_rn(geo.A, geo.C, -w);
        det = __fadd_rn(f, err);
        culled = !(det > 0.f);
    }
    if (culled) {
        out[0] = zero;
        out[1] = zero;
        out[2] = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
        out[3] = zero;
        return;
    }
    float uh, ul, vh, vl;
    proj_df(cam.fx, cam.cx, xh, xl, zh, zl, uh, ul);
    proj_df(cam.fy, cam.cy, yh, yl, zh, zl, vh, vl);
    float ca = geo.C / det, cb = -geo.B / det, cc = geo.A / det;
    float s1 = 1.0f / sqrtf(geo.A);
    float m = geo.B / geo.A;
    float s2 = sqrtf(geo.A / det);
    // Pixel box that can reach alpha >= 1/255: q <= min(9, 2 ln(255 o)), widened by a
    // relative and an absolute margin so float32 evaluation in the walk stays inside.
    float qb = fminf(kQMax, 2.0f * logf(255.0f * o));
    qb = fmaxf(qb, 0.0f) * 1.002f + 0.002f;
    float ex = sqrtf(qb * geo.A) * 1.001f + 0.01f;
    float ey = sqrtf(qb * geo.C) * 1.001f + 0.01f;
    ex = fminf(ex, 65504.f);
    ey = fminf(ey, 65504.f);
    unsigned int hx = __half_as_ushort(__float2half_ru(ex));
    unsigned int hy = __half_as_ushort(__float2half_ru(ey));
    out[0] = make_float4(uh, vh, ul, vl);
    out[1] = make_float4(s1, m, s2, o);
    out[2] = make_float4(rgb[3 * (size_t)g], rgb[3 * (size_t)g + 1], rgb[3 * (size_t)g + 2], zh);
    out[3] = make_float4(ca, cb, cc, __uint_as_float(hx | (hy << 16)));
}

// ------------------------------------------------------------------------------------
// Adjoint: per Gaussian, sum the per-instance partial 2D gradients of each camera,
// then chain through conic -> Sigma2D -> (J R, Sigma3D) -> camera-space mean -> world
// mean.  Partial layout per instance: du, dv, da, db, dc, dopacity, dr, dg, db, dz.
// ------------------------------------------------------------------------------------
// Per-element sums of the re-walk's instance partials (an element's instances are the
// contiguous pre-sort range [elem_off, elem_off + elem_cnt)), skipping the instances the
// re-walk never reached.  One thread per element sums a short range in instance order;
// the ranges longer than kElemSerial (Gaussians near the camera, over many tiles) are
// then taken one at a time by the whole warp (strided lanes, a fixed shuffle tree).
// Either way the order is fixed, so the result is deterministic.
// STEP4: the per-thread loop takes four instances per step, their walked flags and then
// the reached instances' loads issued before the adds (in the same order, so the same
// sums).  It doubles the registers (64 against 32), so it is chosen only for grids of
// under about two waves, which are bound by the loop's latency rather than by occupancy.
constexpr uint32_t kElemSerial = 48;

template <bool STEP4>
__global__ void __launch_bounds__(256) k_elem_grad_sum(long long NE, const uint32_t *__restrict__ elem_off,
                                                       const uint32_t *__restrict__ elem_cnt,
                                                       const float *__restrict__ inst_grad,
                                                       const uint8_t *__restrict__ walked, const int *err,
                                                       float *__restrict__ elem_grad)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    uint32_t o0 = 0, n = 0;
    if (e < NE && *err == 0) {
        o0 = elem_off[e];
        n = elem_cnt[e];
    }
    if (e < NE && n <= kElemSerial) {
        float v[kGradVals];
#pragma unroll
        for (int k = 0; k < kGradVals; ++k) v[k] = 0.f;
        uint32_t i = 0;
        if constexpr (STEP4) {
            for (; i + 4 <= n; i += 4) {
                bool wk[4];
                float2 x[4][kGradVals / 2];
#pragma unroll
                for (int u = 0; u < 4; ++u) wk[u] = walked[o0 + i + u] != 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float2 *pg = (const float2 *)(inst_grad + kGradVals * (size_t)(o0 + i + u));
#pragma unroll
                    for (int k = 0; k < kGradVals / 2; ++k) x[u][k] = wk[u] ? __ldg(pg + k) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (wk[u]) {
#pragma unroll
                        for (int k = 0; k < kGradVals / 2; ++k) {
                            v[2 * k] += x[u][k].x;
                            v[2 * k + 1] += x[u][k].y;
                        }
                    }
            }
        }
        for (; i < n; ++i) {
            if (!walked[o0 + i]) continue;                  // past where its tile's walk stopped
            // 40-byte record, 8-byte aligned: five 8-byte loads
            const float2 *pg = (const float2 *)(inst_grad + kGradVals * (size_t)(o0 + i));
#pragma unroll
            for (int k = 0; k < kGradVals / 2; ++k) {
                const float2 x = __ldg(pg + k);
                v[2 * k] += x.x;
                v[2 * k + 1] += x.y;
            }
        }
        float2 *dst = (float2 *)(elem_grad + kGradVals * (size_t)e);
#pragma unroll
        for (int k = 0; k < kGradVals / 2; ++k) dst[k] = make_float2(v[2 * k], v[2 * k + 1]);
    }
    unsigned long_ones = __ballot_sync(0xffffffffu, n > kElemSerial);
    while (long_ones) {
        const int j = __ffs(long_ones) - 1;
        long_ones &= long_ones - 1;
        const uint32_t oj = __shfl_sync(0xffffffffu, o0, j), nj = __shfl_sync(0xffffffffu, n, j);
        const long long ej = __shfl_sync(0xffffffffu, e, j);
        float v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = 0.f;
        for (uint32_t i = lane; i < nj; i += 32) {
            if (!walked[oj + i]) continue;
            const float2 *pg = (const float2 *)(inst_grad + kGradVals * (size_t)(oj + i));
#pragma unroll
            for (int k = 0; k < kGradVals / 2; ++k) {
                const float2 x = __ldg(pg + k);
                v[2 * k] += x.x;
                v[2 * k + 1] += x.y;
            }
        }
        const float d = warp_reduce16(v, lane);
        const int vi = (lane >> 1) & 15;
        if (!(lane & 1) && vi < kGradVals) elem_grad[kGradVals * ej + vi] = d;
    }
}

__global__ void __launch_bounds__(256) k_project_backward(CamTable ct, int N, const float *__restrict__ mean3d,
                                                          const float *__restrict__ cov3d, const float4 *__restrict__ proj,
                                                          const float *__restrict__ elem_grad, const int *err,
                                                          float *g_opac, float *g_rgb, float *g_mean3d, float *g_cov3d,
                                                          float *g_mean2d, float *g_conic, float *pose_part)
{
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    float go = 0.f, gr[3] = {0.f, 0.f, 0.f}, gm[3] = {0.f, 0.f, 0.f}, gc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    bool bad = *err != 0;
    for (int c = 0; c < ct.n; ++c) {
        const CamDev &cam = ct.c[c];
        size_t e = (size_t)c * N + g;
        float4 r3 = proj[4 * e + 3];
        float acc[kGradVals];
#pragma unroll
        for (int v = 0; v < kGradVals; ++v) acc[v] = 0.f;
        bool live = __float_as_uint(r3.w) != 0u && !bad;
        if (live) {
#pragma unroll
            for (int v = 0; v < kGradVals; ++v) acc[v] = elem_grad[kGradVals * e + v];
        }
        if (g_mean2d) {
            g_mean2d[2 * e] = acc[0];
            g_mean2d[2 * e + 1] = acc[1];
        }
        if (g_conic) {
            g_conic[3 * e] = acc[2];
            g_conic[3 * e + 1] = acc[3];
            g_conic[3 * e + 2] = acc[4];
        }
        if (!live) {
            if (pose_part) {
#pragma unroll
                for (int k = 0; k < 12; ++k) pose_part[12 * e + k] = 0.f;
            }
            continue;
        }
        go += acc[5];
        gr[0] += acc[6]; gr[1] += acc[7]; gr[2] += acc[8];
        float mu[3] = {mean3d[3 * (size_t)g], mean3d[3 * (size_t)g + 1], mean3d[3 * (size_t)g + 2]};
        float xh, xl, yh, yl, zh, zl;
        cam_point(cam, mu, xh, xl, yh, yl, zh, zl);
        Geo geo;
        ewa(cam, xh, yh, zh, cov3d + 6 * (size_t)g, geo);
        float x = geo.x, y = geo.y, z = geo.z;
        // conic -> Sigma2D: dSigma = -Q G Q, G the full-matrix gradient of the conic
        float Q[2][2] = {{r3.x, r3.y}, {r3.y, r3.z}};
        float Gq[2][2] = {{acc[2], 0.5f * acc[3]}, {0.5f * acc[3], acc[4]}};
        float QG[2][2], GS[2][2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) QG[i][j] = Q[i][0] * Gq[0][j] + Q[i][1] * Gq[1][j];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) GS[i][j] = -(QG[i][0] * Q[0][j] + QG[i][1] * Q[1][j]);
        // Sigma3D gradient: T^T GS T
        float GT[2][3];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int b = 0; b < 3; ++b) GT[i][b] = GS[i][0] * geo.T[0][b] + GS[i][1] * geo.T[1][b];
        float G3[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) G3[a][b] = geo.T[0][a] * GT[0][b] + geo.T[1][a] * GT[1][b];
        gc[0] += G3[0][0]; gc[1] += G3[0][1] + G3[1][0]; gc[2] += G3[0][2] + G3[2][0];
        gc[3] += G3[1][1]; gc[4] += G3[1][2] + G3[2][1]; gc[5] += G3[2][2];
        // dT = 2 GS T Sigma3D ; dJ = dT R^T
        float dT[2][3], dJ[2][3];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                dT[i][j] = 2.f * (GT[i][0] * geo.S[0][j] + GT[i][1] * geo.S[1][j] + GT[i][2] * geo.S[2][j]);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                dJ[i][j] = dT[i][0] * cam.R[j * 3 + 0] + dT[i][1] * cam.R[j * 3 + 1] + dT[i][2] * cam.R[j * 3 + 2];
        float iz = 1.f / z, iz2 = iz * iz;
        float drx_dx = geo.clx ? 0.f : iz, drx_dz = geo.clx ? 0.f : -x * iz2;
        float dry_dy = geo.cly ? 0.f : iz, dry_dz = geo.cly ? 0.f : -y * iz2;
        float dpx = 0.f, dpy = 0.f, dpz = 0.f;
        dpz += dJ[0][0] * (-cam.fx * iz2);
        dpz += dJ[1][1] * (-cam.fy * iz2);
        dpx += dJ[0][2] * (-cam.fx * iz) * drx_dx;
        dpz += dJ[0][2] * (cam.fx * geo.rx * iz2 - cam.fx * iz * drx_dz);
        dpy += dJ[1][2] * (-cam.fy * iz) * dry_dy;
        dpz += dJ[1][2] * (cam.fy * geo.ry * iz2 - cam.fy * iz * dry_dz);
        // u = fx x/z + cx, v = fy y/z + cy, depth = z
        dpx += acc[0] * cam.fx * iz;
        dpz += acc[0] * (-cam.fx * x * iz2);
        dpy += acc[1] * cam.fy * iz;
        dpz += acc[1] * (-cam.fy * y * iz2);
        dpz += acc[9];
#pragma unroll
        for (int j = 0; j < 3; ++j) gm[j] += cam.R[0 * 3 + j] * dpx + cam.R[1 * 3 + j] * dpy + cam.R[2 * 3 + j] * dpz;
        if (pose_part) {
            // the camera: dL/dR_ij = dL/dp_i mu_j + (J^T dL/dT)_ij, dL/dt_i = dL/dp_i
            const float J[2][3] = {{cam.fx * iz, 0.f, -cam.fx * geo.rx * iz}, {0.f, cam.fy * iz, -cam.fy * geo.ry * iz}};
            const float dp[3] = {dpx, dpy, dpz};
            float *pp = pose_part + 12 * e;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
#pragma unroll
                for (int j = 0; j < 3; ++j) pp[4 * i + j] = dp[i] * mu[j] + J[0][i] * dT[0][j] + J[1][i] * dT[1][j];
                pp[4 * i + 3] = dp[i];
            }
        }
    }
    g_opac[g] = go;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        g_rgb[3 * (size_t)g + j] = gr[j];
        g_mean3d[3 * (size_t)g + j] = gm[j];
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) g_cov3d[6 * (size_t)g + j] = gc[j];
}

void launch_preprocess(const CamTable &ct, int N, const float *mean3d, const float *cov3d, const float *opac,
                       const float *rgb, float *proj, cudaStream_t s)
{
    long long NE = (long long)ct.n * N;
    if (NE <= 0) return;
    k_preprocess<<<(unsigned)((NE + 255) / 256), 256, 0, s>>>(ct, N, mean3d, cov3d, opac, rgb, (float4 *)proj);
}

// Pose gradient: per camera, each of its 12 partial columns summed over the Gaussians in a
// fixed order (each thread a contiguous run, then a tree over the threads).
__global__ void __launch_bounds__(1024) k_pose_reduce(int N, const float *__restrict__ pose_part, float *g_view)
{
    __shared__ float sm[1024];
    const int c = blockIdx.x / 12, k = blockIdx.x % 12;
    const int per = (N + 1023) / 1024;
    const int b = threadIdx.x * per, e = min(b + per, N);
    float acc = 0.f;
    for (int g = b; g < e; ++g) acc += pose_part[12 * ((size_t)c * N + g) + k];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) g_view[12 * c + k] = sm[0];
}

void launch_project_backward(const CamTable &ct, int N, const float *mean3d, const float *cov3d, const float *proj,
                             const uint32_t *elem_off, const uint32_t *elem_cnt, const float *inst_grad,
                             const uint8_t *walked, float *elem_grad, const int *err, const gs_grads *gr,
                             float *pose_part, cudaStream_t s)
{
    if (N <= 0) return;
    long long NE = (long long)ct.n * N;
    const unsigned nb = (unsigned)((NE + 255) / 256);
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 148;
    // four-instance steps while the grid is under two waves of that form (4 CTAs per SM)
    if (nb <= (unsigned)(2 * 4 * sms))
        k_elem_grad_sum<true><<<nb, 256, 0, s>>>(NE, elem_off, elem_cnt, inst_grad, walked, err, elem_grad);
    else
        k_elem_grad_sum<false><<<nb, 256, 0, s>>>(NE, elem_off, elem_cnt, inst_grad, walked, err, elem_grad);
    float *pp = gr->viewmat ? pose_part : nullptr;
    k_project_backward<<<(N + 255) / 256, 256, 0, s>>>(ct, N, mean3d, cov3d, (const float4 *)proj, elem_grad, err,
                                                      gr->opacity, gr->rgb, gr->mean3d, gr->cov3d, gr->mean2d,
                                                      gr->conic, pp);
    if (pp) k_pose_reduce<<<ct.n * 12, 1024, 0, s>>>(N, pp, gr->viewmat);
}

}  // namespace gs
