/*
 * gs_oracle.c -- FP64 CPU oracle for the Top-K feature render.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's
 * CPU-baseline leg are the only users of this file; the product path never links,
 * loads or calls it.  It shares no code, header or constant table with the CUDA
 * library.
 *
 * It is a plain, slow, per-pixel restatement of what the paper defines:
 *   Sec. 3.1, Eq. 1  alpha blending of colour and depth front to back, with the
 *                    contribution weight w_i = alpha_i * prod_{j<i} (1 - alpha_j);
 *   Sec. 3.2, Eq. 2  the Top-K index set: the K contributors of largest w;
 *   Sec. 3.2, Eq. 3  renormalised weights w'_k = w_k / sum_{j in K} w_j;
 *   Sec. 3.2, Eq. 4  F(p) = sum_{k in K} w'_k f_k.
 * The projection of a 3D Gaussian to the image (EWA splatting) is the one of 3D
 * Gaussian Splatting, which Sec. 3.1 says the geometric rendering follows; the
 * constants the paper leaves to that method (0.3 px^2 low-pass dilation, 0.99
 * opacity clamp, 1/255 minimum alpha, 1e-4 transmittance stop, 1.3 x tan(fov)
 * frustum clamp of the Jacobian) are taken from it.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   R1 pixel (i, j) is sampled at (i + 0.5, j + 0.5); u = fx x/z + cx, v = fy y/z + cy.
 *   R2 a Gaussian takes part at a pixel iff its camera depth z > near, its Mahalanobis
 *      distance q = d^T Sigma2D^-1 d <= 9 (3-sigma ellipse, per pixel, so the result
 *      does not depend on any tiling), alpha >= 1/255 and the walk has not stopped.
 *   R3 the walk stops before the first Gaussian whose use would take the
 *      transmittance below 1e-4; that Gaussian is not used.
 *   R4 depth order: ascending camera z rounded to float32 (the precision the GPU
 *      sorts in), equal values by ascending Gaussian index.
 *   R5 Top-K ties (equal w) keep the Gaussian that comes first in depth order;
 *      fewer than K contributors pad with index -1 and weight 0.
 *   R6 a pixel with no contributor has F = 0; F is not renormalised to unit length.
 *   R7 depth is D = sum w_i z_i (not divided by sum w), colour has no background.
 *   R8 backward: the Top-K set and the contributor set are held fixed (piecewise
 *      constant); the 0.99 clamp passes no gradient while it is active; every
 *      contributor before a Top-K member receives gradient through the
 *      transmittance.  The Jacobian clamp passes no gradient to the clamped
 *      coordinate ratio.
 *
 * Near-decision flags: where a discrete decision (contributor test, stop test, Top-K
 * membership) is taken within a small relative margin of its threshold, the pixel
 * is flagged, since a float32 evaluation of the same definition may take it the
 * other way.  Callers exclude flagged pixels from exact comparison and count them.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* camera: R (row-major world->camera rotation, 9), t (3), fx, fy, cx, cy, W, H, near */
enum { CAM_R = 0, CAM_T = 9, CAM_FX = 12, CAM_FY, CAM_CX, CAM_CY, CAM_W, CAM_H, CAM_NEAR, OR_CAM_LEN };

/* per-Gaussian projection record */
enum {
    P_VALID = 0, P_X, P_Y, P_Z,          /* camera-space mean */
    P_U, P_V,                            /* projected mean (pixels) */
    P_SA, P_SB, P_SC,                    /* Sigma2D = [[SA, SB], [SB, SC]] */
    P_CA, P_CB, P_CC,                    /* conic = Sigma2D^-1 = [[CA, CB], [CB, CC]] */
    P_ZF,                                /* depth rounded to float32 (ordering key) */
    P_RX, P_RY,                          /* clamped x/z, y/z used in the Jacobian */
    P_CLX, P_CLY,                        /* 1 if the ratio was clamped */
    OR_PROJ
};

enum { F_NEAR_Q = 1, F_NEAR_ALPHA = 2, F_NEAR_TERM = 4, F_NEAR_TIE = 8, F_NEAR_CLAMP = 16 };

#define Q_MAX 9.0
#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_CLAMP 0.99
#define T_STOP 1e-4
#define DILATION 0.3
#define FRUSTUM_CLAMP 1.3

int or_proj_len(void) { return OR_PROJ; }
int or_cam_len(void) { return OR_CAM_LEN; }

/* ---------------------------------------------------------------------------------
 * EWA projection (Sec. 3.1, following 3D Gaussian Splatting)
 *   p = R mu + t;  J = d(u,v)/d(x,y,z) with x/z, y/z clamped to 1.3 tan(fov/2);
 *   Sigma2D = (J R) Sigma3D (J R)^T + 0.3 I;  conic = Sigma2D^-1.
 * ------------------------------------------------------------------------------- */
static void cov6_to_mat(const double *c6, double S[3][3])
{
    S[0][0] = c6[0]; S[0][1] = c6[1]; S[0][2] = c6[2];
    S[1][0] = c6[1]; S[1][1] = c6[3]; S[1][2] = c6[4];
    S[2][0] = c6[2]; S[2][1] = c6[4]; S[2][2] = c6[5];
}

static void jacobian(const double *cam, const double *pr, double J[2][3])
{
    double fx = cam[CAM_FX], fy = cam[CAM_FY], z = pr[P_Z];
    J[0][0] = fx / z; J[0][1] = 0.0; J[0][2] = -fx * pr[P_RX] / z;
    J[1][0] = 0.0; J[1][1] = fy / z; J[1][2] = -fy * pr[P_RY] / z;
}

int or_project(int n, const double *mean3d, const double *cov3d, const double *cam, double *out)
{
    const double *R = cam + CAM_R, *t = cam + CAM_T;
    double tanx = cam[CAM_W] / (2.0 * cam[CAM_FX]);
    double tany = cam[CAM_H] / (2.0 * cam[CAM_FY]);
    for (int g = 0; g < n; ++g) {
        double *pr = out + (size_t)g * OR_PROJ;
        const double *mu = mean3d + 3 * (size_t)g;
        memset(pr, 0, sizeof(double) * OR_PROJ);
        double p[3];
        for (int r = 0; r < 3; ++r)
            p[r] = R[3 * r + 0] * mu[0] + R[3 * r + 1] * mu[1] + R[3 * r + 2] * mu[2] + t[r];
        pr[P_X] = p[0]; pr[P_Y] = p[1]; pr[P_Z] = p[2];
        if (!(p[2] > cam[CAM_NEAR])) continue;
        double limx = FRUSTUM_CLAMP * tanx, limy = FRUSTUM_CLAMP * tany;
        double rx = p[0] / p[2], ry = p[1] / p[2];
        pr[P_CLX] = (rx < -limx || rx > limx) ? 1.0 : 0.0;
        pr[P_CLY] = (ry < -limy || ry > limy) ? 1.0 : 0.0;
        pr[P_RX] = rx < -limx ? -limx : (rx > limx ? limx : rx);
        pr[P_RY] = ry < -limy ? -limy : (ry > limy ? limy : ry);
        double J[2][3], T[2][3], S[3][3], TS[2][3], S2[2][2];
        jacobian(cam, pr, J);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                T[i][j] = J[i][0] * R[0 * 3 + j] + J[i][1] * R[1 * 3 + j] + J[i][2] * R[2 * 3 + j];
        cov6_to_mat(cov3d + 6 * (size_t)g, S);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                TS[i][j] = T[i][0] * S[0][j] + T[i][1] * S[1][j] + T[i][2] * S[2][j];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                S2[i][j] = TS[i][0] * T[j][0] + TS[i][1] * T[j][1] + TS[i][2] * T[j][2];
        double A = S2[0][0] + DILATION, B = 0.5 * (S2[0][1] + S2[1][0]), C = S2[1][1] + DILATION;
        double det = A * C - B * B;
        if (!(det > 0.0)) continue;
        pr[P_SA] = A; pr[P_SB] = B; pr[P_SC] = C;
        pr[P_CA] = C / det; pr[P_CB] = -B / det; pr[P_CC] = A / det;
        pr[P_U] = cam[CAM_FX] * p[0] / p[2] + cam[CAM_CX];
        pr[P_V] = cam[CAM_FY] * p[1] / p[2] + cam[CAM_CY];
        pr[P_ZF] = (double)(float)p[2];
        pr[P_VALID] = 1.0;
    }
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Per-pixel walk (Eq. 1) and Top-K (Eqs. 2-4)
 * ------------------------------------------------------------------------------- */
typedef struct { int g; double q, G, ao, alpha, T, w, zf, dx, dy; } contrib_t;

static int cmp_depth(const void *a, const void *b)
{
    const contrib_t *x = (const contrib_t *)a, *y = (const contrib_t *)b;
    if (x->zf < y->zf) return -1;
    if (x->zf > y->zf) return 1;
    return (x->g > y->g) - (x->g < y->g);
}

/* Contributors in walk order; returns their count.  cand is scratch of n entries.
 * *flags gets the near-decision bits for this pixel. */
static int pixel_walk(int n, const double *proj, const double *opac, double px, double py,
                      const double *margin, contrib_t *cand, contrib_t *out, double *T_final, int *flags)
{
    double tq = margin[0], ta = margin[1], tt = margin[2], tc = margin[4];
    int nc = 0, ncand = 0;
    for (int g = 0; g < n; ++g) {
        const double *pr = proj + (size_t)g * OR_PROJ;
        if (pr[P_VALID] == 0.0) continue;
        double dx = px - pr[P_U], dy = py - pr[P_V];
        double q = pr[P_CA] * dx * dx + 2.0 * pr[P_CB] * dx * dy + pr[P_CC] * dy * dy;
        if (q > Q_MAX * (1.0 + tq)) continue;          /* far outside the ellipse */
        contrib_t c;
        c.g = g; c.q = q; c.zf = pr[P_ZF]; c.dx = dx; c.dy = dy;
        cand[ncand++] = c;
    }
    qsort(cand, (size_t)ncand, sizeof(contrib_t), cmp_depth);
    double T = 1.0;
    for (int i = 0; i < ncand; ++i) {
        contrib_t c = cand[i];
        /* the ellipse test only decides anything if the Gaussian would pass the
         * alpha test on the ellipse boundary */
        if (fabs(c.q - Q_MAX) <= tq * Q_MAX && opac[c.g] * exp(-0.5 * Q_MAX) >= ALPHA_MIN * (1.0 - ta))
            *flags |= F_NEAR_Q;
        if (c.q > Q_MAX) continue;
        c.G = exp(-0.5 * c.q);
        c.ao = opac[c.g] * c.G;
        c.alpha = c.ao < ALPHA_CLAMP ? c.ao : ALPHA_CLAMP;
        if (fabs(c.ao - ALPHA_CLAMP) <= tc * ALPHA_CLAMP) *flags |= F_NEAR_CLAMP;
        if (fabs(c.alpha - ALPHA_MIN) <= ta * ALPHA_MIN) *flags |= F_NEAR_ALPHA;
        if (c.alpha < ALPHA_MIN) continue;
        double test_T = T * (1.0 - c.alpha);
        if (fabs(test_T - T_STOP) <= tt * T_STOP) *flags |= F_NEAR_TERM;
        if (test_T < T_STOP) break;
        c.T = T;
        c.w = c.alpha * T;
        out[nc++] = c;
        T = test_T;
    }
    *T_final = T;
    return nc;
}

/* Top-K positions (into the walk order) by descending w, ties to the earlier one. */
static int topk_positions(const contrib_t *c, int nc, int K, int *pos, double ttie, int *flags)
{
    int m = nc < K ? nc : K;
    /* selection by repeated arg-max: plain and obviously correct */
    char *taken = (char *)calloc((size_t)(nc > 0 ? nc : 1), 1);
    for (int k = 0; k < m; ++k) {
        int best = -1;
        for (int i = 0; i < nc; ++i)
            if (!taken[i] && (best < 0 || c[i].w > c[best].w)) best = i;
        taken[best] = 1;
        pos[k] = best;
    }
    if (nc > K) {
        int next = -1;
        for (int i = 0; i < nc; ++i)
            if (!taken[i] && (next < 0 || c[i].w > c[next].w)) next = i;
        double wk = c[pos[K - 1]].w, wn = c[next].w;
        if (wk - wn <= ttie * wk) *flags |= F_NEAR_TIE;
    }
    free(taken);
    return m;
}

/* Forward render of a list of pixel centres.
 * Outputs per pixel: C (3), Dep, T_final, n_contrib, topk idx (K, -1 padded),
 * topk w (K, descending, 0 padded), F (D), flags.
 * margin = {tq, ta, tt, ttie, tclamp}: relative margins for the near-decision flags. */
int or_render(int n, const double *proj, const double *opac, const double *rgb, const double *feat,
              int D, int K, int npix, const double *pxy, const double *margin,
              double *C, double *Dep, double *T_final, int *n_contrib, int *tidx, double *tw,
              double *F, int *flags)
{
    contrib_t *cand = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
    contrib_t *walk = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
    int *pos = (int *)malloc(sizeof(int) * (size_t)(K > 0 ? K : 1));
    for (int p = 0; p < npix; ++p) {
        int fl = 0;
        double Tf;
        int nc = pixel_walk(n, proj, opac, pxy[2 * p], pxy[2 * p + 1], margin, cand, walk, &Tf, &fl);
        double c3[3] = {0, 0, 0}, dep = 0.0;
        for (int i = 0; i < nc; ++i) {          /* Eq. 1 */
            for (int ch = 0; ch < 3; ++ch) c3[ch] += walk[i].w * rgb[3 * (size_t)walk[i].g + ch];
            dep += walk[i].w * proj[(size_t)walk[i].g * OR_PROJ + P_Z];
        }
        int m = topk_positions(walk, nc, K, pos, margin[3], &fl);   /* Eq. 2 */
        double S = 0.0;
        for (int k = 0; k < m; ++k) S += walk[pos[k]].w;           /* Eq. 3 denominator */
        double *Fp = F + (size_t)p * D;
        for (int d = 0; d < D; ++d) Fp[d] = 0.0;
        for (int k = 0; k < m && S > 0.0; ++k) {                    /* Eq. 4 */
            double wp = walk[pos[k]].w / S;
            const double *f = feat + (size_t)walk[pos[k]].g * D;
            for (int d = 0; d < D; ++d) Fp[d] += wp * f[d];
        }
        for (int k = 0; k < K; ++k) {
            tidx[(size_t)p * K + k] = k < m ? walk[pos[k]].g : -1;
            tw[(size_t)p * K + k] = k < m ? walk[pos[k]].w : 0.0;
        }
        for (int ch = 0; ch < 3; ++ch) C[3 * (size_t)p + ch] = c3[ch];
        Dep[p] = dep;
        T_final[p] = Tf;
        n_contrib[p] = nc;
        flags[p] = fl;
    }
    free(cand); free(walk); free(pos);
    return 0;
}

/* Full walk of one pixel for inspection: writes up to cap contributors as
 * (g, alpha, T, w) rows; returns the contributor count. */
int or_pixel_walk(int n, const double *proj, const double *opac, double px, double py,
                  const double *margin, int cap, int *g_out, double *awt_out, double *T_final, int *flags)
{
    contrib_t *cand = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
    contrib_t *walk = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
    int fl = 0;
    int nc = pixel_walk(n, proj, opac, px, py, margin, cand, walk, T_final, &fl);
    for (int i = 0; i < nc && i < cap; ++i) {
        g_out[i] = walk[i].g;
        awt_out[3 * i + 0] = walk[i].alpha;
        awt_out[3 * i + 1] = walk[i].T;
        awt_out[3 * i + 2] = walk[i].w;
    }
    *flags = fl;
    free(cand); free(walk);
    return nc;
}

/* ---------------------------------------------------------------------------------
 * Backward of Eqs. 1-4 (reading R8), accumulated (+=) over the given pixels into
 * per-Gaussian gradients of the 2D quantities:
 *   g_mean2d (n x 2: u, v), g_conic (n x 3: a, b, c with q = a dx^2 + 2 b dx dy + c dy^2),
 *   g_opac (n), g_rgb (n x 3), g_depth (n, through D = sum w z), g_feat (n x D).
 * For contributor i (walk order), with upstream dL/dF, dL/dC, dL/dD at the pixel:
 *   dL/dw_i = dL/dC . c_i + dL/dD z_i + [i in K] dL/dF . (f_i - F) / S
 *   dL/dalpha_i = dL/dw_i T_i - (sum_{m > i} dL/dw_m w_m) / (1 - alpha_i)
 * (the second term: alpha_i enters every later weight through the transmittance).
 * ------------------------------------------------------------------------------- */
int or_backward(int n, const double *proj, const double *opac, const double *rgb, const double *feat,
                int D, int K, int npix, const double *pxy, const double *margin,
                const double *dF, const double *dC, const double *dD,
                double *g_mean2d, double *g_conic, double *g_opac, double *g_rgb, double *g_depth,
                double *g_feat)
{
    contrib_t *cand = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
    contrib_t *walk = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
    int *pos = (int *)malloc(sizeof(int) * (size_t)(K > 0 ? K : 1));
    double *dw = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int *slot = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double *Fp = (double *)malloc(sizeof(double) * (size_t)(D > 0 ? D : 1));
    for (int p = 0; p < npix; ++p) {
        int fl = 0;
        double Tf;
        int nc = pixel_walk(n, proj, opac, pxy[2 * p], pxy[2 * p + 1], margin, cand, walk, &Tf, &fl);
        int m = topk_positions(walk, nc, K, pos, margin[3], &fl);
        double S = 0.0;
        for (int k = 0; k < m; ++k) S += walk[pos[k]].w;
        for (int i = 0; i < nc; ++i) slot[i] = -1;
        for (int k = 0; k < m; ++k) slot[pos[k]] = k;
        for (int d = 0; d < D; ++d) Fp[d] = 0.0;
        for (int k = 0; k < m && S > 0.0; ++k) {
            const double *f = feat + (size_t)walk[pos[k]].g * D;
            for (int d = 0; d < D; ++d) Fp[d] += walk[pos[k]].w / S * f[d];
        }
        const double *dFp = dF + (size_t)p * D, *dCp = dC + 3 * (size_t)p;
        double dDp = dD[p];
        /* dL/dw_i */
        for (int i = 0; i < nc; ++i) {
            int g = walk[i].g;
            double v = dCp[0] * rgb[3 * (size_t)g] + dCp[1] * rgb[3 * (size_t)g + 1] + dCp[2] * rgb[3 * (size_t)g + 2]
                     + dDp * proj[(size_t)g * OR_PROJ + P_Z];
            if (slot[i] >= 0) {
                const double *f = feat + (size_t)g * D;
                double acc = 0.0;
                for (int d = 0; d < D; ++d) acc += dFp[d] * (f[d] - Fp[d]);
                v += acc / S;
            }
            dw[i] = v;
        }
        for (int i = 0; i < nc; ++i) {
            int g = walk[i].g;
            const contrib_t *c = &walk[i];
            double suffix = 0.0;
            for (int mm = i + 1; mm < nc; ++mm) suffix += dw[mm] * walk[mm].w;
            double dalpha = dw[i] * c->T - suffix / (1.0 - c->alpha);
            for (int ch = 0; ch < 3; ++ch) g_rgb[3 * (size_t)g + ch] += c->w * dCp[ch];
            g_depth[g] += c->w * dDp;
            if (slot[i] >= 0) {
                double wp = c->w / S;
                double *gf = g_feat + (size_t)g * D;
                for (int d = 0; d < D; ++d) gf[d] += wp * dFp[d];
            }
            if (c->ao < ALPHA_CLAMP) {
                const double *pr = proj + (size_t)g * OR_PROJ;
                g_opac[g] += dalpha * c->G;
                double dq = -0.5 * c->alpha * dalpha;
                g_conic[3 * (size_t)g + 0] += dq * c->dx * c->dx;
                g_conic[3 * (size_t)g + 1] += dq * 2.0 * c->dx * c->dy;
                g_conic[3 * (size_t)g + 2] += dq * c->dy * c->dy;
                /* d = pixel - mean2d, so d(q)/d(u) = -2 (a dx + b dy) */
                g_mean2d[2 * (size_t)g + 0] += dq * -2.0 * (pr[P_CA] * c->dx + pr[P_CB] * c->dy);
                g_mean2d[2 * (size_t)g + 1] += dq * -2.0 * (pr[P_CB] * c->dx + pr[P_CC] * c->dy);
            }
        }
    }
    free(cand); free(walk); free(pos); free(dw); free(slot); free(Fp);
    return 0;
}

/* Chain the 2D gradients back through the projection to the 3D mean and the
 * 3D covariance (6 entries xx, xy, xz, yy, yz, zz; an off-diagonal entry stands for
 * both symmetric positions), and to the camera: g_view (12, accumulated +=) is the
 * gradient with respect to the world-to-camera matrix [R | t] (row-major 3 x 4), through
 * p = R mu + t and through T = J R -- the rendering-loss gradient of a pose refinement. */
int or_backward_project(int n, const double *mean3d, const double *cov3d, const double *cam, const double *proj,
                        const double *g_mean2d, const double *g_conic, const double *g_depth,
                        double *g_mean3d, double *g_cov3d, double *g_view)
{
    const double *R = cam + CAM_R;
    double fx = cam[CAM_FX], fy = cam[CAM_FY];
    for (int g = 0; g < n; ++g) {
        const double *pr = proj + (size_t)g * OR_PROJ;
        double *gm = g_mean3d + 3 * (size_t)g, *gc = g_cov3d + 6 * (size_t)g;
        for (int i = 0; i < 3; ++i) gm[i] = 0.0;
        for (int i = 0; i < 6; ++i) gc[i] = 0.0;
        if (pr[P_VALID] == 0.0) continue;
        double x = pr[P_X], y = pr[P_Y], z = pr[P_Z];
        /* conic -> Sigma2D:  d Sigma^-1 = -Sigma^-1 dSigma Sigma^-1 */
        double Q[2][2] = {{pr[P_CA], pr[P_CB]}, {pr[P_CB], pr[P_CC]}};
        const double *gq = g_conic + 3 * (size_t)g;
        double Gq[2][2] = {{gq[0], 0.5 * gq[1]}, {0.5 * gq[1], gq[2]}};
        double QG[2][2], GS[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) QG[i][j] = Q[i][0] * Gq[0][j] + Q[i][1] * Gq[1][j];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) GS[i][j] = -(QG[i][0] * Q[0][j] + QG[i][1] * Q[1][j]);
        /* Sigma2D = T Sigma3D T^T + 0.3 I,  T = J R */
        double J[2][3], T[2][3], S[3][3];
        jacobian(cam, pr, J);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                T[i][j] = J[i][0] * R[0 * 3 + j] + J[i][1] * R[1 * 3 + j] + J[i][2] * R[2 * 3 + j];
        cov6_to_mat(cov3d + 6 * (size_t)g, S);
        double GS3[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) acc += T[i][a] * GS[i][j] * T[j][b];
                GS3[a][b] = acc;
            }
        gc[0] = GS3[0][0]; gc[1] = GS3[0][1] + GS3[1][0]; gc[2] = GS3[0][2] + GS3[2][0];
        gc[3] = GS3[1][1]; gc[4] = GS3[1][2] + GS3[2][1]; gc[5] = GS3[2][2];
        /* dL/dT = 2 GS T Sigma3D ;  dL/dJ = dL/dT R^T */
        double dT[2][3], dJ[2][3];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 2; ++k)
                    for (int l = 0; l < 3; ++l) acc += GS[i][k] * T[k][l] * S[l][j];
                dT[i][j] = 2.0 * acc;
            }
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                dJ[i][j] = dT[i][0] * R[j * 3 + 0] + dT[i][1] * R[j * 3 + 1] + dT[i][2] * R[j * 3 + 2];
        /* J = [[fx/z, 0, -fx rx/z], [0, fy/z, -fy ry/z]], rx = clamp(x/z) */
        double drx_dx = pr[P_CLX] != 0.0 ? 0.0 : 1.0 / z;
        double drx_dz = pr[P_CLX] != 0.0 ? 0.0 : -x / (z * z);
        double dry_dy = pr[P_CLY] != 0.0 ? 0.0 : 1.0 / z;
        double dry_dz = pr[P_CLY] != 0.0 ? 0.0 : -y / (z * z);
        double rx = pr[P_RX], ry = pr[P_RY];
        double dpx = 0.0, dpy = 0.0, dpz = 0.0;
        dpz += dJ[0][0] * (-fx / (z * z));
        dpz += dJ[1][1] * (-fy / (z * z));
        dpx += dJ[0][2] * (-fx / z) * drx_dx;
        dpz += dJ[0][2] * (fx * rx / (z * z) - fx / z * drx_dz);
        dpy += dJ[1][2] * (-fy / z) * dry_dy;
        dpz += dJ[1][2] * (fy * ry / (z * z) - fy / z * dry_dz);
        /* u = fx x/z + cx, v = fy y/z + cy, depth = z */
        const double *g2 = g_mean2d + 2 * (size_t)g;
        dpx += g2[0] * fx / z;
        dpz += g2[0] * (-fx * x / (z * z));
        dpy += g2[1] * fy / z;
        dpz += g2[1] * (-fy * y / (z * z));
        dpz += g_depth[g];
        /* p = R mu + t */
        for (int j = 0; j < 3; ++j) gm[j] = R[0 * 3 + j] * dpx + R[1 * 3 + j] * dpy + R[2 * 3 + j] * dpz;
        /* the camera: dL/dR_ij = dL/dp_i mu_j + (J^T dL/dT)_ij, dL/dt_i = dL/dp_i */
        const double dp[3] = {dpx, dpy, dpz};
        const double *mu = mean3d + 3 * (size_t)g;
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j)
                g_view[4 * i + j] += dp[i] * mu[j] + J[0][i] * dT[0][j] + J[1][i] * dT[1][j];
            g_view[4 * i + 3] += dp[i];
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Consistency-pruning statistics (Sec. 3.3), accumulated over the given pixels of one
 * view, for every Gaussian g:
 *   count[g] += the number of pixels whose Top-K set (Eq. 2) holds g
 *               (the Top-K participation that selects the candidate set G_prune);
 *   maxw[g]   = max(maxw[g], w_g(r)) over every pixel r where g is a contributor --
 *               the geometric importance S_g of Eq. 8, a maximum of the alpha-blending
 *               weight of Eq. 1 over all rays, selected or not.
 * flags as in or_render.
 * ------------------------------------------------------------------------------- */
int or_prune_stats(int n, const double *proj, const double *opac, int K, int npix, const double *pxy,
                   const double *margin, long long *count, double *maxw, int *flags)
{
    contrib_t *cand = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
    contrib_t *walk = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
    int *pos = (int *)malloc(sizeof(int) * (size_t)(K > 0 ? K : 1));
    for (int p = 0; p < npix; ++p) {
        int fl = 0;
        double Tf;
        int nc = pixel_walk(n, proj, opac, pxy[2 * p], pxy[2 * p + 1], margin, cand, walk, &Tf, &fl);
        for (int i = 0; i < nc; ++i)
            if (walk[i].w > maxw[walk[i].g]) maxw[walk[i].g] = walk[i].w;
        int m = topk_positions(walk, nc, K, pos, margin[3], &fl);
        for (int k = 0; k < m; ++k) count[walk[pos[k]].g] += 1;
        flags[p] = fl;
    }
    free(cand); free(walk); free(pos);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Vanilla feature render (the full alpha-blending baseline of Sec. 3.2 / Tab. 4, as
 * Feature3DGS renders features): F(p) = sum over every contributor i of w_i f_i --
 * Eq. 1 applied to the feature rows, no Top-K, no renormalisation.
 * ------------------------------------------------------------------------------- */
int or_render_vanilla(int n, const double *proj, const double *opac, const double *feat, int D, int npix,
                      const double *pxy, const double *margin, double *F, int *flags)
{
    contrib_t *cand = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
    contrib_t *walk = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
    for (int p = 0; p < npix; ++p) {
        int fl = 0;
        double Tf;
        int nc = pixel_walk(n, proj, opac, pxy[2 * p], pxy[2 * p + 1], margin, cand, walk, &Tf, &fl);
        double *Fp = F + (size_t)p * D;
        for (int d = 0; d < D; ++d) Fp[d] = 0.0;
        for (int i = 0; i < nc; ++i) {
            const double *f = feat + (size_t)walk[i].g * D;
            for (int d = 0; d < D; ++d) Fp[d] += walk[i].w * f[d];
        }
        flags[p] = fl;
    }
    free(cand); free(walk);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Training loss of the benchmark workloads.  Eqs. 5-7 of Sec. 3.4 name the terms (a
 * feature distance, L1 on colour and on depth) but Eq. 6 is garbled and no weights
 * are given; the reading used here takes, per pixel p,
 *   l_p = w_feat (1 - cos(F_p, G_p)) + w_rgb |C_p - Cgt_p|_1 / 3 + w_depth |D_p - Dgt_p|,
 * with cos(F, G) = F.G / (|F| |G|), and L = (1 / P_total) sum_p l_p.  A pixel with
 * |F_p| = 0 or |G_p| = 0 has no direction: its cosine is taken as 0 (it adds w_feat)
 * and it passes no feature gradient.  Gradients, with sign(0) = 0:
 *   dL/dF_p = (w_feat / P_total) (cos F_p / |F_p|^2 - G_p / (|F_p| |G_p|)),
 *   dL/dC_p = (w_rgb / (3 P_total)) sign(C_p - Cgt_p),
 *   dL/dD_p = (w_depth / P_total) sign(D_p - Dgt_p).
 * P of the P_total pixels are given here; *loss receives their share sum_p l_p / P_total
 * (so the shares of disjoint chunks add up to L).
 * ------------------------------------------------------------------------------- */
static double sgn(double x) { return (x > 0.0) - (x < 0.0); }

int or_loss_cos_l1(int P, long long P_total, int D, const double *F, const double *G, const double *C,
                   const double *Cgt, const double *Dp, const double *Dgt, double w_feat, double w_rgb,
                   double w_depth, double *dF, double *dC, double *dD, double *loss)
{
    double sum = 0.0;
    const double inv = 1.0 / (double)P_total;
    for (int p = 0; p < P; ++p) {
        const double *f = F + (size_t)p * D, *g = G + (size_t)p * D;
        double ff = 0.0, gg = 0.0, fg = 0.0;
        for (int d = 0; d < D; ++d) {
            ff += f[d] * f[d];
            gg += g[d] * g[d];
            fg += f[d] * g[d];
        }
        double cosv = 0.0;
        double *df = dF + (size_t)p * D;
        if (ff > 0.0 && gg > 0.0) {
            const double nf = sqrt(ff), ng = sqrt(gg);
            cosv = fg / (nf * ng);
            for (int d = 0; d < D; ++d) df[d] = w_feat * inv * (cosv * f[d] / ff - g[d] / (nf * ng));
        } else {
            for (int d = 0; d < D; ++d) df[d] = 0.0;
        }
        double l1c = 0.0;
        for (int i = 0; i < 3; ++i) {
            const double e = C[3 * p + i] - Cgt[3 * p + i];
            l1c += fabs(e);
            dC[3 * p + i] = w_rgb * inv / 3.0 * sgn(e);
        }
        const double ed = Dp[p] - Dgt[p];
        dD[p] = w_depth * inv * sgn(ed);
        sum += w_feat * (1.0 - cosv) + w_rgb * l1c / 3.0 + w_depth * fabs(ed);
    }
    *loss = sum * inv;
    return 0;
}
