"""FP64 CPU oracle for the Top-K feature render -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import this
package; the product path (the CUDA library and its binding) never does, and this
package imports nothing from the product.  The arithmetic lives in gs_oracle.c
(plain C, FP64), compiled here with gcc into oracle/_build/liboracle.so.

Functions follow the paper's definitions:
  project   -- EWA projection of each Gaussian (Sec. 3.1, after 3D Gaussian Splatting)
  render    -- per pixel: Eq. 1 colour/depth, Eq. 2 Top-K set, Eq. 3 renormalised
               weights, Eq. 4 feature
  backward  -- the adjoint of the above (no counterpart in the paper; written out from
               Eqs. 1-4 by the chain rule), chained through the projection to the 3D
               mean and covariance.
  prune_stats  -- Sec. 3.3: Top-K participation count and the geometric importance
               S_i = max w_i (Eq. 8) of every Gaussian over a view's pixels
  prune_select -- Sec. 3.3: the candidate set (low Top-K participation) and the weighted
               survival sampling of Eq. 9
  render_vanilla -- the full alpha-blending feature baseline (Sec. 3.2, Tab. 4):
               F = sum over all contributors of w_i f_i
  adam_step  -- the Adam update (Kingma and Ba, with bias correction) of the mapping
               iterations, FP64
  loss_geo   -- the colour/depth L1 loss of the geometry-only iterations and its gradient
  loss_cos_l1 -- the training loss of the benchmark workloads (Sec. 3.4, Eqs. 5-7 read
               as 1 - cosine on features plus L1 on colour and depth) and its gradients
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# near-decision margins (relative): ellipse test, alpha test, stop test, Top-K tie, clamp
DEFAULT_MARGINS = (2e-5, 2e-5, 2e-5, 1e-6, 2e-5)
F_NEAR_Q, F_NEAR_ALPHA, F_NEAR_TERM, F_NEAR_TIE, F_NEAR_CLAMP = 1, 2, 4, 8, 16
F_SET_FRAGILE = F_NEAR_Q | F_NEAR_ALPHA | F_NEAR_TERM   # may change the contributor set
P_VALID, P_X, P_Y, P_Z, P_U, P_V, P_SA, P_SB, P_SC, P_CA, P_CB, P_CC, P_ZF = range(13)


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into a shared library (gcc, -O2, FP64, no fast-math)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        # GS_ORACLE_LIB lets the mutation test load a deliberately broken copy
        lib = ctypes.CDLL(os.environ.get("GS_ORACLE_LIB") or build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        i = ctypes.c_int
        lib.or_project.argtypes = [i, dp, dp, dp, dp]
        lib.or_render.argtypes = [i, dp, dp, dp, dp, i, i, i, dp, dp, dp, dp, dp, ip, ip, dp, dp, ip]
        lib.or_backward.argtypes = [i, dp, dp, dp, dp, i, i, i, dp, dp, dp, dp, dp,
                                    dp, dp, dp, dp, dp, dp]
        lib.or_backward_project.argtypes = [i, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        lib.or_pixel_walk.argtypes = [i, dp, dp, ctypes.c_double, ctypes.c_double, dp, i, ip, dp, dp, ip]
        lib.or_prune_stats.argtypes = [i, dp, dp, i, i, dp, dp, ctypes.POINTER(ctypes.c_longlong), dp, ip]
        lib.or_render_vanilla.argtypes = [i, dp, dp, dp, i, i, dp, dp, dp, ip]
        lib.or_loss_cos_l1.argtypes = [i, ctypes.c_longlong, i, dp, dp, dp, dp, dp, dp, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
        _lib = lib
        global PROJ_LEN, CAM_LEN
        PROJ_LEN = lib.or_proj_len()
        CAM_LEN = lib.or_cam_len()
    return _lib


PROJ_LEN = 17
CAM_LEN = 19


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def cam_array(cam) -> np.ndarray:
    """Camera as the oracle's 19 doubles.  Every value is first rounded to float32,
    the precision in which a renderer receives its camera, so that both sides start
    from identical parameters."""
    vm = np.asarray(cam.viewmat, dtype=np.float32).astype(np.float64)
    intr = np.asarray([cam.fx, cam.fy, cam.cx, cam.cy], dtype=np.float32).astype(np.float64)
    return np.concatenate([vm[:3, :3].ravel(), vm[:3, 3], intr,
                           [cam.width, cam.height, float(np.float32(cam.near))]])


def pixel_centres(cam, pixels=None) -> np.ndarray:
    """(P, 2) pixel-centre coordinates; pixels is None (all, row-major) or flat indices."""
    if pixels is None:
        pixels = np.arange(cam.width * cam.height)
    pixels = np.asarray(pixels, dtype=np.int64)
    return np.stack([pixels % cam.width + 0.5, pixels // cam.width + 0.5], axis=1).astype(np.float64)


def project(scene, cam, cam_arr=None) -> np.ndarray:
    """EWA projection of every Gaussian; cam_arr (float64, cam_array's layout) overrides
    the camera -- e.g. a perturbed pose for finite differences."""
    L = _L()
    n = scene.n
    mean, pm = _d(scene.mean3d)
    cov, pc = _d(scene.cov3d)
    ca, pca = _d(cam_array(cam) if cam_arr is None else np.asarray(cam_arr, np.float64))
    out, po = _d(np.zeros((n, PROJ_LEN)))
    L.or_project(n, pm, pc, pca, po)
    return out


def render(scene, cam, K, pixels=None, proj=None, margins=DEFAULT_MARGINS, feats=None):
    """Forward render at the given pixels (flat row-major indices, default: all).
    feats overrides scene.feats (e.g. with bf16-rounded rows)."""
    L = _L()
    if proj is None:
        proj = project(scene, cam)
    feats = scene.feats if feats is None else feats
    n, D = scene.n, feats.shape[1]
    pxy, ppx = _d(pixel_centres(cam, pixels))
    P = pxy.shape[0]
    pr, ppr = _d(proj)
    op, pop = _d(scene.opacity)
    rgb, prgb = _d(scene.rgb)
    ft, pft = _d(feats)
    mg, pmg = _d(np.asarray(margins, dtype=np.float64))
    C, pC = _d(np.zeros((P, 3)))
    Dp, pD = _d(np.zeros(P))
    T, pT = _d(np.zeros(P))
    nc, pnc = _i(np.zeros(P))
    idx, pidx = _i(np.zeros((P, K)))
    w, pw = _d(np.zeros((P, K)))
    F, pF = _d(np.zeros((P, D)))
    fl, pfl = _i(np.zeros(P))
    L.or_render(n, ppr, pop, prgb, pft, D, K, P, ppx, pmg, pC, pD, pT, pnc, pidx, pw, pF, pfl)
    return dict(C=C, D=Dp, T=T, n=nc, idx=idx, w=w, F=F, flags=fl)


def pixel_walk(scene, cam, px, py, proj=None, margins=DEFAULT_MARGINS, cap=4096):
    """Contributors of one pixel centre (px, py) in walk order: (ids, alpha, T, w), T_final, flags."""
    L = _L()
    if proj is None:
        proj = project(scene, cam)
    pr, ppr = _d(proj)
    op, pop = _d(scene.opacity)
    mg, pmg = _d(np.asarray(margins, dtype=np.float64))
    g, pg = _i(np.zeros(cap))
    awt, pawt = _d(np.zeros((cap, 3)))
    Tf, pTf = _d(np.zeros(1))
    fl, pfl = _i(np.zeros(1))
    nc = L.or_pixel_walk(scene.n, ppr, pop, float(px), float(py), pmg, cap, pg, pawt, pTf, pfl)
    m = min(nc, cap)
    return g[:m].copy(), awt[:m, 0].copy(), awt[:m, 1].copy(), awt[:m, 2].copy(), float(Tf[0]), int(fl[0])


def backward(scene, cam, K, dF, dC, dD, pixels=None, proj=None, margins=DEFAULT_MARGINS, feats=None, cam_arr=None):
    """Gradients of L with upstream dL/dF (P, D), dL/dC (P, 3), dL/dD (P,) at the given
    pixels.  Returns per-Gaussian FP64 arrays: mean2d (n,2), conic (n,3), opac (n),
    rgb (n,3), depth (n), feat (n,D), mean3d (n,3), cov3d (n,6), and viewmat (3,4): the
    gradient with respect to the camera's world-to-camera [R | t].  cam_arr overrides
    the camera array (float64, as cam_array lays it out)."""
    L = _L()
    if proj is None:
        proj = project(scene, cam, cam_arr=cam_arr)
    feats = scene.feats if feats is None else feats
    n, D = scene.n, feats.shape[1]
    pxy, ppx = _d(pixel_centres(cam, pixels))
    P = pxy.shape[0]
    pr, ppr = _d(proj)
    op, pop = _d(scene.opacity)
    rgb, prgb = _d(scene.rgb)
    ft, pft = _d(feats)
    mg, pmg = _d(np.asarray(margins, dtype=np.float64))
    dF_, pdF = _d(np.asarray(dF).reshape(P, D))
    dC_, pdC = _d(np.asarray(dC).reshape(P, 3))
    dD_, pdD = _d(np.asarray(dD).reshape(P))
    g2, pg2 = _d(np.zeros((n, 2)))
    gq, pgq = _d(np.zeros((n, 3)))
    go, pgo = _d(np.zeros(n))
    gr, pgr = _d(np.zeros((n, 3)))
    gz, pgz = _d(np.zeros(n))
    gf, pgf = _d(np.zeros((n, D)))
    L.or_backward(n, ppr, pop, prgb, pft, D, K, P, ppx, pmg, pdF, pdC, pdD, pg2, pgq, pgo, pgr, pgz, pgf)
    mean, pmean = _d(scene.mean3d)
    cov, pcov = _d(scene.cov3d)
    ca, pca = _d(cam_array(cam) if cam_arr is None else cam_arr)
    gm, pgm = _d(np.zeros((n, 3)))
    gc, pgc = _d(np.zeros((n, 6)))
    gv, pgv = _d(np.zeros((3, 4)))
    L.or_backward_project(n, pmean, pcov, pca, ppr, pg2, pgq, pgz, pgm, pgc, pgv)
    return dict(mean2d=g2, conic=gq, opac=go, rgb=gr, depth=gz, feat=gf, mean3d=gm, cov3d=gc, viewmat=gv)


def prune_stats(scene, cam, K, pixels=None, proj=None, margins=DEFAULT_MARGINS, count=None, maxw=None):
    """Sec. 3.3 statistics over one view's pixels (default: all), accumulated into count
    (int64, n) and maxw (float64, n) when given: Top-K participation and S_i = max w_i
    (Eq. 8).  Returns dict(count, maxw, flags)."""
    L = _L()
    if proj is None:
        proj = project(scene, cam)
    n = scene.n
    pxy, ppx = _d(pixel_centres(cam, pixels))
    P = pxy.shape[0]
    pr, ppr = _d(proj)
    op, pop = _d(scene.opacity)
    mg, pmg = _d(np.asarray(margins, dtype=np.float64))
    cnt = np.zeros(n, dtype=np.int64) if count is None else count
    mw = np.zeros(n, dtype=np.float64) if maxw is None else maxw
    assert cnt.dtype == np.int64 and cnt.flags.c_contiguous and mw.dtype == np.float64 and mw.flags.c_contiguous
    fl, pfl = _i(np.zeros(P))
    L.or_prune_stats(n, ppr, pop, K, P, ppx, pmg, cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                     mw.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pfl)
    return dict(count=cnt, maxw=mw, flags=fl)


def prune_select(count, S, tau, ratio, expo):
    """Sec. 3.3, Eq. 9.  Candidates G_prune: Gaussians with Top-K participation count < tau.
    Within G_prune, m = floor(ratio |G_prune| + 1/2) Gaussians survive, drawn by weighted
    sampling without replacement with probability proportional to S_i (Eq. 9): each
    draw picks candidate i with probability S_i / sum of the remaining S.  The draws are
    realised as an exponential race -- candidate i finishes at e_i / S_i with the given
    e_i ~ Exp(1), the m earliest survive (the first finisher is i with probability
    S_i / sum S); S_i = 0 never finishes, equal times go to the smaller id.  The times
    are formed in float32 (as the kernel does), so both sides take the same decision.
    Returns keep (bool, n): every non-candidate is kept."""
    count = np.asarray(count)
    S32 = np.asarray(S, dtype=np.float32)
    e32 = np.asarray(expo, dtype=np.float32)
    n = count.shape[0]
    cand = np.nonzero(count < tau)[0]
    m = int(np.floor(ratio * cand.size + 0.5))
    t = np.full(cand.size, np.inf, dtype=np.float32)
    pos = S32[cand] > 0
    t[pos] = e32[cand][pos] / S32[cand][pos]
    order = np.lexsort((cand, t))          # by time, then id
    keep = np.ones(n, dtype=bool)
    keep[cand] = False
    keep[cand[order[:m]]] = True
    return keep


def render_vanilla(scene, cam, pixels=None, proj=None, margins=DEFAULT_MARGINS, feats=None):
    """Full alpha-blended feature (Eq. 1 on the feature rows, every contributor, no
    renormalisation) at the given pixels.  Returns dict(F, flags)."""
    L = _L()
    if proj is None:
        proj = project(scene, cam)
    feats = scene.feats if feats is None else feats
    n, D = scene.n, feats.shape[1]
    pxy, ppx = _d(pixel_centres(cam, pixels))
    P = pxy.shape[0]
    pr, ppr = _d(proj)
    op, pop = _d(scene.opacity)
    ft, pft = _d(feats)
    mg, pmg = _d(np.asarray(margins, dtype=np.float64))
    F, pF = _d(np.zeros((P, D)))
    fl, pfl = _i(np.zeros(P))
    L.or_render_vanilla(n, ppr, pop, pft, D, P, ppx, pmg, pF, pfl)
    return dict(F=F, flags=fl)


def adam_step(p, g, m, v, lr, beta1, beta2, eps, step):
    """One Adam step in FP64 (Kingma and Ba, Algorithm 1 with bias correction): returns
    the new (p, m, v)."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def loss_geo(C, Cgt, D, Dgt, w_rgb, w_depth):
    """Mean over pixels of w_rgb |C - C_gt|_1 / 3 + w_depth |D - D_gt| (Eq. 6's L1 terms)
    and its gradient (sign convention: 0 at equality).  Returns (loss, dC, dD)."""
    C, Cgt, D, Dgt = (np.asarray(a, np.float64) for a in (C, Cgt, D, Dgt))
    P = D.shape[0]
    loss = (w_rgb * np.abs(C - Cgt).sum(1) / 3 + w_depth * np.abs(D - Dgt)).sum() / P
    return loss, w_rgb / (3 * P) * np.sign(C - Cgt), w_depth / P * np.sign(D - Dgt)


def loss_cos_l1(F, F_gt, C, C_gt, D, D_gt, w_feat=1.0, w_rgb=1.0, w_depth=1.0, n_total=None):
    """Training loss of the workloads and its gradients, FP64 (gs_oracle.c, or_loss_cos_l1):
    L = (1/P) sum_p [w_feat (1 - cos(F_p, Fgt_p)) + w_rgb |C_p - Cgt_p|_1 / 3 + w_depth |D_p - Dgt_p|],
    a pixel with |F_p| = 0 or |Fgt_p| = 0 adding w_feat and no feature gradient.  The
    pixels given may be a chunk of n_total (default: all of them); the returned loss is
    then their share of the mean.  Returns (loss, dF (P, Dim), dC (P, 3), dD (P,))."""
    L = _L()
    F, pF = _d(F)
    G, pG = _d(F_gt)
    P, Dim = F.shape
    assert G.shape == (P, Dim)
    C_, pC = _d(np.asarray(C).reshape(P, 3))
    Cg, pCg = _d(np.asarray(C_gt).reshape(P, 3))
    D_, pD = _d(np.asarray(D).reshape(P))
    Dg, pDg = _d(np.asarray(D_gt).reshape(P))
    dF, pdF = _d(np.zeros((P, Dim)))
    dC, pdC = _d(np.zeros((P, 3)))
    dD, pdD = _d(np.zeros(P))
    lo, plo = _d(np.zeros(1))
    L.or_loss_cos_l1(P, int(P if n_total is None else n_total), Dim, pF, pG, pC, pCg, pD, pDg, float(w_feat),
                     float(w_rgb), float(w_depth), pdF, pdC, pdD, plo)
    return float(lo[0]), dF, dC, dD
