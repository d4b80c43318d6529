"""GPU parity of the training loss against the FP64 oracle (oracle.loss_cos_l1):
gs_loss_cos_l1, the fused gs_feature_blend_loss and gs_loss_cos_l1_noalloc, element by
element, through the C ABI.

Loss (Sec. 3.4, Eqs. 5-7 read as 1 - cosine on the feature, L1 on colour and depth):
L = (1/P) sum_p [w_feat (1 - cos(F_p, Fgt_p)) + w_rgb |C_p - Cgt_p|_1 / 3 + w_depth |D_p - Dgt_p|];
a pixel with |F_p| = 0 or |Fgt_p| = 0 adds w_feat and passes no feature gradient.

Tolerances.  The CUDA path works in float32.  dL/dF_p = a Fgt_p + b F_p with
a = -w_feat / (P |F||Fgt|) and b = w_feat cos / (P |F|^2), from the sums |F|^2, |Fgt|^2
and F.Fgt over D elements.  Float32 sums carry an error of about gamma = sqrt(D) 2^-24
relative to |F|^2, |Fgt|^2 and |F||Fgt| (not to F.Fgt, which is small for nearly orthogonal
rows), so a carries a relative error ~gamma and cos an absolute one ~gamma (1 + |cos|),
and b an error ~gamma (2 + |cos|) w_feat / (P |F|^2).  Each element is held to
1e-5 (|a Fgt_i| + (2 + |cos|) |F_i| w_feat / (P |F|^2)) + 1e-6 |dL/dF_i|, a relative 1e-5 of
the terms' scale (gamma is 1.7e-6 at D = 768).  A bf16-stored dL/dF may further round by
one bf16 ulp of the oracle value.  The plain element-wise relative error (with a floor
of 1e-3 of the pixel's largest element) is reported beside it.  The oracle is given F
and Fgt exactly as stored (float32 or bf16, exact in FP64).  dL/dC, dL/dD: relative 1e-6;
the loss: relative 1e-5 (a float32 sum over the pixels in fixed order).
"""
import ctypes

import numpy as np
import pytest
import torch

import gs_scenes as S
import oracle
import parity_util as U

pytestmark = pytest.mark.gpu

W = (0.8, 0.6, 0.25)          # w_feat, w_rgb, w_depth


def _bf16_ulp(x):
    ax = np.abs(x)
    e = np.floor(np.log2(np.where(ax > 0, ax, 1.0)))
    return np.where(ax > 0, 2.0 ** (e - 7), 0.0)


def check_dF(dF_gpu, dF_or, F, G, P_total, w_feat, bf16):
    """Element-wise bound described in the module docstring; returns the worst ratio."""
    F, G = np.asarray(F, np.float64), np.asarray(G, np.float64)
    ff, gg = (F * F).sum(1, keepdims=True), (G * G).sum(1, keepdims=True)
    ok = (ff > 0) & (gg > 0)
    nfng = np.sqrt(np.where(ok, ff * gg, 1.0))
    cos = np.where(ok, (F * G).sum(1, keepdims=True) / nfng, 0.0)
    term = np.where(ok, w_feat / P_total * (np.abs(G) / nfng + (2 + np.abs(cos)) * np.abs(F) / np.where(ok, ff, 1.0)),
                    0.0)
    tol = 1e-5 * term + 1e-6 * np.abs(dF_or) + (_bf16_ulp(dF_or) if bf16 else 0.0) + 1e-30
    err = np.abs(np.asarray(dF_gpu, np.float64) - dF_or)
    ratio = float((err / tol).max()) if err.size else 0.0
    assert ratio <= 1.0, (ratio, np.unravel_index(np.argmax(err / tol), err.shape))
    # zero-norm pixels pass no gradient, exactly
    assert np.all(np.asarray(dF_gpu)[~ok[:, 0]] == 0.0)
    floor = 1e-3 * np.abs(dF_or).max(1, keepdims=True)
    elem = float((err / (np.abs(dF_or) + floor + 1e-30)).max()) if err.size else 0.0
    return ratio, elem


def _inputs(P, D, tdt, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    F = torch.randn(P, D, generator=g)
    Fgt = torch.randn(P, D, generator=g)
    # nearly parallel and nearly opposite pairs, and empty rows on either side
    F[10:20] = Fgt[10:20] * 3 + 1e-3 * torch.randn(10, D, generator=g)
    F[20:30] = -Fgt[20:30] * 0.5
    F[3] = 0
    Fgt[7] = 0
    F[11], Fgt[11] = 0, 0
    C, Cgt = torch.rand(P, 3, generator=g), torch.rand(P, 3, generator=g)
    Cgt[:50, 1] = C[:50, 1]                      # equal values: sign 0, no gradient
    Dp, Dgt = torch.rand(P, generator=g) * 4 + 1, torch.rand(P, generator=g) * 4 + 1
    Dgt[60:70] = Dp[60:70]
    dev = lambda t, dt=torch.float32: t.to("cuda", dt).contiguous()
    return dev(F, tdt), dev(Fgt, tdt), dev(C), dev(Cgt), dev(Dp), dev(Dgt)


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


def _compare(out, ins, P, D, bf16):
    F, Fgt, C, Cgt, Dp, Dgt = (_np(t) for t in ins)
    lo, dF, dC, dD = oracle.loss_cos_l1(F, Fgt, C, Cgt, Dp, Dgt, *W)
    dF_g, dC_g, dD_g, loss_g = out
    r, _ = check_dF(_np(dF_g), dF, F, Fgt, P, W[0], bf16)
    np.testing.assert_allclose(_np(dC_g), dC, rtol=1e-6, atol=0)
    np.testing.assert_allclose(_np(dD_g), dD, rtol=1e-6, atol=0)
    assert float(loss_g.item()) == pytest.approx(lo, rel=1e-5)
    return r


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("D", [16, 512, 768])
def test_loss_and_noalloc_match_oracle(dtype, D):
    """gs_loss_cos_l1 and gs_loss_cos_l1_noalloc on 5,003 pixels (not a multiple of any
    group or block size) with parallel, opposite and empty rows and L1 ties."""
    from paper_2602_06991_b300 import _abi as A, build
    build()
    lib = A.load()
    P = 5003
    bf16 = dtype == "bf16"
    tdt = torch.bfloat16 if bf16 else torch.float32
    cfg = A.GsConfig(8, D, 16, 16, A.GS_BF16 if bf16 else A.GS_F32, 0)
    ins = _inputs(P, D, tdt, seed=D)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    for noalloc in (False, True):
        out = (torch.empty(P, D, device="cuda", dtype=tdt), torch.empty(P, 3, device="cuda"),
               torch.empty(P, device="cuda"), torch.empty(1, device="cuda"))
        if noalloc:
            st = lib.gs_loss_cos_l1_noalloc(ctypes.byref(cfg), P, *map(p, ins), *W, *map(p, out), stream)
        else:
            scratch = torch.empty(int(lib.gs_loss_scratch_size(P)), dtype=torch.uint8, device="cuda")
            st = lib.gs_loss_cos_l1(ctypes.byref(cfg), P, *map(p, ins), *W, *map(p, out), p(scratch),
                                    scratch.numel(), stream)
        torch.cuda.synchronize()
        assert st == A.GS_OK
        r = _compare(out, ins, P, D, bf16)
        print(dtype, D, "noalloc" if noalloc else "scratch", "worst dF error / bound", r)


def _fused(sc, cams, K, dtype, seed):
    r, ts, out = U.gpu_forward(sc, cams, K, (16, 16), feat_dtype=dtype)
    Fgt, Cgt, Dgt = S.voronoi_targets(seed, cams, sc.d)
    Fgt = torch.from_numpy(Fgt).cuda().to(r.feat_torch_dtype).contiguous()
    Fgt[5] = 0                                       # an empty target row
    Cgt, Dgt = torch.from_numpy(Cgt).cuda(), torch.from_numpy(Dgt).cuda()
    lo = r.blend_loss(ts[4], Fgt, Cgt, Dgt, *W)
    torch.cuda.synchronize()
    return r, out, lo, (Fgt, Cgt, Dgt)


@pytest.mark.parametrize("case", ["small", "planes_f32_512", "planes_bf16_512", "ragged_bf16_768_k16"])
def test_fused_blend_loss_matches_oracle_full_frame(case):
    """gs_feature_blend_loss: the loss and its gradients at every pixel, against the oracle
    given the F the kernel stored (F itself is held to the oracle render elsewhere).
    Covers the per-pixel path (D = 16), the pixel-group path (float32 and bf16, K = 8),
    and K = 16 on two ragged views (groups of 2 straddling rows and the view boundary);
    pixels with no contributor (F = 0) and an empty target row."""
    if case == "small":
        sc, cams, K, _, dtype = S.make_config("small", 0)
    elif case == "ragged_bf16_768_k16":
        sc = S.random_scene_box(11, 2500, 768, box=((-1, 1), (-1, 1), (2, 4)))
        cams, K, dtype = S.orbit_cameras(5, [(37, 23, 40.0), (50, 41, 60.0)], radius=3.0), 16, "bf16"
    else:
        sc = S.planes_scene(7, 6000, 512)
        cams, K, dtype = [S.pinhole(160, 120, 131.25)], 8, case.split("_")[1]
    r, out, lo, (Fgt, Cgt, Dgt) = _fused(sc, cams, K, dtype, seed=3)
    P = r.P
    ins = (out["F"], Fgt, out["rgb"], Cgt, out["depth"], Dgt)
    ratio = _compare((lo["dL_dF"], lo["dL_dC"], lo["dL_dD"], lo["loss"]), ins, P, sc.d, dtype == "bf16")
    print(case, "worst dF error / bound", ratio)


@pytest.mark.parametrize("workload", ["frame", "batched"])
def test_fused_blend_loss_matches_oracle_at_workload_size(workload):
    """The benchmark's workloads at full size: the fused kernel's per-pixel gradients on
    sampled pixels of every view, and the scalar loss over all pixels (the oracle runs
    over the kernel's stored F in chunks of 65,536 pixels, summing their shares)."""
    sc, cams, K, tile, dtype = S.make_config(workload, 0)
    from paper_2602_06991_b300.renderer import TopKRenderer
    r = TopKRenderer(cams, K=K, D=sc.d, tile=tile, feat_dtype=dtype)
    ts = U.tensors(sc, dtype)
    out = r.forward(*ts)
    lab, fv, cv, dv = S.voronoi_sites(100, cams, sc.d)
    lab = torch.from_numpy(lab).cuda().long()
    Fgt = torch.from_numpy(fv).cuda().to(r.feat_torch_dtype)[lab].contiguous()
    Cgt = torch.from_numpy(cv).cuda()[lab].contiguous()
    Dgt = torch.from_numpy(dv).cuda()[lab].contiguous()
    del lab
    lo = r.blend_loss(ts[4], Fgt, Cgt, Dgt, *W)
    torch.cuda.synchronize()
    P = r.P
    rng = np.random.default_rng(9)
    pix = torch.from_numpy(np.sort(rng.choice(P, 4000, replace=False))).cuda()
    sel = lambda t: t.index_select(0, pix)
    F, G = _np(sel(out["F"])), _np(sel(Fgt))
    _, dF, dC, dD = oracle.loss_cos_l1(F, G, _np(sel(out["rgb"])), _np(sel(Cgt)), _np(sel(out["depth"])),
                                       _np(sel(Dgt)), *W, n_total=P)
    ratio, elem = check_dF(_np(sel(lo["dL_dF"])), dF, F, G, P, W[0], dtype == "bf16")
    np.testing.assert_allclose(_np(sel(lo["dL_dC"])), dC, rtol=1e-6, atol=0)
    np.testing.assert_allclose(_np(sel(lo["dL_dD"])), dD, rtol=1e-6, atol=0)
    total = 0.0
    for a in range(0, P, 65536):
        b = min(P, a + 65536)
        total += oracle.loss_cos_l1(_np(out["F"][a:b]), _np(Fgt[a:b]), _np(out["rgb"][a:b]), _np(Cgt[a:b]),
                                    _np(out["depth"][a:b]), _np(Dgt[a:b]), *W, n_total=P)[0]
    assert float(lo["loss"].item()) == pytest.approx(total, rel=1e-5)
    print(workload, "loss", float(lo["loss"].item()), "oracle", total, "worst dF error / bound", ratio,
          "element-wise relative", elem)
