"""GPU parity of the BF16-row form and the multi-view batched form at their workload
sizes, against the FP64 oracle on sampled pixels.

BF16 form: feature rows, F and dL/dF are stored in bf16; weights, transmittance and
all accumulation stay float32.  The oracle is given the bf16-rounded rows and
upstream gradients (exact in FP64), so contributor sets and gradients are held to the
float32 bars, and F to per-pixel cosine >= 0.999 (its bf16 storage rounds it)."""
import numpy as np
import pytest
import torch

import gs_scenes as S
import oracle
import parity_util as U

pytestmark = pytest.mark.gpu


def _bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).float().numpy()


def _cosine_check(g, o, ok):
    Fg, Fo = g["F"][ok].astype(np.float64), o["F"][ok]
    nz = np.linalg.norm(Fo, axis=1) > 0
    cos = (Fg[nz] * Fo[nz]).sum(1) / (np.linalg.norm(Fg[nz], axis=1) * np.linalg.norm(Fo[nz], axis=1))
    return float(cos.min()) if cos.size else 1.0


def _sampled_backward(r, sc, cams, K, pix_per_cam, feats_exact, seed):
    """GPU backward with upstream gradients only at the sampled non-flagged pixels, and
    the oracle gradient from those pixels alone."""
    P = sum(c.n_pix for c in cams)
    o = U.oracle_forward(sc, cams, K, pixels_per_cam=pix_per_cam, feats=feats_exact)
    flags = np.full(P, U.FRAGILE_ANY, dtype=np.int64)
    flags[o["gidx"]] = o["flags"]
    dF, dC, dD = S.upstream_grads(seed, P, sc.d)
    keep = (flags & U.FRAGILE_ANY) == 0
    dF[~keep] = 0; dC[~keep] = 0; dD[~keep] = 0
    dF_t = torch.from_numpy(dF).cuda().to(r.feat_torch_dtype)
    dF_exact = dF_t.float().cpu().numpy()
    g = r.backward(dF_t, torch.from_numpy(dC).cuda(), torch.from_numpy(dD).cuda())
    torch.cuda.synchronize()
    tot = None
    for i, (cam, off) in enumerate(U.cam_slices(cams)):
        pix = np.asarray(pix_per_cam[i])
        sl = off + pix
        og = oracle.backward(sc, cam, K, dF_exact[sl], dC[sl], dD[sl], pixels=pix, feats=feats_exact)
        if tot is None:
            tot = og
        else:
            for k in ("feat", "opac", "rgb", "mean3d", "cov3d"):
                tot[k] += og[k]
    errs = {gk: U.rel_l2(g[gk].cpu().numpy(), tot[ok]) for gk, ok in
            [("feat", "feat"), ("opacity", "opac"), ("rgb", "rgb"), ("mean3d", "mean3d"), ("cov3d", "cov3d")]}
    return errs, o


def test_bf16_1m_sampled_forward_and_backward():
    """'frame_1m_bf16': 1M Gaussians, 640x480, D=512 bf16, K=8."""
    sc, cams, K, tile, fdt = S.make_config("frame_1m_bf16", 0)
    r, ts, out = U.gpu_forward(sc, cams, K, tile, feat_dtype="bf16")
    feats_exact = _bf16_round(sc.feats)
    rng = np.random.default_rng(3)
    pix = [np.sort(rng.choice(cams[0].n_pix, 160, replace=False))]
    errs, o = _sampled_backward(r, sc, cams, K, pix, feats_exact, seed=5)
    g = U.to_np(out)
    ok = (o["flags"] & U.FRAGILE_SET) == 0
    assert np.array_equal(g["n_contrib"][o["gidx"]][ok], o["n"][ok])
    sets_ok = ok & ((o["flags"] & oracle.F_NEAR_TIE) == 0)
    gi = np.sort(g["topk_idx"][o["gidx"]][sets_ok], axis=1)
    assert np.array_equal(gi, np.sort(o["idx"][sets_ok], axis=1))
    cmin = _cosine_check({"F": g["F"][o["gidx"]]}, o, ok)
    # the form's bar: per-pixel cosine against FP64 on the original float32 rows
    o32 = U.oracle_forward(sc, cams, K, pixels_per_cam=pix)
    cmin32 = _cosine_check({"F": g["F"][o["gidx"]]}, o32, ok)
    print("bf16 1M: cos min (bf16 rows)", cmin, "(f32 rows)", cmin32, "grad rel-L2", errs,
          "flagged", int((~ok).sum()), "of", ok.size, "near-ties", int((ok & ~sets_ok).sum()))
    assert cmin >= 0.999 and cmin32 >= 0.999
    for k, e in errs.items():
        assert e <= U.GRAD_TOL, (k, e)


def test_batched_views_sampled_forward_and_backward():
    """'batched': 8 orbit keyframes (3x640x480, 3x1200x680, 2x320x240) of a 1M-Gaussian
    scene in one flat pixel space, bf16 rows, K=8 -- per view against the oracle."""
    sc, cams, K, tile, fdt = S.make_config("batched", 0)
    r, ts, out = U.gpu_forward(sc, cams, K, tile, feat_dtype="bf16")
    feats_exact = _bf16_round(sc.feats)
    rng = np.random.default_rng(4)
    pix = [np.sort(rng.choice(c.n_pix, 24, replace=False)) for c in cams]
    errs, o = _sampled_backward(r, sc, cams, K, pix, feats_exact, seed=6)
    g = U.to_np(out)
    ok = (o["flags"] & U.FRAGILE_SET) == 0
    assert np.array_equal(g["n_contrib"][o["gidx"]][ok], o["n"][ok])
    np.testing.assert_allclose(g["T"][o["gidx"]][ok], o["T"][ok], rtol=1e-5, atol=1e-7)
    cmin = _cosine_check({"F": g["F"][o["gidx"]]}, o, ok)
    o32 = U.oracle_forward(sc, cams, K, pixels_per_cam=pix)
    cmin32 = _cosine_check({"F": g["F"][o["gidx"]]}, o32, ok)
    print("batched: cos min (bf16 rows)", cmin, "(f32 rows)", cmin32, "grad rel-L2", errs, "flagged",
          int((~ok).sum()), "of", ok.size)
    assert cmin >= 0.999 and cmin32 >= 0.999
    for k, e in errs.items():
        assert e <= U.GRAD_TOL, (k, e)


def test_autotuner_picks_a_compiled_shape_and_caches(tmp_path):
    from paper_2602_06991_b300 import autotune
    from paper_2602_06991_b300.renderer import TopKRenderer
    sc, cams, K, tile, _ = S.make_config("small", 0)
    ts = U.tensors(sc)

    def factory(shape, layout):
        r = TopKRenderer(cams, K=K, D=sc.d, tile=shape, topk_layout=layout)
        r.forward(*ts)
        r.check_overflow = False
        return lambda: r.forward(*ts)

    path = str(tmp_path / "tune.json")
    res = autotune.tune(cams, sc.n, K, sc.d, "f32", factory, cache_path=path)
    assert tuple(res["tile"]) in autotune.TILE_SHAPES and res["layout"] in autotune.KBUF_LAYOUTS
    assert not res["cached"]
    assert len(res["ms"]) == len(autotune.TILE_SHAPES) * len(autotune.KBUF_LAYOUTS)
    again = autotune.tune(cams, sc.n, K, sc.d, "f32", factory, cache_path=path)
    assert again["cached"] and tuple(again["tile"]) == tuple(res["tile"]) and again["layout"] == res["layout"]
