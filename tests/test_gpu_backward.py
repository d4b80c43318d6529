"""GPU parity of the adjoint (a5) against the FP64 oracle gradient, through the C ABI.
Upstream gradients are zeroed at pixels the oracle flags (threshold decisions, Top-K
near-ties, the 0.99 clamp), on both sides, so both differentiate the same piecewise
branch; the bar is relative L2 <= 1e-4 per parameter group."""
import numpy as np
import pytest
import torch

import gs_scenes as S
import oracle
import parity_util as U

pytestmark = pytest.mark.gpu

GROUPS = [("feat", "feat"), ("opacity", "opac"), ("rgb", "rgb"), ("mean3d", "mean3d"), ("cov3d", "cov3d")]


def _upstream(cams, D, seed, fl, mask_pixels=None):
    P = sum(c.n_pix for c in cams)
    dF, dC, dD = S.upstream_grads(seed, P, D)
    keep = (fl & U.FRAGILE_ANY) == 0
    if mask_pixels is not None:
        keep &= mask_pixels
    dF[~keep] = 0
    dC[~keep] = 0
    dD[~keep] = 0
    return dF, dC, dD


def _oracle_grads(sc, cams, K, dF, dC, dD, pixels_per_cam=None):
    tot = None
    for i, (cam, off) in enumerate(U.cam_slices(cams)):
        pix = np.arange(cam.n_pix) if pixels_per_cam is None else np.asarray(pixels_per_cam[i])
        sl = off + pix
        g = oracle.backward(sc, cam, K, dF[sl], dC[sl], dD[sl], pixels=pix)
        if tot is None:
            tot = {k: v.copy() for k, v in g.items()}
            tot["mean2d_cams"] = [g["mean2d"]]
            tot["conic_cams"] = [g["conic"]]
        else:
            for k in ("feat", "opac", "rgb", "mean3d", "cov3d"):
                tot[k] += g[k]
            tot["mean2d_cams"].append(g["mean2d"])
            tot["conic_cams"].append(g["conic"])
    return tot


def _check(r, sc, cams, K, dF, dC, dD, og, with_2d=True):
    dev = "cuda"
    gg = r.backward(torch.from_numpy(dF).to(dev).to(r.feat_torch_dtype), torch.from_numpy(dC).to(dev),
                    torch.from_numpy(dD).to(dev), with_2d=with_2d)
    torch.cuda.synchronize()
    errs = {}
    for gk, ok in GROUPS:
        errs[gk] = U.rel_l2(gg[gk].cpu().numpy(), og[ok])
    if with_2d:
        errs["mean2d"] = U.rel_l2(gg["mean2d"].cpu().numpy(), np.stack(og["mean2d_cams"]))
        errs["conic"] = U.rel_l2(gg["conic"].cpu().numpy(), np.stack(og["conic_cams"]))
    print("grad rel-L2", errs)
    for k, e in errs.items():
        assert e <= U.GRAD_TOL, (k, e, errs)
    return gg


def test_small_backward_parity():
    sc, cams, K, tile, _ = S.make_config("small", 0)
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    o = U.oracle_forward(sc, cams, K)
    dF, dC, dD = _upstream(cams, sc.d, 1, o["flags"])
    og = _oracle_grads(sc, cams, K, dF, dC, dD)
    _check(r, sc, cams, K, dF, dC, dD, og)


def test_backward_deterministic():
    sc, cams, K, tile, _ = S.make_config("small", 3)
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    P = cams[0].n_pix
    dF, dC, dD = (torch.from_numpy(a).cuda() for a in S.upstream_grads(2, P, sc.d))
    g1 = {k: v.clone() for k, v in r.backward(dF, dC, dD, with_2d=True).items()}
    g2 = r.backward(dF, dC, dD, with_2d=True)
    for k in g1:
        assert torch.equal(g1[k], g2[k]), k


@pytest.mark.parametrize("K,tile", [(1, (16, 16)), (8, (32, 8)), (16, (8, 8))])
def test_backward_k_and_tiles(K, tile):
    sc, cams, _, _, _ = S.make_config("small", 4)
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    o = U.oracle_forward(sc, cams, K)
    dF, dC, dD = _upstream(cams, sc.d, 5, o["flags"])
    og = _oracle_grads(sc, cams, K, dF, dC, dD)
    _check(r, sc, cams, K, dF, dC, dD, og)


def test_backward_multi_camera_general_poses():
    sc = S.random_scene_box(6, 2500, 24, box=((-1, 1), (-1, 1), (2, 4)))
    cams = S.orbit_cameras(8, [(90, 70, 80.0), (64, 48, 50.0)], radius=3.0)
    r, ts, out = U.gpu_forward(sc, cams, 6, (16, 16))
    o = U.oracle_forward(sc, cams, 6)
    dF, dC, dD = _upstream(cams, sc.d, 7, o["flags"])
    og = _oracle_grads(sc, cams, 6, dF, dC, dD)
    _check(r, sc, cams, 6, dF, dC, dD, og)


def test_backward_crop_1k():
    """The 1k-Gaussian crop of the 'frame' scene (nearest to the optical axis), 640x480,
    D=512, K=8, full frame."""
    sc, cams, K, tile, _ = S.make_config("frame", 0)
    sc = S.crop_scene(sc, cams[0], 1000)
    cams = [S.pinhole(128, 128, 525.0 * 0.2, cx=64, cy=64)]
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    o = U.oracle_forward(sc, cams, K)
    dF, dC, dD = _upstream(cams, sc.d, 11, o["flags"])
    og = _oracle_grads(sc, cams, K, dF, dC, dD)
    _check(r, sc, cams, K, dF, dC, dD, og)


def test_frame_workload_sampled_backward():
    """Full 'frame' workload in the benchmark's launch configuration: upstream gradients
    are non-zero only at 192 seeded pixels, so the oracle can compute the exact
    per-Gaussian gradients from those pixels alone."""
    sc, cams, K, tile, _ = S.make_config("frame", 0)
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    rng = np.random.default_rng(1)
    P = cams[0].n_pix
    pix = np.sort(rng.choice(P, 192, replace=False))
    o = U.oracle_forward(sc, cams, K, pixels_per_cam=[pix])
    flags = np.full(P, U.FRAGILE_ANY, dtype=np.int64)
    flags[pix] = o["flags"]
    dF, dC, dD = _upstream(cams, sc.d, 3, flags)
    og = _oracle_grads(sc, cams, K, dF, dC, dD, pixels_per_cam=[pix])
    _check(r, sc, cams, K, dF, dC, dD, og, with_2d=False)


def test_autograd_function_matches_direct_calls():
    from paper_2602_06991_b300.renderer import TopKRenderer, render
    sc, cams, K, tile, _ = S.make_config("small", 9)
    r = TopKRenderer(cams, K=K, D=sc.d, tile=tile)
    ts = [t.clone().requires_grad_(True) for t in U.tensors(sc)]
    F, C, Dp = render(r, *ts)
    P = cams[0].n_pix
    dF, dC, dD = (torch.from_numpy(a).cuda() for a in S.upstream_grads(4, P, sc.d))
    ((F * dF).sum() + (C * dC).sum() + (Dp * dD).sum()).backward()
    r2, _, _ = U.gpu_forward(sc, cams, K, tile)
    g = r2.backward(dF, dC, dD)
    for t, k in zip(ts, ["mean3d", "cov3d", "opacity", "rgb", "feat"]):
        assert torch.equal(t.grad, g[k]), k


@pytest.mark.parametrize("D,K,dtype", [(1024, 5, "f32"), (768, 16, "bf16"), (136, 32, "f32")])
def test_backward_feature_block_shapes(D, K, dtype):
    """Feature-gradient blocks of every shape and TMA column count: float32 D=1024
    (4x4 blocks, four 256-column boxes), bf16 D=768 K=16 (8x4 blocks, three boxes), and
    D=136 K=32 (a box narrower than 256 columns); two ragged cameras whose blocks run
    past the image edges.  Against the oracle gradient (bf16: the oracle takes the
    bf16-rounded rows and upstream feature gradients)."""
    sc = S.random_scene_box(12, 1500, D, box=((-1, 1), (-1, 1), (2, 4)))
    cams = S.orbit_cameras(13, [(45, 29, 50.0), (38, 31, 45.0)], radius=3.0)
    r, ts, out = U.gpu_forward(sc, cams, K, (16, 16), feat_dtype=dtype)
    feats = None
    if dtype == "bf16":
        feats = torch.from_numpy(sc.feats).to(torch.bfloat16).float().numpy()
    o = U.oracle_forward(sc, cams, K, feats=feats)
    dF, dC, dD = _upstream(cams, sc.d, 14, o["flags"])
    dF_t = torch.from_numpy(dF).cuda().to(r.feat_torch_dtype)
    dF_exact = dF_t.float().cpu().numpy().astype(np.float64)
    gg = r.backward(dF_t, torch.from_numpy(dC).cuda(), torch.from_numpy(dD).cuda())
    torch.cuda.synchronize()
    tot = None
    for i, (cam, off) in enumerate(U.cam_slices(cams)):
        sl = slice(off, off + cam.n_pix)
        g = oracle.backward(sc, cam, K, dF_exact[sl], dC[sl], dD[sl], feats=feats)
        if tot is None:
            tot = {k: v.copy() for k, v in g.items()}
        else:
            for k in ("feat", "opac", "rgb", "mean3d", "cov3d"):
                tot[k] += g[k]
    errs = {gk: U.rel_l2(gg[gk].cpu().numpy(), tot[ok]) for gk, ok in GROUPS}
    print("block shapes", D, K, dtype, errs)
    for k, e in errs.items():
        assert e <= U.GRAD_TOL, (k, e, errs)


@pytest.mark.parametrize("case", ["small_f32", "bf16_groups", "per_pixel_path"])
def test_backward_reuses_loss_h(case):
    """gs_backward_ex with GS_BWD_H_FROM_LOSS reuses the per-slot h = dL/dF . f that the
    fused blend + loss left in the workspace; the gradients are bit-identical to the
    call that recomputes h from dL_dF.  'per_pixel_path' (K = 32) takes the blend path
    that writes no h, so the flag must fall back to recomputing it.  A dL_dF other than
    the loss's own is refused by the binding."""
    if case == "small_f32":
        sc, cams, K, tile, _ = S.make_config("small", 5)
        dtype = "f32"
    else:
        D, K, dtype = (768, 16, "bf16") if case == "bf16_groups" else (136, 32, "f32")
        sc = S.random_scene_box(21, 1500, D, box=((-1, 1), (-1, 1), (2, 4)))
        cams = S.orbit_cameras(22, [(45, 29, 50.0), (38, 31, 45.0)], radius=3.0)
        tile = (16, 16)
    # capacity for the partial feature rows up front, so no retry replaces the workspace
    r, ts, out = U.gpu_forward(sc, cams, K, tile, feat_dtype=dtype, max_instances=256 * len(cams) * sc.n)
    P = sum(c.n_pix for c in cams)
    g = torch.Generator().manual_seed(23)
    F_gt = torch.randn(P, sc.d, generator=g).cuda().to(r.feat_torch_dtype)
    C_gt = torch.rand(P, 3, generator=g).cuda()
    D_gt = (2 + 2 * torch.rand(P, generator=g)).cuda()
    lo = r.blend_loss(ts[4], F_gt, C_gt, D_gt)
    ga = {k: v.clone() for k, v in r.backward(lo["dL_dF"], lo["dL_dC"], lo["dL_dD"], with_2d=True).items()}
    assert r._h_valid, "a capacity retry replaced the workspace"
    gb = r.backward(lo["dL_dF"], lo["dL_dC"], lo["dL_dD"], with_2d=True, h_from_loss=True)
    torch.cuda.synchronize()
    for k in ga:
        assert torch.equal(ga[k], gb[k]), k
    assert float(ga["feat"].abs().sum()) > 0 and float(ga["opacity"].abs().sum()) > 0
    with pytest.raises(ValueError):
        r.backward(lo["dL_dF"].clone(), lo["dL_dC"], lo["dL_dD"], h_from_loss=True)


def test_slot_sort_fallback_matches_warp_path():
    """Scenes of 2^22 Gaussians or more take the shared-memory slot sort (64-bit keys)
    instead of the warp form (32-bit keys).  The 'small' scene is rendered alone and
    again with 2^22 culled Gaussians (behind the camera) appended after it: the visible
    Gaussians keep their ids, so the two paths must give bit-identical gradients for
    them, and zero for the appended ones."""
    sc, cams, K, tile, _ = S.make_config("small", 6)
    n0, extra = sc.n, (1 << 22) + 16 - sc.n
    rng = np.random.default_rng(7)
    far = S.Scene(mean3d=np.concatenate([sc.mean3d, np.column_stack(
                      [rng.uniform(-1, 1, extra), rng.uniform(-1, 1, extra), rng.uniform(-6, -2, extra)])]).astype(np.float32),
                  cov3d=np.concatenate([sc.cov3d, np.tile(sc.cov3d[:1], (extra, 1))]).astype(np.float32),
                  opacity=np.concatenate([sc.opacity, np.full(extra, 0.5, np.float32)]),
                  rgb=np.concatenate([sc.rgb, np.full((extra, 3), 0.5, np.float32)]),
                  feats=np.concatenate([sc.feats, np.tile(sc.feats[:1], (extra, 1))]).astype(np.float32))
    assert far.n >= (1 << 22)
    P = cams[0].n_pix
    dF, dC, dD = (torch.from_numpy(a).cuda() for a in S.upstream_grads(8, P, sc.d))
    grads = []
    for scene in (sc, far):
        r, ts, out = U.gpu_forward(scene, cams, K, tile, max_instances=1 << 20)
        g = r.backward(dF, dC, dD, with_2d=True)
        torch.cuda.synchronize()
        grads.append({k: v.clone() for k, v in g.items()})
        del r, ts, out, g
    a, b = grads
    for k in ("feat", "opacity", "rgb", "mean3d", "cov3d"):
        assert torch.equal(a[k], b[k][:n0]), k
        assert float(b[k][n0:].abs().max()) == 0.0, k
    for k in ("mean2d", "conic"):
        assert torch.equal(a[k], b[k][:, :n0]), k
    assert float(a["feat"].abs().sum()) > 0
