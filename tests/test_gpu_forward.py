"""GPU parity of the forward path (a1-a4) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import gs_scenes as S
import oracle
import parity_util as U

pytestmark = pytest.mark.gpu


def test_small_full_frame_parity():
    """2,000 Gaussians, 128x96, D=16, K=4: every pixel against the oracle."""
    sc, cams, K, tile, _ = S.make_config("small", 0)
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    g = U.to_np(out)
    o = U.oracle_forward(sc, cams, K)
    st = U.compare_forward(g, o, K)
    print("small", st)


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (16, 8), (8, 8)])
@pytest.mark.parametrize("layout", [0, 1, 2])
@pytest.mark.parametrize("K", [4, 16])
def test_tile_shape_and_kbuf_layout_independence(tile, layout, K):
    """The contributor set is defined per pixel, so every tile shape gives bit-identical
    outputs, and so does every K-buffer layout of the walk (registers, shared memory with
    per-thread insertion, shared memory with warp-level insertion); all match the oracle."""
    from paper_2602_06991_b300.renderer import TopKRenderer
    sc, cams, _, _, _ = S.make_config("small", 1)
    _, ts, ref = U.gpu_forward(sc, cams, K, (16, 16))
    r = TopKRenderer(cams, K=K, D=sc.d, tile=tile, topk_layout=layout)
    out = r.forward(*ts)
    torch.cuda.synchronize()
    for k in ("rgb", "depth", "T", "n_contrib", "topk_idx", "topk_w", "F"):
        assert torch.equal(ref[k], out[k]), k
    U.compare_forward(U.to_np(out), U.oracle_forward(sc, cams, K), K)


@pytest.mark.parametrize("K", [3, 8, 16])
def test_kbuf_layouts_identical_on_frame(K):
    """'frame' (every pixel saturates after ~180 contributors, many Top-K replacements):
    the three K-buffer layouts give bit-identical forward outputs."""
    from paper_2602_06991_b300.renderer import TopKRenderer
    sc, cams, _, tile, _ = S.make_config("frame", 0)
    ts = U.tensors(sc)
    outs = []
    for layout in (0, 1, 2):
        r = TopKRenderer(cams, K=K, D=sc.d, tile=tile, topk_layout=layout)
        o = r.forward(*ts)
        torch.cuda.synchronize()
        outs.append({k: o[k].clone() for k in ("rgb", "depth", "T", "n_contrib", "topk_idx", "topk_w", "F")})
        del r, o
    for o in outs[1:]:
        for k in outs[0]:
            assert torch.equal(outs[0][k], o[k]), k


@pytest.mark.parametrize("K", [1, 3, 5, 8, 10, 16, 32])
def test_k_values(K):
    sc, cams, _, tile, _ = S.make_config("small", 2)
    _, _, out = U.gpu_forward(sc, cams, K, tile)
    o = U.oracle_forward(sc, cams, K, pixels_per_cam=[np.arange(0, cams[0].n_pix, 3)])
    U.compare_forward(U.to_np(out), o, K)


@pytest.mark.parametrize("D", [8, 24, 136, 512, 1024])
def test_feature_widths(D):
    sc = S.random_scene_box(3, 1500, D)
    cams = [S.pinhole(96, 64, 80.0)]
    _, _, out = U.gpu_forward(sc, cams, 6)
    o = U.oracle_forward(sc, cams, 6, pixels_per_cam=[np.arange(0, cams[0].n_pix, 5)])
    U.compare_forward(U.to_np(out), o, 6)


def test_ragged_multi_camera_general_poses():
    """Three cameras of uneven, non-tile-multiple sizes on an orbit (general rotations):
    one flat pixel space, each camera against the oracle."""
    sc = S.random_scene_box(4, 3000, 32, box=((-1, 1), (-1, 1), (2, 4)))
    cams = S.orbit_cameras(7, [(100, 75, 90.0), (64, 48, 50.0), (131, 97, 120.0)], radius=3.0)
    _, _, out = U.gpu_forward(sc, cams, 8, (16, 8))
    o = U.oracle_forward(sc, cams, 8)
    st = U.compare_forward(U.to_np(out), o, 8)
    print("multi", st)


def test_empty_and_degenerate_scenes():
    cams = [S.pinhole(40, 30, 40.0)]
    # N = 0
    sc0 = S.random_scene_box(0, 0, 8)
    _, _, out = U.gpu_forward(sc0, cams, 4)
    assert torch.all(out["T"] == 1) and torch.all(out["topk_idx"] == -1) and torch.all(out["F"] == 0)
    assert torch.all(out["n_contrib"] == 0)
    # everything behind the camera or below the opacity floor
    sc = S.random_scene_box(1, 50, 8)
    sc.mean3d[:, 2] = -sc.mean3d[:, 2]
    _, _, out = U.gpu_forward(sc, cams, 4)
    assert torch.all(out["n_contrib"] == 0) and torch.all(out["F"] == 0)
    sc = S.random_scene_box(1, 50, 8)
    sc.opacity[:] = 1e-3
    _, _, out = U.gpu_forward(sc, cams, 4)
    assert torch.all(out["n_contrib"] == 0)
    # a single Gaussian
    sc = S.random_scene_box(2, 1, 8, box=((0, 0), (0, 0), (2, 2)), log_scale_mu=-2.0)
    _, _, out = U.gpu_forward(sc, cams, 4)
    U.compare_forward(U.to_np(out), U.oracle_forward(sc, cams, 4), 4)


def test_overflow_reported_and_recovered():
    """A too-small instance capacity is reported as GS_ERR_OVERFLOW by the device error
    word; the binding then grows the capacity and renders correctly."""
    from paper_2602_06991_b300 import _abi as A
    from paper_2602_06991_b300.renderer import TopKRenderer
    sc, cams, K, tile, _ = S.make_config("small", 0)
    r = TopKRenderer(cams, K=K, D=sc.d, tile=tile, max_instances=4096, check_overflow=False)
    out = r.forward(*U.tensors(sc))
    st, m = r.sync_status()
    assert st == A.GS_ERR_OVERFLOW and m > 4096
    r.check_overflow = True
    out = r.forward(*U.tensors(sc))
    U.compare_forward(U.to_np(out), U.oracle_forward(sc, cams, K), K)


def test_frame_workload_sampled_pixels():
    """The full 'frame' workload (200k Gaussians on planes, 640x480, D=512, K=8) in the
    launch configuration the benchmark times; 384 seeded pixels against the oracle."""
    sc, cams, K, tile, _ = S.make_config("frame", 0)
    _, _, out = U.gpu_forward(sc, cams, K, tile)
    rng = np.random.default_rng(0)
    pix = np.sort(rng.choice(cams[0].n_pix, 384, replace=False))
    o = U.oracle_forward(sc, cams, K, pixels_per_cam=[pix])
    st = U.compare_forward(U.to_np(out), o, K)
    print("frame", st)
    # invariants over every pixel
    w = out["topk_w"]
    assert torch.all(w >= 0) and torch.all(w <= 1)
    assert torch.all(w[:, :-1] >= w[:, 1:])
    nrm = out["F"].norm(dim=1)
    assert torch.all(nrm <= 1 + 1e-5)


def test_bf16_rows_cosine():
    """BF16 feature rows and BF16 F: per-pixel cosine >= 0.999 against the FP64 oracle
    with the float32 rows; index sets as in float32."""
    sc, cams, K, tile, _ = S.make_config("small", 5)
    _, _, out = U.gpu_forward(sc, cams, K, tile, feat_dtype="bf16")
    o = U.oracle_forward(sc, cams, K)
    g = U.to_np(out)
    ok = (o["flags"] & U.FRAGILE_SET) == 0
    Fg, Fo = g["F"][ok].astype(np.float64), o["F"][ok]
    nz = np.linalg.norm(Fo, axis=1) > 0
    cos = (Fg[nz] * Fo[nz]).sum(1) / (np.linalg.norm(Fg[nz], axis=1) * np.linalg.norm(Fo[nz], axis=1))
    assert cos.min() >= 0.999, cos.min()
    assert np.array_equal(g["n_contrib"][ok], o["n"][ok])


@pytest.mark.parametrize("dtype,D", [("f32", 512), ("f32", 24), ("bf16", 64)])
def test_fused_blend_loss_matches_separate_calls(dtype, D):
    """gs_feature_blend_loss gives the same F, loss gradients and loss as
    gs_feature_blend followed by gs_loss_cos_l1."""
    sc = S.planes_scene(7, 6000, D) if D >= 64 else S.random_scene_box(7, 3000, D)
    cams = [S.pinhole(100, 75, 90.0)] if D < 512 else [S.pinhole(160, 120, 131.25)]
    r, ts, out = U.gpu_forward(sc, cams, 8, (16, 16), feat_dtype=dtype)
    Fgt, Cgt, Dgt = (torch.from_numpy(a).cuda() for a in S.voronoi_targets(3, cams, D))
    Fgt = Fgt.to(r.feat_torch_dtype).contiguous()
    sep = r.loss(out["F"], Fgt, out["rgb"], Cgt, out["depth"], Dgt, 1.0, 0.5, 0.25)
    F_sep = out["F"].clone()
    out["F"].zero_()
    fused = r.blend_loss(ts[4], Fgt, Cgt, Dgt, 1.0, 0.5, 0.25)
    torch.cuda.synchronize()
    assert torch.equal(out["F"], F_sep)
    # float32 values agree to summation order; bf16-stored dL/dF may round one ulp apart
    rt = 2.0 ** -7 if dtype == "bf16" else 1e-5
    for k in ("dL_dF", "dL_dC", "dL_dD"):
        torch.testing.assert_close(fused[k].float(), sep[k].float(), rtol=rt if k == "dL_dF" else 1e-5, atol=1e-9)
    torch.testing.assert_close(fused["loss"], sep["loss"], rtol=1e-6, atol=0)


@pytest.mark.parametrize("K,D,dtype", [(3, 256, "f32"), (12, 512, "f32"), (16, 1024, "bf16"), (8, 256, "bf16")])
def test_pixel_group_blend_forms(K, D, dtype):
    """The pixel-group gather-blend (a warp shares the distinct rows of G consecutive
    pixels) at K <= 4, 8, 16 and both row types, on two ragged cameras whose pixel
    counts are not multiples of G, so groups straddle image rows and the camera
    boundary.  F against the oracle; the fused blend+loss gives bit-identical F."""
    sc = S.random_scene_box(11, 2500, D, box=((-1, 1), (-1, 1), (2, 4)))
    cams = S.orbit_cameras(5, [(37, 23, 40.0), (50, 41, 60.0)], radius=3.0)
    r, ts, out = U.gpu_forward(sc, cams, K, (16, 16), feat_dtype=dtype)
    o = U.oracle_forward(sc, cams, K)
    g = U.to_np(out)
    if dtype == "f32":
        U.compare_forward(g, o, K)
    else:
        ok = (o["flags"] & U.FRAGILE_SET) == 0
        Fg, Fo = g["F"][o["gidx"]][ok].astype(np.float64), o["F"][ok]
        nz = np.linalg.norm(Fo, axis=1) > 0
        cos = (Fg[nz] * Fo[nz]).sum(1) / (np.linalg.norm(Fg[nz], axis=1) * np.linalg.norm(Fo[nz], axis=1))
        assert cos.min() >= 0.999, cos.min()
    Fgt, Cgt, Dgt = (torch.from_numpy(a).cuda() for a in S.voronoi_targets(3, cams, D))
    Fgt = Fgt.to(r.feat_torch_dtype).contiguous()
    F_sep = out["F"].clone()
    out["F"].zero_()
    r.blend_loss(ts[4], Fgt, Cgt, Dgt, 1.0, 0.5, 0.25)
    torch.cuda.synchronize()
    assert torch.equal(out["F"], F_sep)
