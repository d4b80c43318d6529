"""GPU parity of the vanilla (full alpha-blending) feature render -- the baseline of
Tab. 4 -- against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import gs_scenes as S
import oracle
import parity_util as U

pytestmark = pytest.mark.gpu


def _check(F_gpu, ov, bf16=False):
    ok = (ov["flags"] & U.FRAGILE_SET) == 0
    Fg, Fo = F_gpu[ok].astype(np.float64), ov["F"][ok]
    if bf16:
        nz = np.linalg.norm(Fo, axis=1) > 1e-6
        cos = (Fg[nz] * Fo[nz]).sum(1) / (np.linalg.norm(Fg[nz], axis=1) * np.linalg.norm(Fo[nz], axis=1))
        assert cos.min() >= 0.999, cos.min()
        return float(cos.min())
    err = np.abs(Fg - Fo).max(1) / np.maximum(np.linalg.norm(Fo, axis=1), 1e-3)
    assert err.max() <= U.F_TOL, err.max()
    return float(err.max())


def test_vanilla_small_full_frame():
    sc, cams, K, tile, _ = S.make_config("small", 0)
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    F = r.forward_vanilla(ts[4])
    torch.cuda.synchronize()
    print("small vanilla", _check(F.cpu().numpy(), oracle.render_vanilla(sc, cams[0])))


@pytest.mark.parametrize("D,dtype,tile", [(136, "f32", (16, 8)), (256, "bf16", (32, 8)), (24, "f32", (8, 8))])
def test_vanilla_ragged_cameras_and_widths(D, dtype, tile):
    """Two ragged cameras; a width that is not a multiple of the 64-column pass (136 =
    64 + 64 + 8), bf16 rows, and every tile shape."""
    sc = S.random_scene_box(17, 2500, D, box=((-1, 1), (-1, 1), (2, 4)))
    cams = S.orbit_cameras(18, [(45, 29, 50.0), (38, 31, 45.0)], radius=3.0)
    r, ts, out = U.gpu_forward(sc, cams, 6, tile, feat_dtype=dtype)
    F = r.forward_vanilla(ts[4]).float().cpu().numpy()
    for cam, off in U.cam_slices(cams):
        _check(F[off:off + cam.n_pix], oracle.render_vanilla(sc, cam), bf16=dtype == "bf16")


def test_vanilla_is_scaled_full_topk_on_gpu():
    """Where K is at least the pixel's contributor count, the Top-K feature is the
    vanilla one divided by 1 - T_final (Eq. 3 renormalises the full blend)."""
    sc = S.random_scene_box(19, 400, 32, box=((-1, 1), (-1, 1), (1.5, 4)), log_scale_mu=-2.5)
    cams = [S.pinhole(48, 40, 50.0)]
    r, ts, out = U.gpu_forward(sc, cams, 32, (16, 16))
    Fv = r.forward_vanilla(ts[4])
    all_in = out["n_contrib"] <= 32
    assert all_in.float().mean() > 0.5
    has = (out["n_contrib"] > 0) & all_in
    want = out["F"][has] * (1 - out["T"][has, None])
    torch.testing.assert_close(Fv[has], want, rtol=2e-5, atol=1e-6)
    assert torch.all(Fv[out["n_contrib"] == 0] == 0)


def test_vanilla_frame_sampled_pixels():
    """'frame' workload (200k Gaussians, 640x480, D=512, ~180 contributors per pixel):
    256 seeded pixels against the oracle."""
    sc, cams, K, tile, _ = S.make_config("frame", 0)
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    F = r.forward_vanilla(ts[4]).cpu().numpy()
    pix = np.sort(np.random.default_rng(2).choice(cams[0].n_pix, 256, replace=False))
    print("frame vanilla", _check(F[pix], oracle.render_vanilla(sc, cams[0], pixels=pix)))
