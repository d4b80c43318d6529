"""Depth-cut binning (gs_config.depth_cut): a workspace that carries per-tile depth cuts
from one render to the next sorts only the instances in front of them, and completes
within the render every tile that the shorter list leaves unsaturated.  Every output --
the forward's colour, depth, transmittance, contributor counts and Top-K, and every
gradient of the adjoint -- must be bit-identical to a renderer that sorts every
instance, on the first render (no cut recorded yet) and on later renders of a changed
scene (opacities lowered, so tiles saturate deeper and must be completed, then raised,
and the means moved)."""
import pytest
import torch

import gs_scenes as S
import parity_util as U
from paper_2602_06991_b300.renderer import TopKRenderer

pytestmark = pytest.mark.gpu

FWD_KEYS = ("proj", "rgb", "depth", "T", "n_contrib", "topk_idx", "topk_w", "F")
GRAD_KEYS = ("feat", "opacity", "rgb", "mean3d", "cov3d")


def _variants(ts, seed):
    """The scene as given, then three changed scenes (float32 tensors on the device)."""
    mean, cov, opac, rgb, feats = ts
    g = torch.Generator(device="cuda").manual_seed(seed)
    moved = (mean + 0.02 * torch.randn(mean.shape, generator=g, device="cuda")).contiguous()
    return [
        list(ts),
        [mean, cov, (opac * 0.55).contiguous(), rgb, feats],          # saturate deeper: completions
        [moved, cov, (opac * 0.55).contiguous(), rgb, feats],
        [moved, cov, (opac * 1.4).clamp(max=0.999).contiguous(), rgb, feats],   # saturate earlier
    ]


def _render(r, t, up):
    out = r.forward(*t)
    g = r.backward(*up)
    torch.cuda.synchronize()
    return ({k: out[k].clone() for k in FWD_KEYS}, {k: g[k].clone() for k in GRAD_KEYS})


def _check_sequence(sc, cams, K, tile, fdt="f32"):
    ts = U.tensors(sc, fdt)
    cut = TopKRenderer(cams, K=K, D=sc.d, tile=tile, feat_dtype=fdt, depth_cut=True)
    ref = TopKRenderer(cams, K=K, D=sc.d, tile=tile, feat_dtype=fdt, depth_cut=False)
    dF, dC, dD = S.upstream_grads(3, cut.P, sc.d)
    up = (torch.from_numpy(dF).cuda().to(cut.feat_torch_dtype), torch.from_numpy(dC).cuda(),
          torch.from_numpy(dD).cuda())
    stats = []
    for i, t in enumerate(_variants(ts, 11)):
        fc, gc = _render(cut, t, up)
        st = cut.binning_stats()
        fr, gr = _render(ref, t, up)
        st_ref = ref.binning_stats()
        assert st_ref["sorted_first"] == st_ref["instances"] and st_ref["sorted_second"] == 0
        # elements behind every cut of their rows take instance slots only when completed
        assert st["instances"] <= st_ref["instances"]
        for k in FWD_KEYS:
            assert torch.equal(fc[k], fr[k]), (i, k)
        for k in GRAD_KEYS:
            assert torch.equal(gc[k], gr[k]), (i, k)
        if i == 0:
            stats_ref0 = st_ref["instances"]
        stats.append(st)
    # the first render has no recorded cut; later ones sort fewer instances
    assert stats[0]["sorted_first"] == stats[0]["instances"] and stats[0]["tiles_completed"] == 0
    assert stats[0]["instances"] == stats_ref0
    assert all(s["sorted_first"] < s["instances"] for s in stats[1:])
    return stats


def test_depth_cut_frame_bit_identical():
    """'frame' (200k Gaussians, 640x480, D=512, K=8): every pixel saturates, so cuts are
    recorded for every tile; lowering the opacities forces completions."""
    sc, cams, K, tile, fdt = S.make_config("frame", 0)
    stats = _check_sequence(sc, cams, K, tile)
    print("depth cut, frame:", stats)
    assert sum(s["tiles_completed"] for s in stats) > 0
    assert stats[-1]["sorted_first"] < 0.5 * stats[-1]["instances"]


@pytest.mark.parametrize("tile,K", [((8, 8), 16), ((32, 8), 4)])
def test_depth_cut_multi_camera_tiles_bit_identical(tile, K):
    """Two orbit views of the 'frame' scene (ragged sizes), other tile shapes and K."""
    sc, _, _, _, _ = S.make_config("frame", 0)
    cams = S.orbit_cameras(31, [(203, 157, 180.0), (160, 121, 140.0)], radius=3.0)
    stats = _check_sequence(sc, cams, K, tile)
    print("depth cut, two views", tile, K, stats)


def test_depth_cut_bf16_rows_bit_identical():
    """bf16 feature rows (the tensor-core blend and feature gradient)."""
    sc, cams, K, tile, fdt = S.make_config("frame", 0)
    _check_sequence(sc, cams, K, tile, fdt="bf16")
