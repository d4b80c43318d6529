"""A training step replayed from a captured CUDA graph gives the same outputs, loss, loss
gradients and parameter gradients, bit for bit, as the same step launched directly.  The
cases cover FP32 rows (the CUDA-core block product, whose re-walk waits on the block records
through an event inside the capture) and BF16 rows (the tensor-core blend and block
product), on one camera and on several cameras of uneven size."""
import pytest
import torch

import gs_scenes as S
import parity_util as U
from paper_2602_06991_b300.renderer import TopKRenderer

pytestmark = pytest.mark.gpu

OUT_KEYS = ("rgb", "depth", "T", "n_contrib", "topk_idx", "topk_w", "F")
LOSS_KEYS = ("dL_dF", "dL_dC", "dL_dD", "loss")
GRAD_KEYS = ("feat", "opacity", "rgb", "mean3d", "cov3d")


def _targets(cams, d, tdt):
    lab, fv, cv, dv = S.voronoi_sites(100, cams, d)
    lab = torch.from_numpy(lab).cuda().long()
    t = lambda a, dt=torch.float32: torch.from_numpy(a).cuda().to(dt)
    return t(fv, tdt)[lab].contiguous(), t(cv)[lab].contiguous(), t(dv)[lab].contiguous()


def _snapshot(o, lo, g):
    return ({k: o[k].clone() for k in OUT_KEYS}, {k: lo[k].clone() for k in LOSS_KEYS},
            {k: g[k].clone() for k in GRAD_KEYS})


def _assert_same(a, b, what):
    for part_a, part_b in zip(a, b):
        for k in part_a:
            assert torch.equal(part_a[k], part_b[k]), f"{what}: {k} differs"


@pytest.mark.parametrize("fdt,views", [("f32", 1), ("f32", 2), ("bf16", 1), ("bf16", 2)])
def test_graph_replay_matches_direct_launches(fdt, views):
    sc, cams, K, tile, _ = S.make_config("frame", 0)
    if views > 1:
        cams = S.orbit_cameras(41, [(203, 157, 180.0), (160, 121, 140.0)], radius=3.0)
    ts = U.tensors(sc, fdt)
    r = TopKRenderer(cams, K=K, D=sc.d, tile=tile, feat_dtype=fdt)
    tgt = _targets(cams, sc.d, r.feat_torch_dtype)
    o, lo, g = r.alloc_outputs(sc.n), r.alloc_loss(), r.alloc_grads(sc.n)
    step = lambda: r.train_step(*ts, *tgt, out=o, lo=lo, grads=g)
    step()                                    # sizes the capacities (host checks)
    r.check_overflow = False
    step()                                    # direct launches, with the recorded depth cut
    torch.cuda.synchronize()
    assert r.sync_status()[0] == 0
    ref = _snapshot(o, lo, g)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()                                # warm on the capture's side stream
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for rep in range(2):
        checked = [o[k] for k in OUT_KEYS] + [lo[k] for k in LOSS_KEYS] + [g[k] for k in GRAD_KEYS]
        for t in checked:
            if t.is_floating_point():
                t.fill_(float("nan"))         # every checked output must be written again
            else:
                t.fill_(-7)
        graph.replay()
        torch.cuda.synchronize()
        assert r.sync_status()[0] == 0
        _assert_same(ref, _snapshot(o, lo, g), f"replay {rep}")
