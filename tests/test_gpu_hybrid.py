"""GPU parity of the hybrid field optimisation pieces (Sec. 3.4): the geometry-only
adjoint, the geometric loss and the fused Adam step, against the FP64 oracle."""
import numpy as np
import pytest
import torch

import gs_scenes as S
import oracle
import parity_util as U

pytestmark = pytest.mark.gpu

GEO = [("opacity", "opac"), ("rgb", "rgb"), ("mean3d", "mean3d"), ("cov3d", "cov3d")]


def test_geometry_only_backward_vs_oracle():
    """dL_dF = None: the oracle gradient with a zero feature upstream, and the feature
    gradient buffer left untouched."""
    sc, cams, K, tile, _ = S.make_config("small", 6)
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    o = U.oracle_forward(sc, cams, K)
    P = cams[0].n_pix
    _, dC, dD = S.upstream_grads(8, P, sc.d)
    keep = (o["flags"] & U.FRAGILE_ANY) == 0
    dC[~keep] = 0
    dD[~keep] = 0
    g = r.alloc_grads(sc.n)
    g["feat"].fill_(7.0)
    r.backward(None, torch.from_numpy(dC).cuda(), torch.from_numpy(dD).cuda(), grads=g)
    torch.cuda.synchronize()
    og = oracle.backward(sc, cams[0], K, np.zeros((P, sc.d)), dC, dD)
    for gk, ok in GEO:
        e = U.rel_l2(g[gk].cpu().numpy(), og[ok])
        assert e <= U.GRAD_TOL, (gk, e)
    assert torch.all(g["feat"] == 7.0)


def test_geometry_only_equals_full_adjoint_with_zero_feature_upstream():
    """The full adjoint with dL/dF = 0 gives bit-identical geometry gradients (h = 0 and
    H = 0, so the feature term of dL/dw vanishes exactly)."""
    sc, cams, K, tile, _ = S.make_config("frame", 0)
    sc = S.crop_scene(sc, cams[0], 5000)
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    P = cams[0].n_pix
    _, dC, dD = S.upstream_grads(9, P, sc.d)
    dCt, dDt = torch.from_numpy(dC).cuda(), torch.from_numpy(dD).cuda()
    g0 = r.backward(None, dCt, dDt)
    g1 = r.backward(torch.zeros(P, sc.d, device="cuda"), dCt, dDt)
    torch.cuda.synchronize()
    for gk, _ in GEO:
        assert torch.equal(g0[gk], g1[gk]), gk
    assert torch.all(g1["feat"] == 0)


def test_geometric_loss_vs_oracle():
    sc, cams, K, tile, _ = S.make_config("small", 7)
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    _, Cgt, Dgt = S.voronoi_targets(4, cams, sc.d)
    lo = r.loss_geo(out["rgb"], torch.from_numpy(Cgt).cuda(), out["depth"], torch.from_numpy(Dgt).cuda(), 1.0, 0.5)
    torch.cuda.synchronize()
    loss, dC, dD = oracle.loss_geo(out["rgb"].cpu().numpy(), Cgt, out["depth"].cpu().numpy(), Dgt, 1.0, 0.5)
    np.testing.assert_allclose(lo["loss"].item(), loss, rtol=1e-5)
    np.testing.assert_allclose(lo["dL_dC"].cpu().numpy(), dC, rtol=1e-6, atol=0)
    np.testing.assert_allclose(lo["dL_dD"].cpu().numpy(), dD, rtol=1e-6, atol=0)


def test_fused_adam_vs_oracle():
    """Five tensors in one launch -- lengths not multiples of 4 and a misaligned view take
    the scalar path -- three steps against FP64 Adam."""
    from paper_2602_06991_b300.hybrid import AdamState, adam_step
    rng = np.random.default_rng(3)
    sizes = {"a": 1001, "b": 4096, "c": 7, "d": 300_000, "e": 33}
    base = torch.from_numpy(rng.standard_normal(sizes["e"] + 1).astype(np.float32)).cuda()
    params = {k: torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda() for k, n in sizes.items() if k != "e"}
    params["e"] = base[1:]                           # 4-byte offset: not 16-byte aligned
    lr = {k: 10.0 ** -(1 + i) for i, k in enumerate(sizes)}
    st = AdamState(params)
    ref = {k: (v.double().cpu().numpy(), np.zeros(v.numel()), np.zeros(v.numel())) for k, v in params.items()}
    for t in (1, 2, 3):
        grads = {k: torch.from_numpy(rng.standard_normal(v.numel()).astype(np.float32)).cuda() for k, v in params.items()}
        adam_step(params, grads, st, lr, beta1=0.9, beta2=0.99, eps=1e-8)
        for k in params:
            p, m, v = ref[k]
            ref[k] = oracle.adam_step(p, grads[k].cpu().numpy(), m, v, lr[k], 0.9, 0.99, 1e-8, t)
    torch.cuda.synchronize()
    # float32 parameters of magnitude ~1 round to ~6e-8 per update: absolute 1e-6
    for k, v in params.items():
        np.testing.assert_allclose(v.cpu().numpy(), ref[k][0], rtol=2e-6, atol=1e-6)
        np.testing.assert_allclose(st.m[k].cpu().numpy(), ref[k][1], rtol=1e-5, atol=1e-7)


def test_fused_adam_bf16_copy():
    """float32 master weights with a bf16 renderer copy: the same launch writes the copy,
    the updated master rounded to nearest (both the float4 and the scalar path)."""
    from paper_2602_06991_b300.hybrid import AdamState, adam_step
    rng = np.random.default_rng(4)
    params = {k: torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda() for k, n in (("f", 4096 + 6),
                                                                                                   ("g", 13))}
    copies = {k: torch.empty(v.numel(), dtype=torch.bfloat16, device="cuda") for k, v in params.items()}
    st = AdamState(params)
    for _ in range(2):
        grads = {k: torch.from_numpy(rng.standard_normal(v.numel()).astype(np.float32)).cuda()
                 for k, v in params.items()}
        adam_step(params, grads, st, {"f": 1e-2, "g": 1e-3}, bf16_copies=copies)
    torch.cuda.synchronize()
    for k, v in params.items():
        assert torch.equal(copies[k], v.to(torch.bfloat16)), k


def test_hybrid_loop_runs_and_lowers_the_loss():
    """Twelve iterations of the hybrid schedule (semantics every third) with Adam on the
    small scene: every loss finite, the geometric loss lower at the end."""
    from paper_2602_06991_b300.hybrid import AdamState, HybridSchedule, adam_step
    from paper_2602_06991_b300.renderer import TopKRenderer
    sc, cams, K, tile, _ = S.make_config("small", 8)
    r = TopKRenderer(cams, K=K, D=sc.d, tile=tile)
    ts = [t.clone() for t in U.tensors(sc)]
    names = ["mean3d", "opacity", "rgb", "feat"]
    params = {"mean3d": ts[0], "opacity": ts[2], "rgb": ts[3], "feat": ts[4]}
    Fgt, Cgt, Dgt = (torch.from_numpy(a).cuda() for a in S.voronoi_targets(5, cams, sc.d))
    sched = HybridSchedule(3)
    geo_state, sem_state = AdamState({k: params[k] for k in names[:3]}), AdamState({"feat": params["feat"]})
    lrs = {"mean3d": 1e-3, "opacity": 1e-2, "rgb": 1e-2, "feat": 1e-2}
    losses = []
    for it in range(12):
        if sched.is_semantic(it):
            o, lo, g = r.train_step(*ts, Fgt, Cgt, Dgt)
            adam_step(params, {"feat": g["feat"]}, sem_state, lrs, names=["feat"])
        else:
            o, lo, g = r.train_step_geometry(*ts[:4], Cgt, Dgt)
        adam_step(params, {"mean3d": g["mean3d"], "opacity": g["opacity"], "rgb": g["rgb"]}, geo_state, lrs,
                  names=names[:3])
        losses.append(float(r.loss_geo(o["rgb"], Cgt, o["depth"], Dgt)["loss"].item()))
    assert all(np.isfinite(losses)) and losses[-1] < losses[0], losses
