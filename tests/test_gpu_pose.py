"""GPU parity of the camera-pose gradient (rendering-loss pose refinement, Sec. 4.1)
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import gs_scenes as S
import oracle
import parity_util as U

pytestmark = pytest.mark.gpu


def _run(sc, cams, K, tile, seed):
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    o = U.oracle_forward(sc, cams, K)
    P = sum(c.n_pix for c in cams)
    dF, dC, dD = S.upstream_grads(seed, P, sc.d)
    keep = (o["flags"] & U.FRAGILE_ANY) == 0
    dF[~keep] = 0
    dC[~keep] = 0
    dD[~keep] = 0
    g = r.backward(torch.from_numpy(dF).cuda(), torch.from_numpy(dC).cuda(), torch.from_numpy(dD).cuda(),
                   with_pose=True)
    torch.cuda.synchronize()
    gv = g["viewmat"].cpu().numpy()
    errs = []
    for i, (cam, off) in enumerate(U.cam_slices(cams)):
        sl = slice(off, off + cam.n_pix)
        ov = oracle.backward(sc, cam, K, dF[sl], dC[sl], dD[sl])["viewmat"]
        errs.append(U.rel_l2(gv[i], ov))
    return errs


def test_pose_gradient_small():
    sc, cams, K, tile, _ = S.make_config("small", 10)
    errs = _run(sc, cams, K, tile, 13)
    print("pose rel-L2", errs)
    assert max(errs) <= U.GRAD_TOL, errs


def test_pose_gradient_ragged_cameras():
    """Three cameras of uneven size on an orbit: one [R | t] gradient per camera."""
    sc = S.random_scene_box(23, 3000, 16, box=((-1, 1), (-1, 1), (2, 4)))
    cams = S.orbit_cameras(24, [(70, 52, 70.0), (48, 40, 50.0), (57, 33, 60.0)], radius=3.0)
    errs = _run(sc, cams, 6, (16, 8), 14)
    print("pose rel-L2", errs)
    assert max(errs) <= U.GRAD_TOL, errs
