"""Kernel timers (gs_timer_enable / gs_timer_read): every timed stage of a render and its
adjoint records a positive device time while enabled, reading waits for the stage's end
event, nothing is recorded while disabled or during a stream capture, and enabling clears
earlier records."""
import pytest
import torch

import gs_scenes as S
import parity_util as U
from paper_2602_06991_b300 import _abi as A
from paper_2602_06991_b300.renderer import TopKRenderer

pytestmark = pytest.mark.gpu

STAGES = (A.GS_TIMER_BINNING, A.GS_TIMER_TILE_SORT, A.GS_TIMER_WALK_FWD, A.GS_TIMER_BLOCK_GRAD,
          A.GS_TIMER_WALK_BWD, A.GS_TIMER_COMPLETE)


def _step(r, ts, up):
    r.forward(*ts)
    r.backward(*up)


def test_timers_record_every_stage():
    # D = 512 float32 rows: the feature gradient takes the per-block pipeline
    sc = S.planes_scene(7, 6000, 512)
    cams = [S.pinhole(160, 120, 131.25)]
    ts = U.tensors(sc)
    r = TopKRenderer(cams, K=8, D=sc.d, tile=(16, 16))
    dF, dC, dD = S.upstream_grads(1, r.P, sc.d)
    up = (torch.from_numpy(dF).cuda(), torch.from_numpy(dC).cuda(), torch.from_numpy(dD).cuda())
    _step(r, ts, up)                              # workspace, capacities
    torch.cuda.synchronize()
    A.timer_enable(False)
    _step(r, ts, up)
    torch.cuda.synchronize()
    assert all(A.timer_read(t) is None for t in STAGES)        # disabled: nothing recorded
    A.timer_enable(True)
    try:
        _step(r, ts, up)
        ms = {t: A.timer_read(t) for t in STAGES}
        assert all(v is not None and v > 0.0 for v in ms.values()), ms
        # a captured step records nothing (the last eager records stay readable)
        A.timer_enable(True)
        r.check_overflow = False
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            _step(r, ts, up)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        A.timer_enable(True)                      # clears the records of that eager step
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            _step(r, ts, up)
        g.replay()
        torch.cuda.synchronize()
        assert all(A.timer_read(t) is None for t in STAGES)
    finally:
        A.timer_enable(False)
