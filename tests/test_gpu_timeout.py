"""Failure detection of the bounded device-side waits, without a GPU fault.

The feature-gradient pipeline of gs_backward (k_block_accum) waits on mbarriers for its
bulk copies.  Each wait has a bound; gs_set_wait_limit lowers it for the current render.
A bound of one cycle makes the first wait of every CTA run out: the kernel records
GS_ERR_TIMEOUT in the workspace error word, waits with the default bound for the copies
it has in flight, and returns; later kernels on the workspace skip their work.  The host
reads the status with gs_sync_status, the context stays usable, and the next render
(gs_preprocess resets the bound and the error word) gives the same gradients as a
render that never timed out."""
import pytest
import torch

import gs_scenes as S
import parity_util as U
from paper_2602_06991_b300 import _abi as A

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32"])
def test_wait_timeout_is_reported_and_recovered(dtype):
    # (float32 rows take the TMA pipeline with its mbarrier waits; bf16 rows of these
    # widths take the tensor-core block product, which waits on nothing)
    sc = S.planes_scene(7, 6000, 512)
    cams = [S.pinhole(160, 120, 131.25)]
    r, ts, out = U.gpu_forward(sc, cams, 8, (16, 16), feat_dtype=dtype, max_instances=1 << 22)
    r.check_overflow = False
    P = r.P
    g = torch.Generator().manual_seed(5)
    dF = torch.randn(P, sc.d, generator=g).cuda().to(r.feat_torch_dtype)
    dC, dD = torch.randn(P, 3, generator=g).cuda(), torch.randn(P, generator=g).cuda()

    ref = {k: v.clone() for k, v in r.backward(dF, dC, dD).items()}
    assert r.sync_status()[0] == A.GS_OK
    assert float(ref["feat"].abs().sum()) > 0

    r.set_wait_limit(1)
    r.backward(dF, dC, dD)
    assert r.sync_status()[0] == A.GS_ERR_TIMEOUT

    # the context is intact: a new render clears the bound and the error word
    r.forward(*ts, out=out)
    got = r.backward(dF, dC, dD)
    assert r.sync_status()[0] == A.GS_OK
    for k in ref:
        assert torch.equal(ref[k], got[k]), k
