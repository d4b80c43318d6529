"""The loss entry point that allocates nothing (gs_loss_cos_l1_noalloc), against the
regular one (gs_loss_cos_l1, which takes caller scratch).

Some callers cannot allocate device memory: code in a real-time loop where cudaMalloc
may stall the device, a plug-in inside a framework that owns all device memory, or a
component handed only its buffers.  For them the library keeps the loss's partial sums
in a fixed array of its own.  This file is collected last on purpose, so that a run
stopping at its first failure has already run every other test; it also passes on its
own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _inputs(P, D, dtype, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    F = torch.randn(P, D, generator=g).to("cuda", dtype).contiguous()
    Fgt = torch.randn(P, D, generator=g).to("cuda", dtype).contiguous()
    F[3] = 0          # a pixel with an empty feature: no gradient, loss term w_feat
    C, Cgt = torch.rand(P, 3, generator=g).cuda(), torch.rand(P, 3, generator=g).cuda()
    Dp, Dgt = torch.rand(P, generator=g).cuda() * 4 + 1, torch.rand(P, generator=g).cuda() * 4 + 1
    return F, Fgt, C, Cgt, Dp, Dgt


def _outs(P, D, dtype):
    return (torch.empty(P, D, device="cuda", dtype=dtype), torch.empty(P, 3, device="cuda"),
            torch.empty(P, device="cuda"), torch.empty(1, device="cuda"))


def _ptrs(*ts):
    return [ctypes.c_void_p(t.data_ptr()) for t in ts]


def _run(lib, A, cfg, P, ins, outs, noalloc, weights=(1.0, 0.7, 0.3)):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if noalloc:
        st = lib.gs_loss_cos_l1_noalloc(ctypes.byref(cfg), P, *_ptrs(*ins), *weights, *_ptrs(*outs), stream)
    else:
        scratch = torch.empty(int(lib.gs_loss_scratch_size(P)), dtype=torch.uint8, device="cuda")
        st = lib.gs_loss_cos_l1(ctypes.byref(cfg), P, *_ptrs(*ins), *weights, *_ptrs(*outs),
                                ctypes.c_void_p(scratch.data_ptr()), scratch.numel(), stream)
    torch.cuda.synchronize()
    return st


def test_noalloc_loss_matches_regular_entry_point_twice_in_a_row():
    from paper_2602_06991_b300 import _abi as A, build
    build()
    lib = A.load()
    # two calls in a row on the shared array, the second smaller than the first, so any
    # stale partial sums left by the first call would show up in the second
    for (P, D, dt, seed) in [(20000, 64, torch.float32, 0), (7001, 32, torch.bfloat16, 1)]:
        cfg = A.GsConfig(8, D, 16, 16, A.GS_BF16 if dt == torch.bfloat16 else A.GS_F32, 0)
        ins = _inputs(P, D, dt, seed)
        ref, got = _outs(P, D, dt), _outs(P, D, dt)
        assert _run(lib, A, cfg, P, ins, ref, noalloc=False) == A.GS_OK
        assert _run(lib, A, cfg, P, ins, got, noalloc=True) == A.GS_OK
        for a, b in zip(got, ref):
            np.testing.assert_allclose(a.float().cpu().numpy(), b.float().cpu().numpy(), rtol=1e-6, atol=1e-7)
        assert torch.isfinite(got[3]).all()


def test_noalloc_loss_rejects_oversize_without_launching():
    from paper_2602_06991_b300 import _abi as A, build
    build()
    lib = A.load()
    cfg = A.GsConfig(8, 16, 16, 16, A.GS_F32, 0)
    small = _inputs(8, 16, torch.float32, 2)
    outs = _outs(8, 16, torch.float32)
    st = lib.gs_loss_cos_l1_noalloc(ctypes.byref(cfg), A.GS_LOSS_NOALLOC_MAX_PIX + 1, *_ptrs(*small),
                                    1.0, 1.0, 1.0, *_ptrs(*outs), None)
    assert st == A.GS_ERR_WORKSPACE
