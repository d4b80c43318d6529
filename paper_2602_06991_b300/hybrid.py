"""Hybrid field optimisation (Sec. 3.4): geometry every iteration, semantics at a lower
rate, and a fused Adam step over all parameter tensors.

The paper gives no rates; HybridSchedule takes the semantic period as a parameter.  A
semantic iteration runs the full Top-K training step (feature loss and its adjoint);
the others run TopKRenderer.train_step_geometry (colour and depth only, the adjoint
without its feature part).  adam_step updates every tensor in one launch
(gs_adam_step); its moment buffers live in AdamState.
"""
from __future__ import annotations

import ctypes
from typing import Dict, Sequence

import torch

from . import _abi as A


class HybridSchedule:
    """Iteration i is semantic when i % semantic_every == semantic_every - 1 (so the
    geometry leads); semantic_every = 1 is the plain schedule (features every step)."""

    def __init__(self, semantic_every: int = 1):
        if int(semantic_every) < 1:
            raise ValueError("semantic_every must be >= 1")
        self.semantic_every = int(semantic_every)

    def is_semantic(self, it: int) -> bool:
        return it % self.semantic_every == self.semantic_every - 1

    def semantic_fraction(self) -> float:
        return 1.0 / self.semantic_every


class AdamState:
    """First and second moments for a set of named float32 parameter tensors."""

    def __init__(self, params: Dict[str, torch.Tensor]):
        self.m = {k: torch.zeros_like(v) for k, v in params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in params.items()}
        self.step = 0


def adam_step(params: Dict[str, torch.Tensor], grads: Dict[str, torch.Tensor], state: AdamState,
              lr: Dict[str, float], names: Sequence[str] = None, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-15, bf16_copies: Dict[str, torch.Tensor] = None):
    """One Adam step (in place) over the named tensors, all in a single launch.  Only the
    tensors in `names` (default: all) are stepped; their moments advance together, so a
    semantic-rate tensor keeps its own step count by being passed only on semantic
    iterations with its own AdamState.  bf16_copies: for float32 master weights whose
    renderer copy is bf16 (the BF16 feature rows), the bf16 tensor the same launch
    refreshes from the updated master."""
    bf16_copies = bf16_copies or {}
    names = list(params) if names is None else list(names)
    if len(names) > A.GS_ADAM_MAX_TENSORS:
        raise ValueError("too many tensors for one Adam launch")
    state.step += 1
    arr = (A.GsAdamTensor * max(1, len(names)))()
    for i, k in enumerate(names):
        p, g = params[k], grads[k]
        for t, nm in ((p, "param"), (g, "grad"), (state.m[k], "exp_avg"), (state.v[k], "exp_avg_sq")):
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                raise TypeError(f"{k}.{nm} must be a contiguous float32 CUDA tensor")
        if g.numel() != p.numel():
            raise ValueError(f"gradient of {k} has {g.numel()} elements, parameter {p.numel()}")
        cp = bf16_copies.get(k)
        if cp is not None and (cp.dtype != torch.bfloat16 or cp.numel() != p.numel() or not cp.is_contiguous()):
            raise TypeError(f"bf16 copy of {k} must be a contiguous bfloat16 tensor of {p.numel()} elements")
        arr[i] = A.GsAdamTensor(p.data_ptr(), g.data_ptr(), state.m[k].data_ptr(), state.v[k].data_ptr(), p.numel(),
                                float(lr[k]), cp.data_ptr() if cp is not None else None)
    lib = A.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream(params[names[0]].device).cuda_stream)
    A.check(lib.gs_adam_step(arr, len(names), state.step, float(beta1), float(beta2), float(eps), stream),
            "gs_adam_step")
