"""Torch-facing wrapper of the C ABI: device memory, streams and argument marshalling.

    r = TopKRenderer(cameras, K=8, D=512)
    out = r.forward(mean3d, cov3d, opacity, rgb, feats)          # F, rgb, depth, Top-K ...
    g = r.backward(dL_dF, dL_dC, dL_dD)                         # per-Gaussian gradients

or through autograd with ``render(renderer, mean3d, cov3d, opacity, rgb, feats)``.
Every stage runs in the CUDA library; torch only allocates tensors and provides the
stream.  Tensors must be contiguous CUDA tensors: float32 for geometry, float32 or
bfloat16 for feature rows (the renderer's feat dtype).
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import torch

from . import _abi as A

_DT = {"f32": A.GS_F32, "bf16": A.GS_BF16}
_TORCH_DT = {A.GS_F32: torch.float32, A.GS_BF16: torch.bfloat16}


def _p(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need(t: torch.Tensor, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class TopKRenderer:
    """One configuration (cameras, K, D, tile, feature dtype) and its workspace."""

    def __init__(self, cameras: Sequence, K: int, D: int, tile=(16, 16), feat_dtype: str = "f32",
                 max_instances: int = 0, device=None, check_overflow: bool = True, max_feature_rows: int = 0,
                 topk_layout: int = 0, depth_cut: bool = True):
        self.lib = A.load()
        self.cams = A.make_cameras(list(cameras))
        self.n_cams = len(cameras)
        self.K, self.D = int(K), int(D)
        self.tile = (int(tile[0]), int(tile[1]))
        self.dtype = _DT[feat_dtype] if isinstance(feat_dtype, str) else int(feat_dtype)
        self.feat_torch_dtype = _TORCH_DT[self.dtype]
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.check_overflow = check_overflow
        self.cfg = A.GsConfig(self.K, self.D, self.tile[0], self.tile[1], self.dtype, int(max_instances),
                              int(max_feature_rows), int(topk_layout), 1 if depth_cut else 0)
        self.P = int(self.lib.gs_pixel_count(self.cams, self.n_cams))
        if self.P < 0:
            raise ValueError("bad cameras")
        self.ws = None
        self.ws_n = -1
        self.state = None

    # ------------------------------------------------------------------ workspace
    def workspace_bytes(self, N: int) -> int:
        b = int(self.lib.gs_workspace_size(ctypes.byref(self.cfg), self.cams, self.n_cams, int(N)))
        if b == 0:
            raise A.GsError(A.GS_ERR_ARG, "gs_workspace_size")
        return b

    def _ensure_ws(self, N: int):
        if self.ws is None or self.ws_n != N:
            self.ws = torch.empty(self.workspace_bytes(N), dtype=torch.uint8, device=self.device)
            # a zeroed header: the first render records depth cuts instead of reading
            # whatever an earlier tenant of the memory left
            self.ws[:256].zero_()
            self.ws_n = N

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def set_wait_limit(self, cycles: int):
        """Bound (SM clock cycles) of the device-side pipeline waits of the current
        render (gs_set_wait_limit); the next forward resets it to the default."""
        A.check(self.lib.gs_set_wait_limit(_p(self.ws), self.ws.numel(), int(cycles), self._stream()),
                "gs_set_wait_limit")

    def counts(self):
        """(instances of the last binning, partial feature rows the last backward needed)."""
        n, m = ctypes.c_int64(0), ctypes.c_int64(0)
        A.check(self.lib.gs_workspace_counts(_p(self.ws), self.ws.numel(), self._stream(), ctypes.byref(n),
                                             ctypes.byref(m)), "gs_workspace_counts")
        return int(n.value), int(m.value)

    def binning_stats(self):
        """Of the last render: {instances, sorted_first, sorted_second, tiles_completed}."""
        out = (ctypes.c_int64 * 4)()
        A.check(self.lib.gs_binning_stats(_p(self.ws), self.ws.numel(), self._stream(), out), "gs_binning_stats")
        return {"instances": int(out[0]), "sorted_first": int(out[1]), "sorted_second": int(out[2]),
                "tiles_completed": int(out[3])}

    def sync_status(self):
        n = ctypes.c_int64(0)
        st = self.lib.gs_sync_status(_p(self.ws), self.ws.numel(), self._stream(), ctypes.byref(n))
        return st, int(n.value)

    # ------------------------------------------------------------------ forward
    def alloc_outputs(self, N: int):
        dev, P, K = self.device, self.P, self.K
        return dict(proj=torch.empty(self.n_cams * N * A.GS_PROJ_FLOATS, dtype=torch.float32, device=dev),
                    rgb=torch.empty(P, 3, dtype=torch.float32, device=dev),
                    depth=torch.empty(P, dtype=torch.float32, device=dev),
                    T=torch.empty(P, dtype=torch.float32, device=dev),
                    n_contrib=torch.empty(P, dtype=torch.int32, device=dev),
                    topk_idx=torch.empty(P, K, dtype=torch.int32, device=dev),
                    topk_w=torch.empty(P, K, dtype=torch.float32, device=dev),
                    F=torch.empty(P, self.D, dtype=self.feat_torch_dtype, device=dev))

    def forward(self, mean3d, cov3d, opacity, rgb, feats, out=None):
        N = int(mean3d.shape[0])
        f32 = torch.float32
        _need(mean3d, f32, (N, 3), "mean3d"); _need(cov3d, f32, (N, 6), "cov3d")
        _need(opacity, f32, (N,), "opacity"); _need(rgb, f32, (N, 3), "rgb")
        _need(feats, self.feat_torch_dtype, (N, self.D), "feats")
        self._ensure_ws(N)
        o = out if out is not None else self.alloc_outputs(N)
        self._forward_into(N, mean3d, cov3d, opacity, rgb, feats, o)
        if self.check_overflow:
            st, m = self.sync_status()
            while st == A.GS_ERR_OVERFLOW:
                self.cfg.max_instances = int(min(2 ** 31 - 1, max(2 * m, 1024)))
                self.ws = None
                self._ensure_ws(N)
                self._forward_into(N, mean3d, cov3d, opacity, rgb, feats, o)
                st, m = self.sync_status()
            A.check(st, "render")
        self.state = dict(N=N, mean3d=mean3d, cov3d=cov3d, opacity=opacity, rgb=rgb, feats=feats, out=o)
        return o

    def _forward_into(self, N, mean3d, cov3d, opacity, rgb, feats, o):
        L, cfg, s = self.lib, ctypes.byref(self.cfg), self._stream()
        ws, wsb = _p(self.ws), self.ws.numel()
        A.check(L.gs_preprocess(cfg, self.cams, self.n_cams, N, _p(mean3d), _p(cov3d), _p(opacity), _p(rgb),
                                _p(o["proj"]), ws, wsb, s), "gs_preprocess")
        A.check(L.gs_bin_sort(cfg, self.cams, self.n_cams, N, _p(o["proj"]), ws, wsb, s), "gs_bin_sort")
        A.check(L.gs_topk_select(cfg, self.cams, self.n_cams, N, _p(o["proj"]), ws, wsb, _p(o["rgb"]),
                                 _p(o["depth"]), _p(o["T"]), _p(o["n_contrib"]), _p(o["topk_idx"]),
                                 _p(o["topk_w"]), s), "gs_topk_select")
        A.check(L.gs_feature_blend(cfg, self.P, N, _p(o["topk_idx"]), _p(o["topk_w"]), _p(feats), _p(o["F"]), s),
                "gs_feature_blend")

    def _select_into(self, N, mean3d, cov3d, opacity, rgb, o):
        """a1-a3 only (projection, binning, Top-K walk)."""
        self._h_valid = False                    # a new Top-K (or workspace): no h from a loss
        L, cfg, s = self.lib, ctypes.byref(self.cfg), self._stream()
        ws, wsb = _p(self.ws), self.ws.numel()
        A.check(L.gs_preprocess(cfg, self.cams, self.n_cams, N, _p(mean3d), _p(cov3d), _p(opacity), _p(rgb),
                                _p(o["proj"]), ws, wsb, s), "gs_preprocess")
        A.check(L.gs_bin_sort(cfg, self.cams, self.n_cams, N, _p(o["proj"]), ws, wsb, s), "gs_bin_sort")
        A.check(L.gs_topk_select(cfg, self.cams, self.n_cams, N, _p(o["proj"]), ws, wsb, _p(o["rgb"]),
                                 _p(o["depth"]), _p(o["T"]), _p(o["n_contrib"]), _p(o["topk_idx"]),
                                 _p(o["topk_w"]), s), "gs_topk_select")

    def alloc_loss(self):
        P, dev = self.P, self.device
        return dict(dL_dF=torch.empty(P, self.D, dtype=self.feat_torch_dtype, device=dev),
                    dL_dC=torch.empty(P, 3, dtype=torch.float32, device=dev),
                    dL_dD=torch.empty(P, dtype=torch.float32, device=dev),
                    loss=torch.empty(1, dtype=torch.float32, device=dev),
                    scratch=torch.empty(int(self.lib.gs_loss_scratch_size(P)), dtype=torch.uint8, device=dev))

    def blend_loss(self, feats, F_gt, rgb_gt, depth_gt, w_feat=1.0, w_rgb=1.0, w_depth=1.0, lo=None):
        """Fused gather-blend + loss after a forward (or _select_into): writes out['F']
        and the loss gradients (gs_feature_blend_loss)."""
        st = self.state
        N, o = st["N"], st["out"]
        lo = lo if lo is not None else self.alloc_loss()
        A.check(self.lib.gs_feature_blend_loss(
            ctypes.byref(self.cfg), self.cams, self.n_cams, N, _p(o["topk_idx"]), _p(o["topk_w"]), _p(feats),
            _p(F_gt), _p(o["rgb"]), _p(rgb_gt), _p(o["depth"]), _p(depth_gt), float(w_feat), float(w_rgb),
            float(w_depth), _p(o["F"]), _p(lo["dL_dF"]), _p(lo["dL_dC"]), _p(lo["dL_dD"]), _p(lo["loss"]),
            _p(self.ws), self.ws.numel(), _p(lo["scratch"]), lo["scratch"].numel(), self._stream()),
            "gs_feature_blend_loss")
        # that call also left h = dL/dF . f in the workspace for this dL_dF
        self._loss_dLdF, self._h_valid = lo["dL_dF"].data_ptr(), True
        return lo

    def train_step(self, mean3d, cov3d, opacity, rgb, feats, F_gt, rgb_gt, depth_gt, out=None, lo=None, grads=None,
                   weights=(1.0, 1.0, 1.0)):
        """One training step with every buffer supplied (no allocation, no host sync when
        check_overflow is off): a1-a3, fused a4 + loss, a5."""
        N = int(mean3d.shape[0])
        self._ensure_ws(N)
        o = out if out is not None else self.alloc_outputs(N)
        self._select_into(N, mean3d, cov3d, opacity, rgb, o)
        self.state = dict(N=N, mean3d=mean3d, cov3d=cov3d, opacity=opacity, rgb=rgb, feats=feats, out=o)
        lo = self.blend_loss(feats, F_gt, rgb_gt, depth_gt, *weights, lo=lo)
        g = self.backward(lo["dL_dF"], lo["dL_dC"], lo["dL_dD"], grads=grads, h_from_loss=True)
        return o, lo, g

    # ------------------------------------------------------------------ backward
    def alloc_grads(self, N: int, with_2d: bool = False, with_pose: bool = False):
        dev = self.device
        g = dict(feat=torch.empty(N, self.D, dtype=torch.float32, device=dev),
                 opacity=torch.empty(N, dtype=torch.float32, device=dev),
                 rgb=torch.empty(N, 3, dtype=torch.float32, device=dev),
                 mean3d=torch.empty(N, 3, dtype=torch.float32, device=dev),
                 cov3d=torch.empty(N, 6, dtype=torch.float32, device=dev))
        if with_2d:
            g["mean2d"] = torch.empty(self.n_cams, N, 2, dtype=torch.float32, device=dev)
            g["conic"] = torch.empty(self.n_cams, N, 3, dtype=torch.float32, device=dev)
        if with_pose:
            g["viewmat"] = torch.empty(self.n_cams, 3, 4, dtype=torch.float32, device=dev)
        return g

    def backward(self, dL_dF, dL_dC, dL_dD, grads=None, with_2d=False, with_pose=False, h_from_loss=False):
        """The adjoint (gs_backward_ex).  dL_dF = None is the geometry-only adjoint of the
        hybrid schedule: no feature loss, so grads['feat'] is left as it is.
        h_from_loss: dL_dF is the tensor the last blend_loss wrote, unmodified since, so
        the per-slot terms that call left in the workspace are reused (recomputed if a
        capacity retry has replaced the workspace since)."""
        st = self.state
        if st is None:
            raise RuntimeError("backward before forward")
        if h_from_loss and (dL_dF is None or getattr(self, "_loss_dLdF", None) != dL_dF.data_ptr()):
            raise ValueError("h_from_loss: dL_dF is not the gradient the last blend_loss wrote")
        h_reuse = h_from_loss and getattr(self, "_h_valid", False)
        N, o = st["N"], st["out"]
        if dL_dF is not None:
            _need(dL_dF, self.feat_torch_dtype, (self.P, self.D), "dL_dF")
        _need(dL_dC, torch.float32, (self.P, 3), "dL_dC")
        _need(dL_dD, torch.float32, (self.P,), "dL_dD")
        g = grads if grads is not None else self.alloc_grads(N, with_2d, with_pose)
        gg = A.GsGrads(g["feat"].data_ptr() if dL_dF is not None else None, g["opacity"].data_ptr(),
                       g["rgb"].data_ptr(), g["mean3d"].data_ptr(),
                       g["cov3d"].data_ptr(), g["mean2d"].data_ptr() if "mean2d" in g else None,
                       g["conic"].data_ptr() if "conic" in g else None,
                       g["viewmat"].data_ptr() if "viewmat" in g else None)
        def run(flags):
            A.check(self.lib.gs_backward_ex(ctypes.byref(self.cfg), self.cams, self.n_cams, N, _p(st["mean3d"]),
                                            _p(st["cov3d"]), _p(st["opacity"]), _p(st["rgb"]), _p(st["feats"]),
                                            _p(o["proj"]), _p(o["rgb"]), _p(o["depth"]), _p(o["topk_idx"]),
                                            _p(o["topk_w"]), _p(dL_dF), _p(dL_dC), _p(dL_dD), ctypes.byref(gg),
                                            flags, _p(self.ws), self.ws.numel(), self._stream()), "gs_backward_ex")

        run(A.GS_BWD_H_FROM_LOSS if h_reuse else 0)
        if self.check_overflow:
            # the per-block partial feature rows have a capacity: on overflow, size it to
            # the rows needed (with a margin), redo a1-a3 into the new workspace (same
            # Top-K, deterministic) and the adjoint
            code, _ = self.sync_status()
            tries = 0
            while code == A.GS_ERR_OVERFLOW and tries < 4:
                _, need = self.counts()
                self.cfg.max_feature_rows = int(min(2 ** 31 - 1, max(need + need // 4, 2 * self.cfg.max_feature_rows)))
                self.ws = None
                self._ensure_ws(N)
                self._select_into(N, st["mean3d"], st["cov3d"], st["opacity"], st["rgb"], o)
                run(0)                  # the new workspace holds no h from the loss
                code, _ = self.sync_status()
                tries += 1
            A.check(code, "backward")
        return g

    # ------------------------------------------------------------------ hybrid schedule (Sec. 3.4)
    def loss_geo(self, rgb, rgb_gt, depth, depth_gt, w_rgb=1.0, w_depth=1.0, out=None):
        """Geometric loss of the geometry-only iterations (gs_loss_geo_l1)."""
        P = self.P
        o = out if out is not None else dict(
            dL_dC=torch.empty(P, 3, dtype=torch.float32, device=self.device),
            dL_dD=torch.empty(P, dtype=torch.float32, device=self.device),
            loss=torch.empty(1, dtype=torch.float32, device=self.device),
            scratch=torch.empty(int(self.lib.gs_loss_scratch_size(P)), dtype=torch.uint8, device=self.device))
        A.check(self.lib.gs_loss_geo_l1(P, _p(rgb), _p(rgb_gt), _p(depth), _p(depth_gt), float(w_rgb), float(w_depth),
                                        _p(o["dL_dC"]), _p(o["dL_dD"]), _p(o["loss"]), _p(o["scratch"]),
                                        o["scratch"].numel(), self._stream()), "gs_loss_geo_l1")
        return o

    def train_step_geometry(self, mean3d, cov3d, opacity, rgb, rgb_gt, depth_gt, out=None, lo=None, grads=None,
                            weights=(1.0, 1.0)):
        """A geometry-only iteration: a1-a3, the colour/depth loss, the adjoint without its
        feature part (the feature gradient is left untouched)."""
        N = int(mean3d.shape[0])
        self._ensure_ws(N)
        o = out if out is not None else self.alloc_outputs(N)
        self._select_into(N, mean3d, cov3d, opacity, rgb, o)
        feats = self.state["feats"] if self.state is not None else None
        self.state = dict(N=N, mean3d=mean3d, cov3d=cov3d, opacity=opacity, rgb=rgb, feats=feats, out=o)
        lo = self.loss_geo(o["rgb"], rgb_gt, o["depth"], depth_gt, *weights, out=lo)
        g = self.backward(None, lo["dL_dC"], lo["dL_dD"], grads=grads)
        return o, lo, g

    # ------------------------------------------------------------------ vanilla baseline
    def forward_vanilla(self, feats, F=None):
        """Full alpha-blended feature of the last forward's views (gs_feature_blend_vanilla):
        F = sum over all contributors of w_i f_i -- the baseline Top-K rendering replaces."""
        st = self.state
        if st is None:
            raise RuntimeError("forward_vanilla before forward")
        N, o = st["N"], st["out"]
        _need(feats, self.feat_torch_dtype, (N, self.D), "feats")
        F = F if F is not None else torch.empty(self.P, self.D, dtype=self.feat_torch_dtype, device=self.device)
        A.check(self.lib.gs_feature_blend_vanilla(ctypes.byref(self.cfg), self.cams, self.n_cams, N, _p(o["proj"]),
                                                  _p(feats), _p(F), _p(self.ws), self.ws.numel(), self._stream()),
                "gs_feature_blend_vanilla")
        return F

    # ------------------------------------------------------------------ pruning (Sec. 3.3)
    def alloc_prune_stats(self, N: int):
        """Zeroed accumulators for a pruning window: Top-K count (int32) and S (float32)."""
        return dict(count=torch.zeros(N, dtype=torch.int32, device=self.device),
                    S=torch.zeros(N, dtype=torch.float32, device=self.device))

    def prune_stats(self, acc):
        """Accumulate the statistics of the last forward's views into acc (gs_prune_stats):
        acc['count'] += Top-K participation, acc['S'] = max(acc['S'], max w) (Eq. 8)."""
        st = self.state
        if st is None:
            raise RuntimeError("prune_stats before forward")
        N, o = st["N"], st["out"]
        _need(acc["count"], torch.int32, (N,), "count")
        _need(acc["S"], torch.float32, (N,), "S")
        A.check(self.lib.gs_prune_stats(ctypes.byref(self.cfg), self.cams, self.n_cams, N, _p(o["proj"]),
                                        _p(o["topk_idx"]), _p(self.ws), self.ws.numel(), _p(acc["count"]),
                                        _p(acc["S"]), self._stream()), "gs_prune_stats")
        return acc

    # ------------------------------------------------------------------ loss
    def loss(self, F, F_gt, rgb, rgb_gt, depth, depth_gt, w_feat=1.0, w_rgb=1.0, w_depth=1.0, out=None):
        P = self.P
        o = out if out is not None else dict(
            dL_dF=torch.empty(P, self.D, dtype=self.feat_torch_dtype, device=self.device),
            dL_dC=torch.empty(P, 3, dtype=torch.float32, device=self.device),
            dL_dD=torch.empty(P, dtype=torch.float32, device=self.device),
            loss=torch.empty(1, dtype=torch.float32, device=self.device),
            scratch=torch.empty(int(self.lib.gs_loss_scratch_size(P)), dtype=torch.uint8, device=self.device))
        A.check(self.lib.gs_loss_cos_l1(ctypes.byref(self.cfg), P, _p(F), _p(F_gt), _p(rgb), _p(rgb_gt),
                                        _p(depth), _p(depth_gt), float(w_feat), float(w_rgb), float(w_depth),
                                        _p(o["dL_dF"]), _p(o["dL_dC"]), _p(o["dL_dD"]), _p(o["loss"]),
                                        _p(o["scratch"]), o["scratch"].numel(), self._stream()), "gs_loss_cos_l1")
        return o


class _TopKRenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, mean3d, cov3d, opacity, rgb, feats):
        o = renderer.forward(mean3d.detach(), cov3d.detach(), opacity.detach(), rgb.detach(), feats.detach())
        ctx.renderer = renderer
        ctx.feat_dtype = feats.dtype
        return o["F"], o["rgb"], o["depth"]

    @staticmethod
    def backward(ctx, dF, dC, dD):
        r = ctx.renderer
        dF = (dF if dF is not None else torch.zeros(r.P, r.D, device=r.device)).to(r.feat_torch_dtype).contiguous()
        dC = (dC if dC is not None else torch.zeros(r.P, 3, device=r.device)).float().contiguous()
        dD = (dD if dD is not None else torch.zeros(r.P, device=r.device)).float().contiguous()
        g = r.backward(dF, dC, dD)
        return None, g["mean3d"], g["cov3d"], g["opacity"], g["rgb"], g["feat"].to(ctx.feat_dtype)


def render(renderer: TopKRenderer, mean3d, cov3d, opacity, rgb, feats):
    """Differentiable Top-K render: returns (F, rgb, depth) with gradients to every input."""
    return _TopKRenderFn.apply(renderer, mean3d, cov3d, opacity, rgb, feats)


def prune_select(count, S, tau: int, ratio: float, expo):
    """Survival selection of Sec. 3.3 (Eq. 9) on the device (gs_prune_select): candidates
    have count < tau; floor(ratio |candidates| + 1/2) of them survive by weighted
    sampling without replacement with probability proportional to S, drawn as an
    exponential race with the given Exp(1) variates expo.  Returns keep (uint8, N)."""
    lib = A.load()
    N = int(count.shape[0])
    dev = count.device
    _need(count, torch.int32, (N,), "count")
    _need(S, torch.float32, (N,), "S")
    _need(expo, torch.float32, (N,), "expo")
    keep = torch.empty(N, dtype=torch.uint8, device=dev)
    ws = torch.empty(max(1, int(lib.gs_prune_select_workspace_size(N))), dtype=torch.uint8, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    A.check(lib.gs_prune_select(N, _p(count), _p(S), int(tau), float(ratio), _p(expo), _p(keep), _p(ws), ws.numel(),
                                stream), "gs_prune_select")
    return keep
