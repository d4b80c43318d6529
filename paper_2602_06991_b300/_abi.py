"""ctypes declarations of the C ABI in include/gs_topk.h (argument marshalling only).

Every stage of the render runs in libgs_topk.so; there is no Python or CPU
fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgs_topk.so")

GS_OK, GS_ERR_ARG, GS_ERR_WORKSPACE, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_OVERFLOW, GS_ERR_UNSUPPORTED = range(7)
GS_BWD_H_FROM_LOSS = 1      # gs_backward_ex flag: reuse the h terms gs_feature_blend_loss left in ws
GS_F32, GS_BF16 = 0, 1
GS_MAX_CAMERAS = 16
GS_MAX_K = 32
GS_PROJ_FLOATS = 16
GS_LOSS_NOALLOC_MAX_PIX = 1 << 22
# kernel timers (gs_timer_enable / gs_timer_read)
(GS_TIMER_BINNING, GS_TIMER_TILE_SORT, GS_TIMER_WALK_FWD, GS_TIMER_BLOCK_GRAD, GS_TIMER_WALK_BWD,
 GS_TIMER_COMPLETE) = range(6)
GS_TIMER_COUNT = 6

c_float_p = ctypes.c_void_p
vp = ctypes.c_void_p


class GsCamera(ctypes.Structure):
    _fields_ = [("viewmat", ctypes.c_float * 16), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("near_z", ctypes.c_float)]


class GsConfig(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("D", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("tile_h", ctypes.c_int32), ("feat_dtype", ctypes.c_int32), ("max_instances", ctypes.c_int32),
                ("max_feature_rows", ctypes.c_int32), ("topk_layout", ctypes.c_int32),
                ("depth_cut", ctypes.c_int32)]


class GsGrads(ctypes.Structure):
    _fields_ = [("feat", vp), ("opacity", vp), ("rgb", vp), ("mean3d", vp), ("cov3d", vp),
                ("mean2d", vp), ("conic", vp), ("viewmat", vp)]


class GsAdamTensor(ctypes.Structure):
    _fields_ = [("param", vp), ("grad", vp), ("exp_avg", vp), ("exp_avg_sq", vp), ("n", ctypes.c_int64),
                ("lr", ctypes.c_float), ("param_bf16", vp)]


GS_ADAM_MAX_TENSORS = 16


class GsError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


# exported symbols and their prototypes: (restype, argtypes)
PROTOTYPES = {
    "gs_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gs_version": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)] * 3),
    "gs_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(GsConfig), ctypes.POINTER(GsCamera), ctypes.c_int32,
                                            ctypes.c_int32]),
    "gs_pixel_count": (ctypes.c_int64, [ctypes.POINTER(GsCamera), ctypes.c_int32]),
    "gs_preprocess": (ctypes.c_int, [ctypes.POINTER(GsConfig), ctypes.POINTER(GsCamera), ctypes.c_int32,
                                     ctypes.c_int32, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]),
    "gs_bin_sort": (ctypes.c_int, [ctypes.POINTER(GsConfig), ctypes.POINTER(GsCamera), ctypes.c_int32,
                                   ctypes.c_int32, vp, vp, ctypes.c_size_t, vp]),
    "gs_topk_select": (ctypes.c_int, [ctypes.POINTER(GsConfig), ctypes.POINTER(GsCamera), ctypes.c_int32,
                                      ctypes.c_int32, vp, vp, ctypes.c_size_t, vp, vp, vp, vp, vp, vp, vp]),
    "gs_feature_blend": (ctypes.c_int, [ctypes.POINTER(GsConfig), ctypes.c_int64, ctypes.c_int32, vp, vp, vp, vp,
                                        vp]),
    "gs_backward": (ctypes.c_int, [ctypes.POINTER(GsConfig), ctypes.POINTER(GsCamera), ctypes.c_int32,
                                   ctypes.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                   ctypes.POINTER(GsGrads), vp, ctypes.c_size_t, vp]),
    "gs_backward_ex": (ctypes.c_int, [ctypes.POINTER(GsConfig), ctypes.POINTER(GsCamera), ctypes.c_int32,
                                      ctypes.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                      ctypes.POINTER(GsGrads), ctypes.c_uint32, vp, ctypes.c_size_t, vp]),
    "gs_loss_scratch_size": (ctypes.c_size_t, [ctypes.c_int64]),
    "gs_loss_cos_l1": (ctypes.c_int, [ctypes.POINTER(GsConfig), ctypes.c_int64, vp, vp, vp, vp, vp, vp,
                                      ctypes.c_float, ctypes.c_float, ctypes.c_float, vp, vp, vp, vp, vp,
                                      ctypes.c_size_t, vp]),
    "gs_feature_blend_loss": (ctypes.c_int, [ctypes.POINTER(GsConfig), ctypes.POINTER(GsCamera), ctypes.c_int32,
                                             ctypes.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_float,
                                             ctypes.c_float, ctypes.c_float, vp, vp, vp, vp, vp, vp, ctypes.c_size_t,
                                             vp, ctypes.c_size_t, vp]),
    "gs_loss_cos_l1_noalloc": (ctypes.c_int, [ctypes.POINTER(GsConfig), ctypes.c_int64, vp, vp, vp, vp, vp, vp,
                                              ctypes.c_float, ctypes.c_float, ctypes.c_float, vp, vp, vp, vp, vp]),
    "gs_loss_geo_l1": (ctypes.c_int, [ctypes.c_int64, vp, vp, vp, vp, ctypes.c_float, ctypes.c_float, vp, vp, vp, vp,
                                      ctypes.c_size_t, vp]),
    "gs_adam_step": (ctypes.c_int, [ctypes.POINTER(GsAdamTensor), ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, vp]),
    "gs_feature_blend_vanilla": (ctypes.c_int, [ctypes.POINTER(GsConfig), ctypes.POINTER(GsCamera), ctypes.c_int32,
                                                ctypes.c_int32, vp, vp, vp, vp, ctypes.c_size_t, vp]),
    "gs_prune_stats": (ctypes.c_int, [ctypes.POINTER(GsConfig), ctypes.POINTER(GsCamera), ctypes.c_int32,
                                      ctypes.c_int32, vp, vp, vp, ctypes.c_size_t, vp, vp, vp]),
    "gs_prune_select_workspace_size": (ctypes.c_size_t, [ctypes.c_int32]),
    "gs_prune_select": (ctypes.c_int, [ctypes.c_int32, vp, vp, ctypes.c_int32, ctypes.c_double, vp, vp, vp,
                                       ctypes.c_size_t, vp]),
    "gs_set_wait_limit": (ctypes.c_int, [vp, ctypes.c_size_t, ctypes.c_int64, vp]),
    "gs_workspace_counts": (ctypes.c_int, [vp, ctypes.c_size_t, vp, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_int64)]),
    "gs_sync_status": (ctypes.c_int, [vp, ctypes.c_size_t, vp, ctypes.POINTER(ctypes.c_int64)]),
    "gs_binning_stats": (ctypes.c_int, [vp, ctypes.c_size_t, vp, ctypes.POINTER(ctypes.c_int64)]),
    "gs_timer_enable": (ctypes.c_int, [ctypes.c_int]),
    "gs_timer_read": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libgs_topk.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run `python -m paper_2602_06991_b300.build`)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load().gs_status_string(int(status)).decode()
    except Exception:
        return "unknown"


def check(status: int, what: str):
    if status != GS_OK:
        raise GsError(status, what)


def make_cameras(cams):
    """Array of GsCamera from objects with viewmat (4x4), fx, fy, cx, cy, width,
    height and near (or near_z)."""
    if len(cams) < 1 or len(cams) > GS_MAX_CAMERAS:
        raise ValueError(f"1..{GS_MAX_CAMERAS} cameras, got {len(cams)}")
    arr = (GsCamera * len(cams))()
    for a, c in zip(arr, cams):
        vm = [float(v) for row in c.viewmat for v in row] if hasattr(c.viewmat, "__len__") and \
            len(c.viewmat) == 4 else [float(v) for v in c.viewmat]
        a.viewmat[:] = vm
        a.fx, a.fy, a.cx, a.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        a.width, a.height = int(c.width), int(c.height)
        a.near_z = float(getattr(c, "near", getattr(c, "near_z", 0.2)))
    return arr


def timer_enable(on: bool):
    """Turn the library's kernel timers on (clearing earlier records) or off."""
    check(load().gs_timer_enable(1 if on else 0), "gs_timer_enable")


def timer_read(timer_id: int):
    """Milliseconds of the last recorded launch of a timed stage, or None if none was recorded."""
    ms = ctypes.c_float(0.0)
    st = load().gs_timer_read(int(timer_id), ctypes.byref(ms))
    if st == GS_ERR_ARG:
        return None
    check(st, "gs_timer_read")
    return float(ms.value)
