"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/gs_topk.h declares, and its pure host logic (workspace sizing, pixel
counts, argument validation, status strings) behaves.  No call here launches work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs_topk.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2602_06991_b300 import build, _abi
    build()
    return _abi.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_stage_calls():
    names = declared_functions()
    for stage in ("gs_preprocess", "gs_bin_sort", "gs_topk_select", "gs_feature_blend", "gs_backward"):
        assert stage in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2602_06991_b300 import _abi
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported"
        assert name in _abi.PROTOTYPES, f"{name} has no ctypes prototype"


def test_built_for_sm103(lib):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert lib.gs_version(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)) == 0
    assert c.value == 103


def _cams(*sizes):
    import gs_scenes as S
    from paper_2602_06991_b300 import _abi
    return _abi.make_cameras([S.pinhole(w, h, 100.0) for (w, h) in sizes])


def test_pixel_count_and_workspace(lib):
    from paper_2602_06991_b300 import _abi as A
    cams = _cams((128, 96), (100, 75))
    assert lib.gs_pixel_count(cams, 2) == 128 * 96 + 100 * 75
    assert lib.gs_pixel_count(cams, 0) == -1
    cfg = A.GsConfig(4, 16, 16, 16, A.GS_F32, 0)
    w1 = lib.gs_workspace_size(ctypes.byref(cfg), cams, 2, 1000)
    w2 = lib.gs_workspace_size(ctypes.byref(cfg), cams, 2, 2000)
    assert 0 < w1 < w2 and w1 % 256 == 0
    cfg.max_instances = 1 << 20
    assert lib.gs_workspace_size(ctypes.byref(cfg), cams, 2, 1000) > w1
    assert lib.gs_workspace_size(ctypes.byref(cfg), cams, 2, 0) > 0     # empty scene is valid


@pytest.mark.parametrize("field,value", [("K", 0), ("K", 33), ("D", 12), ("D", 0), ("D", 2048),
                                         ("tile_w", 12), ("feat_dtype", 7), ("max_instances", -1),
                                         ("max_feature_rows", -1), ("depth_cut", 2), ("depth_cut", -1),
                                         ("topk_layout", 3), ("topk_layout", -1)])
def test_bad_config_rejected_on_host(lib, field, value):
    from paper_2602_06991_b300 import _abi as A
    cams = _cams((64, 48))
    cfg = A.GsConfig(4, 16, 16, 16, A.GS_F32, 0)
    setattr(cfg, field, value)
    assert lib.gs_workspace_size(ctypes.byref(cfg), cams, 1, 10) == 0
    st = lib.gs_preprocess(ctypes.byref(cfg), cams, 1, 10, None, None, None, None, None, None, 0, None)
    assert st == A.GS_ERR_ARG
    st = lib.gs_feature_blend(ctypes.byref(cfg), 10, 10, None, None, None, None, None)
    assert st == A.GS_ERR_ARG


def test_bad_workspace_rejected_on_host(lib):
    from paper_2602_06991_b300 import _abi as A
    cams = _cams((64, 48))
    cfg = A.GsConfig(4, 16, 16, 16, A.GS_F32, 0)
    need = lib.gs_workspace_size(ctypes.byref(cfg), cams, 1, 10)
    fake = ctypes.c_void_p(1 << 40)           # never dereferenced: rejected before any launch
    for ws, nbytes in [(None, need), (fake, need - 1), (ctypes.c_void_p((1 << 40) + 16), need)]:
        st = lib.gs_bin_sort(ctypes.byref(cfg), cams, 1, 10, fake, ws, nbytes, None)
        assert st == A.GS_ERR_WORKSPACE


def test_bad_cameras_rejected(lib):
    import gs_scenes as S
    from paper_2602_06991_b300 import _abi as A
    cfg = A.GsConfig(4, 16, 16, 16, A.GS_F32, 0)
    bad = A.make_cameras([S.pinhole(64, 48, -1.0)])
    assert lib.gs_workspace_size(ctypes.byref(cfg), bad, 1, 10) == 0
    ok = A.make_cameras([S.pinhole(64, 48, 50.0)] * 3)
    assert lib.gs_workspace_size(ctypes.byref(cfg), ok, 17, 10) == 0


def test_status_strings(lib):
    from paper_2602_06991_b300 import _abi as A
    for s in range(7):
        assert lib.gs_status_string(s).decode()
    assert "capacity" in lib.gs_status_string(A.GS_ERR_OVERFLOW).decode()


def test_missing_library_fails_loudly(tmp_path):
    from paper_2602_06991_b300 import _abi as A
    saved = A._lib
    try:
        A._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            A.load(str(tmp_path / "nope.so"))
    finally:
        A._lib = saved


def test_timers_without_records(lib):
    """The kernel timers answer 'nothing recorded' (and reject unknown ids) without any
    device work: enabling clears the records, reads need a recorded launch."""
    from paper_2602_06991_b300 import _abi as A
    A.timer_enable(True)
    try:
        for t in range(A.GS_TIMER_COUNT):
            assert A.timer_read(t) is None
        ms = ctypes.c_float(0.0)
        assert lib.gs_timer_read(A.GS_TIMER_COUNT, ctypes.byref(ms)) == A.GS_ERR_ARG
        assert lib.gs_timer_read(-1, ctypes.byref(ms)) == A.GS_ERR_ARG
        assert lib.gs_timer_read(0, None) == A.GS_ERR_ARG
    finally:
        A.timer_enable(False)
