"""GPU parity of the consistency-pruning statistics and survival selection (Sec. 3.3,
Eqs. 8-9) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import gs_scenes as S
import oracle
import parity_util as U

pytestmark = pytest.mark.gpu


def _touched_by_flagged(sc, cam, flags):
    """Gaussians that contribute at a pixel whose decisions sit within the oracle's
    margins (an FP32 walk may decide those the other way)."""
    ids = set()
    for p in np.nonzero((flags & (U.FRAGILE_SET | oracle.F_NEAR_TIE)) != 0)[0]:
        g, *_ = oracle.pixel_walk(sc, cam, p % cam.width + 0.5, p // cam.width + 0.5)
        ids.update(int(x) for x in g)
    return np.array(sorted(ids), dtype=np.int64)


def _compare(sc, cams, K, acc, runs):
    cnt = np.zeros(sc.n, np.int64)
    mw = np.zeros(sc.n)
    skip = []
    for cam in runs:
        r = oracle.prune_stats(sc, cam, K, count=cnt, maxw=mw)
        skip.append(_touched_by_flagged(sc, cam, r["flags"]))
    skip = np.unique(np.concatenate(skip)) if skip else np.zeros(0, np.int64)
    ok = np.ones(sc.n, bool)
    ok[skip] = False
    g_cnt = acc["count"].cpu().numpy().astype(np.int64)
    g_S = acc["S"].cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(g_cnt[ok], cnt[ok])
    rel = np.abs(g_S[ok] - mw[ok]) / np.maximum(mw[ok], 1e-12)
    assert rel.max() <= 1e-5, rel.max()
    assert (g_S[ok] > 0).sum() == (mw[ok] > 0).sum()
    return int((~ok).sum())


def test_prune_stats_small_vs_oracle():
    sc, cams, K, tile, _ = S.make_config("small", 0)
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    acc = r.prune_stats(r.alloc_prune_stats(sc.n))
    torch.cuda.synchronize()
    skipped = _compare(sc, cams, K, acc, cams)
    print("skipped", skipped, "of", sc.n)


def test_prune_stats_accumulate_over_views():
    """Two renders of two ragged cameras each, accumulated into one window: counts add
    and S keeps the maximum, as the oracle over the four views."""
    sc = S.random_scene_box(14, 2500, 8, box=((-1, 1), (-1, 1), (2, 4)))
    views1 = S.orbit_cameras(15, [(61, 45, 60.0), (40, 33, 45.0)], radius=3.0)
    views2 = S.orbit_cameras(16, [(52, 37, 55.0), (33, 29, 40.0)], radius=3.0)
    r1, ts, _ = U.gpu_forward(sc, views1, 5, (16, 8))
    acc = r1.prune_stats(r1.alloc_prune_stats(sc.n))
    r2, _, _ = U.gpu_forward(sc, views2, 5, (8, 8))
    r2.prune_stats(acc)
    torch.cuda.synchronize()
    _compare(sc, views1 + views2, 5, acc, views1 + views2)


def test_prune_stats_frame_properties():
    """'frame' workload (200k Gaussians, 640x480, K=8) in the benchmark's launch
    configuration: the counts are the histogram of the Top-K ids; S bounds every Top-K
    weight of its Gaussian from above, lies in (0, 0.99] exactly where the Gaussian
    contributes, and is the same for every tile shape."""
    sc, cams, K, tile, _ = S.make_config("frame", 0)
    r, ts, out = U.gpu_forward(sc, cams, K, tile)
    acc = r.prune_stats(r.alloc_prune_stats(sc.n))
    idx = out["topk_idx"].long()
    sel = idx >= 0
    want = torch.bincount(idx[sel], minlength=sc.n)
    assert torch.equal(acc["count"].long(), want)
    wmax = torch.zeros(sc.n, device="cuda").scatter_reduce(0, idx[sel], out["topk_w"][sel], reduce="amax")
    assert torch.all(acc["S"] >= wmax)
    assert torch.all(acc["S"] <= 0.99) and torch.all(acc["S"][want > 0] > 0)
    r2, _, _ = U.gpu_forward(sc, cams, K, (32, 8))
    acc2 = r2.prune_stats(r2.alloc_prune_stats(sc.n))
    torch.cuda.synchronize()
    assert torch.equal(acc["S"], acc2["S"]) and torch.equal(acc["count"], acc2["count"])


@pytest.mark.parametrize("N,tau,ratio", [(1, 1, 0.5), (1000, 2, 0.5), (1000, 3, 0.0), (1000, 3, 1.0),
                                         (1_000_003, 2, 0.5), (200_000, 5, 0.3)])
def test_prune_select_matches_oracle(N, tau, ratio):
    """Seeded synthetic statistics (integer counts, S with zeros and repeated values,
    Exp(1) variates): the kept set equals the oracle's, bit for bit."""
    from paper_2602_06991_b300.renderer import prune_select
    rng = np.random.default_rng(N + tau)
    count = rng.integers(0, 8, N).astype(np.int32)
    Sv = rng.random(N).astype(np.float32)
    Sv[rng.random(N) < 0.05] = 0.0
    Sv[rng.random(N) < 0.05] = 0.5                      # repeated values
    e = rng.exponential(size=N).astype(np.float32)
    keep = prune_select(torch.from_numpy(count).cuda(), torch.from_numpy(Sv).cuda(), tau, ratio,
                        torch.from_numpy(e).cuda())
    want = oracle.prune_select(count, Sv, tau, ratio, e)
    got = keep.cpu().numpy().astype(bool)
    assert np.array_equal(got, want), (np.nonzero(got != want)[0][:10], got.sum(), want.sum())
