"""Pins for the oracle's consistency-pruning statistics and survival sampling (Sec. 3.3,
Eqs. 8-9): closed forms of one and two on-axis Gaussians worked out by hand, a brute
force over a tiny scene, and the sampling law of Eq. 9 checked by frequency.  CPU only."""
import numpy as np
import pytest

import gs_scenes as S
import oracle
from test_oracle_pins import axis_cam, iso, scene_from


def test_single_gaussian_count_and_importance_closed_form():
    """One isotropic on-axis Gaussian (Sigma2D = ((f s / z)^2 + 0.3) I): it takes part
    at exactly the pixel centres with q <= 9 and o exp(-q/2) >= 1/255, is the Top-1
    there (so its count is that pixel number), and its importance S (Eq. 8) is its
    largest weight, o at the principal point (w = alpha, T = 1)."""
    f, s, z, o = 20.0, 0.1, 2.0, 0.8
    cam = axis_cam(f, 16, 16)
    sc = scene_from([0, 0, z], iso(s), [o], [1, 1, 1], [[1.0]])
    var = (f * s / z) ** 2 + 0.3
    xs = np.arange(16) + 0.5
    dx, dy = np.meshgrid(xs - cam.cx, xs - cam.cy)
    q = (dx ** 2 + dy ** 2) / var
    alpha = np.minimum(0.99, o * np.exp(-0.5 * q))
    takes_part = (q <= 9) & (alpha >= 1 / 255)
    r = oracle.prune_stats(sc, cam, K=1)
    assert r["count"][0] == takes_part.sum()
    np.testing.assert_allclose(r["maxw"][0], o, rtol=1e-15)


def test_two_stacked_count_and_importance_closed_form():
    """Front A (o = 0.3) over back B (o = 0.9) on the axis, both wide: at the principal
    point w_A = 0.3 and w_B = 0.9 (1 - 0.3) = 0.63, so the Top-1 there is B; S_B = 0.63
    and S_A = 0.3 are the weights at the centre.  With K = 2 both are counted at every
    pixel where both take part."""
    cam = axis_cam(20.0, 8, 8)
    oa, ob = 0.3, 0.9
    sc = scene_from([[0, 0, 1.5], [0, 0, 2.5]], [iso(0.4), iso(0.6)], [oa, ob], [[1, 0, 0]] * 2, [[1.0]] * 2)
    r1 = oracle.prune_stats(sc, cam, K=1)
    np.testing.assert_allclose(r1["maxw"], [oa, ob * (1 - oa)], rtol=1e-14)
    centre = oracle.prune_stats(sc, cam, K=1, pixels=[(cam.height // 2) * cam.width + cam.width // 2])
    np.testing.assert_array_equal(centre["count"], [0, 1])
    r2 = oracle.prune_stats(sc, cam, K=2)
    assert r2["count"][0] == r2["count"][1] == cam.n_pix      # both wide: every pixel holds both


def test_counts_and_importance_brute_force():
    """Tiny random scene: the counts equal, Gaussian by Gaussian, the number of pixels
    whose rendered Top-K set holds it, and S equals the largest walk weight found by
    walking every pixel -- two independent routes through the per-pixel definition."""
    sc = S.random_scene_box(21, 40, 4, box=((-0.5, 0.5), (-0.5, 0.5), (1.5, 3)), log_scale_mu=-2.0)
    cam = S.pinhole(24, 18, 30.0)
    K = 3
    r = oracle.prune_stats(sc, cam, K)
    rend = oracle.render(sc, cam, K)
    want_count = np.zeros(sc.n, np.int64)
    for row in rend["idx"]:
        for g in row[row >= 0]:
            want_count[g] += 1
    np.testing.assert_array_equal(r["count"], want_count)
    want_S = np.zeros(sc.n)
    for p in range(cam.n_pix):
        ids, a, T, w, _, _ = oracle.pixel_walk(sc, cam, p % cam.width + 0.5, p // cam.width + 0.5)
        for g, wi in zip(ids, w):
            want_S[g] = max(want_S[g], wi)
    np.testing.assert_allclose(r["maxw"], want_S, rtol=1e-15)
    assert (r["maxw"] <= 1).all() and (r["count"] <= cam.n_pix).all()
    # accumulation over views: two calls add counts and keep the maximum
    acc_c, acc_s = np.zeros(sc.n, np.int64), np.zeros(sc.n)
    oracle.prune_stats(sc, cam, K, pixels=np.arange(0, cam.n_pix, 2), count=acc_c, maxw=acc_s)
    oracle.prune_stats(sc, cam, K, pixels=np.arange(1, cam.n_pix, 2), count=acc_c, maxw=acc_s)
    np.testing.assert_array_equal(acc_c, r["count"])
    np.testing.assert_allclose(acc_s, r["maxw"], rtol=0)


def test_survival_sampling_first_draw_follows_eq9():
    """With one survivor the chance that candidate i survives is S_i / sum S (Eq. 9):
    checked by frequency over 40k seeded exponential draws (5 sigma)."""
    S_ = np.array([0.05, 0.1, 0.2, 0.4, 0.25], dtype=np.float32)
    count = np.zeros(5, np.int64)                     # all candidates (count < tau = 1)
    rng = np.random.default_rng(5)
    trials = 40000
    hits = np.zeros(5)
    for _ in range(trials):
        keep = oracle.prune_select(count, S_, tau=1, ratio=0.2, expo=rng.exponential(size=5))
        assert keep.sum() == 1
        hits[np.argmax(keep)] += 1
    p = S_ / S_.sum()
    sigma = np.sqrt(trials * p * (1 - p))
    assert np.all(np.abs(hits - trials * p) < 5 * sigma), (hits / trials, p)


def test_survival_sampling_is_without_replacement():
    """Two survivors of three candidates: P({i, j}) = p_i p_j / (1 - p_i) + p_j p_i / (1 - p_j),
    the law of two successive draws without replacement with p = S / sum S."""
    S_ = np.array([0.6, 0.3, 0.1], dtype=np.float32)
    count = np.zeros(3, np.int64)
    rng = np.random.default_rng(6)
    trials = 40000
    pairs = {}
    for _ in range(trials):
        keep = oracle.prune_select(count, S_, tau=1, ratio=2 / 3, expo=rng.exponential(size=3))
        assert keep.sum() == 2
        key = tuple(np.nonzero(keep)[0])
        pairs[key] = pairs.get(key, 0) + 1
    p = S_.astype(np.float64) / S_.sum()
    for (i, j) in [(0, 1), (0, 2), (1, 2)]:
        want = p[i] * p[j] / (1 - p[i]) + p[j] * p[i] / (1 - p[j])
        got = pairs.get((i, j), 0) / trials
        assert abs(got - want) < 5 * np.sqrt(want * (1 - want) / trials), ((i, j), got, want)


def test_survival_selection_rules():
    """Non-candidates (count >= tau) always survive; exactly floor(ratio |G_prune| + 1/2)
    candidates survive; a candidate with S = 0 is never chosen before one with S > 0;
    ratio 0 prunes every candidate and ratio 1 keeps all."""
    rng = np.random.default_rng(7)
    n = 50
    count = rng.integers(0, 6, n)
    S_ = rng.random(n).astype(np.float32)
    S_[::7] = 0.0
    e = rng.exponential(size=n)
    for tau, ratio in [(2, 0.5), (3, 0.3), (6, 0.25), (0, 0.5), (3, 0.0), (3, 1.0)]:
        keep = oracle.prune_select(count, S_, tau, ratio, e)
        cand = count < tau
        assert keep[~cand].all()
        m = int(np.floor(ratio * cand.sum() + 0.5))
        assert keep[cand].sum() == m
        pos = cand & (S_ > 0)
        if m <= pos.sum():
            assert not (keep & cand & (S_ == 0)).any()


# ----------------------------------------------------------------------------------
# vanilla (full alpha-blending) feature render
# ----------------------------------------------------------------------------------
def test_vanilla_two_stacked_closed_form():
    """Front A over back B on the axis: F = w_A f_A + w_B f_B with w_A = o_A and
    w_B = o_B (1 - o_A) -- unnormalised, unlike Top-K's Eq. 3."""
    cam = axis_cam()
    oa, ob = 0.3, 0.9
    fa, fb = np.array([1.0, 0.0, 0.5]), np.array([0.0, 1.0, -0.5])
    sc = scene_from([[0, 0, 1.5], [0, 0, 2.5]], [iso(0.05)] * 2, [oa, ob], [[1, 0, 0]] * 2, [fa, fb])
    c = [(cam.height // 2) * cam.width + cam.width // 2]
    r = oracle.render_vanilla(sc, cam, pixels=c)
    np.testing.assert_allclose(r["F"][0], oa * fa + ob * (1 - oa) * fb, rtol=1e-14)


def test_vanilla_is_scaled_full_topk():
    """With K at least the contributor count, Top-K renormalises the full blend:
    F_topK = F_vanilla / (1 - T_final), pixel by pixel (and F_vanilla = 0 where nothing
    contributes)."""
    sc = S.random_scene_box(22, 300, 6, box=((-1, 1), (-1, 1), (1.5, 4)), log_scale_mu=-2.5)
    cam = S.pinhole(32, 24, 40.0)
    v = oracle.render_vanilla(sc, cam)
    t = oracle.render(sc, cam, K=400)
    assert t["n"].max() < 400
    has = t["n"] > 0
    np.testing.assert_allclose(v["F"][has], t["F"][has] * (1 - t["T"][has, None]), rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(v["F"][~has], 0.0)
