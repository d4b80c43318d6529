"""Pins of the oracle's training loss (Sec. 3.4, Eqs. 5-7 read as 1 - cosine on the
feature plus L1 on colour and depth, weights w_feat, w_rgb, w_depth, mean over pixels).

Each pin is fixed by something other than the oracle's own formula: hand-derived
closed forms (parallel, antiparallel, orthogonal and 45-degree vectors, zero rows, L1
of known differences), SciPy's independent cosine distance, central finite differences
of the scalar loss, and invariants of the cosine (scale invariance, hence a gradient
orthogonal to F).  CPU only."""
import numpy as np
import pytest
from scipy.spatial import distance

import oracle


def _one(F, G, C=(0.0, 0.0, 0.0), Cg=(0.0, 0.0, 0.0), D=0.0, Dg=0.0, **w):
    F = np.asarray(F, np.float64)[None]
    G = np.asarray(G, np.float64)[None]
    return oracle.loss_cos_l1(F, G, np.asarray([C]), np.asarray([Cg]), np.asarray([D]), np.asarray([Dg]), **w)


def test_parallel_and_antiparallel_closed_form():
    rng = np.random.default_rng(1)
    f = rng.standard_normal(16)
    lo, dF, _, _ = _one(f, 2.5 * f)                  # same direction: cos = 1
    assert abs(lo) < 1e-14 and np.abs(dF).max() < 1e-14
    lo, dF, _, _ = _one(f, -0.3 * f)                 # opposite: cos = -1, a maximum of 1 - cos
    assert abs(lo - 2.0) < 1e-14 and np.abs(dF).max() < 1e-14


def test_orthogonal_closed_form():
    # |F| = 2, |G| = 3, F.G = 0: loss 1, dL/dF = -G / (|F||G|) = -(0, 3, 0) / 6
    lo, dF, _, _ = _one([2.0, 0.0, 0.0], [0.0, 3.0, 0.0])
    assert lo == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(dF[0], [0.0, -0.5, 0.0], atol=1e-15)


def test_45_degrees_closed_form():
    # F = (1, 0), G = (1, 1): cos = 1/sqrt2, dL/dF = cos F / |F|^2 - G / (|F||G|) = (0, -1/sqrt2)
    lo, dF, _, _ = _one([1.0, 0.0], [1.0, 1.0], w_feat=3.0)
    assert lo == pytest.approx(3.0 * (1.0 - 2 ** -0.5), abs=1e-15)
    np.testing.assert_allclose(dF[0], [0.0, -3.0 * 2 ** -0.5], atol=1e-15)


def test_zero_rows_add_w_feat_and_no_gradient():
    for F, G in (([0.0, 0.0, 0.0], [1.0, 2.0, 3.0]), ([1.0, 2.0, 3.0], [0.0, 0.0, 0.0]), ([0.0] * 3, [0.0] * 3)):
        lo, dF, _, _ = _one(F, G, w_feat=0.7)
        assert lo == pytest.approx(0.7, abs=1e-15)
        assert np.all(dF == 0.0)


def test_l1_closed_form():
    # C - Cgt = (0.5, -0.25, 0): L1/3 = 0.25, dC = (1, -1, 0) w_rgb / 3; D - Dgt = -2: dD = -w_depth
    lo, dF, dC, dD = _one([1.0, 0.0], [1.0, 0.0], C=(1.5, 0.25, 0.4), Cg=(1.0, 0.5, 0.4), D=1.0, Dg=3.0,
                          w_rgb=0.6, w_depth=0.2)
    assert lo == pytest.approx(0.6 * 0.25 + 0.2 * 2.0, abs=1e-15)
    np.testing.assert_allclose(dC[0], [0.2, -0.2, 0.0], atol=1e-15)
    assert dD[0] == pytest.approx(-0.2, abs=1e-15)


def _random(P, Dim, seed):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((P, Dim))
    G = rng.standard_normal((P, Dim))
    C, Cg = rng.random((P, 3)), rng.random((P, 3))
    D, Dg = 1 + 4 * rng.random(P), 1 + 4 * rng.random(P)
    # keep every L1 argument at least 0.02 away from its kink
    C = np.where(np.abs(C - Cg) < 0.02, Cg + 0.05, C)
    D = np.where(np.abs(D - Dg) < 0.02, Dg + 0.05, D)
    return F, G, C, Cg, D, Dg


def test_feature_term_matches_scipy_cosine_distance():
    F, G, C, Cg, D, Dg = _random(9, 33, 2)
    lo, *_ = oracle.loss_cos_l1(F, G, C, C, D, D, w_feat=1.0, w_rgb=5.0, w_depth=5.0)
    want = np.mean([distance.cosine(F[p], G[p]) for p in range(9)])
    assert lo == pytest.approx(want, rel=1e-13)


def test_mean_over_pixels_and_chunk_shares():
    F, G, C, Cg, D, Dg = _random(12, 20, 3)
    w = dict(w_feat=1.3, w_rgb=0.4, w_depth=2.0)
    full, dF, dC, dD = oracle.loss_cos_l1(F, G, C, Cg, D, Dg, **w)
    singles = [oracle.loss_cos_l1(F[p:p + 1], G[p:p + 1], C[p:p + 1], Cg[p:p + 1], D[p:p + 1], Dg[p:p + 1], **w)
               for p in range(12)]
    assert full == pytest.approx(np.mean([s[0] for s in singles]), rel=1e-14)
    # per-pixel gradients of the mean are the single-pixel gradients / P
    np.testing.assert_allclose(dF, np.concatenate([s[1] for s in singles]) / 12, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(dC, np.concatenate([s[2] for s in singles]) / 12, rtol=1e-13)
    np.testing.assert_allclose(dD, np.concatenate([s[3] for s in singles]) / 12, rtol=1e-13)
    parts = [oracle.loss_cos_l1(F[a:a + 5], G[a:a + 5], C[a:a + 5], Cg[a:a + 5], D[a:a + 5], Dg[a:a + 5],
                                n_total=12, **w) for a in (0, 5, 10)]
    assert sum(p[0] for p in parts) == pytest.approx(full, rel=1e-14)
    np.testing.assert_array_equal(np.concatenate([p[1] for p in parts]), dF)


def test_central_differences():
    F, G, C, Cg, D, Dg = _random(4, 12, 4)
    w = dict(w_feat=0.9, w_rgb=1.7, w_depth=0.3)
    lo, dF, dC, dD = oracle.loss_cos_l1(F, G, C, Cg, D, Dg, **w)
    h = 1e-6

    def fd(arr, name):
        g = np.zeros_like(arr)
        for i in np.ndindex(arr.shape):
            a, b = arr.copy(), arr.copy()
            a[i] += h
            b[i] -= h
            args = dict(F=F, C=C, D=D)
            args[name] = a
            la = oracle.loss_cos_l1(args["F"], G, args["C"], Cg, args["D"], Dg, **w)[0]
            args[name] = b
            lb = oracle.loss_cos_l1(args["F"], G, args["C"], Cg, args["D"], Dg, **w)[0]
            g[i] = (la - lb) / (2 * h)
        return g

    np.testing.assert_allclose(dF, fd(F, "F"), rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(dC, fd(C, "C"), rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(dD, fd(D, "D"), rtol=1e-6, atol=1e-9)


def test_scale_invariance_and_orthogonal_gradient():
    F, G, C, Cg, D, Dg = _random(6, 24, 5)
    lo, dF, _, _ = oracle.loss_cos_l1(F, G, C, Cg, D, Dg)
    # the cosine does not change along F, so its gradient is orthogonal to F
    dots = np.abs((dF * F).sum(1)) / (np.linalg.norm(dF, axis=1) * np.linalg.norm(F, axis=1))
    assert dots.max() < 1e-13
    a = 3.7
    lo2, dF2, _, _ = oracle.loss_cos_l1(a * F, G, C, Cg, D, Dg)
    assert lo2 == pytest.approx(lo, rel=1e-14)
    np.testing.assert_allclose(dF2, dF / a, rtol=1e-12, atol=1e-18)
