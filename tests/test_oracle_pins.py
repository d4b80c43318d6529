"""Pins for the FP64 oracle: each test fixes part of it against something other than
itself -- closed forms of special cases, a hand-derived golden fixture, invariants
the paper's definitions imply, brute force on tiny scenes, a finite-difference
Jacobian of the pinhole projection, and central finite differences of the forward
for the backward.  CPU only."""
import itertools
import json
import os

import numpy as np
import pytest

import gs_scenes as S
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def scene_from(mean, cov6, opac, rgb, feats, dtype=np.float64):
    return S.Scene(np.asarray(mean, dtype).reshape(-1, 3), np.asarray(cov6, dtype).reshape(-1, 6),
                   np.asarray(opac, dtype).reshape(-1), np.asarray(rgb, dtype).reshape(-1, 3),
                   np.asarray(feats, dtype).reshape(len(opac), -1))


def iso(s):
    return [s * s, 0, 0, s * s, 0, s * s]


def axis_cam(f=20.0, w=16, h=16):
    # principal point on the centre of pixel (w//2, h//2)
    return S.pinhole(w, h, f, cx=w // 2 + 0.5, cy=h // 2 + 0.5)


def centre_pixel(cam):
    return [(cam.height // 2) * cam.width + cam.width // 2]


# ----------------------------------------------------------------------------------
# closed forms
# ----------------------------------------------------------------------------------
def test_single_isotropic_gaussian_closed_form():
    """On the optical axis, an isotropic Gaussian of std s at depth z projects to
    Sigma2D = ((f s / z)^2 + 0.3) I; at the principal point alpha = opacity, the
    only contributor has w = alpha and its row is the feature exactly (S = w)."""
    f, s, z, o = 30.0, 0.04, 2.0, 0.7
    cam = axis_cam(f)
    sc = scene_from([0, 0, z], iso(s), [o], [0.2, 0.5, 0.9], [[0.6, -0.8, 0.0]])
    pr = oracle.project(sc, cam)[0]
    var = (f * s / z) ** 2 + 0.3
    assert pr[oracle.P_VALID] == 1
    np.testing.assert_allclose([pr[oracle.P_SA], pr[oracle.P_SB], pr[oracle.P_SC]], [var, 0, var], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose([pr[oracle.P_U], pr[oracle.P_V]], [cam.cx, cam.cy], rtol=1e-15)
    r = oracle.render(sc, cam, K=4, pixels=centre_pixel(cam))
    assert r["n"][0] == 1
    np.testing.assert_allclose(r["w"][0], [o, 0, 0, 0], rtol=1e-15)
    np.testing.assert_array_equal(r["idx"][0], [0, -1, -1, -1])
    np.testing.assert_allclose(r["T"][0], 1 - o, rtol=1e-15)
    np.testing.assert_allclose(r["F"][0], [0.6, -0.8, 0.0], rtol=1e-15)
    np.testing.assert_allclose(r["C"][0], o * np.array([0.2, 0.5, 0.9]), rtol=1e-15)
    np.testing.assert_allclose(r["D"][0], o * z, rtol=1e-15)
    # off-centre along x by 2 px: alpha = o exp(-(2^2) / (2 var))
    px = centre_pixel(cam)[0] + 2
    r2 = oracle.render(sc, cam, K=1, pixels=[px])
    np.testing.assert_allclose(r2["w"][0, 0], o * np.exp(-4.0 / (2 * var)), rtol=1e-14)


def test_ellipse_cutoff_closed_form():
    """q <= 9 decides participation: with Sigma2D = 1.3 I a pixel 3 px away has
    q = 9/1.3 < 9 and takes part, one 4 px away has q = 16/1.3 > 9 and does not."""
    f, z = 20.0, 2.0
    s = z / f                        # (f s / z)^2 = 1  ->  var = 1.3
    cam = axis_cam(f)
    sc = scene_from([0, 0, z], iso(s), [0.9], [1, 1, 1], [[1.0, 0.0]])
    c = centre_pixel(cam)[0]
    r = oracle.render(sc, cam, K=2, pixels=[c + 3, c + 4, c + 3 * cam.width])
    np.testing.assert_array_equal(r["n"], [1, 0, 1])
    np.testing.assert_allclose(r["w"][0, 0], 0.9 * np.exp(-9 / 2.6), rtol=1e-14)
    np.testing.assert_allclose(r["F"][1], [0, 0])


def test_alpha_cutoff_and_clamp():
    """alpha < 1/255 is skipped (pixel stays empty, F = 0); opacity above 0.99 is
    clamped to 0.99."""
    cam = axis_cam()
    c = centre_pixel(cam)
    low = scene_from([0, 0, 2], iso(0.05), [0.003], [1, 1, 1], [[1.0, 0.0]])
    r = oracle.render(low, cam, K=2, pixels=c)
    assert r["n"][0] == 0 and r["T"][0] == 1.0
    np.testing.assert_array_equal(r["idx"][0], [-1, -1])
    np.testing.assert_array_equal(r["F"][0], [0, 0])
    high = scene_from([0, 0, 2], iso(0.05), [0.999], [1, 1, 1], [[1.0, 0.0]])
    r = oracle.render(high, cam, K=2, pixels=c)
    np.testing.assert_allclose(r["w"][0, 0], 0.99, rtol=1e-15)
    np.testing.assert_allclose(r["T"][0], 0.01, rtol=1e-13)


def test_termination_closed_form():
    """Five on-axis Gaussians of opacity 0.95: T goes 1, 0.05, 0.0025, 1.25e-4; the
    fourth would take it to 6.25e-6 < 1e-4, so the walk stops before it."""
    cam = axis_cam()
    sc = scene_from([[0, 0, z] for z in (1, 2, 3, 4, 5)], [iso(0.05)] * 5, [0.95] * 5,
                    [[1, 0, 0]] * 5, [[1.0]] * 5)
    r = oracle.render(sc, cam, K=8, pixels=centre_pixel(cam))
    assert r["n"][0] == 3
    np.testing.assert_allclose(r["T"][0], 0.05 ** 3, rtol=1e-12)
    np.testing.assert_allclose(r["w"][0, :3], [0.95, 0.95 * 0.05, 0.95 * 0.0025], rtol=1e-12)


def test_two_stacked_closed_form():
    """Two on-axis Gaussians: w2 = alpha2 (1 - alpha1); Top-1 keeps the arg-max,
    Top-2 blends with weights w / (w1 + w2)."""
    cam = axis_cam()
    o1, o2 = 0.3, 0.9
    f1, f2 = np.array([1.0, 0.0]), np.array([0.0, 1.0])
    sc = scene_from([[0, 0, 1.5], [0, 0, 2.5]], [iso(0.05)] * 2, [o1, o2], [[1, 0, 0], [0, 1, 0]], [f1, f2])
    w1, w2 = o1, o2 * (1 - o1)
    r1 = oracle.render(sc, cam, K=1, pixels=centre_pixel(cam))
    assert r1["idx"][0, 0] == 1                      # w2 = 0.63 > w1 = 0.3
    np.testing.assert_allclose(r1["F"][0], f2, rtol=1e-15)
    r2 = oracle.render(sc, cam, K=2, pixels=centre_pixel(cam))
    np.testing.assert_array_equal(r2["idx"][0], [1, 0])
    np.testing.assert_allclose(r2["F"][0], (w1 * f1 + w2 * f2) / (w1 + w2), rtol=1e-14)
    np.testing.assert_allclose(r2["D"][0], w1 * 1.5 + w2 * 2.5, rtol=1e-14)


def test_golden_three_on_axis():
    with open(os.path.join(GOLDEN, "three_on_axis.json")) as fh:
        gd = json.load(fh)
    c, g, e = gd["camera"], gd["gaussians"], gd["expected"]
    cam = S.pinhole(c["width"], c["height"], c["fx"], c["fy"], c["cx"], c["cy"])
    sc = scene_from(g["mean3d"], [iso(s) for s in g["scale"]], g["opacity"], g["rgb"], g["feats"])
    pix = [gd["pixel"][1] * c["width"] + gd["pixel"][0]]
    ids, alpha, T, w, Tf, fl = oracle.pixel_walk(sc, cam, pix[0] % c["width"] + 0.5, pix[0] // c["width"] + 0.5)
    np.testing.assert_allclose(w, e["w_walk"], rtol=1e-14)
    np.testing.assert_allclose(Tf, e["T_final"], rtol=1e-14)
    for K in (1, 2, 3, 4):
        r = oracle.render(sc, cam, K=K, pixels=pix)
        ek = e[f"K{K}"]
        np.testing.assert_array_equal(r["idx"][0], ek["idx"])
        np.testing.assert_allclose(r["w"][0], ek["w"], rtol=1e-14)
        np.testing.assert_allclose(r["F"][0], ek["F"], rtol=1e-14, atol=1e-16)
        np.testing.assert_allclose(r["C"][0], e["C"], rtol=1e-14)
        np.testing.assert_allclose(r["D"][0], e["D"], rtol=1e-14)
        assert r["n"][0] == e["n_contrib"]


# ----------------------------------------------------------------------------------
# projection against an independent derivation
# ----------------------------------------------------------------------------------
def _proj_uv(cam, mu):
    vm = cam.viewmat.astype(np.float64)
    p = vm[:3, :3] @ mu + vm[:3, 3]
    return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])


@pytest.mark.parametrize("seed", [0, 1])
def test_projection_matches_numerical_jacobian(seed):
    """Sigma2D must equal J_num Sigma3D J_num^T + 0.3 I with J_num the central-difference
    Jacobian of the pinhole map mu -> (u, v) (inside the frustum clamp), under a
    general camera pose."""
    rng = np.random.default_rng(seed)
    cams = S.orbit_cameras(seed, [(320, 240, 262.5)], radius=3.0)
    cam = cams[0]
    sc = S.random_scene_box(seed, 64, 4, box=((-0.5, 0.5), (-0.4, 0.4), (2.5, 3.5)))
    sc = scene_from(sc.mean3d, sc.cov3d, sc.opacity, sc.rgb, sc.feats)
    pr = oracle.project(sc, cam)
    checked = 0
    for g in range(sc.n):
        if pr[g, oracle.P_VALID] == 0 or pr[g, 15] or pr[g, 16]:
            continue
        mu = sc.mean3d[g]
        h = 1e-6
        Jn = np.stack([(_proj_uv(cam, mu + h * e) - _proj_uv(cam, mu - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        c6 = sc.cov3d[g]
        Sg = np.array([[c6[0], c6[1], c6[2]], [c6[1], c6[3], c6[4]], [c6[2], c6[4], c6[5]]])
        S2 = Jn @ Sg @ Jn.T + 0.3 * np.eye(2)
        np.testing.assert_allclose([pr[g, oracle.P_SA], pr[g, oracle.P_SB], pr[g, oracle.P_SC]],
                                   [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=2e-6, atol=1e-9)
        np.testing.assert_allclose(pr[g, oracle.P_U:oracle.P_V + 1], _proj_uv(cam, mu), rtol=1e-13)
        conic = np.linalg.inv(S2)
        np.testing.assert_allclose([pr[g, oracle.P_CA], pr[g, oracle.P_CB], pr[g, oracle.P_CC]],
                                   [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=2e-5)
        checked += 1
    assert checked > 10


def test_projection_frustum_clamp_closed_form():
    """Outside 1.3 tan(fov/2) the Jacobian uses the clamped ratio: for an isotropic
    Gaussian at y = 0 and x/z beyond the limit, Sigma2D = s^2 diag(fx^2 (1 + l^2),
    fy^2) / z^2 + 0.3 I with l = 1.3 W / (2 fx)."""
    cam = S.pinhole(64, 48, 40.0)
    z, s = 2.0, 0.05
    lim = 1.3 * cam.width / (2 * cam.fx)
    sc = scene_from([2.0 * lim * z, 0, z], iso(s), [0.5], [1, 1, 1], [[1.0]])
    pr = oracle.project(sc, cam)[0]
    exp_a = s * s * cam.fx ** 2 * (1 + lim ** 2) / z ** 2 + 0.3
    exp_c = s * s * cam.fy ** 2 / z ** 2 + 0.3
    np.testing.assert_allclose([pr[oracle.P_SA], pr[oracle.P_SB], pr[oracle.P_SC]], [exp_a, 0, exp_c], rtol=1e-14, atol=1e-15)


def test_near_plane_cull():
    cam = axis_cam()
    sc = scene_from([[0, 0, 0.1], [0, 0, -1.0]], [iso(0.05)] * 2, [0.9, 0.9], [[1, 1, 1]] * 2, [[1.0]] * 2)
    pr = oracle.project(sc, cam)
    assert pr[0, oracle.P_VALID] == 0 and pr[1, oracle.P_VALID] == 0


# ----------------------------------------------------------------------------------
# invariants on seeded scenes
# ----------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_scene():
    sc, cams, K, tile, _ = S.make_config("small", 0)
    return sc, cams[0], K


def test_invariants_small(small_scene):
    sc, cam, K = small_scene
    r = oracle.render(sc, cam, K)
    w = r["w"]
    assert np.all(w >= 0) and np.all(w <= 1)
    assert np.all(np.diff(w, axis=1) <= 0)                       # descending slots
    valid = r["idx"] >= 0
    assert np.all(valid.sum(1) == np.minimum(r["n"], K))
    for row in r["idx"]:
        v = row[row >= 0]
        assert len(set(v.tolist())) == len(v)
    assert np.all(np.linalg.norm(r["F"], axis=1) <= 1 + 1e-12)   # convex blend of unit rows
    assert np.all((r["T"] >= 1e-4) & (r["T"] <= 1))
    # Eq. 1 telescoping: sum of all weights = 1 - T_final; transmittance is non-increasing
    rng = np.random.default_rng(0)
    for p in rng.choice(cam.n_pix, 64, replace=False):
        ids, alpha, T, ww, Tf, fl = oracle.pixel_walk(sc, cam, p % cam.width + 0.5, p // cam.width + 0.5)
        np.testing.assert_allclose(ww.sum(), 1 - Tf, rtol=1e-12, atol=1e-15)
        assert np.all(np.diff(T) <= 0) and np.all(ww == alpha * T)
        assert len(ids) == r["n"][p]


def test_large_k_is_normalised_alpha_blend(small_scene):
    """With K at least the contributor count, Eq. 4 with Eq. 3's renormalisation is the
    full alpha blend divided by its total weight 1 - T_final."""
    sc, cam, _ = small_scene
    pix = np.arange(0, cam.n_pix, 37)
    r = oracle.render(sc, cam, K=256, pixels=pix)
    for j, p in enumerate(pix):
        ids, alpha, T, w, Tf, fl = oracle.pixel_walk(sc, cam, p % cam.width + 0.5, p // cam.width + 0.5)
        if len(ids) == 0:
            np.testing.assert_array_equal(r["F"][j], 0)
            continue
        full = (w[:, None] * sc.feats[ids].astype(np.float64)).sum(0) / (1 - Tf)
        np.testing.assert_allclose(r["F"][j], full, rtol=1e-10, atol=1e-12)


def test_k1_is_argmax(small_scene):
    sc, cam, _ = small_scene
    pix = np.arange(0, cam.n_pix, 41)
    r = oracle.render(sc, cam, K=1, pixels=pix)
    for j, p in enumerate(pix):
        ids, alpha, T, w, Tf, fl = oracle.pixel_walk(sc, cam, p % cam.width + 0.5, p // cam.width + 0.5)
        if len(ids) == 0:
            continue
        best = ids[int(np.argmax(w))]
        assert r["idx"][j, 0] == best
        np.testing.assert_allclose(r["F"][j], sc.feats[best], rtol=1e-7)


def test_compositing_split_identity():
    """Eq. 1 is front-to-back 'over' compositing: rendering the Gaussians nearer than
    z0 and those beyond separately, C = C_front + T_front C_back and
    T = T_front T_back (no early stop at these opacities)."""
    sc = S.random_scene_box(3, 40, 4, box=((-0.3, 0.3), (-0.3, 0.3), (1.0, 4.0)))
    sc = scene_from(sc.mean3d, sc.cov3d, np.minimum(sc.opacity, 0.4), sc.rgb, sc.feats)
    cam = S.pinhole(24, 24, 30.0)
    z0 = 2.5
    front = np.nonzero(sc.mean3d[:, 2] < z0)[0]
    back = np.nonzero(sc.mean3d[:, 2] >= z0)[0]
    ra = oracle.render(sc, cam, 4)
    rf = oracle.render(sc.subset(front), cam, 4)
    rb = oracle.render(sc.subset(back), cam, 4)
    ok = (ra["T"] > 1e-3)
    assert ok.mean() > 0.9
    np.testing.assert_allclose(ra["C"][ok], (rf["C"] + rf["T"][:, None] * rb["C"])[ok], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(ra["T"][ok], (rf["T"] * rb["T"])[ok], rtol=1e-12)
    np.testing.assert_allclose(ra["D"][ok], (rf["D"] + rf["T"] * rb["D"])[ok], rtol=1e-12, atol=1e-14)


def test_permutation_invariance(small_scene):
    sc, cam, K = small_scene
    perm = np.random.default_rng(5).permutation(sc.n)
    inv = np.argsort(perm)
    pix = np.arange(0, cam.n_pix, 7)
    ra = oracle.render(sc, cam, K, pixels=pix)
    rb = oracle.render(sc.subset(perm), cam, K, pixels=pix)
    np.testing.assert_allclose(rb["F"], ra["F"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(rb["C"], ra["C"], rtol=1e-12, atol=1e-14)
    mapped = np.where(rb["idx"] >= 0, perm[np.maximum(rb["idx"], 0)], -1)
    np.testing.assert_array_equal(mapped, ra["idx"])
    del inv


def test_topk_brute_force_subsets():
    """On a tiny scene every K-subset of each pixel's contributors is enumerated: the
    oracle's Top-K set is the unique subset of largest total weight (Eq. 2), unless
    flagged as a near-tie."""
    sc = S.random_scene_box(11, 30, 3, box=((-0.4, 0.4), (-0.4, 0.4), (1.0, 3.0)),
                            log_scale_mu=-2.5)
    cam = S.pinhole(16, 16, 20.0)
    K = 3
    r = oracle.render(sc, cam, K)
    checked = 0
    for p in range(cam.n_pix):
        ids, alpha, T, w, Tf, fl = oracle.pixel_walk(sc, cam, p % 16 + 0.5, p // 16 + 0.5)
        if len(ids) <= K or (r["flags"][p] & oracle.F_NEAR_TIE):
            continue
        best = max(itertools.combinations(range(len(ids)), K), key=lambda c: sum(w[i] for i in c))
        assert set(ids[list(best)].tolist()) == set(r["idx"][p].tolist())
        checked += 1
    assert checked > 50


# ----------------------------------------------------------------------------------
# backward against central finite differences of the forward
# ----------------------------------------------------------------------------------
def _fd_scene():
    rng = np.random.default_rng(21)
    n, D = 8, 4
    mean = np.stack([rng.uniform(-0.25, 0.25, n), rng.uniform(-0.25, 0.25, n), rng.uniform(1.5, 3.0, n)], 1)
    base = S._random_cov6(rng, n, -2.3, 0.3)
    opac = rng.uniform(0.2, 0.8, n)
    rgb = rng.uniform(0, 1, (n, 3))
    feats = rng.standard_normal((n, D))
    feats /= np.linalg.norm(feats, axis=1, keepdims=True)
    return scene_from(mean, base, opac, rgb, feats), S.pinhole(12, 12, 16.0)


def _loss_and_signature(sc, cam, K, up):
    dF, dC, dD = up
    r = oracle.render(sc, cam, K)
    L = float((dF * r["F"]).sum() + (dC * r["C"]).sum() + (dD * r["D"]).sum())
    sig = []
    for p in range(cam.n_pix):
        ids, alpha, T, w, Tf, fl = oracle.pixel_walk(sc, cam, p % cam.width + 0.5, p // cam.width + 0.5)
        sig.append((tuple(ids.tolist()), tuple((alpha >= 0.99).tolist())))
    sig.append(tuple(map(tuple, np.sort(r["idx"], axis=1).tolist())))
    return L, sig


@pytest.mark.parametrize("K", [2, 16])
def test_backward_matches_central_differences(K):
    sc, cam = _fd_scene()
    D = sc.d
    up = S.upstream_grads(4, cam.n_pix, D)
    up = tuple(a.astype(np.float64) for a in up)
    g = oracle.backward(sc, cam, K, *up)
    _, sig0 = _loss_and_signature(sc, cam, K, up)
    fields = [("mean3d", "mean3d"), ("cov3d", "cov3d"), ("opacity", "opac"), ("rgb", "rgb"), ("feats", "feat")]
    n_checked = n_skipped = 0
    for attr, key in fields:
        arr = getattr(sc, attr)
        flat = arr.reshape(-1)
        ga = g[key].reshape(-1)
        for i in range(flat.size):
            h = 1e-7 * max(1.0, abs(flat[i])) if attr != "cov3d" else 1e-9
            old = flat[i]
            flat[i] = old + h
            Lp, sp = _loss_and_signature(sc, cam, K, up)
            flat[i] = old - h
            Lm, sm = _loss_and_signature(sc, cam, K, up)
            flat[i] = old
            if sp != sig0 or sm != sig0:
                n_skipped += 1
                continue
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - ga[i]) <= 2e-6 * max(1.0, abs(fd)), (attr, i, fd, ga[i])
            n_checked += 1
    assert n_checked > 0.8 * (n_checked + n_skipped)


def test_backward_2d_gradients_by_perturbing_projection():
    """The 2D gradients (mean2d, conic, opacity) against central differences taken
    directly on the projected record."""
    sc, cam = _fd_scene()
    K = 2
    up = tuple(a.astype(np.float64) for a in S.upstream_grads(9, cam.n_pix, sc.d))
    proj = oracle.project(sc, cam)
    g = oracle.backward(sc, cam, K, *up, proj=proj)

    def loss(pr):
        r = oracle.render(sc, cam, K, proj=pr)
        return float((up[0] * r["F"]).sum() + (up[1] * r["C"]).sum() + (up[2] * r["D"]).sum()), r["n"].copy(), r["idx"].copy()

    L0, n0, i0 = loss(proj)
    for gidx in range(sc.n):
        for col, ref in [(oracle.P_U, g["mean2d"][gidx, 0]), (oracle.P_V, g["mean2d"][gidx, 1]),
                         (oracle.P_CA, g["conic"][gidx, 0]), (oracle.P_CB, g["conic"][gidx, 1]),
                         (oracle.P_CC, g["conic"][gidx, 2])]:
            h = 1e-7 * max(1.0, abs(proj[gidx, col]))
            pp = proj.copy(); pp[gidx, col] += h
            pm = proj.copy(); pm[gidx, col] -= h
            Lp, np_, ip = loss(pp)
            Lm, nm, im = loss(pm)
            if not (np.array_equal(np_, n0) and np.array_equal(nm, n0) and np.array_equal(ip, i0) and np.array_equal(im, i0)):
                continue
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - ref) <= 2e-6 * max(1.0, abs(fd)), (gidx, col, fd, ref)


def test_pose_gradient_matches_central_differences():
    """The gradient with respect to the world-to-camera [R | t] (pose refinement) against
    central differences of the FP64 forward, the camera perturbed entry by entry in
    float64; entries whose perturbation changes a discrete decision are skipped."""
    sc, cam = _fd_scene()
    K = 2
    up = tuple(a.astype(np.float64) for a in S.upstream_grads(12, cam.n_pix, sc.d))
    ca0 = oracle.cam_array(cam)
    g = oracle.backward(sc, cam, K, *up)["viewmat"]

    def loss(ca):
        r = oracle.render(sc, cam, K, proj=oracle.project(sc, cam, cam_arr=ca))
        return (float((up[0] * r["F"]).sum() + (up[1] * r["C"]).sum() + (up[2] * r["D"]).sum()),
                r["n"].copy(), np.sort(r["idx"], axis=1))

    L0, n0, i0 = loss(ca0)
    checked = 0
    for i in range(3):
        for j in range(4):
            k = 3 * i + j if j < 3 else 9 + i                 # R row-major, then t
            h = 1e-7
            cp, cm = ca0.copy(), ca0.copy()
            cp[k] += h
            cm[k] -= h
            Lp, np_, ip = loss(cp)
            Lm, nm, im = loss(cm)
            if not (np.array_equal(np_, n0) and np.array_equal(nm, n0) and np.array_equal(ip, i0)
                    and np.array_equal(im, i0)):
                continue
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[i, j]) <= 2e-5 * max(1.0, abs(fd)), (i, j, fd, g[i, j])
            checked += 1
    assert checked >= 9
